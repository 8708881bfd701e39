"""Differentiable bundle adjustment: a torch.autograd.Function around the library.

Forward: Levenberg-Marquardt to convergence on the GPU (ba_create, ba_lm_solve).  Backward: the
implicit-differentiation adjoint (ba_adjoint) solved with the same power-series Schur kernels at
the damping `adjoint_lambda` (default: the LM's final lambda), giving the gradients of the
converged cameras and landmarks with respect to the observations and the per-observation
weights.  The initial state is not differentiated (a local minimiser does not depend on it).

The adjoint series converges more slowly as its damping falls (its ratio approaches 1 along the
gauge directions), and the LM's final lambda is often tiny (down to its floor of 1e-10).  With
the default 20 terms the backward solve is then truncated and the gradient is only an
approximation: the series state of each backward (terms, stopped, stop value) is kept in
`BundleAdjustment.last_adjoint_info`, and a RuntimeWarning is raised when the stop rule did
not fire.  Pass a larger adjoint_lambda and / or adjoint_options with a larger max_inner (and a
smaller eps) for an accurate gradient.
"""
from __future__ import annotations

import warnings
from typing import Optional

import torch

from . import (BA_FP64, Options, ba_adjoint, ba_create, ba_default_options, ba_get_lm_state,
               ba_get_params, ba_lm_solve, ba_set_options)


class BundleAdjustment(torch.autograd.Function):
    # series state of the most recent backward solve ({"inner_iters", "stopped", "stop_value",
    # "x_norm", "lam"}), or None before the first backward
    last_adjoint_info: Optional[dict] = None

    @staticmethod
    def forward(ctx, obs, weights, cams0, lms0, cam_idx, lm_idx, precision, options,
                adjoint_lambda, adjoint_options):
        opts = options if options is not None else ba_default_options()
        h = ba_create(cams0.detach().contiguous(), lms0.detach().contiguous(),
                      obs.detach().contiguous(), cam_idx.contiguous(), lm_idx.contiguous(),
                      None if weights is None else weights.detach().contiguous(),
                      precision=precision, options=opts,
                      stream=torch.cuda.current_stream(obs.device))
        steps = ba_lm_solve(h, max_lm=opts.max_lm)
        cams = torch.empty_like(cams0, dtype=torch.float64)
        lms = torch.empty_like(lms0, dtype=torch.float64)
        ba_get_params(h, cams, lms)
        ctx.h = h
        ctx.options = opts
        ctx.lam = float(adjoint_lambda) if adjoint_lambda else ba_get_lm_state(h)["lam"]
        ctx.adjoint_options = adjoint_options
        ctx.has_weights = weights is not None
        ctx.steps = len(steps)
        return cams, lms

    @staticmethod
    def backward(ctx, g_cams, g_lms):
        h = ctx.h
        if g_cams is None:
            g_cams = torch.zeros((h.n_cams, 9), dtype=torch.float64, device="cuda")
        if g_lms is None:
            g_lms = torch.zeros((h.n_lms, 3), dtype=torch.float64, device=g_cams.device)
        want_w = ctx.has_weights and ctx.needs_input_grad[1]
        if ctx.adjoint_options is not None:
            ba_set_options(h, ctx.adjoint_options)
        try:
            d_obs, d_w, info = ba_adjoint(h, ctx.lam, g_cams.to(torch.float64).contiguous(),
                                          g_lms.to(torch.float64).contiguous(),
                                          want_weights=want_w)
        finally:
            # the handle keeps the forward's options (the adjoint's apply to this solve only)
            if ctx.adjoint_options is not None:
                ba_set_options(h, ctx.options)
        BundleAdjustment.last_adjoint_info = info
        if not info["stopped"]:
            warnings.warn(f"bundle_adjust backward: the adjoint series stopped at its term cap "
                          f"({info['inner_iters']} terms, stop value {info['stop_value']:.3g}) "
                          f"at lambda {ctx.lam:.3g}; the gradient is truncated (pass a larger "
                          f"adjoint_lambda or adjoint_options with a larger max_inner)",
                          RuntimeWarning, stacklevel=2)
        return (d_obs if ctx.needs_input_grad[0] else None, d_w if want_w else None,
                None, None, None, None, None, None, None, None)


def bundle_adjust(obs: torch.Tensor, cams0: torch.Tensor, lms0: torch.Tensor,
                  cam_idx: torch.Tensor, lm_idx: torch.Tensor,
                  weights: Optional[torch.Tensor] = None, precision: int = BA_FP64,
                  options: Optional[Options] = None, adjoint_lambda: Optional[float] = None,
                  adjoint_options: Optional[Options] = None):
    """(cams*, lms*) = argmin F; differentiable with respect to obs and weights (CUDA float64
    tensors).  adjoint_options (eps, max_inner, ...) apply to the backward solve only.  The
    backward solves the adjoint system with the power series at adjoint_lambda (default: the
    LM's final lambda, often tiny); where the series hits its term cap before its stop rule the
    gradient is truncated, a RuntimeWarning says so, and BundleAdjustment.last_adjoint_info
    holds the series state.  For accurate gradients pass adjoint_lambda (e.g. 1e-2) and
    adjoint_options with a larger max_inner (hundreds of terms) and a smaller eps."""
    return BundleAdjustment.apply(obs, weights, cams0, lms0, cam_idx, lm_idx, precision, options,
                                  adjoint_lambda, adjoint_options)
