"""FP64 CPU oracle for Power Bundle Adjustment (Weber et al., "Power Bundle Adjustment for
Large-Scale 3D Reconstruction").

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct restatement of the
method that the CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import it; the library in
``paper_2204_12834_gb300`` never does, and the two share no code (the seeded problem generator
``bal_synth`` is the only module both read).

Layout (each function cites the passage it restates):
  camera_model   -- BAL projection, residuals r, Jacobians J_p, J_l by forward-mode dual numbers
                    (Sec. 4: objective F(x) = 1/2 ||r(x)||^2, d_p = 9)
  normal_eq      -- J assembly, U_lambda, V_lambda, W, b (Sec. 4.1 eq. `normal`), damping,
                    block Cholesky inverses, Schur complement S and b~ (Sec. 4.2 eqs. `Sx`,
                    `Schur`), back-substitution (Sec. 4.2 eq. `back_substitution`, sign derived)
  power_series   -- truncated inverse expansion x(m) (Sec. 4.3 eqs. `S_approx`, `x_approx`) and
                    the stop rule (eq. `qcriterion`), plus the operator P = U^-1 W V^-1 W^T
  direct         -- exact solves of S dx_p = -b~: dense Cholesky, Schur-Jacobi PCG
  lm             -- Levenberg-Marquardt outer loop with the settings of Sec. 5.1 ("LM loop")
  pcg            -- conjugate gradients on the reduced system, matrix-free, with the Schur-Jacobi
                    (Sec. 5) or the truncated power-series (eq. `S_approx`) preconditioner
  adjoint        -- implicit-differentiation adjoint of the solution (no paper counterpart):
                    H_lam a = dL/dx through the Schur complement, gradients w.r.t. observations
                    and weights

Parity status: every function above is pinned by ``tests/test_oracle_*.py`` against closed
forms, finite differences, brute-force dense solves, Lemma 1 / Prop. 1 / Prop. 2 identities,
library routines (matrix exponential, dense Cholesky) or scripted sequences, and
``tests/test_oracle_planted_mistakes.py`` checks that one-line mistakes planted in every function
that computes a step of the method make those pins fail.  The one exception is the LM trajectory itself (the lambda-update rule is
not printed in the paper): "parity unpinned" against the paper, pinned only by invariants
(cost never increases on accepted steps, convergence to the noise floor).
"""
from . import camera_model, normal_eq, power_series, direct, lm, pcg, adjoint  # noqa: F401
