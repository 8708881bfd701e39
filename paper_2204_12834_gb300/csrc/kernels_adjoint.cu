// Implicit-differentiation adjoint kernels of libpoba.  The paper has no adjoint; the method
// reuses its solver.  The solution x* satisfies g(x*, theta) = sum_o w_o J_o^T r_o = 0 with
// theta = (obs, w).  With the damped Gauss-Newton matrix H_lam of eq. `normal` standing in for
// dg/dx, a scalar L(x*) has
//   a = H_lam^-1 dL/dx   (solved by the Schur complement and the power series, with the
//                         right-hand side -(dL/dx) in place of b),
//   dL/dobs_o = w_o J_o a_o,   dL/dw_o = -r_o^T J_o a_o,
// where a_o is the part of a at observation o's camera and landmark.
#include "poba_internal.cuh"

namespace poba {

// adj_p = -g_p (cameras, caller order = internal order); adj_l[i] = -g_l[lm_order[i]].
__global__ void adjoint_rhs_kernel(int n_cams, int n_lms, const int32_t* __restrict__ lm_order,
                                   const double* __restrict__ g_p, const double* __restrict__ g_l,
                                   double* __restrict__ adj_p, double* __restrict__ adj_l) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_cams * 9) adj_p[i] = -g_p[i];
  if (i < n_lms * 3) {
    const int l = i / 3, k = i - 3 * l;
    adj_l[i] = -g_l[(size_t)lm_order[l] * 3 + k];
  }
}

void launch_adjoint_rhs(int n_cams, int n_lms, const int32_t* lm_order, const double* g_p,
                        const double* g_l, double* adj_p, double* adj_l, cudaStream_t s) {
  const int n = n_cams * 9 > n_lms * 3 ? n_cams * 9 : n_lms * 3;
  adjoint_rhs_kernel<<<(n + 255) / 256, 256, 0, s>>>(n_cams, n_lms, lm_order, g_p, g_l, adj_p,
                                                     adj_l);
}

// One thread per (sorted) observation: u = sqrt(w) J a (the stored J and r carry sqrt(w)),
// d_obs[caller] = sqrt(w) u, d_w[caller] = -(sqrt(w) r) . u / w.  Accumulation in float64.
template <typename T>
__global__ void obs_gradient_kernel(Topology tp, const T* __restrict__ J, const T* __restrict__ r,
                                    const double* __restrict__ sqrt_w,
                                    const double* __restrict__ a_p, const double* __restrict__ a_l,
                                    const int32_t* __restrict__ obs_caller,
                                    double* __restrict__ d_obs, double* __restrict__ d_w) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= tp.n_obs) return;
  const size_t pad = (size_t)tp.n_obs_pad;
  const int c = tp.cam_of[o], l = tp.lm_of[o];
  double ap[9], al[3];
#pragma unroll
  for (int j = 0; j < 9; ++j) ap[j] = a_p[(size_t)c * 9 + j];
#pragma unroll
  for (int j = 0; j < 3; ++j) al[j] = a_l[(size_t)l * 3 + j];
  double u[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < 9; ++j) v += (double)J[jidx<T>(9 * i + j, o, pad)] * ap[j];
#pragma unroll
    for (int j = 0; j < 3; ++j) v += (double)J[jidx<T>(18 + 3 * i + j, o, pad)] * al[j];
    u[i] = v;
  }
  const double sw = sqrt_w ? sqrt_w[o] : 1.0;
  const int oc = obs_caller[o];
  d_obs[(size_t)oc * 2 + 0] = sw * u[0];
  d_obs[(size_t)oc * 2 + 1] = sw * u[1];
  if (d_w) d_w[oc] = -((double)r[o] * u[0] + (double)r[pad + o] * u[1]) / (sw * sw);
}

template <typename T>
void launch_obs_gradient(const Topology& tp, const T* J, const T* r, const double* sqrt_w,
                         const double* a_p, const double* a_l, const int32_t* obs_caller,
                         double* d_obs, double* d_w, cudaStream_t s) {
  if (tp.n_obs == 0) return;
  obs_gradient_kernel<T><<<(tp.n_obs + 255) / 256, 256, 0, s>>>(tp, J, r, sqrt_w, a_p, a_l,
                                                                 obs_caller, d_obs, d_w);
}

template void launch_obs_gradient<double>(const Topology&, const double*, const double*, const double*, const double*, const double*, const int32_t*, double*, double*, cudaStream_t);
template void launch_obs_gradient<float>(const Topology&, const float*, const float*, const double*, const double*, const double*, const int32_t*, double*, double*, cudaStream_t);

}  // namespace poba
