// Device access to the Jacobian planes in their 16-byte plane groups (layout: jidx in
// poba_internal.cuh).  One observation's 24 values move with 6 (float) or 12 (double) 16-byte
// loads or stores, and a warp's access to one group covers 512 contiguous bytes.
#pragma once

#include <cstddef>
#include <cstdint>

#include "poba_internal.cuh"

namespace poba {

template <typename T> struct Vec16Of;
template <> struct Vec16Of<float> { using type = float4; };
template <> struct Vec16Of<double> { using type = double2; };
template <typename T> using vec16 = typename Vec16Of<T>::type;

// The 24 planes of observation o as 16-byte groups: group q of o at G[q * pad + o].
template <typename T>
__device__ __forceinline__ const vec16<T>* jgroups(const T* J) {
  return reinterpret_cast<const vec16<T>*>(J);
}

__device__ __forceinline__ void unpack16(const float4& v, float* d) {
  d[0] = v.x;
  d[1] = v.y;
  d[2] = v.z;
  d[3] = v.w;
}
__device__ __forceinline__ void unpack16(const double2& v, double* d) {
  d[0] = v.x;
  d[1] = v.y;
}
__device__ __forceinline__ float4 pack16(const float* s) { return make_float4(s[0], s[1], s[2], s[3]); }
__device__ __forceinline__ double2 pack16(const double* s) { return make_double2(s[0], s[1]); }

// Reads of data that an FP64 series term streams once (the Jacobians, chunk records and V^-1 rows)
// carry an L2 evict-first policy, so that the small state read again every term -- partial
// rows, t, x, U^-1 -- stays in L2 while the Jacobians pass through it.  (Measured on GB300: the
// FP64 term gains about 4 %; FP32-bulk terms lose a little with it and read without it.)
__device__ __forceinline__ uint64_t l2_stream_policy() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ double2 ldg_stream(const double2* p, uint64_t pol) {
  double2 v;
  asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
      : "=d"(v.x), "=d"(v.y)
      : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ldg_stream(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

// J_p (18 values, row-major) and J_l (6) of observation o.
template <typename T>
__device__ __forceinline__ void load_J(const T* __restrict__ J, size_t pad, int o, T (&jp)[18],
                                       T (&jl)[6]) {
  constexpr int V = jgroup<T>();
  const vec16<T>* G = jgroups(J);
  T all[24];
#pragma unroll
  for (int q = 0; q < 24 / V; ++q) unpack16(__ldg(G + (size_t)q * pad + o), all + q * V);
#pragma unroll
  for (int p = 0; p < 18; ++p) jp[p] = all[p];
#pragma unroll
  for (int p = 0; p < 6; ++p) jl[p] = all[18 + p];
}

// load_J of FP64 planes with the streaming policy.
__device__ __forceinline__ void load_J_stream(const double* __restrict__ J, size_t pad, int o,
                                              double (&jp)[18], double (&jl)[6], uint64_t pol) {
  const double2* G = jgroups(J);
  double all[24];
#pragma unroll
  for (int q = 0; q < 12; ++q) unpack16(ldg_stream(G + (size_t)q * pad + o, pol), all + 2 * q);
#pragma unroll
  for (int p = 0; p < 18; ++p) jp[p] = all[p];
#pragma unroll
  for (int p = 0; p < 6; ++p) jl[p] = all[18 + p];
}

template <typename T>
__device__ __forceinline__ void store_J(T* __restrict__ J, size_t pad, int o, const T (&jp)[18],
                                        const T (&jl)[6]) {
  constexpr int V = jgroup<T>();
  vec16<T>* G = reinterpret_cast<vec16<T>*>(J);
  T all[24];
#pragma unroll
  for (int p = 0; p < 18; ++p) all[p] = jp[p];
#pragma unroll
  for (int p = 0; p < 6; ++p) all[18 + p] = jl[p];
#pragma unroll
  for (int q = 0; q < 24 / V; ++q) G[(size_t)q * pad + o] = pack16(all + q * V);
}

}  // namespace poba
