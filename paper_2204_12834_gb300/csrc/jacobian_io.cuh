// Device access to the Jacobian planes in their 16-byte plane groups (layout: jidx in
// poba_internal.cuh).  One observation's 24 values move with 6 (float) or 12 (double) 16-byte
// loads or stores, and a warp's access to one group covers 512 contiguous bytes.
#pragma once

#include <cstddef>

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
