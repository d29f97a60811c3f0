// Small device helpers: vector loads, warp/CTA reductions in FP64.
#pragma once

#include <cuda_runtime.h>
#include "ax_internal.cuh"

namespace ax {

template <typename T> struct VecT;
template <> struct VecT<float> { using type = float4; static constexpr int n = 4; };
template <> struct VecT<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void load_vec(const T *p, T (&v)[VecT<T>::n]);
template <>
__device__ __forceinline__ void load_vec<float>(const float *p, float (&v)[4]) {
  float4 t = *reinterpret_cast<const float4 *>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void load_vec<double>(const double *p, double (&v)[2]) {
  double2 t = *reinterpret_cast<const double2 *>(p);
  v[0] = t.x; v[1] = t.y;
}
template <typename T>
__device__ __forceinline__ void store_vec(T *p, const T (&v)[VecT<T>::n]);
template <>
__device__ __forceinline__ void store_vec<float>(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store_vec<double>(double *p, const double (&v)[2]) {
  *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic CTA sum (fixed order); result valid in thread 0.
// `red` must hold blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += red[w];
  }
  return s;
}

__device__ __forceinline__ bool rhs_selected(const RhsState *st, int mask, int m) {
  return mask < 0 || st[m].state == mask;
}

}  // namespace ax
