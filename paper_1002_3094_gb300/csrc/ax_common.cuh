// Small device helpers: vector loads, warp/CTA reductions in FP64.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
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
  if (mask == kDue) return st[m].state == kActive && st[m].due != 0;
  return mask < 0 || st[m].state == mask;
}

// ---- mbarrier and bulk-copy primitives (PTX) --------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity (at most `polls` tries);
// false when it expired.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned polls) {
  for (unsigned i = 0; i < polls; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// ---------------------------------------------------------------------------
// BF16 operand of the tensor-core transform ("split" layout).  A field x is
// stored as x = hi + lo, hi = bf16(x), lo = bf16(x - hi), in tiles of 128 rows
// x 64 positions per right-hand side: tile (m, row / 128, pos / 64) is 32 KB,
// the 16 KB of high parts and then the 16 KB of low parts, each as 8 x 8 core
// matrices of 16-byte rows, element (row, pos) at byte
//   (row % 128 / 8) 1024 + (pos % 64 / 8) 128 + (row % 8) 16 + (pos % 8) 2.
// Columns are stored even ones first (the operand order of the transform's
// even / odd split): column c at position c / 2 if c is even, else at
// kbe 64 + c / 2, with kbe = ceil(n8 / 2 / 64) tiles of even columns and as
// many of odd ones, n8 = n rounded up to 8.  Writers store whole chunks of 8
// columns c < n8 only (chunk starts c < n), which keeps every position inside.
// A tile is copied to shared memory as it is.  Padding rows and positions
// hold zeros (the buffer is zeroed when allocated and never written there).
// ---------------------------------------------------------------------------
constexpr int kSplitTileBytes = 32768;

__device__ __forceinline__ int split_pos(int c, int kbe) { return (c & 1) ? kbe * 64 + (c >> 1) : (c >> 1); }
__device__ __forceinline__ size_t split_byte(int m, int row, int pos, int mtiles, int ktiles) {
  return (((size_t)m * mtiles + (row >> 7)) * ktiles + (pos >> 6)) * (size_t)kSplitTileBytes +
         ((row & 127) >> 3) * 1024 + ((pos & 63) >> 3) * 128 + (row & 7) * 16 + (pos & 7) * 2;
}
__device__ __forceinline__ unsigned bf16_pack2(float a, float b) {
  // round-to-nearest-even BF16 of a (low half, lower address) and b, by the
  // packed conversion instruction
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const unsigned *>(&h);
}
__device__ __forceinline__ float bf16_round(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }
// The two BF16 halves of a packed pair as FP32 (exact).
__device__ __forceinline__ float bf16_lo(unsigned p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16_hi(unsigned p) { return __uint_as_float(p & 0xFFFF0000u); }
// Writes the 8 consecutive columns col .. col + 7 (col % 8 == 0) of one row:
// the 4 even ones and the 4 odd ones each as 8 bytes of high and of low parts.
__device__ __forceinline__ void split_store8(unsigned char *split, int m, int row, int col, int mtiles, int ktiles,
                                             int kbe, const float (&x)[8]) {
  unsigned he[2], le[2], ho[2], lo[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    he[e] = bf16_pack2(x[4 * e], x[4 * e + 2]);
    ho[e] = bf16_pack2(x[4 * e + 1], x[4 * e + 3]);
    le[e] = bf16_pack2(x[4 * e] - bf16_lo(he[e]), x[4 * e + 2] - bf16_hi(he[e]));
    lo[e] = bf16_pack2(x[4 * e + 1] - bf16_lo(ho[e]), x[4 * e + 3] - bf16_hi(ho[e]));
  }
  unsigned char *te = split + split_byte(m, row, split_pos(col, kbe), mtiles, ktiles);
  unsigned char *to = split + split_byte(m, row, split_pos(col + 1, kbe), mtiles, ktiles);
  *reinterpret_cast<uint2 *>(te) = make_uint2(he[0], he[1]);
  *reinterpret_cast<uint2 *>(te + kSplitTileBytes / 2) = make_uint2(le[0], le[1]);
  *reinterpret_cast<uint2 *>(to) = make_uint2(ho[0], ho[1]);
  *reinterpret_cast<uint2 *>(to + kSplitTileBytes / 2) = make_uint2(lo[0], lo[1]);
}

// Writes the 4 consecutive columns col .. col + 3 (col % 4 == 0) of one row:
// the 2 even ones and the 2 odd ones each as 4 bytes of high and of low parts.
__device__ __forceinline__ void split_store4(unsigned char *split, int m, int row, int col, int mtiles, int ktiles,
                                             int kbe, const float (&x)[4]) {
  const unsigned he = bf16_pack2(x[0], x[2]), ho = bf16_pack2(x[1], x[3]);
  unsigned char *te = split + split_byte(m, row, split_pos(col, kbe), mtiles, ktiles);
  unsigned char *to = split + split_byte(m, row, split_pos(col + 1, kbe), mtiles, ktiles);
  *reinterpret_cast<unsigned *>(te) = he;
  *reinterpret_cast<unsigned *>(te + kSplitTileBytes / 2) = bf16_pack2(x[0] - bf16_lo(he), x[2] - bf16_hi(he));
  *reinterpret_cast<unsigned *>(to) = ho;
  *reinterpret_cast<unsigned *>(to + kSplitTileBytes / 2) = bf16_pack2(x[1] - bf16_lo(ho), x[3] - bf16_hi(ho));
}

// Folded input of the tensor-core cosine forward transform for the 8
// positions k0 .. k0 + 7 (k0 % 8 == 0) of one row, from x[e] = r_{k0+e} and
// xm[e] = r_{n-1-k0-e}: u_k = r_k + r_{n-1-k} at position k of the first K
// half, w_k = r_k - r_{n-1-k} at position kbe 64 + k of the second, for
// k < ceil(n/2) (the middle entry of odd n: u = r, w = 0), zeros after.
__device__ __forceinline__ void fold_store8(unsigned char *split, int m, int row, int k0, int n, int mtiles,
                                            int ktiles, int kbe, const float (&x)[8], const float (&xm)[8]) {
  const int ne = (n + 1) >> 1;
  unsigned uh[4], ul[4], wh[4], wl[4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    float u2[2], w2[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int k = k0 + e + j;
      const bool mid = 2 * k + 1 == n;
      u2[j] = k < ne ? (mid ? x[e + j] : x[e + j] + xm[e + j]) : 0.f;
      w2[j] = (k < ne && !mid) ? x[e + j] - xm[e + j] : 0.f;
    }
    const float uh0 = bf16_round(u2[0]), uh1 = bf16_round(u2[1]);
    const float wh0 = bf16_round(w2[0]), wh1 = bf16_round(w2[1]);
    uh[e / 2] = bf16_pack2(uh0, uh1);
    ul[e / 2] = bf16_pack2(u2[0] - uh0, u2[1] - uh1);
    wh[e / 2] = bf16_pack2(wh0, wh1);
    wl[e / 2] = bf16_pack2(w2[0] - wh0, w2[1] - wh1);
  }
  unsigned char *pu = split + split_byte(m, row, k0, mtiles, ktiles);
  unsigned char *pw = split + split_byte(m, row, kbe * 64 + k0, mtiles, ktiles);
  *reinterpret_cast<uint4 *>(pu) = make_uint4(uh[0], uh[1], uh[2], uh[3]);
  *reinterpret_cast<uint4 *>(pu + kSplitTileBytes / 2) = make_uint4(ul[0], ul[1], ul[2], ul[3]);
  *reinterpret_cast<uint4 *>(pw) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
  *reinterpret_cast<uint4 *>(pw + kSplitTileBytes / 2) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
}

}  // namespace ax
