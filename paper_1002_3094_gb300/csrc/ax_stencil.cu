// Variable-coefficient cylindrical 5-point stencil (Section 2.1, Eqs.
// poisson_diff_2, scheme_op_r_z, diff_approx1, sign-reversed so A > 0):
//
//   (A y)_{i,k} = CR_i (y_{i,k} - y_{i+1,k}) + CR_{i-1} (y_{i,k} - y_{i-1,k})
//               + CZ_{i,k} (y_{i,k} - y_{i,k+1}) + CZ_{i,k-1} (y_{i,k} - y_{i,k-1})
//               + W_{i,k} y_{i,k}
//
// with CR = KR / h_r^2, CZ = KZ / h_z^2 precomputed, CR_0 = 0 on the axis and
// zero values beyond the Dirichlet boundaries r = lr, z = 0, z = lz.
//
// One CTA owns kStencilRows consecutive r-rows and a strip of z-columns of one
// right-hand side.  Each lane holds a short vector (4 FP32 / 2 FP64) of
// consecutive z-nodes and walks down the rows with a three-row register
// window, so every input element is read from memory once (plus one halo row
// per CTA edge).  z-neighbours across lanes come from warp shuffles; the two
// warp-edge lanes fetch one extra element.  blockIdx.x is the right-hand side,
// so CTAs that share a coefficient tile run together and the tile is served
// from L2.
#include "ax_common.cuh"

namespace ax {

namespace {

template <typename T, int MODE>
struct StencilValue {
  // Value of the grid function the operator is applied to, at element e.
  __device__ __forceinline__ static T at(const T *in, const T *p_old, size_t e, T beta) {
    if (MODE == kStencilPcg) return in[e] + beta * p_old[e];
    return in[e];
  }
};

// Hint: bring the line holding p into L2 (no register, no completion; p must
// be a valid global address).
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <typename T, int MODE>
__global__ void __launch_bounds__(256) stencil_kernel(const StencilArgs<T> a) {
  constexpr int V = VecT<T>::n;
  __shared__ double red[8];
  const int m = blockIdx.x;
  if (!rhs_selected(a.st, a.mask, m)) return;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int k0 = ((blockIdx.z * nwarps + warp) * 32 + lane) * V;
  const int nr = a.nr, nz = a.nz;
  const int i0 = blockIdx.y * kStencilRows;
  const int i1 = min(i0 + kStencilRows, nr);
  const size_t base = (size_t)m * (size_t)a.field;
  const bool col_ok = k0 < nz;
  const T *__restrict__ CR = a.CR + (size_t)m * a.cstride;
  const T *__restrict__ CZ = a.CZ + (size_t)m * a.czstride;
  const T *__restrict__ Wc = a.W + (size_t)m * a.cstride;
  T beta = T(0);
  const T *p_old = nullptr;
  T *p_new = nullptr;
  const T *src = a.in;  // the grid function (before the direction update in mode Pcg)
  if (MODE == kStencilPcg) {
    beta = (T)a.st[m].beta;
    const bool odd = a.st[m].iters & 1;
    p_old = odd ? a.pb : a.pa;
    p_new = odd ? a.pa : a.pb;
  } else if (MODE == kStencilPcgP) {
    src = (a.st[m].iters & 1) ? a.pa : a.pb;
  }

  auto load_row = [&](int i, T (&v)[V]) {
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = T(0);
    if (!col_ok) return;
    const size_t off = base + (size_t)i * a.pitch + k0;
    T t[V];
    load_vec<T>(src + off, t);
    if (MODE == kStencilPcg) {
      T po[V];
      load_vec<T>(p_old + off, po);
#pragma unroll
      for (int e = 0; e < V; ++e) t[e] += beta * po[e];
    }
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = (k0 + e < nz) ? t[e] : T(0);
  };
  auto load_coef = [&](const T *c, int i, T (&v)[V]) {
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = T(0);
    if (!col_ok) return;
    load_vec<T>(c + (size_t)i * a.pitch + k0, v);
  };

  // Everything row i + 1 needs (values, its CR / CZ / W rows and the two
  // warp-edge halo values) is loaded one row ahead, while row i is computed.
  auto load_halo = [&](int i, T &left, T &right, T &czlast) {
    const size_t rowoff = base + (size_t)i * a.pitch;
    left = right = czlast = T(0);
    if (lane == 0 && col_ok && k0 > 0) left = StencilValue<T, MODE>::at(src, p_old, rowoff + k0 - 1, beta);
    if (lane == 31) {
      if (k0 + V < nz) right = StencilValue<T, MODE>::at(src, p_old, rowoff + k0 + V, beta);
      if (k0 + V <= nz) czlast = CZ[(size_t)i * a.pitchz + k0 + V];
    }
  };
  auto load_cz = [&](int i, T (&v)[V]) {
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = T(0);
    // Faces run to index nz, so the lane just past the last node still loads
    // its first face (the upper face of node nz - 1, fetched by the shuffle).
    if (k0 <= nz) load_vec<T>(CZ + (size_t)i * a.pitchz + k0, v);
  };

  // every row of the DRAM stream(s) this CTA reads, into L2 at once: the
  // register loads below then wait on L2 instead of DRAM
  if (col_ok)
    for (int i = max(i0 - 1, 0); i <= i1 && i < nr; ++i) {
      const size_t off = base + (size_t)i * a.pitch + k0;
      prefetch_l2(src + off);
      if (MODE == kStencilPcg) prefetch_l2(p_old + off);
      if ((MODE == kStencilResidual || MODE == kStencilCheb) && i >= i0 && i < i1) prefetch_l2(a.phi + off);
    }
  T pm[V], pc[V], pn[V], crl[V], crh[V], czl[V], w[V];
  T left, right, czlast;
  if (i0 > 0) {
    load_row(i0 - 1, pm);
    load_coef(CR, i0 - 1, crl);
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) { pm[e] = T(0); crl[e] = T(0); }
  }
  load_row(i0, pc);
  load_coef(CR, i0, crh);
  load_cz(i0, czl);
  load_coef(Wc, i0, w);
  load_halo(i0, left, right, czlast);

  // FP32 partials per thread are short sums (<= 64 terms); the CTA and grid
  // combination is FP64.
  T acc = T(0);
  for (int i = i0; i < i1; ++i) {
    T crn[V], czn[V], wn[V], leftn = T(0), rightn = T(0), czlastn = T(0);
    if (i + 1 < nr) {
      load_row(i + 1, pn);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) pn[e] = T(0);
    }
    if (i + 1 < i1) {
      load_coef(CR, i + 1, crn);
      load_cz(i + 1, czn);
      load_coef(Wc, i + 1, wn);
      load_halo(i + 1, leftn, rightn, czlastn);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) crn[e] = czn[e] = wn[e] = T(0);
    }
    const size_t rowoff = base + (size_t)i * a.pitch;
    // z-neighbours of the lane's first and last node.
    T l = __shfl_up_sync(0xffffffffu, pc[V - 1], 1);
    T r = __shfl_down_sync(0xffffffffu, pc[0], 1);
    T czh_last = __shfl_down_sync(0xffffffffu, czl[0], 1);
    if (lane == 0) l = left;
    if (lane == 31) {
      r = right;
      czh_last = czlast;
    }

    T o[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const T yl = (e == 0) ? l : pc[e - 1];
      const T yr = (e == V - 1) ? r : pc[e + 1];
      const T czh = (e == V - 1) ? czh_last : czl[e + 1];
      const T y = pc[e];
      T v = w[e] * y;
      v = fma(crh[e], y - pn[e], v);
      v = fma(crl[e], y - pm[e], v);
      v = fma(czh, y - yr, v);
      v = fma(czl[e], y - yl, v);
      o[e] = (k0 + e < nz) ? v : T(0);
    }
    if (col_ok) {
      if (MODE == kStencilApply) {
        store_vec<T>(a.out + rowoff + k0, o);
      } else if (MODE == kStencilPcg || MODE == kStencilPcgP) {
        if (MODE == kStencilPcg) store_vec<T>(p_new + rowoff + k0, pc);
        store_vec<T>(a.out + rowoff + k0, o);
#pragma unroll
        for (int e = 0; e < V; ++e) acc = fma(pc[e], o[e], acc);
      } else {
        T ph[V];
        load_vec<T>(a.phi + rowoff + k0, ph);
        T res[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
          res[e] = (k0 + e < nz) ? ((MODE == kStencilResidual) ? ph[e] - o[e] : o[e] - ph[e]) : T(0);
          acc = fma(res[e], res[e], acc);
        }
        if (MODE == kStencilResidual) {
          if (a.out_res) store_vec<T>(a.out_res + rowoff + k0, res);
          if (a.out32) {
            float r32[4];
#pragma unroll
            for (int e = 0; e < V; ++e) r32[e] = (float)res[e];
            if (V == 4) {
              *reinterpret_cast<float4 *>(a.out32 + rowoff + k0) = make_float4(r32[0], r32[1], r32[2], r32[3]);
            } else {
              *reinterpret_cast<float2 *>(a.out32 + rowoff + k0) = make_float2(r32[0], r32[1]);
            }
          }
        } else {
          store_vec<T>(a.out + rowoff + k0, res);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
      pm[e] = pc[e];
      pc[e] = pn[e];
      crl[e] = crh[e];
      crh[e] = crn[e];
      czl[e] = czn[e];
      w[e] = wn[e];
    }
    left = leftn;
    right = rightn;
    czlast = czlastn;
  }
  if (MODE != kStencilApply && a.partial != nullptr) {  // uniform over the CTA
    const double s = block_sum((double)acc, red);
    if (threadIdx.x == 0)
      a.partial[(size_t)m * kPartialStride + blockIdx.y * gridDim.z + blockIdx.z] = s;
  }
}

// ---- q = A p with the rows of p staged by bulk copies (fused FP32 iteration;
// also y -> A y) --------------------------------------------------------------
// The register-window kernel keeps about one row of DRAM loads in flight per
// thread, and ncu shows it waiting on them (long scoreboard).  Here one thread
// issues, as the CTA starts, one bulk copy (cp.async.bulk) per row of the
// CTA's strip of p, its R rows and the halo row on each side, each completing
// on its own mbarrier: the CTA has R + 2 row strips of reads in flight at
// once, moved by the copy engine without registers.  The threads then walk
// down the rows with the same register window, taking each row of p from
// shared memory once its barrier has completed; the coefficient rows
// (L2-resident, shared by all right-hand sides of an operator) are still
// loaded one row ahead.  Waits are bounded: on expiry a thread sets *err and
// stops, and thread 0 waits (bounded) for every copy before the CTA exits.
constexpr int kBulkBarBytes = 256;            // room for the mbarriers of up to 32 rows
constexpr unsigned kBulkPolls = 1u << 22;

__host__ __device__ constexpr int bulk_rows(int variant) { return variant == 2 ? 8 : 16; }

template <int R, int MODE>
__global__ void __launch_bounds__(256) stencil_bulk_kernel(const StencilArgs<float> a) {
  static_assert(MODE == kStencilPcgP || MODE == kStencilApply, "modes without a second input field");
  static_assert((R + 2) * 8 <= kBulkBarBytes, "barrier area");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[8];
  const int m = blockIdx.x;
  if (!rhs_selected(a.st, a.mask, m)) return;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  float *rows = reinterpret_cast<float *>(smem + kBulkBarBytes);
  const int W = blockDim.x * 4;  // strip width (floats)
  const int lane = threadIdx.x & 31;
  const int c = threadIdx.x * 4;
  const int ks = blockIdx.z * W;
  const int k0 = ks + c;
  const int nr = a.nr, nz = a.nz;
  const int i0 = blockIdx.y * R, i1 = min(i0 + R, nr);
  const int ilo = max(i0 - 1, 0), ihi = min(i1, nr - 1);  // staged rows
  const size_t base = (size_t)m * (size_t)a.field;
  const float *src = MODE == kStencilApply ? a.in : ((a.st[m].iters & 1) ? a.pa : a.pb);
  const float *__restrict__ CR = a.CR + (size_t)m * a.cstride;
  const float *__restrict__ CZ = a.CZ + (size_t)m * a.czstride;
  const float *__restrict__ Wc = a.W + (size_t)m * a.cstride;
  const unsigned polls = a.polls ? a.polls : kBulkPolls;
  // whole padded rows: pitch - ks is a multiple of 32 floats (128 bytes), the
  // source and destination addresses are 16-byte aligned
  const unsigned bytes = (unsigned)min(W, a.pitch - ks) * 4u;
  if (threadIdx.x == 0) {
    for (int j = 0; j <= ihi - ilo; ++j) mbar_init(&bar[j], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !a.stall)
    for (int i = ilo; i <= ihi; ++i) {
      mbar_arrive_tx(&bar[i - ilo], bytes);
      bulk_g2s(rows + (size_t)(i - ilo) * W, src + base + (size_t)i * a.pitch + ks, bytes, &bar[i - ilo]);
    }
  const bool col_ok = k0 < nz;
  bool ok = true;
  // row i of p (zero outside the grid and beyond nz), once its copy has landed
  auto get_row = [&](int i, float (&v)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = 0.f;
    if (i < 0 || i >= nr || !col_ok || !ok) return;
    if (!mbar_wait(&bar[i - ilo], 0u, polls)) {
      ok = false;
      atomicExch(a.err, 1);
      return;
    }
    const float4 t = *reinterpret_cast<const float4 *>(rows + (size_t)(i - ilo) * W + c);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = (k0 + e < nz) ? v[e] : 0.f;
  };
  auto load_coef = [&](const float *cf, int i, float (&v)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = 0.f;
    if (col_ok) load_vec<float>(cf + (size_t)i * a.pitch + k0, v);
  };
  auto load_cz = [&](int i, float (&v)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = 0.f;
    if (k0 <= nz) load_vec<float>(CZ + (size_t)i * a.pitchz + k0, v);
  };
  // upper face of the lane's last node (lane 31 only; the others shuffle it)
  auto load_czlast = [&](int i) {
    return (lane == 31 && k0 + 4 <= nz) ? CZ[(size_t)i * a.pitchz + k0 + 4] : 0.f;
  };
  float pm[4], pc[4], pn[4], crl[4], crh[4], czl[4], w[4];
  if (i0 > 0) {
    get_row(i0 - 1, pm);
    load_coef(CR, i0 - 1, crl);
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) pm[e] = crl[e] = 0.f;
  }
  get_row(i0, pc);
  load_coef(CR, i0, crh);
  load_cz(i0, czl);
  load_coef(Wc, i0, w);
  float czlast = load_czlast(i0);
  float acc = 0.f;
  for (int i = i0; i < i1; ++i) {
    float crn[4], czn[4], wn[4], czlastn = 0.f;
    if (i + 1 < i1) {
      load_coef(CR, i + 1, crn);
      load_cz(i + 1, czn);
      load_coef(Wc, i + 1, wn);
      czlastn = load_czlast(i + 1);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) crn[e] = czn[e] = wn[e] = 0.f;
    }
    get_row(i + 1, pn);
    // z-neighbours: shuffles inside the warp; the warp-edge lanes read the
    // neighbouring warp's column from shared memory, or the next strip's from
    // global memory at the strip edges
    float l = __shfl_up_sync(0xffffffffu, pc[3], 1);
    float r = __shfl_down_sync(0xffffffffu, pc[0], 1);
    float czh_last = __shfl_down_sync(0xffffffffu, czl[0], 1);
    if (lane == 0) {
      l = 0.f;
      if (col_ok && ok && k0 > 0)
        l = c > 0 ? rows[(size_t)(i - ilo) * W + c - 1] : src[base + (size_t)i * a.pitch + k0 - 1];
    }
    if (lane == 31) {
      r = 0.f;
      if (col_ok && ok && k0 + 4 < nz)
        r = c + 4 < W ? rows[(size_t)(i - ilo) * W + c + 4] : src[base + (size_t)i * a.pitch + k0 + 4];
      czh_last = czlast;
    }
    float o[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float yl = (e == 0) ? l : pc[e - 1];
      const float yr = (e == 3) ? r : pc[e + 1];
      const float czh = (e == 3) ? czh_last : czl[e + 1];
      const float y = pc[e];
      float v = w[e] * y;
      v = fmaf(crh[e], y - pn[e], v);
      v = fmaf(crl[e], y - pm[e], v);
      v = fmaf(czh, y - yr, v);
      v = fmaf(czl[e], y - yl, v);
      o[e] = (k0 + e < nz) ? v : 0.f;
    }
    if (col_ok) {
      store_vec<float>(a.out + base + (size_t)i * a.pitch + k0, o);
#pragma unroll
      for (int e = 0; e < 4; ++e) acc = fmaf(pc[e], o[e], acc);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      pm[e] = pc[e];
      pc[e] = pn[e];
      crl[e] = crh[e];
      crh[e] = crn[e];
      czl[e] = czn[e];
      w[e] = wn[e];
    }
    czlast = czlastn;
  }
  // no copy may still be writing shared memory when the CTA exits
  if (threadIdx.x == 0 && !a.stall)
    for (int j = 0; j <= ihi - ilo; ++j)
      if (!mbar_wait(&bar[j], 0u, polls)) atomicExch(a.err, 1);
  if (MODE == kStencilPcgP && a.partial != nullptr) {
    const double sm = block_sum((double)acc, red);
    if (threadIdx.x == 0)
      a.partial[(size_t)m * kPartialStride + blockIdx.y * gridDim.z + blockIdx.z] = sm;
  }
}

// ---- q = A p for two right-hand sides per thread (FP32; the fused iteration's
// q = A p and y -> A y) ---------------------------------------------------------
// The coefficient rows (CR, CZ, W) are the same for every right-hand side of
// one operator.  A thread that applies the stencil at the same nodes of two
// right-hand sides loads each coefficient row once for both, and keeps two
// independent rows of p in flight instead of one.  CTA tile, partial-sum
// layout (one partial per right-hand side and tile) and the arithmetic per
// node are those of the register-window kernel, so the results are the same
// bit for bit.  Operators whose tables differ per right-hand side (stacked
// batch groups) take the register-window kernel.
template <int MODE>
__global__ void __launch_bounds__(256, 3) stencil_pair_kernel(const StencilArgs<float> a) {
  static_assert(MODE == kStencilPcgP || MODE == kStencilApply, "modes without a second input field");
  __shared__ double red[8];
  const int m0 = 2 * blockIdx.x;
  const bool sel0 = rhs_selected(a.st, a.mask, m0);
  const bool sel1 = m0 + 1 < a.m && rhs_selected(a.st, a.mask, m0 + 1);
  if (!sel0 && !sel1) return;
  const bool sel[2] = {sel0, sel1};
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int k0 = ((blockIdx.z * nwarps + warp) * 32 + lane) * 4;
  const int nr = a.nr, nz = a.nz;
  const int i0 = blockIdx.y * kStencilRows;
  const int i1 = min(i0 + kStencilRows, nr);
  const bool col_ok = k0 < nz;
  const float *src[2];
  size_t base[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    base[j] = (size_t)(m0 + j) * (size_t)a.field;
    src[j] = a.in;
    if (MODE == kStencilPcgP && sel[j]) src[j] = (a.st[m0 + j].iters & 1) ? a.pa : a.pb;
  }
  const float *__restrict__ CR = a.CR;
  const float *__restrict__ CZ = a.CZ;
  const float *__restrict__ Wc = a.W;

  auto load_row = [&](int j, int i, float (&v)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = 0.f;
    if (!col_ok || !sel[j]) return;
    load_vec<float>(src[j] + base[j] + (size_t)i * a.pitch + k0, v);
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = (k0 + e < nz) ? v[e] : 0.f;
  };
  auto load_coef = [&](const float *c, int i, float (&v)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = 0.f;
    if (col_ok) load_vec<float>(c + (size_t)i * a.pitch + k0, v);
  };
  auto load_cz = [&](int i, float (&v)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = 0.f;
    if (k0 <= nz) load_vec<float>(CZ + (size_t)i * a.pitchz + k0, v);
  };
  auto load_halo = [&](int i, float (&left)[2], float (&right)[2], float &czlast) {
    left[0] = left[1] = right[0] = right[1] = czlast = 0.f;
    if (lane == 0 && col_ok && k0 > 0) {
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (sel[j]) left[j] = src[j][base[j] + (size_t)i * a.pitch + k0 - 1];
    }
    if (lane == 31) {
      if (k0 + 4 < nz) {
#pragma unroll
        for (int j = 0; j < 2; ++j)
          if (sel[j]) right[j] = src[j][base[j] + (size_t)i * a.pitch + k0 + 4];
      }
      if (k0 + 4 <= nz) czlast = CZ[(size_t)i * a.pitchz + k0 + 4];
    }
  };

  if (col_ok)
    for (int i = max(i0 - 1, 0); i <= i1 && i < nr; ++i) {
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (sel[j]) prefetch_l2(src[j] + base[j] + (size_t)i * a.pitch + k0);
    }
  float pm[2][4], pc[2][4], pn[2][4], crl[4], crh[4], czl[4], w[4];
  float left[2], right[2], czlast;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (i0 > 0) {
      load_row(j, i0 - 1, pm[j]);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) pm[j][e] = 0.f;
    }
    load_row(j, i0, pc[j]);
  }
  if (i0 > 0) {
    load_coef(CR, i0 - 1, crl);
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) crl[e] = 0.f;
  }
  load_coef(CR, i0, crh);
  load_cz(i0, czl);
  load_coef(Wc, i0, w);
  load_halo(i0, left, right, czlast);

  float acc[2] = {0.f, 0.f};
  for (int i = i0; i < i1; ++i) {
    float crn[4], czn[4], wn[4], leftn[2] = {0.f, 0.f}, rightn[2] = {0.f, 0.f}, czlastn = 0.f;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (i + 1 < nr) {
        load_row(j, i + 1, pn[j]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) pn[j][e] = 0.f;
      }
    }
    if (i + 1 < i1) {
      load_coef(CR, i + 1, crn);
      load_cz(i + 1, czn);
      load_coef(Wc, i + 1, wn);
      load_halo(i + 1, leftn, rightn, czlastn);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) crn[e] = czn[e] = wn[e] = 0.f;
    }
    float czh_last = __shfl_down_sync(0xffffffffu, czl[0], 1);
    if (lane == 31) czh_last = czlast;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float l = __shfl_up_sync(0xffffffffu, pc[j][3], 1);
      float r = __shfl_down_sync(0xffffffffu, pc[j][0], 1);
      if (lane == 0) l = left[j];
      if (lane == 31) r = right[j];
      float o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float yl = (e == 0) ? l : pc[j][e - 1];
        const float yr = (e == 3) ? r : pc[j][e + 1];
        const float czh = (e == 3) ? czh_last : czl[e + 1];
        const float y = pc[j][e];
        float v = w[e] * y;
        v = fmaf(crh[e], y - pn[j][e], v);
        v = fmaf(crl[e], y - pm[j][e], v);
        v = fmaf(czh, y - yr, v);
        v = fmaf(czl[e], y - yl, v);
        o[e] = (k0 + e < nz) ? v : 0.f;
      }
      if (col_ok && sel[j]) {
        store_vec<float>(a.out + base[j] + (size_t)i * a.pitch + k0, o);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j] = fmaf(pc[j][e], o[e], acc[j]);
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        pm[j][e] = pc[j][e];
        pc[j][e] = pn[j][e];
      }
      crl[e] = crh[e];
      crh[e] = crn[e];
      czl[e] = czn[e];
      w[e] = wn[e];
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      left[j] = leftn[j];
      right[j] = rightn[j];
    }
    czlast = czlastn;
  }
  if (MODE == kStencilPcgP && a.partial != nullptr) {  // uniform over the CTA
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const double sm = block_sum((double)acc[j], red);
      if (threadIdx.x == 0 && sel[j])
        a.partial[(size_t)(m0 + j) * kPartialStride + blockIdx.y * gridDim.z + blockIdx.z] = sm;
    }
  }
}

// ---- double-float residual -------------------------------------------------
// Pairs (h, l) of FP32 numbers carry about 48 significant bits: sums by Knuth's
// two-sum and Dekker's fast two-sum, products by the FMA two-product (the exact
// error of a*b is fma(a, b, -a*b)).  GB300 runs FP32 about 58 times faster
// than FP64, so the true residual of the mixed method costs a few FP32
// operations per flop instead of FP64 ones.
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF df_fast(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = df_two_sum(a.h, b.h);
  return df_fast(s.h, s.l + (a.l + b.l));
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.h, -a.l}; }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_fast(p, e);
}

constexpr int kDfRows = 16;      // rows per CTA (short: few right-hand sides are due at a time)
constexpr int kDfThreads = 256;  // 4 z-nodes per thread

__global__ void __launch_bounds__(kDfThreads) residual_df_kernel(const DfResidualArgs a) {
  __shared__ double red[8];
  const int m = blockIdx.z;
  if (!rhs_selected(a.st, a.mask, m)) return;
  const int nr = a.nr, nz = a.nz, P = a.pitch, PZ = a.pitchz;
  const int k0 = (blockIdx.x * kDfThreads + threadIdx.x) * 4;
  const int i0 = blockIdx.y * kDfRows, i1 = min(i0 + kDfRows, nr);
  const bool col_ok = k0 < nz;
  const size_t base = (size_t)m * (size_t)a.field;
  const float *crh = a.CRh + (size_t)m * a.cstride, *crl = a.CRl + (size_t)m * a.cstride;
  const float *czh = a.CZh + (size_t)m * a.czstride, *czl = a.CZl + (size_t)m * a.czstride;
  const float *wh = a.Wh + (size_t)m * a.cstride, *wl = a.Wl + (size_t)m * a.cstride;
  // 4 consecutive values of a field row (zero outside the grid; padding
  // columns hold zeros)
  auto ld4 = [&](const float *p, size_t off, bool ok, float (&v)[4]) {
    if (ok) {
      const float4 t = *reinterpret_cast<const float4 *>(p + off);
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
      v[0] = v[1] = v[2] = v[3] = 0.f;
    }
  };
  float ymh[4], yml[4], ych[4], ycl[4], ynh[4], ynl[4], cph[4], cpl[4];
  ld4(a.xh, base + (size_t)(i0 - 1) * P + k0, col_ok && i0 > 0, ymh);
  ld4(a.xl, base + (size_t)(i0 - 1) * P + k0, col_ok && i0 > 0, yml);
  ld4(crh, (size_t)(i0 - 1) * P + k0, col_ok && i0 > 0, cph);  // CR_{i-1}: 0 on the axis
  ld4(crl, (size_t)(i0 - 1) * P + k0, col_ok && i0 > 0, cpl);
  ld4(a.xh, base + (size_t)i0 * P + k0, col_ok, ych);
  ld4(a.xl, base + (size_t)i0 * P + k0, col_ok, ycl);
  float acc = 0.f;
  for (int i = i0; i < i1; ++i) {
    const size_t ro = (size_t)i * P + k0;
    ld4(a.xh, base + ro + P, col_ok && i + 1 < nr, ynh);
    ld4(a.xl, base + ro + P, col_ok && i + 1 < nr, ynl);
    float cch[4], ccl[4], w4h[4], w4l[4], fh[4], fl[4], zh[4], zl[4];
    ld4(crh, ro, col_ok, cch);
    ld4(crl, ro, col_ok, ccl);
    ld4(wh, ro, col_ok, w4h);
    ld4(wl, ro, col_ok, w4l);
    ld4(a.ph, base + ro, col_ok, fh);
    ld4(a.pl, base + ro, col_ok, fl);
    ld4(czh, (size_t)i * PZ + k0, col_ok, zh);  // faces k0 .. k0 + 3
    ld4(czl, (size_t)i * PZ + k0, col_ok, zl);
    // face k0 + 4 and the z-neighbours outside the 4 nodes
    const bool up_ok = col_ok && k0 + 4 <= nz;
    const DF z4 = {up_ok ? czh[(size_t)i * PZ + k0 + 4] : 0.f, up_ok ? czl[(size_t)i * PZ + k0 + 4] : 0.f};
    const bool left_ok = col_ok && k0 > 0, right_ok = col_ok && k0 + 4 < nz;
    const DF yleft = {left_ok ? a.xh[base + ro - 1] : 0.f, left_ok ? a.xl[base + ro - 1] : 0.f};
    const DF yright = {right_ok ? a.xh[base + ro + 4] : 0.f, right_ok ? a.xl[base + ro + 4] : 0.f};
    float res[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const DF y = {ych[e], ycl[e]};
      const DF yl = (e == 0) ? yleft : DF{ych[e - 1], ycl[e - 1]};
      const DF yr = (e == 3) ? yright : DF{ych[e + 1], ycl[e + 1]};
      const DF czlo = {zh[e], zl[e]};
      const DF czhi = (e == 3) ? z4 : DF{zh[e + 1], zl[e + 1]};
      // A y = W y + CR_i (y - y_{i+1}) + CR_{i-1} (y - y_{i-1})
      //           + CZ_{k+1} (y - y_{k+1}) + CZ_k (y - y_{k-1})
      DF v = df_mul({w4h[e], w4l[e]}, y);
      v = df_add(v, df_mul({cch[e], ccl[e]}, df_add(y, df_neg({ynh[e], ynl[e]}))));
      v = df_add(v, df_mul({cph[e], cpl[e]}, df_add(y, df_neg({ymh[e], yml[e]}))));
      v = df_add(v, df_mul(czhi, df_add(y, df_neg(yr))));
      v = df_add(v, df_mul(czlo, df_add(y, df_neg(yl))));
      const DF r = df_add({fh[e], fl[e]}, df_neg(v));
      res[e] = (k0 + e < nz) ? r.h + r.l : 0.f;
      acc = fmaf(res[e], res[e], acc);
    }
    if (col_ok) *reinterpret_cast<float4 *>(a.r32 + base + ro) = make_float4(res[0], res[1], res[2], res[3]);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ymh[e] = ych[e]; yml[e] = ycl[e];
      ych[e] = ynh[e]; ycl[e] = ynl[e];
      cph[e] = cch[e]; cpl[e] = ccl[e];
    }
  }
  const double sum = block_sum((double)acc, red);
  if (threadIdx.x == 0) a.partial[(size_t)m * kPartialStride + blockIdx.y * gridDim.x + blockIdx.x] = sum;
}

int column_warps(int nz, int vec) {
  int w = (nz + 32 * vec - 1) / (32 * vec);
  return w < kStencilWarps ? (w < 1 ? 1 : w) : kStencilWarps;
}

}  // namespace

int stencil_blocks_per_rhs(int nr, int nz, int vec, int variant) {
  const int wx = column_warps(nz, vec);
  const int rows = (variant == 1 || variant == 2) ? bulk_rows(variant) : kStencilRows;
  const int gz = (nz + 32 * vec * wx - 1) / (32 * vec * wx);
  const int gy = (nr + rows - 1) / rows;
  return gy * gz;
}

template <int R, int MODE>
void launch_stencil_bulk(const StencilArgs<float> &a, cudaStream_t s) {
  const int wx = column_warps(a.nz, 4);
  const int W = 128 * wx;
  const size_t smem = kBulkBarBytes + (size_t)(R + 2) * W * sizeof(float);
  ensure_smem_attr((const void *)stencil_bulk_kernel<R, MODE>, smem);
  dim3 grid(a.m, (a.nr + R - 1) / R, (a.nz + W - 1) / W);
  note_launch();
  stencil_bulk_kernel<R, MODE><<<grid, 32 * wx, smem, s>>>(a);
}

template <typename T>
void launch_stencil(int mode, const StencilArgs<T> &a, cudaStream_t s) {
  constexpr int V = VecT<T>::n;
  if constexpr (sizeof(T) == 4) {
    if ((mode == kStencilPcgP || mode == kStencilApply) && a.variant == 3 && a.cstride == 0 && a.czstride == 0) {
      const int wx = column_warps(a.nz, V);
      dim3 grid((a.m + 1) / 2, (a.nr + kStencilRows - 1) / kStencilRows, (a.nz + 32 * V * wx - 1) / (32 * V * wx));
      note_launch();
      if (mode == kStencilPcgP)
        stencil_pair_kernel<kStencilPcgP><<<grid, 32 * wx, 0, s>>>(a);
      else
        stencil_pair_kernel<kStencilApply><<<grid, 32 * wx, 0, s>>>(a);
      return;
    }
    if ((mode == kStencilPcgP || mode == kStencilApply) && (a.variant == 1 || a.variant == 2) && a.err != nullptr) {
      if (mode == kStencilPcgP)
        a.variant == 2 ? launch_stencil_bulk<8, kStencilPcgP>(a, s) : launch_stencil_bulk<16, kStencilPcgP>(a, s);
      else
        a.variant == 2 ? launch_stencil_bulk<8, kStencilApply>(a, s) : launch_stencil_bulk<16, kStencilApply>(a, s);
      return;
    }
  }
  const int wx = column_warps(a.nz, V);
  dim3 grid(a.m, (a.nr + kStencilRows - 1) / kStencilRows, (a.nz + 32 * V * wx - 1) / (32 * V * wx));
  dim3 block(32 * wx);
  note_launch();
  switch (mode) {
    case kStencilApply: stencil_kernel<T, kStencilApply><<<grid, block, 0, s>>>(a); break;
    case kStencilPcg: stencil_kernel<T, kStencilPcg><<<grid, block, 0, s>>>(a); break;
    case kStencilPcgP: stencil_kernel<T, kStencilPcgP><<<grid, block, 0, s>>>(a); break;
    case kStencilResidual: stencil_kernel<T, kStencilResidual><<<grid, block, 0, s>>>(a); break;
    default: stencil_kernel<T, kStencilCheb><<<grid, block, 0, s>>>(a); break;
  }
}

int residual_df_blocks(int nr, int nz) {
  return ((nz + 4 * kDfThreads - 1) / (4 * kDfThreads)) * ((nr + kDfRows - 1) / kDfRows);
}

void launch_residual_df(const DfResidualArgs &a, cudaStream_t s) {
  dim3 grid((a.nz + 4 * kDfThreads - 1) / (4 * kDfThreads), (a.nr + kDfRows - 1) / kDfRows, a.m);
  note_launch();
  residual_df_kernel<<<grid, kDfThreads, 0, s>>>(a);
}

template void launch_stencil<float>(int, const StencilArgs<float> &, cudaStream_t);
template void launch_stencil<double>(int, const StencilArgs<double> &, cudaStream_t);

}  // namespace ax
