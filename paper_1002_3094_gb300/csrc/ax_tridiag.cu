// Per-mode tridiagonal solves along r (Section 4.2, Eq. eq_trid; the series
// of systems with one fixed matrix per mode l, Section 3, Eq. main_eq3):
//
//     T_l y = b,   T_l = Lr(kappa~) + diag(r_i (kappa~ lambda_l + q~)),
//
// for every right-hand side m and every mode column l of a transformed field.
// The matrix of each mode is fixed for the whole solve, so its LU factors are
// computed once at set-up (in FP64): IP[i][l] = 1 / delta_i(l) and the
// off-diagonal E[i] (the same for all l).  With them Thomas is two first-order
// linear recurrences:
//
//     g_i = b_i IP_i + alpha_i g_{i-1},   alpha_i = -E_{i-1} IP_i     (forward)
//     y_i = g_i + beta_i y_{i+1},         beta_i  = -E_i IP_i         (backward)
//
// GPU mapping.  A CTA owns W consecutive mode columns of one right-hand side
// and the whole r-range; lanes run along l, so every row access is one
// coalesced segment.  The r-range is cut into P chunks of C rows, one thread
// per (column, chunk), each holding its C values in registers.  A chunk first
// runs its recurrence with zero carry-in, which yields an affine map
// carry_out = a + mu * carry_in (mu = product of the chunk's alpha); the P
// maps of a column are composed by a log-depth scan in shared memory, and a
// second pass applies the true carry-in.  This is the same observation as the
// paper's dichotomy algorithm (Section 3: with a fixed matrix, the unknowns at
// sub-system boundaries follow from precomputable linear combinations), laid
// out for one CTA instead of a multicomputer.  The data are read and written
// once; IP is re-read from L1/L2.
#include <algorithm>
#include "ax_common.cuh"

namespace ax {

namespace {

// Read-only loads that the compiler may not merge across the kernel's passes
// (keeping every factor live in registers would spill the chunk's data).
__device__ __forceinline__ float ld_nc(const float *p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_nc(const double *p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

// Returns x unchanged, but hides its value from the optimiser, so addresses
// built from it are recomputed per pass instead of being kept live in
// registers across passes (which would spill the chunk's data).
template <typename X>
__device__ __forceinline__ X launder(X x) {
  asm volatile("" : "+l"(x));
  return x;
}
__device__ __forceinline__ int launder_i(int x) {
  asm volatile("" : "+r"(x));
  return x;
}


template <typename T>
__device__ __forceinline__ void scan_affine(T *sa, T *sm, int P, int W, int c, int w, T &a, T &mu,
                                            bool reverse) {
  // Inclusive scan of affine maps f_c(x) = a_c + mu_c x composed in chunk
  // order (reverse = from the last chunk down).  On return (a, mu) of thread
  // (c, w) describe the composition of chunks 0..c (or c..P-1).
  const int pos = reverse ? (P - 1 - c) : c;
  for (int off = 1; off < P; off <<= 1) {
    sa[pos * W + w] = a;
    sm[pos * W + w] = mu;
    __syncthreads();
    if (pos >= off) {
      const T pa = sa[(pos - off) * W + w], pm = sm[(pos - off) * W + w];
      a = fma(mu, pa, a);
      mu = mu * pm;
    }
    __syncthreads();
  }
}

template <typename T, int C>
__global__ void __launch_bounds__(1024) tridiag_kernel(const TriArgs<T> a, int W, int P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sa = reinterpret_cast<T *>(smem_raw);
  T *sm = sa + P * W;
  const int m = blockIdx.x;
  if (!rhs_selected(a.st, a.mask, m)) return;
  const int w = threadIdx.x % W;
  const int c = threadIdx.x / W;
  const int col = blockIdx.y * W + w;
  const int nr = a.nr;
  const int s0 = c * C;
  // rows of this chunk that exist (0 for padding columns)
  const int cnt = (col < a.nz) ? max(0, min(C, nr - s0)) : 0;
  const int pitch = a.pitch;
  const T *__restrict__ in = a.in + (size_t)m * (size_t)a.field + (size_t)s0 * pitch + col;
  T *__restrict__ out = a.out + (size_t)m * (size_t)a.field + (size_t)s0 * pitch + col;
  const T *__restrict__ ipc = a.IP + (size_t)m * a.cstride + (size_t)s0 * pitch + col;
  const T *__restrict__ E0 = a.E + (size_t)m * a.estride;
  const T *__restrict__ E = E0 + s0;   // E[t] couples rows s0 + t and s0 + t + 1
  const T e_before = (s0 > 0 && cnt > 0) ? ld_nc(E0 + s0 - 1) : T(0);

  T v[C];
  {
  const T *ip_in = launder(in);
  const int pt = launder_i(pitch);
#pragma unroll
  for (int t = 0; t < C; ++t) v[t] = (t < cnt) ? ip_in[t * pt] : T(0);
  }

  // forward, zero carry-in: g_t = v_t ip_t + alpha_t g_{t-1}
  T g = T(0), mu = T(1), eprev = e_before;
  {
  const T *ipp = launder(ipc);
  const int pt = launder_i(pitch);
#pragma unroll
  for (int t = 0; t < C; ++t) {
    const T ip = (t < cnt) ? ld_nc(ipp + t * pt) : T(0);
    const T al = -eprev * ip;
    g = fma(v[t], ip, al * g);
    mu *= al;
    v[t] = g;
    eprev = (t < cnt) ? ld_nc(E + t) : T(0);
  }
  }
  T A = g, M = mu;
  scan_affine(sa, sm, P, W, c, w, A, M, false);
  sa[c * W + w] = A;
  __syncthreads();
  const T gin = (c > 0) ? sa[(c - 1) * W + w] : T(0);
  __syncthreads();
  mu = T(1);
  eprev = e_before;
  {
  const T *ipp = launder(ipc);
  const int pt = launder_i(pitch);
#pragma unroll
  for (int t = 0; t < C; ++t) {
    const T ip = (t < cnt) ? ld_nc(ipp + t * pt) : T(0);
    mu *= -eprev * ip;
    v[t] = fma(mu, gin, v[t]);
    eprev = (t < cnt) ? ld_nc(E + t) : T(0);
  }
  }

  // backward, zero carry-in: y_t = g_t + beta_t y_{t+1}, beta_t = -E_t ip_t
  T y = T(0);
  mu = T(1);
  {
  const T *ipp = launder(ipc);
  const int pt = launder_i(pitch);
#pragma unroll
  for (int t = C - 1; t >= 0; --t) {
    const T be = (t < cnt) ? -ld_nc(E + t) * ld_nc(ipp + t * pt) : T(0);
    y = fma(be, y, v[t]);
    mu *= be;
    v[t] = y;
  }
  }
  A = y;
  M = mu;
  scan_affine(sa, sm, P, W, c, w, A, M, true);
  sa[c * W + w] = A;
  __syncthreads();
  const T yin = (c + 1 < P) ? sa[(c + 1) * W + w] : T(0);
  mu = T(1);
  {
  const T *ipp = launder(ipc);
  const int pt = launder_i(pitch);
#pragma unroll
  for (int t = C - 1; t >= 0; --t) {
    const T be = (t < cnt) ? -ld_nc(E + t) * ld_nc(ipp + t * pt) : T(0);
    mu *= be;
    v[t] = fma(mu, yin, v[t]);
  }
  }
  {
  T *op = launder(out);
  const int pt = launder_i(pitch);
#pragma unroll
  for (int t = 0; t < C; ++t)
    if (t < cnt) op[t * pt] = v[t];
  }
}

// Tiles of the register kernel below: a CTA stages an nr x CW column tile in
// shared memory; idx(row, col) = row CW + col + row / C2 is padded by one word
// per chunk of C2 rows, so the lanes of a warp (rows c C2 + t of one column,
// c = lane) fall in distinct banks: the bank is ((CW C2 + 1) c + CW t + col)
// mod 32, and CW C2 + 1 is odd.

// 4-byte asynchronous global -> shared copy (zero fill when !ok); the whole
// tile is in flight at once instead of one row per round trip.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Register kernel (FP32, nr <= 32 WPC C2): a CTA stages an nr x CW column
// tile of IP and the data of one right-hand side in shared memory (cp.async,
// padded to 32 WPC chunks of C2 rows with one word per chunk); one column
// system per group of WPC warps, lane c of warp h owning rows (32 h + c) C2 ..
// (32 h + c) C2 + C2 - 1, so a chunk, its alpha_t = -E_{t-1} ip_t and
// beta_t = -E_t ip_t stay in registers after one pass over the shared tile.
// The couplings are E_i = E_0 (i + 1) (faces rbar_{i+1} = (i + 1) h_r of
// Eq. eq_trid), so they are formed from the row index instead of being
// loaded; the last row's coupling to the Dirichlet row nr, 0 in the table,
// only ever multiplies that row's value 0 (a zero padding row, or the zero
// carry into the last chunk) and needs no special case.  The affine carry maps of the chunks are composed with
// shuffles inside each warp, and the WPC warp totals of a column through
// shared memory.  Padding rows carry IP = E = 0 and solve to zero, so every
// lane runs the same unpredicated recurrences.  For the tensor-core transform
// the result is written in the BF16 split layout.
// Shapes: <C2, 2, 8> for nr <= 64 C2 (C2 = 4, 8, 16), <16, 4, 8> for
// nr <= 2048 and <16, 8, 4> for nr <= 4096 (1024 threads).
template <int C2, int WPC, int CW>
__global__ void __launch_bounds__(32 * WPC * CW, (32 * WPC * CW <= 512) ? 2 : 1)
    tridiag_reg_kernel(const TriArgs<float> a) {
  constexpr int NT = 32 * WPC * CW;  // threads
  constexpr int NCH = 32 * WPC;      // chunks per column
  constexpr int NP = NCH * C2;       // padded rows
  constexpr int kTileWords = NP * CW + NCH;
  static_assert(NT <= 1024 && (CW == 4 || CW == 8), "tile shape");
  extern __shared__ __align__(16) float tsm[];
  // per column and warp: the warp's composed map (A, M), forward and backward
  __shared__ float xfa[CW][WPC], xfm[CW][WPC], xba[CW][WPC], xbm[CW][WPC];
  const int nr = a.nr, pitch = a.pitch;
  float *ips = tsm;
  float *ds = ips + kTileWords;
  const int col0 = blockIdx.x * CW;
  const int m = blockIdx.y;
  const int ncol = min(CW, a.nz - col0);
  if (!rhs_selected(a.st, a.mask, m)) return;  // uniform over the CTA
  // ---- stage the tiles (coalesced rows, cp.async) ----
  const int cw = threadIdx.x % CW;
  {
    const bool colok = cw < ncol;
    const int cc = colok ? cw : 0;
    const float *ipg = a.IP + (size_t)m * a.cstride + col0 + cc;
    const float *ing = a.in + (size_t)m * a.field + col0 + cc;
    for (int row = threadIdx.x / CW; row < NP; row += NT / CW) {
      const bool ok = colok && row < nr;
      const int rs = ok ? row : 0;
      const int si = row * CW + cw + row / C2;
      cp_async4(ips + si, ipg + (size_t)rs * pitch, ok);
      cp_async4(ds + si, ing + (size_t)rs * pitch, ok);
    }
    cp_async_wait_all();
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = warp / WPC, h = warp % WPC;  // column, segment of the r-range
  const int ci = h * 32 + lane;               // chunk index 0 .. NCH - 1
  const bool active = w < ncol;
  float *pd = ds + ci * (CW * C2 + 1) + w;
  const float *pip = ips + ci * (CW * C2 + 1) + w;
  const float e0 = nr > 1 ? a.E[(size_t)m * a.estride] : 0.f;  // E_0
  const int rbase = ci * C2;                                   // first row of the chunk
  float v[C2], al[C2], be[C2];
  // forward, zero carry-in (one pass over the shared tile)
  float g = 0.f, mu = 1.f;
  float rowf = (float)rbase;  // row index, exact in FP32
#pragma unroll
  for (int t = 0; t < C2; ++t) {
    const float ip = pip[CW * t];
    const float f = -e0 * ip;  // padding rows: ip = 0
    al[t] = f * rowf;          // -E_{row-1} ip (0 on the axis row)
    rowf += 1.f;
    be[t] = f * rowf;          // -E_row ip (on the last row it multiplies y_nr = 0)
    g = fmaf(pd[CW * t], ip, al[t] * g);
    mu *= al[t];
    v[t] = g;
  }
  // inclusive scan of the maps over the 32 chunks of this warp
  float A = g, M = mu;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float pa = __shfl_up_sync(0xffffffffu, A, off), pm = __shfl_up_sync(0xffffffffu, M, off);
    if (lane >= off) {
      A = fmaf(M, pa, A);
      M *= pm;
    }
  }
  float Ae = __shfl_up_sync(0xffffffffu, A, 1), Me = __shfl_up_sync(0xffffffffu, M, 1);
  if (lane == 0) {
    Ae = 0.f;
    Me = 1.f;
  }
  if (lane == 31 && active) {  // map of all 32 chunks of this warp
    xfa[w][h] = A;
    xfm[w][h] = M;
  }
  __syncthreads();
  float cin = 0.f;  // carry into this warp's first chunk: the maps of warps 0 .. h-1
  if (active)
    for (int j = 0; j < h; ++j) cin = fmaf(xfm[w][j], cin, xfa[w][j]);
  const float gin = fmaf(Me, cin, Ae);
  mu = 1.f;
#pragma unroll
  for (int t = 0; t < C2; ++t) {
    mu *= al[t];
    v[t] = fmaf(mu, gin, v[t]);
  }
  // backward, zero carry-in
  float y = 0.f;
  mu = 1.f;
#pragma unroll
  for (int t = C2 - 1; t >= 0; --t) {
    y = fmaf(be[t], y, v[t]);
    mu *= be[t];
    v[t] = y;
  }
  A = y;
  M = mu;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float pa = __shfl_down_sync(0xffffffffu, A, off), pm = __shfl_down_sync(0xffffffffu, M, off);
    if (lane + off < 32) {
      A = fmaf(M, pa, A);
      M *= pm;
    }
  }
  Ae = __shfl_down_sync(0xffffffffu, A, 1);
  Me = __shfl_down_sync(0xffffffffu, M, 1);
  if (lane == 31) {
    Ae = 0.f;
    Me = 1.f;
  }
  if (lane == 0 && active) {  // map of all 32 chunks of this warp, from its last row up
    xba[w][h] = A;
    xbm[w][h] = M;
  }
  __syncthreads();
  cin = 0.f;  // carry into this warp's last chunk: the maps of warps WPC-1 .. h+1
  if (active)
    for (int j = WPC - 1; j > h; --j) cin = fmaf(xbm[w][j], cin, xba[w][j]);
  const float yin = fmaf(Me, cin, Ae);
  mu = 1.f;
#pragma unroll
  for (int t = C2 - 1; t >= 0; --t) {
    mu *= be[t];
    v[t] = fmaf(mu, yin, v[t]);
  }
  float dot = 0.f;
  if (active) {
#pragma unroll
    for (int t = 0; t < C2; ++t) {
      dot = fmaf(pd[CW * t], v[t], dot);  // (input, solution) of this chunk
      pd[CW * t] = v[t];
    }
  }
  if (a.partial != nullptr) {
    __shared__ double red[NT / 32];
    const double sw = warp_sum((double)dot);
    if (lane == 0) red[warp] = sw;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int i = 0; i < NT / 32; ++i) tot += red[i];
      a.partial[(size_t)m * kPartialStride + blockIdx.x] = tot;
    }
  }
  __syncthreads();
  // ---- write back: one thread per row, its CW columns at once ----
  // (CW shared loads with a 4-way bank conflict, but every lane does useful
  // work; rows go to 16- or 32-byte segments of the output, or to the even
  // and odd halves of the split layout)
  for (int row = threadIdx.x; row < nr; row += NT) {
    float x[CW];
    const int r0 = row * CW + row / C2;
#pragma unroll
    for (int c = 0; c < CW; ++c) x[c] = ds[r0 + c];
    if (a.split != nullptr) {
      if constexpr (CW == 8) split_store8(a.split, m, row, col0, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
      else split_store4(a.split, m, row, col0, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
    } else {
      float *o = a.out + (size_t)m * a.field + (size_t)row * pitch + col0;
      if (ncol == CW) {
#pragma unroll
        for (int c = 0; c < CW; c += 4) *reinterpret_cast<float4 *>(o + c) = make_float4(x[c], x[c + 1], x[c + 2], x[c + 3]);
      } else {
        for (int c = 0; c < ncol; ++c) o[c] = x[c];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Pipelined column-tile kernel (FP32, nr <= 16 NT / CW).
//
// Scaled systems.  With the row scaling D = diag(s_i), s_i s_{i+1} |E_i| = 1
// (E_i the coupling of rows i and i + 1, the same for every mode), each mode
// matrix becomes T'_l = D T_l D with off-diagonal -1, and
//     T_l y = b   <=>   T'_l y' = b',  b' = D b,  y = D y'.
// Its LU factors are the pivots delta'_i = d'_i - 1 / delta'_{i-1} of the
// scaled diagonal d'_i = s_i^2 d_i(l); with ips = 1 / delta' (computed in FP64
// at set-up) Thomas is
//     g_i = ips_i (b'_i + g_{i-1})       (forward)
//     y'_i = g_i + ips_i y'_{i+1}        (backward),
// one or two operations per step and no per-row coupling.  T'_l is symmetric
// positive definite like T_l, so the elimination needs no pivoting.  The
// kernel solves T'_l y' = b' for data already scaled by D: D acts along r and
// the sine / cosine transform along z, so D commutes with them and the
// preconditioner B^-1 = S^T T^-1 S = D S^T T'^-1 S D takes the scaling in the
// epilogues of the two transforms (GemmDstArgs::rowscale); the (rhat, yhat)
// partials are unchanged, (b', y') = (b, y).
//
// Work.  Persistent CTAs walk groups of items; an item is (right-hand side,
// tile of CW mode columns), a group R right-hand sides of one tile (the factors
// ips are the same for all of them and are read once per group).  Lanes run
// along l: thread (c, w) owns column w of the tile and the chunk of C = 16 rows
// c C .. c C + 15, so every shared-memory row access of a warp is one
// conflict-free wavefront and ips comes by coalesced row segments from global
// memory (L2) into registers.  Groups go round-robin over the CTAs, tiles
// fastest, so CTAs that run at the same time read neighbouring tiles of the
// same rows (whole 128-byte lines).  The data tile of the next item is copied
// to shared memory with 16-byte cp.async while the current one is solved
// (two stages).
//
// Chunks.  Each chunk runs its forward (then backward) recurrence with zero
// carry-in, yielding the affine map carry_out = A + M carry_in (M the product
// of the chunk's ips); the maps of a column are composed by CW scan warps (one
// column each, 32 chunks per shuffle round), and the true carry-ins are
// applied in a second pass over the registers.  Rows past nr carry ips = 0
// and data 0: they solve to zero and cut the carry chain (M = 0), so the
// recurrences run unpredicated.
//
// Shared-memory tile: row `row`, column `col` at word (row + row / 16) CW +
// col (one spare row per chunk), so the 32 / CW chunks held by one warp
// (chunk c = 32 j / CW + i) hit distinct banks: the bank is
// (CW (c + t) + col) mod 32.
// Map buffers: column w, chunk c at word w (P + 1) + c.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// Writes columns col .. col + 15 (col % 16 == 0) of one row in the split
// layout: the 8 even ones are one 16-byte row of a core matrix (high parts,
// then low parts), the 8 odd ones another.
__device__ __forceinline__ void split_store16(unsigned char *split, int m, int row, int col, int mtiles, int ktiles,
                                              int kbe, const float (&x)[16]) {
  unsigned he[4], le[4], ho[4], lo[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    he[e] = bf16_pack2(x[4 * e], x[4 * e + 2]);
    ho[e] = bf16_pack2(x[4 * e + 1], x[4 * e + 3]);
    le[e] = bf16_pack2(x[4 * e] - bf16_lo(he[e]), x[4 * e + 2] - bf16_hi(he[e]));
    lo[e] = bf16_pack2(x[4 * e + 1] - bf16_lo(ho[e]), x[4 * e + 3] - bf16_hi(ho[e]));
  }
  unsigned char *te = split + split_byte(m, row, split_pos(col, kbe), mtiles, ktiles);
  unsigned char *to = split + split_byte(m, row, split_pos(col + 1, kbe), mtiles, ktiles);
  *reinterpret_cast<uint4 *>(te) = make_uint4(he[0], he[1], he[2], he[3]);
  *reinterpret_cast<uint4 *>(te + kSplitTileBytes / 2) = make_uint4(le[0], le[1], le[2], le[3]);
  *reinterpret_cast<uint4 *>(to) = make_uint4(ho[0], ho[1], ho[2], ho[3]);
  *reinterpret_cast<uint4 *>(to + kSplitTileBytes / 2) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

template <int CW, int NT>
struct PipeShape {
  static constexpr int C = 16;                     // rows per chunk
  static constexpr int P = NT / CW;                // chunks per column
  static constexpr int kRows = P * C;              // rows covered
  static constexpr int kStageWords = P * (C + 1) * CW;
  static constexpr int kMapWords = CW * (P + 1);
  static constexpr int kMaxList = 8192;            // right-hand sides in the item list
  static constexpr size_t smem = sizeof(float) * (2 * kStageWords + 2 * kMapWords) + sizeof(int) * kMaxList;
  static_assert(P >= 32 && P % 32 == 0 && CW <= 32 && 32 % CW == 0, "pipe shape");
};

// Exclusive scan of the affine maps of one column (warp-wide, called by one
// warp per column): on entry ma/mm[k] hold chunk k's map (A, M); on return
// ma[k] holds the carry into chunk k, in chunk order 0, 1, .. (reverse =
// false) or P-1, P-2, .. (reverse = true).
template <int P>
__device__ __forceinline__ void column_scan(float *ma, const float *mm, int lane, bool reverse) {
  float carry = 0.f;
#pragma unroll
  for (int j = 0; j < P / 32; ++j) {
    const int k = reverse ? (P - 1 - (32 * j + lane)) : (32 * j + lane);
    float A = ma[k], M = mm[k];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float pa = __shfl_up_sync(0xffffffffu, A, off), pm = __shfl_up_sync(0xffffffffu, M, off);
      if (lane >= off) {
        A = fmaf(M, pa, A);
        M *= pm;
      }
    }
    float Ae = __shfl_up_sync(0xffffffffu, A, 1), Me = __shfl_up_sync(0xffffffffu, M, 1);
    if (lane == 0) {
      Ae = 0.f;
      Me = 1.f;
    }
    ma[k] = fmaf(Me, carry, Ae);
    carry = __shfl_sync(0xffffffffu, fmaf(M, carry, A), 31);
  }
}

template <int CW, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) tridiag_pipe_kernel(const TriArgs<float> a) {
  using S = PipeShape<CW, NT>;
  constexpr int C = S::C, P = S::P;
  extern __shared__ __align__(16) float psm[];
  float *mapA = psm + 2 * S::kStageWords;
  float *mapM = mapA + S::kMapWords;
  int *act = reinterpret_cast<int *>(mapM + S::kMapWords);
  __shared__ double red[NT / 32];
  __shared__ int nact_s;
  const int nr = a.nr, nz = a.nz, pitch = a.pitch;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // right-hand sides selected by the mask, in order
  if (warp == 0) {
    int n = 0;
    for (int b = 0; b < a.m; b += 32) {
      const int mm = b + lane;
      const bool sel = mm < a.m && rhs_selected(a.st, a.mask, mm);
      const unsigned bal = __ballot_sync(0xffffffffu, sel);
      if (sel) act[n + __popc(bal & ((1u << lane) - 1u))] = mm;
      n += __popc(bal);
    }
    if (lane == 0) nact_s = n;
  }
  __syncthreads();
  const int nact = nact_s;
  if (nact == 0) return;
  const int ntiles = (nz + CW - 1) / CW;
  // R right-hand sides per group: the R <= 8 with the shortest longest CTA
  // (groups per CTA times R items), the larger R on ties
  int R = 1;
  {
    long long best = -1;
    for (int r = 1; r <= 8 && r <= nact; ++r) {
      const long long ng = (long long)((nact + r - 1) / r) * ntiles;
      const long long span = (ng + gridDim.x - 1) / gridDim.x * r;
      if (best < 0 || span <= best) {
        best = span;
        R = r;
      }
    }
  }
  const int nblk = (nact + R - 1) / R;
  const int ngroups = nblk * ntiles;
  if ((int)blockIdx.x >= ngroups) return;

  const int w = threadIdx.x % CW, c = threadIdx.x / CW;
  const int rbase = c * C;

  // item (group g, index j) -> tile, right-hand side
  auto item_of = [&](int g, int j, int &tile, int &mm) {
    tile = g % ntiles;
    mm = act[(g / ntiles) * R + j];
  };
  auto group_size = [&](int g) { return min(R, nact - (g / ntiles) * R); };
  auto issue = [&](int g, int j, float *dst) {
    int tile, mm;
    item_of(g, j, tile, mm);
    const float *src = a.in + (size_t)mm * a.field + (size_t)tile * CW;
    constexpr int kParts = CW / 4;  // 16-byte pieces per tile row
#pragma unroll
    for (int i = 0; i < S::kRows * kParts / NT; ++i) {
      const int q = threadIdx.x + i * NT;
      const int row = q / kParts, part = q % kParts;
      const bool ok = row < nr;
      cp_async16(dst + (row + row / C) * CW + part * 4, src + (size_t)(ok ? row : 0) * pitch + part * 4, ok);
    }
    cp_async_commit();
  };

  int g = blockIdx.x, j = 0, buf = 0;
  issue(g, 0, psm);
  float ip[C];
  int loaded = -1;  // group (stacked tables: item) whose factors are in ip
  while (g < ngroups) {
    int tile, mm;
    item_of(g, j, tile, mm);
    const int col = tile * CW + w;
    const int gs = group_size(g);
    // next item
    int gn = g, jn = j + 1;
    if (jn == gs) {
      gn = g + gridDim.x;
      jn = 0;
    }
    const int key = a.cstride != 0 ? g * R + j : g;
    if (key != loaded) {
      loaded = key;
      const float *ipg = a.IP + (size_t)mm * a.cstride + (size_t)rbase * pitch + col;
#pragma unroll
      for (int t = 0; t < C; ++t) ip[t] = (rbase + t < nr && col < nz) ? __ldg(ipg + (size_t)t * pitch) : 0.f;
    }
    if (jn == 0 && gn < ngroups && a.cstride == 0) {  // last item of the group: next group's factors into L1
      const int coln = (gn % ntiles) * CW + w;
      if (coln < nz) {
        const float *ipn = a.IP + (size_t)rbase * pitch + coln;
#pragma unroll
        for (int t = 0; t < C; ++t)
          if (rbase + t < nr) prefetch_l1(ipn + (size_t)t * pitch);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();  // this item's tile is in place; the other stage is free
    float *sbuf = psm + buf * S::kStageWords;
    if (gn < ngroups) issue(gn, jn, psm + (buf ^ 1) * S::kStageWords);
    float *sd = sbuf + (c * (C + 1)) * CW + w;  // row rbase + t at sd[t CW]
    float v[C];
#pragma unroll
    for (int t = 0; t < C; ++t) v[t] = sd[t * CW];
    // forward with zero carry-in
    float gg = 0.f, mu = 1.f;
#pragma unroll
    for (int t = 0; t < C; ++t) {
      gg = ip[t] * (v[t] + gg);
      mu *= ip[t];
      v[t] = gg;
    }
    mapA[w * (P + 1) + c] = gg;
    mapM[w * (P + 1) + c] = mu;
    __syncthreads();
    if (warp < CW) column_scan<P>(mapA + warp * (P + 1), mapM + warp * (P + 1), lane, false);
    __syncthreads();
    const float gin = mapA[w * (P + 1) + c];
    // apply the carry, then the backward recurrence with zero carry-in
    float pr = 1.f;
#pragma unroll
    for (int t = 0; t < C; ++t) {
      pr *= ip[t];
      v[t] = fmaf(pr, gin, v[t]);
    }
    float y = 0.f;
    mu = 1.f;
#pragma unroll
    for (int t = C - 1; t >= 0; --t) {
      y = fmaf(ip[t], y, v[t]);
      mu *= ip[t];
      v[t] = y;
    }
    mapA[w * (P + 1) + c] = y;  // each thread rewrites only its own slot
    mapM[w * (P + 1) + c] = mu;
    __syncthreads();
    if (warp < CW) column_scan<P>(mapA + warp * (P + 1), mapM + warp * (P + 1), lane, true);
    __syncthreads();
    const float yin = mapA[w * (P + 1) + c];
    // apply the carry; (b', y') partial
    pr = 1.f;
    float dot = 0.f;
#pragma unroll
    for (int t = C - 1; t >= 0; --t) {
      pr *= ip[t];
      v[t] = fmaf(pr, yin, v[t]);
      dot = fmaf(sd[t * CW], v[t], dot);
    }
    if (a.partial != nullptr) {
      const double sw = warp_sum((double)dot);
      if (lane == 0) red[warp] = sw;
    }
    if (a.split == nullptr) {
      if (col < nz) {
        float *o = a.out + (size_t)mm * a.field + (size_t)rbase * pitch + col;
#pragma unroll
        for (int t = 0; t < C; ++t)
          if (rbase + t < nr) o[(size_t)t * pitch] = v[t];
      }
      if (a.partial != nullptr) {
        __syncthreads();
        if (threadIdx.x == 0) {
          double tot = 0.0;
          for (int i = 0; i < NT / 32; ++i) tot += red[i];
          a.partial[(size_t)mm * kPartialStride + tile] = tot;
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < C; ++t) sd[t * CW] = v[t];
      __syncthreads();
      if (a.partial != nullptr && threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < NT / 32; ++i) tot += red[i];
        a.partial[(size_t)mm * kPartialStride + tile] = tot;
      }
      // write back in the split layout: one row segment of min(CW, 16)
      // columns per thread and step
      constexpr int kSeg = CW < 16 ? CW : 16;
      constexpr int kSegs = CW / kSeg;
      const int c0 = tile * CW;
      for (int q = threadIdx.x; q < nr * kSegs; q += NT) {
        const int row = q / kSegs, sg = q % kSegs;
        const int cs = c0 + sg * kSeg;
        if (cs >= nz) continue;
        const float *src = sbuf + (row + row / C) * CW + sg * kSeg;
        if constexpr (kSeg == 16) {
          float x[16];
#pragma unroll
          for (int e = 0; e < 16; e += 4) {
            const float4 f = *reinterpret_cast<const float4 *>(src + e);
            x[e] = f.x; x[e + 1] = f.y; x[e + 2] = f.z; x[e + 3] = f.w;
          }
          if (cs + 8 < nz) {
            split_store16(a.split, mm, row, cs, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
          } else {  // only the first 8 columns are inside n8
            float x8[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) x8[e] = x[e];
            split_store8(a.split, mm, row, cs, a.split_mtiles, a.split_ktiles, a.split_kbe, x8);
          }
        } else if constexpr (kSeg == 8) {
          float x[8];
          const float4 f0 = *reinterpret_cast<const float4 *>(src), f1 = *reinterpret_cast<const float4 *>(src + 4);
          x[0] = f0.x; x[1] = f0.y; x[2] = f0.z; x[3] = f0.w; x[4] = f1.x; x[5] = f1.y; x[6] = f1.z; x[7] = f1.w;
          split_store8(a.split, mm, row, cs, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
        } else {
          float x[4];
          const float4 f0 = *reinterpret_cast<const float4 *>(src);
          x[0] = f0.x; x[1] = f0.y; x[2] = f0.z; x[3] = f0.w;
          split_store4(a.split, mm, row, cs, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
        }
      }
    }
    g = gn;
    j = jn;
    buf ^= 1;
  }
}

// ---------------------------------------------------------------------------
// Staged register kernel on the row-scaled systems (FP32, variant 9).
//
// The layout of tridiag_reg_kernel (a CTA stages an nr x CW column tile of
// one right-hand side and of the factors in shared memory; WPC warps per
// column, lane c of warp h owning chunk (32 h + c) of C2 rows in registers;
// chunk carries by warp shuffles, across the warps of a column through
// shared memory), but on the systems T'_l = D T_l D with unit couplings (see
// the pipelined kernels above: g = ips (b' + g), y' = g + ips y'), so a chunk
// keeps only its values and factors in registers and each recurrence step is
// one or two operations.  Tiles are staged with 8-byte cp.async (two columns
// per copy); the column pair p = col / 2 of row `row` sits at pair
// p ^ sw(row), sw(row) = (row / (32 / CW)) mod (CW / 2), so row `row`, column `col`
// is at word row CW + 2 (p ^ sw(row)) + col % 2 + 2 (row / C2).  The two spare
// words per chunk keep the pieces 8-byte aligned, and the chunks of a warp's
// lanes (stride C2 CW + 2 words; sw is the same for all of them) fall into 16
// distinct bank pairs (a two-way conflict at most); the XOR spreads the
// write-back, where the lanes of a warp read consecutive rows, over distinct
// bank pairs instead of every fourth row sharing one.
// ---------------------------------------------------------------------------
template <int CW>
__device__ __forceinline__ int reg2_sw(int row) { return (row / (32 / CW)) & (CW / 2 - 1); }
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(ok ? 8 : 0) : "memory");
}

template <int C2, int WPC, int CW>
__global__ void __launch_bounds__(32 * WPC * CW, (32 * WPC * CW <= 512) ? 2 : 1)
    tridiag_reg2_kernel(const TriArgs<float> a) {
  constexpr int NT = 32 * WPC * CW;  // threads
  constexpr int NCH = 32 * WPC;      // chunks per column
  constexpr int NP = NCH * C2;       // padded rows
  constexpr int kChunkWords = C2 * CW + 2;
  constexpr int kTileWords = NCH * kChunkWords;
  static_assert(NT <= 1024 && (CW == 4 || CW == 8 || CW == 16), "tile shape");
  extern __shared__ __align__(16) float tsm2[];
  __shared__ float xfa[CW][WPC], xfm[CW][WPC], xba[CW][WPC], xbm[CW][WPC];
  __shared__ double red[NT / 32];
  const int nr = a.nr, pitch = a.pitch;
  float *ips = tsm2;
  float *ds = ips + kTileWords;
  const int col0 = blockIdx.x * CW;
  const int m = blockIdx.y;
  if (!rhs_selected(a.st, a.mask, m)) return;  // uniform over the CTA
  // ---- stage the tiles: 8-byte pieces, rows of the tile in order ----
  {
    constexpr int kParts = CW / 2;
    const int part = threadIdx.x % kParts;
    const float *ipg = a.IP + (size_t)m * a.cstride + col0 + 2 * part;
    const float *ing = a.in + (size_t)m * a.field + col0 + 2 * part;
#pragma unroll 4
    for (int row = threadIdx.x / kParts; row < NP; row += NT / kParts) {
      const bool ok = row < nr;
      const size_t go = (size_t)(ok ? row : 0) * pitch;
      const int si = row * CW + 2 * (part ^ reg2_sw<CW>(row)) + 2 * (row / C2);
      cp_async8(ips + si, ipg + go, ok);
      cp_async8(ds + si, ing + go, ok);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = warp / WPC, h = warp % WPC;  // column, segment of the r-range
  const int ci = h * 32 + lane;               // chunk index 0 .. NCH - 1
  // column w of row ci C2 + t at word ci kChunkWords + CW t + wc(t)
  float *pd = ds + ci * kChunkWords;
  const float *pip = ips + ci * kChunkWords;
  const int rbase = ci * C2;
  auto wc = [&](int t) { return 2 * ((w >> 1) ^ reg2_sw<CW>(rbase + t)) + (w & 1); };
  float v[C2], ip[C2];
  // forward, zero carry-in
  float g = 0.f, mu = 1.f;
#pragma unroll
  for (int t = 0; t < C2; ++t) {
    ip[t] = pip[CW * t + wc(t)];
    g = ip[t] * (pd[CW * t + wc(t)] + g);
    mu *= ip[t];
    v[t] = g;
  }
  float A = g, M = mu;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float pa = __shfl_up_sync(0xffffffffu, A, off), pm = __shfl_up_sync(0xffffffffu, M, off);
    if (lane >= off) {
      A = fmaf(M, pa, A);
      M *= pm;
    }
  }
  float Ae = __shfl_up_sync(0xffffffffu, A, 1), Me = __shfl_up_sync(0xffffffffu, M, 1);
  if (lane == 0) {
    Ae = 0.f;
    Me = 1.f;
  }
  if (WPC > 1) {
    if (lane == 31) {
      xfa[w][h] = A;
      xfm[w][h] = M;
    }
    __syncthreads();
  }
  float cin = 0.f;  // carry into this warp's first chunk: the maps of warps 0 .. h-1
  for (int j = 0; j < h; ++j) cin = fmaf(xfm[w][j], cin, xfa[w][j]);
  const float gin = fmaf(Me, cin, Ae);
  float pr = 1.f;
#pragma unroll
  for (int t = 0; t < C2; ++t) {
    pr *= ip[t];
    v[t] = fmaf(pr, gin, v[t]);
  }
  // backward, zero carry-in
  float y = 0.f;
  mu = 1.f;
#pragma unroll
  for (int t = C2 - 1; t >= 0; --t) {
    y = fmaf(ip[t], y, v[t]);
    mu *= ip[t];
    v[t] = y;
  }
  A = y;
  M = mu;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float pa = __shfl_down_sync(0xffffffffu, A, off), pm = __shfl_down_sync(0xffffffffu, M, off);
    if (lane + off < 32) {
      A = fmaf(M, pa, A);
      M *= pm;
    }
  }
  Ae = __shfl_down_sync(0xffffffffu, A, 1);
  Me = __shfl_down_sync(0xffffffffu, M, 1);
  if (lane == 31) {
    Ae = 0.f;
    Me = 1.f;
  }
  if (WPC > 1) {
    if (lane == 0) {
      xba[w][h] = A;
      xbm[w][h] = M;
    }
    __syncthreads();
  }
  cin = 0.f;  // carry into this warp's last chunk: the maps of warps WPC-1 .. h+1
  for (int j = WPC - 1; j > h; --j) cin = fmaf(xbm[w][j], cin, xba[w][j]);
  const float yin = fmaf(Me, cin, Ae);
  pr = 1.f;
  float dot = 0.f;
#pragma unroll
  for (int t = C2 - 1; t >= 0; --t) {
    pr *= ip[t];
    v[t] = fmaf(pr, yin, v[t]);
    dot = fmaf(pd[CW * t + wc(t)], v[t], dot);  // (b', y') of this chunk: the (rhat, yhat) partial
    pd[CW * t + wc(t)] = v[t];
  }
  if (a.partial != nullptr) {
    const double sw = warp_sum((double)dot);
    if (lane == 0) red[warp] = sw;
  }
  __syncthreads();
  if (a.partial != nullptr && threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < NT / 32; ++i) tot += red[i];
    a.partial[(size_t)m * kPartialStride + blockIdx.x] = tot;
  }
  // ---- write back: one thread per row, its CW columns ----
  const int ncol = min(CW, a.nz - col0);
  for (int row = threadIdx.x; row < nr; row += NT) {
    float x[CW];
    const float *src = ds + row * CW + 2 * (row / C2);
    const int sw = reg2_sw<CW>(row);
#pragma unroll
    for (int c = 0; c < CW; c += 2) {
      const float2 f2 = *reinterpret_cast<const float2 *>(src + 2 * ((c >> 1) ^ sw));
      x[c] = f2.x;
      x[c + 1] = f2.y;
    }
    if (a.split != nullptr) {
      if constexpr (CW == 16) {
        if (col0 + 8 < a.nz) {
          split_store16(a.split, m, row, col0, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
        } else {  // only the first 8 columns are inside n8
          float x8[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) x8[e] = x[e];
          split_store8(a.split, m, row, col0, a.split_mtiles, a.split_ktiles, a.split_kbe, x8);
        }
      } else if constexpr (CW == 8) {
        split_store8(a.split, m, row, col0, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
      } else {
        split_store4(a.split, m, row, col0, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
      }
    } else {
      float *o = a.out + (size_t)m * a.field + (size_t)row * pitch + col0;
      if (ncol == CW) {
#pragma unroll
        for (int c = 0; c < CW; c += 4) *reinterpret_cast<float4 *>(o + c) = make_float4(x[c], x[c + 1], x[c + 2], x[c + 3]);
      } else {
        for (int c = 0; c < ncol; ++c) o[c] = x[c];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Variant 14: the kernel above fed mode-major (FP32, row-scaled systems).
//
// The forward tensor-core transform writes rhat mode-major (tout): column l of
// right-hand side m is a contiguous run of rows, and the factors IPS have the
// same layout (IPST).  A lane's chunk of C2 rows of one column is then C2
// contiguous floats, and the lanes of a warp (consecutive chunks of the same
// column) read one contiguous run: data and factors go straight from global
// memory to registers with 16-byte loads, with no shared-memory staging (the
// staged kernels are bound by the shared-memory pipe).  Recurrences, carries,
// partials and the write-back of the result through the CTA's shared tile into
// the split operand are those of tridiag_reg2_kernel, whose layout the tile
// keeps.
// ---------------------------------------------------------------------------
template <int C2, int WPC, int CW, bool LOOP>
__global__ void __launch_bounds__(32 * WPC * CW, (32 * WPC * CW <= 512) ? 2 : 1)
    tridiag_tr_kernel(const TriArgs<float> a) {
  constexpr int NT = 32 * WPC * CW;
  constexpr int kChunkWords = C2 * CW + 2;
  static_assert(NT <= 1024 && (CW == 4 || CW == 8) && C2 % 4 == 0, "tile shape");
  extern __shared__ __align__(16) float tsm3[];
  __shared__ float xfa[CW][WPC], xfm[CW][WPC], xba[CW][WPC], xbm[CW][WPC];
  __shared__ double red[NT / 32];
  // one tile: column group cg (columns cg CW ..) of right-hand side m
  auto tile = [&](const int cg, const int m) {
  const int nr = a.nr;
  float *ds = tsm3;
  const int col0 = cg * CW;
  if (!rhs_selected(a.st, a.mask, m)) return;  // uniform over the CTA
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = warp / WPC, h = warp % WPC;  // column, segment of the r-range
  const int ci = h * 32 + lane;               // chunk index 0 .. NCH - 1
  const int rbase = ci * C2;
  const int col = col0 + w;
  const bool cok = col < a.nz;
  // the chunk's data and factors: C2 contiguous floats each (zeros past nr
  // and past nz)
  float v[C2], ip[C2];
  {
    const int colc = cok ? col : a.nz - 1;
    const float *pv = a.in + ((size_t)m * a.nz + colc) * a.tpitch + rbase;
    const float *pi = a.IPST + (size_t)m * a.tcstride + (size_t)colc * a.tpitch + rbase;
#pragma unroll
    for (int t = 0; t < C2; t += 4) {
      const bool ok = cok && rbase + t < nr;  // a group of 4 rows lies inside tpitch (a multiple of 32)
      const float4 d4 = ok ? *reinterpret_cast<const float4 *>(pv + t) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 f4 = ok ? __ldg(reinterpret_cast<const float4 *>(pi + t)) : make_float4(0.f, 0.f, 0.f, 0.f);
      v[t] = d4.x; v[t + 1] = d4.y; v[t + 2] = d4.z; v[t + 3] = d4.w;
      ip[t] = f4.x; ip[t + 1] = f4.y; ip[t + 2] = f4.z; ip[t + 3] = f4.w;
    }
#pragma unroll
    for (int t = 0; t < C2; ++t)
      if (rbase + t >= nr) v[t] = ip[t] = 0.f;  // padding rows solve to zero
  }
  float b[C2];
#pragma unroll
  for (int t = 0; t < C2; ++t) b[t] = v[t];
  // forward, zero carry-in
  float g = 0.f, mu = 1.f;
#pragma unroll
  for (int t = 0; t < C2; ++t) {
    g = ip[t] * (v[t] + g);
    mu *= ip[t];
    v[t] = g;
  }
  float A = g, M = mu;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float pa = __shfl_up_sync(0xffffffffu, A, off), pm = __shfl_up_sync(0xffffffffu, M, off);
    if (lane >= off) {
      A = fmaf(M, pa, A);
      M *= pm;
    }
  }
  float Ae = __shfl_up_sync(0xffffffffu, A, 1), Me = __shfl_up_sync(0xffffffffu, M, 1);
  if (lane == 0) {
    Ae = 0.f;
    Me = 1.f;
  }
  if (WPC > 1) {
    if (lane == 31) {
      xfa[w][h] = A;
      xfm[w][h] = M;
    }
    __syncthreads();
  }
  float cin = 0.f;
  for (int j = 0; j < h; ++j) cin = fmaf(xfm[w][j], cin, xfa[w][j]);
  const float gin = fmaf(Me, cin, Ae);
  float pr = 1.f;
#pragma unroll
  for (int t = 0; t < C2; ++t) {
    pr *= ip[t];
    v[t] = fmaf(pr, gin, v[t]);
  }
  // backward, zero carry-in
  float y = 0.f;
  mu = 1.f;
#pragma unroll
  for (int t = C2 - 1; t >= 0; --t) {
    y = fmaf(ip[t], y, v[t]);
    mu *= ip[t];
    v[t] = y;
  }
  A = y;
  M = mu;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float pa = __shfl_down_sync(0xffffffffu, A, off), pm = __shfl_down_sync(0xffffffffu, M, off);
    if (lane + off < 32) {
      A = fmaf(M, pa, A);
      M *= pm;
    }
  }
  Ae = __shfl_down_sync(0xffffffffu, A, 1);
  Me = __shfl_down_sync(0xffffffffu, M, 1);
  if (lane == 31) {
    Ae = 0.f;
    Me = 1.f;
  }
  if (WPC > 1) {
    if (lane == 0) {
      xba[w][h] = A;
      xbm[w][h] = M;
    }
    __syncthreads();
  }
  cin = 0.f;
  for (int j = WPC - 1; j > h; --j) cin = fmaf(xbm[w][j], cin, xba[w][j]);
  const float yin = fmaf(Me, cin, Ae);
  pr = 1.f;
  float dot = 0.f;
  float *pd = ds + ci * kChunkWords;
  auto wc = [&](int t) { return 2 * ((w >> 1) ^ reg2_sw<CW>(rbase + t)) + (w & 1); };
#pragma unroll
  for (int t = C2 - 1; t >= 0; --t) {
    pr *= ip[t];
    v[t] = fmaf(pr, yin, v[t]);
    dot = fmaf(b[t], v[t], dot);  // (b', y') of this chunk: the (rhat, yhat) partial
    pd[CW * t + wc(t)] = v[t];
  }
  if (a.partial != nullptr) {
    const double sw = warp_sum((double)dot);
    if (lane == 0) red[warp] = sw;
  }
  __syncthreads();
  if (a.partial != nullptr && threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < NT / 32; ++i) tot += red[i];
    a.partial[(size_t)m * kPartialStride + cg] = tot;
  }
  // ---- write back: one thread per row, its CW columns (as tridiag_reg2_kernel)
  const int ncol = min(CW, a.nz - col0);
  for (int row = threadIdx.x; row < nr; row += NT) {
    float x[CW];
    const float *src = ds + row * CW + 2 * (row / C2);
    const int sw = reg2_sw<CW>(row);
#pragma unroll
    for (int c = 0; c < CW; c += 2) {
      const float2 f2 = *reinterpret_cast<const float2 *>(src + 2 * ((c >> 1) ^ sw));
      x[c] = f2.x;
      x[c + 1] = f2.y;
    }
    if (a.split != nullptr) {
      if constexpr (CW == 8) {
        split_store8(a.split, m, row, col0, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
      } else {
        split_store4(a.split, m, row, col0, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
      }
    } else {
      float *o = a.out + (size_t)m * a.field + (size_t)row * a.pitch + col0;
      if (ncol == CW) {
#pragma unroll
        for (int c = 0; c < CW; c += 4) *reinterpret_cast<float4 *>(o + c) = make_float4(x[c], x[c + 1], x[c + 2], x[c + 3]);
      } else {
        for (int c = 0; c < ncol; ++c) o[c] = x[c];
      }
    }
  }
  };
  if constexpr (LOOP) {
    // a launch that rarely selects a right-hand side (TriArgs::short_grid):
    // a few CTAs per SM loop over the tiles t = (right-hand side t / ncg,
    // column group t % ncg), after the gate (TriArgs::gate) if there is one
    if (a.gate != nullptr && *a.gate == 0) return;  // nothing selected
    const int ncg = (a.nz + CW - 1) / CW, ntiles = ncg * a.m;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      tile(t % ncg, t / ncg);
      __syncthreads();  // the tile's shared arrays are read before the next tile writes them
    }
  } else {
    tile(blockIdx.x, blockIdx.y);  // one CTA per tile
  }
}

template <int C2, int WPC, int CW>
void launch_tridiag_tr(const TriArgs<float> &a, cudaStream_t s) {
  constexpr int NT = 32 * WPC * CW;
  const size_t smem = (size_t)(32 * WPC) * (C2 * CW + 2) * sizeof(float);
  if (a.short_grid) {
    ensure_smem_attr((const void *)tridiag_tr_kernel<C2, WPC, CW, true>, smem);
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms <= 0) sms = 148;
    }
    const long long tiles = (long long)((a.nz + CW - 1) / CW) * a.m;
    const int grid = (int)std::min<long long>(tiles, (long long)sms * (NT <= 512 ? 2 : 1));
    tridiag_tr_kernel<C2, WPC, CW, true><<<grid, NT, smem, s>>>(a);
    return;
  }
  ensure_smem_attr((const void *)tridiag_tr_kernel<C2, WPC, CW, false>, smem);
  dim3 grid((a.nz + CW - 1) / CW, a.m);
  tridiag_tr_kernel<C2, WPC, CW, false><<<grid, NT, smem, s>>>(a);
}

// ---------------------------------------------------------------------------
// Variants 10 and 11: the kernel above with the factors kept across right-hand
// sides.  A CTA owns one column tile and R consecutive right-hand sides
// (R = 4 or 8): it stages the factors of the tile once and keeps each lane's
// C2 of them in registers, then solves the selected right-hand sides in turn,
// the data tile of the next one copied into the second of two shared-memory
// stages while the current one is solved.  Same layout, arithmetic and
// partials as tridiag_reg2_kernel.
// ---------------------------------------------------------------------------
template <int C2, int WPC, int CW>
__global__ void __launch_bounds__(32 * WPC * CW, (32 * WPC * CW <= 512) ? 2 : 1)
    tridiag_reg3_kernel(const TriArgs<float> a, int R) {
  constexpr int NT = 32 * WPC * CW;
  constexpr int NCH = 32 * WPC;
  constexpr int NP = NCH * C2;
  constexpr int kChunkWords = C2 * CW + 2;
  constexpr int kTileWords = NCH * kChunkWords;
  constexpr int kParts = CW / 2;
  static_assert(NT <= 1024 && (CW == 4 || CW == 8), "tile shape");
  extern __shared__ __align__(16) float tsm3[];
  __shared__ float xfa[CW][WPC], xfm[CW][WPC], xba[CW][WPC], xbm[CW][WPC];
  __shared__ double red[NT / 32];
  const int nr = a.nr, pitch = a.pitch;
  float *ips = tsm3;
  auto dbuf = [&](int b) { return tsm3 + (1 + b) * kTileWords; };
  const int col0 = blockIdx.x * CW;
  const int m0 = blockIdx.y * R, m1 = min(a.m, m0 + R);
  auto next_sel = [&](int from) {  // first selected right-hand side >= from (m1 if none)
    int mm = from;
    while (mm < m1 && !rhs_selected(a.st, a.mask, mm)) ++mm;
    return mm;
  };
  int mc = next_sel(m0);
  if (mc >= m1) return;  // uniform over the CTA
  const int part = threadIdx.x % kParts;
  auto stage = [&](const float *g, float *dst) {
#pragma unroll 4
    for (int row = threadIdx.x / kParts; row < NP; row += NT / kParts) {
      const bool ok = row < nr;
      cp_async8(dst + row * CW + 2 * (part ^ reg2_sw<CW>(row)) + 2 * (row / C2),
                g + (size_t)(ok ? row : 0) * pitch + 2 * part, ok);
    }
  };
  // factors (one table for all right-hand sides of an operator; a stacked
  // group has one per right-hand side and is not launched here)
  stage(a.IP + col0, ips);
  stage(a.in + (size_t)mc * a.field + col0, dbuf(0));
  cp_async_commit();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = warp / WPC, h = warp % WPC;
  const int ci = h * 32 + lane;
  const int rbase = ci * C2;
  auto wc = [&](int t) { return 2 * ((w >> 1) ^ reg2_sw<CW>(rbase + t)) + (w & 1); };
  const int ncol = min(CW, a.nz - col0);
  float ip[C2];
  bool have_ip = false;
  int buf = 0;
  while (mc < m1) {
    const int mn = next_sel(mc + 1);
    if (mn < m1) {
      stage(a.in + (size_t)mn * a.field + col0, dbuf(buf ^ 1));
      cp_async_commit();
      asm volatile("cp.async.wait_group 1;" ::: "memory");  // all but the newest group
    } else {
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncthreads();
    if (!have_ip) {
      const float *pip = ips + ci * kChunkWords;
#pragma unroll
      for (int t = 0; t < C2; ++t) ip[t] = pip[CW * t + wc(t)];
      have_ip = true;
    }
    float *pd = dbuf(buf) + ci * kChunkWords;
    float v[C2];
    float g = 0.f, mu = 1.f;
#pragma unroll
    for (int t = 0; t < C2; ++t) {
      g = ip[t] * (pd[CW * t + wc(t)] + g);
      mu *= ip[t];
      v[t] = g;
    }
    float A = g, M = mu;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float pa = __shfl_up_sync(0xffffffffu, A, off), pm = __shfl_up_sync(0xffffffffu, M, off);
      if (lane >= off) {
        A = fmaf(M, pa, A);
        M *= pm;
      }
    }
    float Ae = __shfl_up_sync(0xffffffffu, A, 1), Me = __shfl_up_sync(0xffffffffu, M, 1);
    if (lane == 0) {
      Ae = 0.f;
      Me = 1.f;
    }
    if (WPC > 1) {
      if (lane == 31) {
        xfa[w][h] = A;
        xfm[w][h] = M;
      }
      __syncthreads();
    }
    float cin = 0.f;
    for (int j = 0; j < h; ++j) cin = fmaf(xfm[w][j], cin, xfa[w][j]);
    const float gin = fmaf(Me, cin, Ae);
    float pr = 1.f;
#pragma unroll
    for (int t = 0; t < C2; ++t) {
      pr *= ip[t];
      v[t] = fmaf(pr, gin, v[t]);
    }
    float y = 0.f;
    mu = 1.f;
#pragma unroll
    for (int t = C2 - 1; t >= 0; --t) {
      y = fmaf(ip[t], y, v[t]);
      mu *= ip[t];
      v[t] = y;
    }
    A = y;
    M = mu;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const float pa = __shfl_down_sync(0xffffffffu, A, off), pm = __shfl_down_sync(0xffffffffu, M, off);
      if (lane + off < 32) {
        A = fmaf(M, pa, A);
        M *= pm;
      }
    }
    Ae = __shfl_down_sync(0xffffffffu, A, 1);
    Me = __shfl_down_sync(0xffffffffu, M, 1);
    if (lane == 31) {
      Ae = 0.f;
      Me = 1.f;
    }
    if (WPC > 1) {
      if (lane == 0) {
        xba[w][h] = A;
        xbm[w][h] = M;
      }
      __syncthreads();
    }
    cin = 0.f;
    for (int j = WPC - 1; j > h; --j) cin = fmaf(xbm[w][j], cin, xba[w][j]);
    const float yin = fmaf(Me, cin, Ae);
    pr = 1.f;
    float dot = 0.f;
#pragma unroll
    for (int t = C2 - 1; t >= 0; --t) {
      pr *= ip[t];
      v[t] = fmaf(pr, yin, v[t]);
      dot = fmaf(pd[CW * t + wc(t)], v[t], dot);
      pd[CW * t + wc(t)] = v[t];
    }
    if (a.partial != nullptr) {
      const double sw = warp_sum((double)dot);
      if (lane == 0) red[warp] = sw;
    }
    __syncthreads();
    if (a.partial != nullptr && threadIdx.x == 0) {
      double tot = 0.0;
      for (int i = 0; i < NT / 32; ++i) tot += red[i];
      a.partial[(size_t)mc * kPartialStride + blockIdx.x] = tot;
    }
    for (int row = threadIdx.x; row < nr; row += NT) {
      float x[CW];
      const float *src = dbuf(buf) + row * CW + 2 * (row / C2);
      const int sw = reg2_sw<CW>(row);
#pragma unroll
      for (int c = 0; c < CW; c += 2) {
        const float2 f2 = *reinterpret_cast<const float2 *>(src + 2 * ((c >> 1) ^ sw));
        x[c] = f2.x;
        x[c + 1] = f2.y;
      }
      if (a.split != nullptr) {
        if constexpr (CW == 8) split_store8(a.split, mc, row, col0, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
        else split_store4(a.split, mc, row, col0, a.split_mtiles, a.split_ktiles, a.split_kbe, x);
      } else {
        float *o = a.out + (size_t)mc * a.field + (size_t)row * pitch + col0;
        if (ncol == CW) {
#pragma unroll
          for (int c = 0; c < CW; c += 4)
            *reinterpret_cast<float4 *>(o + c) = make_float4(x[c], x[c + 1], x[c + 2], x[c + 3]);
        } else {
          for (int c = 0; c < ncol; ++c) o[c] = x[c];
        }
      }
    }
    __syncthreads();  // the stage is read; the next copy into it may start
    mc = mn;
    buf ^= 1;
  }
}

}  // namespace

// Chunk length C: short enough that the chunk stays in registers without
// spilling (16 FP32 / 8 FP64 values); very tall systems use twice that so
// that a CTA still spans >= 8 mode columns (32-byte row segments).
template <typename T> struct TriChunk;
template <> struct TriChunk<float> { static constexpr int small = 16, large = 32, switch_nr = 2048; };
template <> struct TriChunk<double> { static constexpr int small = 8, large = 16, switch_nr = 1024; };

template <typename T, int C>
void launch_tridiag_c(const TriArgs<T> &a, cudaStream_t s) {
  const int P = (a.nr + C - 1) / C;
  // CTAs of at most 512 threads while that still spans >= 8 mode columns, so
  // two CTAs share an SM (one loads while the other scans); else up to 1024.
  const int max_threads = (P <= 64) ? 512 : 1024;
  int W = 32;
  while (W > 1 && W * P > max_threads) W >>= 1;
  // P <= 1024 holds for nr <= 8192 (the set-up limit).
  const size_t smem = 2ull * P * W * sizeof(T);
  dim3 grid(a.m, (a.nz + W - 1) / W);
  if (smem > 48 * 1024) ensure_smem_attr((const void *)tridiag_kernel<T, C>, smem);
  tridiag_kernel<T, C><<<grid, W * P, smem, s>>>(a, W, P);
}

template <int C2, int WPC, int CW>
void launch_tridiag_reg2(const TriArgs<float> &a, cudaStream_t s) {
  constexpr int NCH = 32 * WPC;
  const size_t smem = sizeof(float) * 2 * NCH * (C2 * CW + 2);
  ensure_smem_attr((const void *)tridiag_reg2_kernel<C2, WPC, CW>, smem);
  dim3 grid((a.nz + CW - 1) / CW, a.m);
  TriArgs<float> b = a;  // the scaled factors through IP
  b.IP = a.IPS;
  tridiag_reg2_kernel<C2, WPC, CW><<<grid, 32 * WPC * CW, smem, s>>>(b);
}

template <int C2, int WPC, int CW>
void launch_tridiag_reg3(const TriArgs<float> &a, int R, cudaStream_t s) {
  constexpr int NCH = 32 * WPC;
  const size_t smem = sizeof(float) * 3 * NCH * (C2 * CW + 2);
  ensure_smem_attr((const void *)tridiag_reg3_kernel<C2, WPC, CW>, smem);
  dim3 grid((a.nz + CW - 1) / CW, (a.m + R - 1) / R);
  TriArgs<float> b = a;
  b.IP = a.IPS;
  tridiag_reg3_kernel<C2, WPC, CW><<<grid, 32 * WPC * CW, smem, s>>>(b, R);
}

template <int C2, int WPC, int CW>
void launch_tridiag_reg(const TriArgs<float> &a, cudaStream_t s) {
  // mirrors the kernel's layout: the IP and data tiles
  constexpr int NCH = 32 * WPC, NP = NCH * C2;
  const size_t smem = sizeof(float) * 2 * (NP * CW + NCH);
  ensure_smem_attr((const void *)tridiag_reg_kernel<C2, WPC, CW>, smem);
  dim3 grid((a.nz + CW - 1) / CW, a.m);
  tridiag_reg_kernel<C2, WPC, CW><<<grid, 32 * WPC * CW, smem, s>>>(a);
}

// FP32 kernel variants: 1 the staged register kernel; 2.. the pipelined
// column-tile kernels <CW columns, NT threads>.
struct PipeVariant { int id, cw, nt; };
constexpr PipeVariant kPipeVariants[] = {{2, 32, 1024}, {3, 16, 512}, {4, 16, 1024}, {5, 8, 512},
                                         {6, 8, 1024}, {7, 4, 512}, {8, 4, 1024}};

int pipe_max_rows(const PipeVariant &v) { return 16 * v.nt / v.cw; }

int tridiag_variants(int nr, int *ids) {
  // the default first: the staged kernel on the row-scaled systems fed
  // mode-major by the forward transform (14; measured 8.25 ms per
  // 1024^2 x 64 solve and 99.9 ms per 4096^2 x 16 solve, against 9.7 and
  // 140.6 for the same kernel staging a row-major input, 9, which runs where
  // the input is row-major), then the others (10.4 ms for the plain register
  // kernel 1, 11.3 to 12.5 for the pipelined kernels and for 10, 11, 12);
  // paths that cannot scale the rows (the FFT transforms) take kernel 1
  // (tridiag_effective)
  int n = 0;
  if (nr <= 4096) {
    ids[n++] = 14;
    ids[n++] = 9;
    ids[n++] = 1;
    ids[n++] = 10;
    ids[n++] = 11;
  }
  if (nr <= 1024) ids[n++] = 12;
  for (const PipeVariant &v : kPipeVariants)
    if (nr <= pipe_max_rows(v) && 2 * nr > pipe_max_rows(v)) ids[n++] = v.id;
  return n;
}

static const PipeVariant *find_pipe(int id) {
  for (const PipeVariant &v : kPipeVariants)
    if (v.id == id) return &v;
  return nullptr;
}

// The variant that runs for nr rows: `variant` if it covers nr, else the
// default (0 when no FP32 tile kernel covers nr).
static int resolve_variant(int nr, int variant) {
  int ids[16];
  const int n = tridiag_variants(nr, ids);
  if (n == 0) return 0;
  for (int i = 0; i < n; ++i)
    if (ids[i] == variant) return variant;
  return ids[0];
}

// Columns per CTA of the register kernel for nr rows (0: not covered).
static int reg_cols(int nr) { return nr <= 2048 ? 8 : (nr <= 4096 ? 4 : 0); }

int tridiag_reg_cols(int nr, int variant) {
  const int v = resolve_variant(nr, variant);
  if (v == 0) return 0;
  if (v == 12) return 16;
  if (v == 1 || v >= 9) return reg_cols(nr);
  return find_pipe(v)->cw;
}

template <int CW, int NT>
void launch_tridiag_pipe(const TriArgs<float> &a, cudaStream_t s) {
  using S = PipeShape<CW, NT>;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  ensure_smem_attr((const void *)tridiag_pipe_kernel<CW, NT>, S::smem);
  const long long items = (long long)a.m * ((a.nz + CW - 1) / CW);
  const int grid = (int)std::min<long long>(items, (long long)sms * (1024 / NT));
  TriArgs<float> b = a;  // the kernel reads the scaled tables through IP and E
  b.IP = a.IPS;
  b.E = a.RS;
  tridiag_pipe_kernel<CW, NT><<<grid, NT, S::smem, s>>>(b);
}

int tridiag_effective(int nr, int variant, int m, bool scaled_tables) {
  const int v = resolve_variant(nr, variant);
  if (v >= 2 && (!scaled_tables || (v < 9 && m > PipeShape<16, 1024>::kMaxList))) return 1;
  return v;
}

bool launch_tridiag_tile(const TriArgs<float> &a, cudaStream_t s) {
  int v = resolve_variant(a.nr, a.variant);
  if (v == 0) return false;
  // the pipelined kernels solve the row-scaled systems; plain data takes the
  // register kernel
  if (!a.prescaled) v = 1;
  if (v == 10 || v == 11) {
    if (a.cstride != 0) {
      v = 9;  // a stacked group: factors per right-hand side
    } else {
      const int R = v == 10 ? 4 : 8;
      const int c2 = (a.nr + 63) / 64;
      if (c2 <= 4) launch_tridiag_reg3<4, 2, 8>(a, R, s);
      else if (c2 <= 8) launch_tridiag_reg3<8, 2, 8>(a, R, s);
      else if (c2 <= 16) launch_tridiag_reg3<16, 2, 8>(a, R, s);
      else if (a.nr <= 2048) launch_tridiag_reg3<16, 4, 8>(a, R, s);
      else launch_tridiag_reg3<16, 8, 4>(a, R, s);
      return true;
    }
  }
  if (v == 14) {  // mode-major input (the forward transform wrote it so)
    if (a.IPST == nullptr || a.tpitch == 0) {
      v = 9;
    } else {
      const int c2 = (a.nr + 63) / 64;
      if (c2 <= 4) launch_tridiag_tr<4, 2, 8>(a, s);
      else if (c2 <= 8) launch_tridiag_tr<8, 2, 8>(a, s);
      else if (c2 <= 16) launch_tridiag_tr<16, 2, 8>(a, s);
      else if (a.nr <= 2048) launch_tridiag_tr<16, 4, 8>(a, s);
      else launch_tridiag_tr<16, 8, 4>(a, s);
      return true;
    }
  }
  if (v == 12) {  // the same on 16-column tiles (one 1024-thread CTA per SM)
    const int c2 = (a.nr + 63) / 64;
    if (c2 <= 4) launch_tridiag_reg2<4, 2, 16>(a, s);
    else if (c2 <= 8) launch_tridiag_reg2<8, 2, 16>(a, s);
    else launch_tridiag_reg2<16, 2, 16>(a, s);
    return true;
  }
  if (v == 9) {  // the staged register kernel on the row-scaled systems
    const int c2 = (a.nr + 63) / 64;
    if (c2 <= 4) launch_tridiag_reg2<4, 2, 8>(a, s);
    else if (c2 <= 8) launch_tridiag_reg2<8, 2, 8>(a, s);
    else if (c2 <= 16) launch_tridiag_reg2<16, 2, 8>(a, s);
    else if (a.nr <= 2048) launch_tridiag_reg2<16, 4, 8>(a, s);
    else launch_tridiag_reg2<16, 8, 4>(a, s);
    return true;
  }
  switch (v) {
    case 2: launch_tridiag_pipe<32, 1024>(a, s); return true;
    case 3: launch_tridiag_pipe<16, 512>(a, s); return true;
    case 4: launch_tridiag_pipe<16, 1024>(a, s); return true;
    case 5: launch_tridiag_pipe<8, 512>(a, s); return true;
    case 6: launch_tridiag_pipe<8, 1024>(a, s); return true;
    case 7: launch_tridiag_pipe<4, 512>(a, s); return true;
    case 8: launch_tridiag_pipe<4, 1024>(a, s); return true;
    default: break;
  }
  // the staged register kernel: chunks of up to 16 rows in registers; 2, 4 or
  // 8 warps per column system
  const int c2 = (a.nr + 63) / 64;
  if (c2 <= 4) launch_tridiag_reg<4, 2, 8>(a, s);
  else if (c2 <= 8) launch_tridiag_reg<8, 2, 8>(a, s);
  else if (c2 <= 16) launch_tridiag_reg<16, 2, 8>(a, s);
  else if (a.nr <= 2048) launch_tridiag_reg<16, 4, 8>(a, s);
  else if (a.nr <= 4096) launch_tridiag_reg<16, 8, 4>(a, s);
  else return false;
  return true;
}

bool tridiag_split_ok(int nr) { return reg_cols(nr) != 0; }

template <typename T>
void launch_tridiag(const TriArgs<T> &a, cudaStream_t s) {
  note_launch();
  if constexpr (sizeof(T) == 4) {
    if (launch_tridiag_tile(a, s)) return;
  }
  if (a.nr > TriChunk<T>::switch_nr) launch_tridiag_c<T, TriChunk<T>::large>(a, s);
  else launch_tridiag_c<T, TriChunk<T>::small>(a, s);
}

template void launch_tridiag<float>(const TriArgs<float> &, cudaStream_t);
template void launch_tridiag<double>(const TriArgs<double> &, cudaStream_t);

}  // namespace ax
