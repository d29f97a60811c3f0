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

// Tiled variant (FP32, nr <= 32 C): a CTA stages an nr x CW column tile of
// IP, of the couplings E and of the data of MR right-hand sides in shared
// memory with coalesced row loads.  Each warp then owns one (column,
// right-hand side) system: lane c holds rows c C .. c C + C - 1 in registers,
// and the affine carry maps of the 32 chunks are composed with warp shuffles
// (no CTA-wide barrier inside the solve).  The shared layouts are padded by
// one word per chunk, idx(row, col) = row CW + col + row / C, so that the 32
// lanes of a warp (rows c C + t, one column) fall in 32 distinct banks: the
// bank is ((8 C + 1) c + 8 t + col) mod 32 for CW = 8, and 8 C + 1 is odd.
constexpr int kTileCW = 8;   // columns per CTA (one 32-byte sector per row)

__device__ __forceinline__ int tidx(int row, int col, int C) { return row * kTileCW + col + row / C; }

// 4-byte asynchronous global -> shared copy (zero fill when !ok); the whole
// tile is in flight at once instead of one row per round trip.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// MR right-hand sides per CTA: 2 when they share one operator (the IP tile is
// staged once for both), 1 when each has its own factors (batched groups).
// The tile is padded to NP = 32 C rows with IP = E = 0 (and zero data): a
// padding row then has alpha = beta = 0 and solves to 0, so every lane runs
// the same unpredicated recurrences.  EA[row] = E[row - 1] (0 on row 0) and
// EB[row] = E[row] are stored at row + row / C, so that lane c finds its
// chunk's couplings at the fixed offsets c (C + 1) + t.
template <int C, int MR>
__global__ void __launch_bounds__(32 * kTileCW * MR, 4 / MR) tridiag_tile_kernel(const TriArgs<float> a) {
  constexpr int NP = 32 * C;
  constexpr int kTileWords = NP * kTileCW + 32;
  constexpr int kEWords = NP + 32;
  extern __shared__ __align__(16) float tsm[];
  const int nr = a.nr, pitch = a.pitch;
  float *ips = tsm;                  // [tile] IP
  float *ea = ips + kTileWords;      // E[row - 1]
  float *eb = ea + kEWords;          // E[row]
  float *ds = eb + kEWords;          // [MR][tile] data
  const int col0 = blockIdx.x * kTileCW;
  const int m0 = blockIdx.y * MR;
  const int mcount = min(MR, a.m - m0);
  const int ncol = min(kTileCW, a.nz - col0);
  // which of this CTA's right-hand sides are selected (uniform over the CTA)
  bool sel[MR];
  bool any = false;
#pragma unroll
  for (int j = 0; j < MR; ++j) {
    sel[j] = j < mcount && rhs_selected(a.st, a.mask, m0 + j);
    any = any || sel[j];
  }
  if (!any) return;
  // ---- stage the tiles (coalesced: 8 consecutive threads read one row) ----
  const int cw = threadIdx.x % kTileCW;
  {
    const bool colok = cw < ncol;
    const int cc = colok ? cw : 0;  // a valid source address for the zero-filled lanes
    const float *ipg = a.IP + (size_t)m0 * a.cstride + col0 + cc;
    for (int row = threadIdx.x / kTileCW; row < NP; row += blockDim.x / kTileCW) {
      const bool ok = colok && row < nr;
      const int rs = ok ? row : 0;
      const int si = tidx(row, cw, C);
      cp_async4(ips + si, ipg + (size_t)rs * pitch, ok);
#pragma unroll
      for (int j = 0; j < MR; ++j)
        if (sel[j]) cp_async4(ds + j * kTileWords + si, a.in + (size_t)(m0 + j) * a.field + (size_t)rs * pitch + col0 + cc, ok);
    }
    const float *eg = a.E + (size_t)m0 * a.estride;
    for (int row = threadIdx.x; row < NP; row += blockDim.x) {
      const int ei = row + row / C;
      cp_async4(ea + ei, eg + (row > 0 && row - 1 < nr ? row - 1 : 0), row > 0 && row - 1 < nr);
      cp_async4(eb + ei, eg + (row < nr ? row : 0), row < nr);
    }
    cp_async_wait_all();
  }
  __syncthreads();
  // ---- one system per warp ----
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = warp % kTileCW, j = warp / kTileCW;
  if (sel[j] && w < ncol) {
    // lane c: rows c C + t, tile offset c (8 C + 1) + w + 8 t
    float *pd = ds + j * kTileWords + lane * (kTileCW * C + 1) + w;
    const float *pip = ips + lane * (kTileCW * C + 1) + w;
    const float *pea = ea + lane * (C + 1);
    const float *peb = eb + lane * (C + 1);
    // The chunk's values live in registers for C <= 16; 32-row chunks work in
    // the shared tile itself (32 more registers would spill).
    constexpr bool kRegs = C <= 16;
    float v[kRegs ? C : 1];
    if constexpr (kRegs) {
#pragma unroll
      for (int t = 0; t < C; ++t) v[t] = pd[kTileCW * t];
    }
    auto rd = [&](int t) -> float {
      if constexpr (kRegs) return v[t];
      else return pd[kTileCW * t];
    };
    auto wr = [&](int t, float x) {
      if constexpr (kRegs) v[t] = x;
      else pd[kTileCW * t] = x;
    };
    // forward, zero carry-in: g_t = v_t ip_t + alpha_t g_{t-1}, alpha_t = -E_{t-1} ip_t
    float g = 0.f, mu = 1.f;
#pragma unroll
    for (int t = 0; t < C; ++t) {
      // fences every 8 rows keep the unrolled loads near their use
      if ((t & 7) == 0) asm volatile("" ::: "memory");
      const float ip = pip[kTileCW * t];
      const float al = -pea[t] * ip;
      g = fmaf(rd(t), ip, al * g);
      mu *= al;
      wr(t, g);
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
    float gin = __shfl_up_sync(0xffffffffu, A, 1);
    if (lane == 0) gin = 0.f;
    mu = 1.f;
#pragma unroll
    for (int t = 0; t < C; ++t) {
      if ((t & 7) == 0) asm volatile("" ::: "memory");
      mu *= -pea[t] * pip[kTileCW * t];
      wr(t, fmaf(mu, gin, rd(t)));
    }
    // backward, zero carry-in: y_t = g_t + beta_t y_{t+1}, beta_t = -E_t ip_t
    float y = 0.f;
    mu = 1.f;
#pragma unroll
    for (int t = C - 1; t >= 0; --t) {
      if ((t & 7) == 7) asm volatile("" ::: "memory");
      const float be = -peb[t] * pip[kTileCW * t];
      y = fmaf(be, y, rd(t));
      mu *= be;
      wr(t, y);
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
    float yin = __shfl_down_sync(0xffffffffu, A, 1);
    if (lane == 31) yin = 0.f;
    mu = 1.f;
#pragma unroll
    for (int t = C - 1; t >= 0; --t) {
      if ((t & 7) == 7) asm volatile("" ::: "memory");
      mu *= -peb[t] * pip[kTileCW * t];
      pd[kTileCW * t] = fmaf(mu, yin, rd(t));
    }
  }
  __syncthreads();
  // ---- write back (coalesced) ----
  if (a.split != nullptr) {
    // the 8 columns of a row (8 consecutive lanes) become, for the even and
    // for the odd columns, 8 bytes of BF16 high parts and 8 of low parts:
    // every lane splits its value, lanes 0, 1, 4, 5 pair theirs with lane + 2
    // (the next column of the same parity) and store 4 bytes of each
    for (int base = 0; base < nr; base += blockDim.x / kTileCW) {
      const int row = base + threadIdx.x / kTileCW;
#pragma unroll
      for (int j = 0; j < MR; ++j) {
        if (!sel[j]) continue;
        const float v = (row < nr) ? ds[j * kTileWords + tidx(row, cw, C)] : 0.f;
        const float hi = bf16_round(v), lo = v - hi;
        const float hi2 = __shfl_down_sync(0xffffffffu, hi, 2), lo2 = __shfl_down_sync(0xffffffffu, lo, 2);
        if ((cw & 2) == 0 && row < nr) {
          unsigned char *t = a.split + split_byte(m0 + j, row, split_pos(col0 + cw, a.split_kbe), a.split_mtiles,
                                                  a.split_ktiles);
          *reinterpret_cast<unsigned *>(t) = bf16_pack2(hi, hi2);
          *reinterpret_cast<unsigned *>(t + kSplitTileBytes / 2) = bf16_pack2(lo, lo2);
        }
      }
    }
  } else if (cw < ncol) {
    for (int row = threadIdx.x / kTileCW; row < nr; row += blockDim.x / kTileCW) {
      const int si = tidx(row, cw, C);
#pragma unroll
      for (int j = 0; j < MR; ++j)
        if (sel[j]) a.out[(size_t)(m0 + j) * a.field + (size_t)row * pitch + col0 + cw] = ds[j * kTileWords + si];
    }
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

template <int C, int MR>
void launch_tridiag_tile_cm(const TriArgs<float> &a, cudaStream_t s) {
  // mirrors the kernel's layout: (1 + MR) padded tiles and the two E arrays
  const size_t smem = sizeof(float) * ((1 + MR) * (32 * C * kTileCW + 32) + 2 * (32 * C + 32));
  ensure_smem_attr((const void *)tridiag_tile_kernel<C, MR>, smem);
  dim3 grid((a.nz + kTileCW - 1) / kTileCW, (a.m + MR - 1) / MR);
  tridiag_tile_kernel<C, MR><<<grid, 32 * kTileCW * MR, smem, s>>>(a);
}

template <int C>
void launch_tridiag_tile_c(const TriArgs<float> &a, cudaStream_t s) {
  if (a.cstride == 0 && a.estride == 0) launch_tridiag_tile_cm<C, 2>(a, s);
  else launch_tridiag_tile_cm<C, 1>(a, s);
}

// FP32 systems of up to 1024 rows use the tiled kernel (chunks of at most 32
// rows per lane, held in registers); the CTA-chunk kernel takes the rest.
bool launch_tridiag_tile(const TriArgs<float> &a, cudaStream_t s) {
  const int cneed = (a.nr + 31) / 32;
  if (cneed <= 4) launch_tridiag_tile_c<4>(a, s);
  else if (cneed <= 8) launch_tridiag_tile_c<8>(a, s);
  else if (cneed <= 16) launch_tridiag_tile_c<16>(a, s);
  else if (cneed <= 32) launch_tridiag_tile_c<32>(a, s);
  else return false;
  return true;
}

bool tridiag_split_ok(int nr) { return nr <= 32 * 32; }

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
