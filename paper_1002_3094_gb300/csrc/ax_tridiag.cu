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

template <typename T>
void launch_tridiag(const TriArgs<T> &a, cudaStream_t s) {
  note_launch();
  if (a.nr > TriChunk<T>::switch_nr) launch_tridiag_c<T, TriChunk<T>::large>(a, s);
  else launch_tridiag_c<T, TriChunk<T>::small>(a, s);
}

template void launch_tridiag<float>(const TriArgs<float> &, cudaStream_t);
template void launch_tridiag<double>(const TriArgs<double> &, cudaStream_t);

}  // namespace ax
