// Orthonormal sine transform (DST-I) along z of every r-row, the
// Dirichlet-z counterpart of the paper's separation of variables (Section 4.2,
// Eq. fft_phi, computed there with a sequential FFT):
//
//     out[l] = sqrt(2/L) * sum_{k=1}^{L-1} in[k] sin(pi k l / L),   L = nz + 1.
//
// Method: the odd extension x of a row (x_0 = x_L = 0, x_k = in[k],
// x_{2L-k} = -in[k]) has the DFT X_l = -2i sum_k in[k] sin(pi k l / L).  The
// length-2L real sequence is packed into L complex numbers z_j = x_{2j} +
// i x_{2j+1}, transformed by a mixed-radix Stockham FFT of length L in shared
// memory, and split into X_l with the standard real-FFT post-processing; only
// Im X_l is kept.  Radices 2, 3, 4, 5, 8 run as unrolled register butterflies;
// any other odd prime radix R runs as a paired direct DFT (outputs o and R - o
// share the sums and differences of inputs r and R - r), eight output pairs
// per thread.
//
// The zero-flux z boundary (the paper's own) uses the cosine pair of
// Eq. fft_phi instead, in orthonormal form (the paper's forward sum with its
// first mode divided by sqrt 2, and its inverse with the 1/2 weight times
// sqrt 2: B^-1 = C^T T^-1 C is the same operator).  Both go through the same
// complex FFT, now of length L = nz:
//   forward (DCT-II): the even extension y (y_k = y_{2n-1-k} = in[k]) is
//     packed as z_j = y_{2j} + i y_{2j+1}; with Z = FFT(z), E_l, O_l the
//     transforms of the even / odd samples of y, Y_l = E_l + e^{-i 2 phi} O_l
//     and out[l] = s_l Re(e^{-i phi} Y_l) / 2, phi = pi l / (2 n);
//   inverse (DCT-III): the spectrum of that even extension,
//     Y_l = 2 e^{i phi} X_l, is split back into E_l and O_l, packed as
//     Z_l = E_l + i O_l, and z = IDFT(Z) = conj(FFT(conj Z)) / n holds
//     out[2j] = Re z_j, out[2j+1] = Im z_j.
//
// One CTA transforms `rpb` rows of one right-hand side (blockIdx.x = RHS).
// The fused variants update the CG iterate and residual while loading the
// rows (forward) or form the (r, z) partial while storing (inverse).
#pragma once
#include <cmath>
#include "ax_common.cuh"

namespace ax {

namespace {

template <typename T> struct CplxT;
template <> struct CplxT<float> { using type = float2; };
template <> struct CplxT<double> { using type = double2; };

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// a * exp(-i theta) with (c, s) = (cos theta, sin theta)
template <typename C, typename T>
__device__ __forceinline__ C crot(C a, T c, T s) {
  C r;
  r.x = fma(a.x, c, a.y * s);
  r.y = fma(a.y, c, -a.x * s);
  return r;
}
// -i * a
template <typename C>
__device__ __forceinline__ C cmi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

template <typename T, int R> struct Butterfly;

template <typename T> struct Butterfly<T, 2> {
  template <typename C> __device__ __forceinline__ static void run(C *v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename T> struct Butterfly<T, 4> {
  template <typename C> __device__ __forceinline__ static void run(C *v) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = cmi(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <typename T> struct Butterfly<T, 8> {
  template <typename C> __device__ __forceinline__ static void run(C *v) {
    const T h = T(0.70710678118654752440);
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Butterfly<T, 4>::run(e);
    Butterfly<T, 4>::run(o);
    C w1, w2, w3;
    w1.x = (o[1].x + o[1].y) * h; w1.y = (o[1].y - o[1].x) * h;
    w2 = cmi(o[2]);
    w3.x = (o[3].y - o[3].x) * h; w3.y = -(o[3].x + o[3].y) * h;
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], w1);   v[5] = csub(e[1], w1);
    v[2] = cadd(e[2], w2);   v[6] = csub(e[2], w2);
    v[3] = cadd(e[3], w3);   v[7] = csub(e[3], w3);
  }
};

template <typename T> struct Butterfly<T, 3> {
  template <typename C> __device__ __forceinline__ static void run(C *v) {
    const T h = T(0.86602540378443864676);  // sin(2 pi / 3)
    C s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    C m0;
    m0.x = v[0].x - T(0.5) * s.x;
    m0.y = v[0].y - T(0.5) * s.y;
    v[0] = cadd(v[0], s);
    v[1].x = m0.x + h * d.y; v[1].y = m0.y - h * d.x;
    v[2].x = m0.x - h * d.y; v[2].y = m0.y + h * d.x;
  }
};

template <typename T> struct Butterfly<T, 5> {
  template <typename C> __device__ __forceinline__ static void run(C *v) {
    const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);  // cos 2pi/5, cos 4pi/5
    const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);   // sin 2pi/5, sin 4pi/5
    C s_1 = cadd(v[1], v[4]), d_1 = csub(v[1], v[4]);
    C s_2 = cadd(v[2], v[3]), d_2 = csub(v[2], v[3]);
    C x0 = v[0];
    C a1, b1, a2, b2;
    a1.x = x0.x + c1 * s_1.x + c2 * s_2.x;  a1.y = x0.y + c1 * s_1.y + c2 * s_2.y;
    b1.x = s1 * d_1.x + s2 * d_2.x;         b1.y = s1 * d_1.y + s2 * d_2.y;
    a2.x = x0.x + c2 * s_1.x + c1 * s_2.x;  a2.y = x0.y + c2 * s_1.y + c1 * s_2.y;
    b2.x = s2 * d_1.x - s1 * d_2.x;         b2.y = s2 * d_1.y - s1 * d_2.y;
    v[0] = cadd(x0, cadd(s_1, s_2));
    v[1].x = a1.x + b1.y; v[1].y = a1.y - b1.x;
    v[4].x = a1.x - b1.y; v[4].y = a1.y + b1.x;
    v[2].x = a2.x + b2.y; v[2].y = a2.y - b2.x;
    v[3].x = a2.x - b2.y; v[3].y = a2.y + b2.x;
  }
};

// cos / sin(2 pi j / R), j < R, for the prime radices whose paired DFT is
// fully unrolled (every coefficient then becomes a constant-bank operand).
// Filled once per device by dst_prepare_device().
constexpr int kUnrolledPrimes[] = {7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47};
constexpr int kNumUnrolled = 12;
constexpr int prime_offset(int R) {
  int off = 0;
  for (int i = 0; i < kNumUnrolled; ++i) {
    if (kUnrolledPrimes[i] == R) return off;
    off += 2 * kUnrolledPrimes[i];
  }
  return -1;
}
constexpr int kPrimeTable = prime_offset(47) + 2 * 47;
__constant__ float c_prime_f[kPrimeTable];
__constant__ double c_prime_d[kPrimeTable];

template <typename T> __device__ __forceinline__ T prime_coef(int i);
template <> __device__ __forceinline__ float prime_coef<float>(int i) { return c_prime_f[i]; }
template <> __device__ __forceinline__ double prime_coef<double>(int i) { return c_prime_d[i]; }

// One block of G output pairs (o = 1 + B G ...) of the paired radix-R DFT of
// the R inputs col[r Tn]; B = 0 also produces the DC output.
template <typename T, int R, int G, int B, typename C>
__device__ __forceinline__ void prime_item(const C *__restrict__ col, int Tn, C *__restrict__ out, int Ns) {
  constexpr int H = (R - 1) / 2;
  constexpr int OFF = prime_offset(R);
  constexpr int O0 = 1 + B * G;
  constexpr int GN = (O0 + G - 1 <= H) ? G : (H - O0 + 1);
  const C t0 = col[0];
  C A[G], Bq[G];
#pragma unroll
  for (int g = 0; g < G; ++g) A[g].x = A[g].y = Bq[g].x = Bq[g].y = T(0);
  C dc;
  dc.x = dc.y = T(0);
#pragma unroll
  for (int r = 1; r <= H; ++r) {
    // Keeps the compiler from hoisting all R loads ahead of the sums (which
    // would hold every input in registers at once).
    asm volatile("" ::: "memory");
    const C tr = col[r * Tn], tm = col[(R - r) * Tn];
    const C s = cadd(tr, tm), d = csub(tr, tm);
    if (B == 0) dc = cadd(dc, s);
#pragma unroll
    for (int g = 0; g < GN; ++g) {
      const int idx = (r * (O0 + g)) % R;
      const T c = prime_coef<T>(OFF + 2 * idx), sn = prime_coef<T>(OFF + 2 * idx + 1);
      A[g].x = fma(s.x, c, A[g].x);
      A[g].y = fma(s.y, c, A[g].y);
      Bq[g].x = fma(d.x, sn, Bq[g].x);
      Bq[g].y = fma(d.y, sn, Bq[g].y);
    }
  }
  if (B == 0) out[0] = cadd(t0, dc);
#pragma unroll
  for (int g = 0; g < GN; ++g) {
    const int o = O0 + g;
    C xo, xm;
    xo.x = t0.x + A[g].x + Bq[g].y; xo.y = t0.y + A[g].y - Bq[g].x;
    xm.x = t0.x + A[g].x - Bq[g].y; xm.y = t0.y + A[g].y + Bq[g].x;
    out[o * Ns] = xo;
    out[(R - o) * Ns] = xm;
  }
}

template <typename T, typename C>
__device__ __forceinline__ void twiddle_in_place(C *__restrict__ src, int nrows, int L, int Ns, int R,
                                                 const FastDiv &tn, const FastDiv &nsd, const T *__restrict__ TW) {
  const int tstep = L / (Ns * R);
  for (int rr = 0; rr < nrows; ++rr) {
    C *row = src + rr * L;
    for (int idx = threadIdx.x; idx < L; idx += blockDim.x) {
      const int r = fdiv(idx, tn);
      const int j = idx - r * tn.d;
      if (r > 0) {
        const int k = j - fdiv(j, nsd) * Ns;
        const int ti = (int)(((long long)k * r * tstep) % L);
        row[idx] = crot(row[idx], __ldg(TW + 2 * ti), __ldg(TW + 2 * ti + 1));
      }
    }
  }
  __syncthreads();
}

// Stage with an unrolled prime radix R (FP32 only: in FP64 the DFMA rate, not
// the coefficient loads, bounds the stage, and the unrolled form spills).
template <typename T, int R, typename C>
__device__ __forceinline__ void prime_stage(C *__restrict__ src, C *__restrict__ dst, int nrows, int L, int Ns,
                                            const FastDiv &tn, const FastDiv &nsd, const T *__restrict__ TW) {
  constexpr int H = (R - 1) / 2;
  constexpr int G = H < 10 ? H : 10;
  constexpr int NB = (H + G - 1) / G;
  static_assert(NB <= 6, "prime radix too large for the unrolled stage");
  const int Tn = tn.d;
  if (Ns > 1) twiddle_in_place<T>(src, nrows, L, Ns, R, tn, nsd, TW);
  // Items are grouped by output block b, each group padded to whole warps,
  // so that b (the unrolled code path) is the same across a warp.
  const int per_b = nrows * Tn;
  const int per_b_pad = (per_b + 31) & ~31;
  {
    for (int item = threadIdx.x; item < NB * per_b_pad; item += blockDim.x) {
      int b = 0, w = item;
      while (w >= per_b_pad) {
        w -= per_b_pad;
        ++b;
      }
      if (w >= per_b) continue;
      const int rr = fdiv(w, tn);
      const int j = w - rr * Tn;
      const int q = fdiv(j, nsd);
      const C *col = src + rr * L + j;
      C *out = dst + rr * L + q * Ns * R + (j - q * Ns);
      switch (b) {
        case 0: prime_item<T, R, G, 0>(col, Tn, out, Ns); break;
        case 1: if (NB > 1) prime_item<T, R, G, (NB > 1 ? 1 : 0)>(col, Tn, out, Ns); break;
        case 2: if (NB > 2) prime_item<T, R, G, (NB > 2 ? 2 : 0)>(col, Tn, out, Ns); break;
        case 3: if (NB > 3) prime_item<T, R, G, (NB > 3 ? 3 : 0)>(col, Tn, out, Ns); break;
        case 4: if (NB > 4) prime_item<T, R, G, (NB > 4 ? 4 : 0)>(col, Tn, out, Ns); break;
        default: if (NB > 5) prime_item<T, R, G, (NB > 5 ? 5 : 0)>(col, Tn, out, Ns); break;
      }
    }
  }
}

// One Stockham stage with a small radix: butterfly j of row rr reads
// src[j + r T] (T = L / R), applies the twiddles exp(-2 pi i k r / (Ns R)),
// k = j mod Ns, and writes dst[(j / Ns) Ns R + k + o Ns].
template <typename T, int R, typename C>
__device__ __forceinline__ void small_stage(const C *__restrict__ src, C *__restrict__ dst, int nrows, int L,
                                            int Ns, const FastDiv &tn, const FastDiv &nsd,
                                            const T *__restrict__ TW) {
  const int Tn = tn.d;
  const int tstep = L / (Ns * R);
  {
    for (int item = threadIdx.x; item < nrows * Tn; item += blockDim.x) {
      const int rr = fdiv(item, tn);
      const int j = item - rr * Tn;
      const int q = fdiv(j, nsd);
      const int k = j - q * Ns;
      const C *s = src + rr * L + j;
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = s[r * Tn];
      if (Ns > 1) {
        // w = exp(-2 pi i k / (Ns R)); the r-th twiddle is w^r, formed by
        // repeated complex multiplication (a few roundings, no further lookups).
        const int idx = k * tstep;  // < L
        const T c1 = __ldg(TW + 2 * idx), s1 = __ldg(TW + 2 * idx + 1);
        T cr = c1, sr = s1;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          v[r] = crot(v[r], cr, sr);
          const T cn = cr * c1 - sr * s1;
          sr = fma(sr, c1, cr * s1);
          cr = cn;
        }
      }
      Butterfly<T, R>::run(v);
      C *d = dst + rr * L + q * Ns * R + k;
#pragma unroll
      for (int o = 0; o < R; ++o) d[o * Ns] = v[o];
    }
  }
}

// Generic odd radix R (prime > 5): paired direct DFT.  Twiddles are applied in
// place first (skipped on the first stage, where Ns = 1).
template <typename T, typename C>
__device__ __forceinline__ void generic_stage(C *__restrict__ src, C *__restrict__ dst, int nrows, int L,
                                              int Ns, int R, const FastDiv &tn, const FastDiv &nsd,
                                              const T *__restrict__ TW) {
  constexpr int G = 8;  // output pairs per thread
  const int Tn = tn.d;
  if (Ns > 1) twiddle_in_place<T>(src, nrows, L, Ns, R, tn, nsd, TW);
  const int H = (R - 1) / 2;
  const int NB = (H + G - 1) / G;
  const int cstep = L / R;
  // FP32: output blocks b grouped and warp-aligned, as in prime_stage.  FP64
  // keeps the row-major item order, which needs fewer registers there (the
  // warp-aligned form spills in the FP64 kernels).
  constexpr bool kAligned = sizeof(T) == 4;
  const int per_b = nrows * Tn;
  const int per_b_pad = kAligned ? ((per_b + 31) & ~31) : per_b;
  const FastDiv nid = make_fastdiv_dev(NB * Tn);  // items per row (row-major order)
  {
    for (int item = threadIdx.x; item < NB * per_b_pad; item += blockDim.x) {
      int b, rr, j;
      if (kAligned) {
        int w = item;
        b = 0;
        while (w >= per_b_pad) {
          w -= per_b_pad;
          ++b;
        }
        if (w >= per_b) continue;
        rr = fdiv(w, tn);
        j = w - rr * Tn;
      } else {
        rr = fdiv(item, nid);
        const int it = item - rr * NB * Tn;
        b = fdiv(it, tn);
        j = it - b * Tn;
      }
      const int q = fdiv(j, nsd);
      const C *col = src + rr * L + j;
      const C t0 = col[0];
      C A[G], B[G];
      int idx[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        A[g].x = A[g].y = B[g].x = B[g].y = T(0);
        idx[g] = 0;
      }
      C dc;
      dc.x = dc.y = T(0);
      const int o0 = 1 + b * G;
      for (int r = 1; r <= H; ++r) {
        const C tr = col[r * Tn], tm = col[(R - r) * Tn];
        const C s = cadd(tr, tm), d = csub(tr, tm);
        dc = cadd(dc, s);
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int o = o0 + g;
          int v = idx[g] + o;
          v = (v >= R) ? v - R : v;
          idx[g] = v;
          const T c = __ldg(TW + 2 * v * cstep), sn = __ldg(TW + 2 * v * cstep + 1);
          A[g].x = fma(s.x, c, A[g].x);
          A[g].y = fma(s.y, c, A[g].y);
          B[g].x = fma(d.x, sn, B[g].x);
          B[g].y = fma(d.y, sn, B[g].y);
        }
      }
      C *out = dst + rr * L + q * Ns * R + (j - q * Ns);
      if (b == 0) out[0] = cadd(t0, dc);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int o = o0 + g;
        if (o <= H) {
          C xo, xm;
          xo.x = t0.x + A[g].x + B[g].y; xo.y = t0.y + A[g].y - B[g].x;
          xm.x = t0.x + A[g].x - B[g].y; xm.y = t0.y + A[g].y + B[g].x;
          out[o * Ns] = xo;
          out[(R - o) * Ns] = xm;
        }
      }
    }
  }
}

// First stage by Rader's algorithm (prime R, Ns = 1): for every butterfly j
// the inputs a_p = x_{g^p} (p < P = R - 1) are transformed, multiplied by the
// spectrum of the permuted kernel c'_m = W^(g^-m), and transformed again
// (inverse via conjugation), which gives X_{g^-q} = x_0 + (a * c')_q; X_0 =
// x_0 + sum a.  The P-point transforms reuse the small-radix Stockham stages
// on sub-rows of length P laid out in the two shared buffers.  x0s holds 2
// values per butterfly (x_0 and X_0).
template <typename T, typename C>
__device__ __forceinline__ void rader_stage(C *__restrict__ src, C *__restrict__ dst, C *__restrict__ x0s, int nrows,
                                            int L, int R, const FftPlan &pl, const T *__restrict__ RK,
                                            const T *__restrict__ RT, const int *__restrict__ RP) {
  const int P = R - 1;
  const FastDiv &tn = pl.tn_div[0];
  const int Tn = tn.d;
  const int nsub = nrows * Tn;
  for (int item = threadIdx.x; item < nsub * P; item += blockDim.x) {
    const int sub = fdiv(item, pl.p_div);
    const int p = item - sub * P;
    const int rr = fdiv(sub, tn);
    const int j = sub - rr * Tn;
    dst[item] = src[rr * L + j + __ldg(RP + p) * Tn];
  }
  for (int sub = threadIdx.x; sub < nsub; sub += blockDim.x) {
    const int rr = fdiv(sub, tn);
    x0s[sub] = src[rr * L + (sub - rr * Tn)];
  }
  __syncthreads();
  C *a = dst, *b = src;
  for (int pass = 0; pass < 2; ++pass) {
    int ns = 1;
    for (int k = 0; k < pl.sub_n; ++k) {
      const int Rk = pl.sub_radix[k];
      switch (Rk) {
        case 2: small_stage<T, 2>(a, b, nsub, P, ns, pl.sub_tn[k], pl.sub_ns[k], RT); break;
        case 3: small_stage<T, 3>(a, b, nsub, P, ns, pl.sub_tn[k], pl.sub_ns[k], RT); break;
        case 4: small_stage<T, 4>(a, b, nsub, P, ns, pl.sub_tn[k], pl.sub_ns[k], RT); break;
        case 5: small_stage<T, 5>(a, b, nsub, P, ns, pl.sub_tn[k], pl.sub_ns[k], RT); break;
        default: small_stage<T, 8>(a, b, nsub, P, ns, pl.sub_tn[k], pl.sub_ns[k], RT); break;
      }
      C *t = a; a = b; b = t;
      ns *= Rk;
      __syncthreads();
    }
    if (pass == 0) {
      // Z = conj(A * C'); X_0 = x_0 + A_0
      for (int item = threadIdx.x; item < nsub * P; item += blockDim.x) {
        const int sub = fdiv(item, pl.p_div);
        const int k = item - sub * P;
        const C v = a[item];
        const T cr = __ldg(RK + 2 * k), ci = __ldg(RK + 2 * k + 1);
        C z;
        z.x = v.x * cr - v.y * ci;
        z.y = -(v.x * ci + v.y * cr);
        b[item] = z;
        if (k == 0) {
          C x0 = x0s[sub];
          x0.x += v.x;
          x0.y += v.y;
          x0s[nsub + sub] = x0;
        }
      }
      C *t = a; a = b; b = t;
      __syncthreads();
    }
  }
  // a == src here (an odd number of buffer moves): scatter into the stage output
  const T inv = T(1) / T(P);
  for (int item = threadIdx.x; item < nsub * P; item += blockDim.x) {
    const int sub = fdiv(item, pl.p_div);
    const int q = item - sub * P;
    const int rr = fdiv(sub, tn);
    const int j = sub - rr * Tn;
    const C v = a[item];
    const C x0 = x0s[sub];
    C o;
    o.x = x0.x + v.x * inv;
    o.y = x0.y - v.y * inv;
    dst[rr * L + j * R + __ldg(RP + P + q)] = o;
  }
  for (int sub = threadIdx.x; sub < nsub; sub += blockDim.x) {
    const int rr = fdiv(sub, tn);
    dst[rr * L + (sub - rr * Tn) * R] = x0s[nsub + sub];
  }
}

template <typename T> struct DstOcc;
template <> struct DstOcc<float> { static constexpr int min_blocks = 3; };
template <> struct DstOcc<double> { static constexpr int min_blocks = 2; };

template <typename T, int MODE>
__global__ void __launch_bounds__(256, DstOcc<T>::min_blocks) dst_kernel(const DstArgs<T> a) {
  using C = typename CplxT<T>::type;
  constexpr int V = VecT<T>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8];
  const int m = blockIdx.x;
  if (!rhs_selected(a.st, a.mask, m)) return;
  const int L = a.plan.L, n = a.n;
  const int LB = dst_buffer_len(L, n);
  const bool cosine = a.cosine != 0;
  const bool inv = cosine && (a.inverse != 0 || MODE == kDstPcgInverse || MODE == kDstChebInverse);
  const int row0 = blockIdx.y * a.rpb;
  const int nrows = min(a.rpb, a.rows - row0);
  C *buf0 = reinterpret_cast<C *>(smem_raw);
  C *buf1 = buf0 + ((a.rpb * LB + 1) & ~1);  // 16-byte aligned (vector staging stores)
  C *x0s = buf1 + a.rpb * LB;                 // Rader: 2 values per first-stage butterfly
  T *pk = reinterpret_cast<T *>(buf0);  // packed real view: pk[rr * 2L + idx] = x_idx
  const size_t base = (size_t)m * (size_t)a.field + (size_t)row0 * a.pitch;
  T alpha = T(0);
  const T *__restrict__ p = nullptr;
  if (MODE == kDstPcgForward) {
    alpha = (T)a.st[m].alpha;
    p = (a.st[m].iters & 1) ? a.pa : a.pb;
  }
  T acc = T(0);

  // ---- load rows: short vectors from global memory into a plain staging
  // copy of the rows (aligned vector stores into the second buffer), then the
  // packed odd extension is built from it with unit-stride accesses.
  // Padding columns beyond n hold zeros in every field and stay zero. ----
  T *__restrict__ xg = a.x;
  T *__restrict__ rg = a.r;
  const T *__restrict__ ing = a.in;
  const int spitch = (n + 3) & ~3;  // staging row length (16-byte aligned rows)
  T *stg = reinterpret_cast<T *>(buf1);
  for (int rr = 0; rr < nrows; ++rr) {
    const size_t rb = base + (size_t)rr * a.pitch;
    for (int k0 = threadIdx.x * V; k0 < n; k0 += blockDim.x * V) {
      const size_t e = rb + k0;
      T v[V];
      if (MODE == kDstPcgForward) {
        T xv[V], pv[V], rv[V], qv[V];
        load_vec<T>(xg + e, xv);
        load_vec<T>(p + e, pv);
        load_vec<T>(rg + e, rv);
        load_vec<T>(ing + e, qv);
#pragma unroll
        for (int t = 0; t < V; ++t) {
          xv[t] = fma(alpha, pv[t], xv[t]);
          rv[t] = fma(-alpha, qv[t], rv[t]);
          acc = fma(rv[t], rv[t], acc);
          v[t] = rv[t];
        }
        store_vec<T>(xg + e, xv);
        store_vec<T>(rg + e, rv);
      } else {
        load_vec<T>(ing + e, v);
      }
      store_vec<T>(stg + rr * spitch + k0, v);
    }
  }
  __syncthreads();
  for (int rr = 0; rr < nrows; ++rr) {
    T *px = pk + rr * 2 * L;
    const T *sr = stg + rr * spitch;
    if (!cosine) {  // odd extension of length 2L
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const T v = sr[k];
        px[k + 1] = v;
        px[2 * L - k - 1] = -v;
      }
      if (threadIdx.x == 0) {
        px[0] = T(0);
        px[L] = T(0);
      }
    } else if (!inv) {  // even extension of length 2n (L = n)
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const T v = sr[k];
        px[k] = v;
        px[2 * L - k - 1] = v;
      }
    } else {  // conj(Z_l), Z_l = E_l + i O_l from X_l and X_{n-l} (X_n = 0)
      C *zr = buf0 + rr * L;
      for (int l = threadIdx.x; l < n; l += blockDim.x) {
        const T xl = sr[l], xm = l ? sr[n - l] : T(0);
        const T c = __ldg(a.CW + 8 * l + 4), sn = __ldg(a.CW + 8 * l + 5);
        const T c2 = __ldg(a.CW + 8 * l + 6), s2 = __ldg(a.CW + 8 * l + 7);
        const T ex = fma(xl, c, xm * sn), ey = fma(xl, sn, -xm * c);
        const T dx = fma(xl, c, -xm * sn), dy = fma(xl, sn, xm * c);
        const T ox = fma(dx, c2, -dy * s2), oy = fma(dx, s2, dy * c2);
        C zc;
        zc.x = ex - oy;
        zc.y = -(ey + ox);
        zr[l] = zc;
      }
    }
  }

  // ---- complex FFT of length L (Stockham, ping-pong) ----
  C *src = buf0, *dst = buf1;
  int Ns = 1;
  for (int s = 0; s < a.plan.nstages; ++s) {
    const int R = a.plan.radix[s];
    const FastDiv tn = a.plan.tn_div[s], nsd = a.plan.ns_div[s];
    __syncthreads();
    if (s == 0 && a.plan.rader) {
      rader_stage<T>(src, dst, x0s, nrows, L, R, a.plan, a.RK, a.RT, a.RP);
      C *t = src; src = dst; dst = t;
      Ns *= R;
      continue;
    }
    switch (R) {
      case 2: small_stage<T, 2>(src, dst, nrows, L, Ns, tn, nsd, a.TW); break;
      case 3: small_stage<T, 3>(src, dst, nrows, L, Ns, tn, nsd, a.TW); break;
      case 4: small_stage<T, 4>(src, dst, nrows, L, Ns, tn, nsd, a.TW); break;
      case 5: small_stage<T, 5>(src, dst, nrows, L, Ns, tn, nsd, a.TW); break;
      case 8: small_stage<T, 8>(src, dst, nrows, L, Ns, tn, nsd, a.TW); break;
      case 7: if (sizeof(T) == 4) prime_stage<T, 7>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 11: if (sizeof(T) == 4) prime_stage<T, 11>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 13: if (sizeof(T) == 4) prime_stage<T, 13>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 17: if (sizeof(T) == 4) prime_stage<T, 17>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 19: if (sizeof(T) == 4) prime_stage<T, 19>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 23: if (sizeof(T) == 4) prime_stage<T, 23>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 29: if (sizeof(T) == 4) prime_stage<T, 29>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 31: if (sizeof(T) == 4) prime_stage<T, 31>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 37: if (sizeof(T) == 4) prime_stage<T, 37>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 41: if (sizeof(T) == 4) prime_stage<T, 41>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 43: if (sizeof(T) == 4) prime_stage<T, 43>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      case 47: if (sizeof(T) == 4) prime_stage<T, 47>(src, dst, nrows, L, Ns, tn, nsd, a.TW); else generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
      default: generic_stage<T>(src, dst, nrows, L, Ns, R, tn, nsd, a.TW); break;
    }
    C *t = src; src = dst; dst = t;
    Ns *= R;
  }
  __syncthreads();

  // ---- split into the sine coefficients and store.  Consecutive threads take
  // consecutive k, so the reads of Z[k] and Z[L - k] are free of bank
  // conflicts and every global access of a warp is one contiguous segment;
  // the half-angle pair is read once per column for all rows.  Padding
  // columns are not written (they hold zeros and stay zero). ----
  const T sc = (T)a.scale;
  T *__restrict__ outg = a.out;
  T cheb_a = T(0), tau = T(0);
  if (MODE == kDstChebInverse) {
    cheb_a = (T)a.st[m].cheb_a;
    tau = (T)a.chp[2 * m];
  }
  for (int o = threadIdx.x; o < n; o += blockDim.x) {
    // per-column factors: sine (c, sn) = half-angle pair of k = o + 1; cosine
    // forward: the four scaled factors of mode o
    T c = T(0), sn = T(0), f2 = T(0), f3 = T(0);
    if (!cosine) {
      c = __ldg(a.HW + 2 * (o + 1));
      sn = __ldg(a.HW + 2 * (o + 1) + 1);
    } else if (!inv) {
      c = __ldg(a.CW + 8 * o);
      sn = __ldg(a.CW + 8 * o + 1);
      f2 = __ldg(a.CW + 8 * o + 2);
      f3 = __ldg(a.CW + 8 * o + 3);
    }
    for (int rr = 0; rr < nrows; ++rr) {
      const C *Z = src + rr * L;
      T v;
      if (!cosine) {
        const C zk = Z[o + 1], zm = Z[L - o - 1];
        v = ((zm.y - zk.y) + c * (zk.x - zm.x) + sn * (zk.y + zm.y)) * sc;
      } else if (!inv) {
        const C zl = Z[o], zm = Z[o ? n - o : 0];
        v = (zl.x + zm.x) * c + (zl.y - zm.y) * sn + (zl.y + zm.y) * f2 - (zl.x - zm.x) * f3;
      } else {
        const C w = Z[o >> 1];
        v = ((o & 1) ? -w.y : w.x) * sc;
      }
      const size_t e = base + (size_t)rr * a.pitch + o;
      if (MODE == kDstPlain || MODE == kDstPcgForward) {
        outg[e] = v;
      } else if (MODE == kDstPcgInverse) {
        const T rv = a.r[e];
        outg[e] = v;
        acc = fma(rv, v, acc);
      } else {  // Chebyshev: y_{k+1} = a (y_k - tau B^-1 res) + (1 - a) y_{k-1}
        const T yb = fma(-tau, v, a.y[e]);
        const T pv = a.yprev[e];
        a.yprev[e] = fma(cheb_a, yb - pv, pv);
      }
    }
  }
  if (MODE == kDstPcgForward || MODE == kDstPcgInverse) {
    const double s = block_sum((double)acc, red);
    if (threadIdx.x == 0) a.partial[(size_t)m * kPartialStride + blockIdx.y] = s;
  }
}

constexpr size_t kDstSmemBudget = 67584;

}  // namespace

}  // namespace ax
