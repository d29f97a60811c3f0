// Persistent FP64 PCG for one right-hand side on a small grid (Section 2.2,
// Eq. main-scheme: textbook PCG; the preconditioner of Section 4.2,
// B^-1 = F^T T^-1 F with the orthonormal z-transform F and the per-mode
// tridiagonal systems T_l of Eq. eq_trid).
//
// At 64 x 64 an iteration is a few hundred thousand FP64 operations, and the
// graph-replayed path spends most of its time between its ~20 launches per
// iteration.  Here the whole solve is one cooperative launch: the CTAs run the
// iteration's phases back to back and meet at grid barriers (a counter and a
// generation word in global memory).  Every wait is bounded: on expiry a CTA
// sets *err and leaves, the others then run out their own waits, and the call
// reports AX_ERR_TIMEOUT.  An iteration has four barriers:
//   1. p = z + beta p_old and q = A p at every node (the neighbours' p formed
//      on the fly from z and p_old; p is double-buffered), (p, q) partials;
//   2. alpha = rho / (p, q); per row r_new = r - alpha q, x += alpha p,
//      ||r_new||^2, and the forward transform of the row, rhat = F r_new
//      (dense FP64: one dot product of length nz per output; a row's outputs
//      may be split over several CTAs, each forming r_new itself; r is
//      double-buffered so that they all read the old one);
//   3. the mode solves T_l yhat = rhat, one warp per mode column: Thomas with
//      the precomputed factors (g_i = b_i IP_i - E_{i-1} IP_i g_{i-1},
//      y_i = g_i - E_i IP_i y_{i+1}), each lane a chunk of rows run with zero
//      carry-in, the chunks' affine carry maps composed by warp shuffles, then
//      the true carries applied (the dichotomy observation of Section 3: with
//      a fixed matrix the chunk-boundary unknowns follow from precomputable
//      linear combinations);
//   4. z = F^T yhat per row and the (r, z) partials; beta = (r, z) / rho.
// Every CTA sums the partial sums in one fixed order, so all CTAs take the same
// decisions (stop, breakdown) without a broadcast.  The stop rule is the FP64
// path's: when the recursive residual passes, the true residual phi - A x is
// formed and tested, and replaces r when it fails.  Data written during the
// launch are read with ld.global.cg (L2), never from a stale L1 line.
#include <cmath>
#include <mutex>
#include <vector>
#include "ax_common.cuh"

namespace ax {

namespace {

constexpr int kSmallThreads = 256;
constexpr unsigned kSmallPolls = 1u << 24;  // spins of an L2 load each: a second or so
constexpr int kPartPQ = 0, kPartRR = 1, kPartRZ = 2;
constexpr size_t kSmallSmem = 100 * 1024;  // bound of the shared-memory copy of the transform rows

// Grid barrier with a bounded wait; false on every thread of the CTA when the
// wait expired (or, with skip, when the CTA left without arriving).  bar[0]
// counts arrivals over the whole launch: a CTA adds 1 (a release reduction,
// no round trip) and waits until the count reaches G times the number of
// barriers it has passed (acquire loads; unsigned differences, so the count
// may wrap).
__device__ bool grid_sync(unsigned *bar, unsigned G, unsigned &gen, unsigned polls, int *err, bool skip) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = G * (gen + 1);
    if (skip) {
      ok = 0;
    } else {
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
      unsigned i = 0;
      for (;;) {
        unsigned c;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(bar) : "memory");
        if ((int)(c - target) >= 0) break;
        if (++i >= polls) {
          ok = 0;
          break;
        }
      }
    }
    if (!ok) atomicExch(err, 1);
    gen += 1;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Thomas on mode column l of a.t (in place), one warp: lane L owns rows
// L C .. L C + C - 1.  Forward g_i = b_i IP_i + al_i g_{i-1}, al_i =
// -E_{i-1} IP_i, and backward y_i = g_i + be_i y_{i+1}, be_i = -E_i IP_i, each
// run per chunk with zero carry-in; the chunks' affine carry maps
// (out = A + M in) are composed over the lanes by shuffles and the true
// carries applied.  C is a template parameter so that no FP64 operation is
// issued for rows a lane does not own (GB300's FP64 pipe is narrow).
template <int C>
__device__ __forceinline__ void thomas_warp(const SmallPcgArgs &a, int l, int lane) {
  const int nr = a.nr, P = a.pitch, i0 = lane * C;
  double v[C], al[C], be[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int i = i0 + j;
    v[j] = 0.0;
    al[j] = 0.0;
    be[j] = 0.0;
    if (i < nr) {
      const double ip = __ldg(a.IP + (size_t)i * P + l);
      al[j] = i > 0 ? -__ldg(a.E + i - 1) * ip : 0.0;
      be[j] = -__ldg(a.E + i) * ip;
      v[j] = __ldcg(a.t + (size_t)i * P + l) * ip;
    }
  }
  double g = 0.0, mu = 1.0;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    g = fma(al[j], g, v[j]);
    mu *= al[j];
    v[j] = g;
  }
  double A = g, M = mu;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double Ap = __shfl_up_sync(0xffffffffu, A, off), Mp = __shfl_up_sync(0xffffffffu, M, off);
    if (lane >= off) {
      A = fma(M, Ap, A);
      M *= Mp;
    }
  }
  double d = __shfl_up_sync(0xffffffffu, A, 1);
  if (lane == 0) d = 0.0;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    d *= al[j];
    v[j] += d;
  }
  double y = 0.0, nu = 1.0;
#pragma unroll
  for (int j = C - 1; j >= 0; --j) {
    y = fma(be[j], y, v[j]);
    nu *= be[j];
    v[j] = y;
  }
  A = y;
  M = nu;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double An = __shfl_down_sync(0xffffffffu, A, off), Mn = __shfl_down_sync(0xffffffffu, M, off);
    if (lane + off < 32) {
      A = fma(M, An, A);
      M *= Mn;
    }
  }
  double e = __shfl_down_sync(0xffffffffu, A, 1);
  if (lane == 31) e = 0.0;
#pragma unroll
  for (int j = C - 1; j >= 0; --j) {
    e *= be[j];
    const int i = i0 + j;
    if (i < nr) a.t[(size_t)i * P + l] = v[j] + e;
  }
}

__global__ void __launch_bounds__(kSmallThreads) pcg_small_kernel(const SmallPcgArgs a) {
  __shared__ double red[kSmallThreads / 32];
  __shared__ double row[kSmallMaxNz];
  extern __shared__ double msm[];  // a.msm: this CTA's rows of F and F^T, row stride nz + 1
  __shared__ double bc;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nr = a.nr, nz = a.nz, P = a.pitch, PZ = a.pitchz;
  const unsigned polls = a.polls ? a.polls : kSmallPolls;
  unsigned gen = 0;
  bool stall = a.stall != 0 && b == 0;
  RhsState s = *a.st;  // the same state in every thread (overwritten below with a.f)
  if (a.f == nullptr && s.state != kActive) return;

  auto sync = [&]() {
    const bool ok = grid_sync(a.bar, (unsigned)G, gen, polls, a.err, stall);
    stall = false;
    return ok;
  };
  // CTA partial of `kind` (thread 0 writes it)
  auto put = [&](int kind, double v) {
    const double sm = block_sum(v, red);
    if (tid == 0) a.part[kind * G + b] = sm;
  };
  // the sum of the G partials of `kind`, in one fixed order, on every thread
  auto total = [&](int kind) {
    __syncthreads();
    if (warp == 0) {
      // G <= 256: up to 8 loads per lane, all issued before the sum
      double t[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) t[j] = lane + 32 * j < G ? __ldcg(a.part + kind * G + lane + 32 * j) : 0.0;
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < 8; ++j) v += t[j];
      v = warp_sum(v);
      if (lane == 0) bc = v;
    }
    __syncthreads();
    return bc;
  };

  // Every CTA transforms one output chunk c (see small_pcg_grid): with a.msm
  // its rows of F and F^T are read once into shared memory.
  const int CHs = (nz + a.nch - 1) / a.nch, c_own = b % a.nch;
  if (a.msm) {
    const int o0 = c_own * CHs, rows_m = min(CHs, nz - o0);
    for (int e = tid; e < rows_m * nz; e += kSmallThreads) {
      const int o = e / nz, k = e % nz;
      msm[o * (nz + 1) + k] = __ldg(a.F + (size_t)(o0 + o) * nz + k);
      msm[(CHs + o) * (nz + 1) + k] = __ldg(a.Ft + (size_t)(o0 + o) * nz + k);
    }
    __syncthreads();
  }

  // r is double-buffered: rbuf[rsel] is the current residual
  double *rbuf[2] = {a.r, a.r2};
  int rsel = 0;

  // ---- dense transforms over items (row i, output chunk c)
  // mode 0: row = r - alpha q (r_new; chunk 0 writes r_new and x += alpha p
  //         and adds ||r_new||^2), out t = F row;
  // mode 1: row = r, out t = F row;
  // mode 2: row = t, out z = F^T row, adds (r, z).
  auto transform = [&](int mode, double alpha, const double *pcur, double &acc) {
    const int nch = a.nch, CH = (nz + nch - 1) / nch;
    const double *M = mode == 2 ? a.Ft : a.F;
    const double *rcur = rbuf[rsel];  // the current residual (mode 0: before the update)
    double *rnew = rbuf[rsel ^ 1];
    for (int item = b; item < nr * nch; item += G) {
      const int i = item / nch, c = item % nch;
      const size_t ro = (size_t)i * P;
      __syncthreads();  // the previous item's outputs have read `row`
      for (int k = tid; k < nz; k += blockDim.x) {
        double v;
        if (mode == 0) {
          v = fma(-alpha, __ldcg(a.q + ro + k), __ldcg(rcur + ro + k));
          if (c == 0) {
            rnew[ro + k] = v;
            a.x[ro + k] = fma(alpha, __ldcg(pcur + ro + k), __ldcg(a.x + ro + k));
            acc = fma(v, v, acc);
          }
        } else if (mode == 1) {
          v = __ldcg(rcur + ro + k);
        } else {
          v = __ldcg(a.t + ro + k);
        }
        row[k] = v;
      }
      __syncthreads();
      const int o0 = c * CH, o1 = min(o0 + CH, nz);
      const int grp = tid >> 3, sub = tid & 7;
      for (int ob = o0; ob < o1; ob += kSmallThreads / 8) {
        const int o = ob + grp;
        const bool valid = o < o1;
        double v = 0.0;
        if (valid) {
          if (a.msm) {
            const double *mr = msm + (size_t)((mode == 2 ? CHs : 0) + (o - o0)) * (nz + 1);
            for (int k = sub; k < nz; k += 8) v = fma(mr[k], row[k], v);
          } else {
            for (int k = sub; k < nz; k += 8) v = fma(__ldg(M + (size_t)o * nz + k), row[k], v);
          }
        }
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        if (valid && sub == 0) {
          if (mode == 2) {
            a.z[ro + o] = v;
            acc = fma(__ldcg(rcur + ro + o), v, acc);
          } else {
            a.t[ro + o] = v;
          }
        }
      }
    }
  };

  // ---- mode solves on t, one warp per mode column (columns spread over the
  // CTAs first: GB300's FP64 pipe is narrow, so one SM should not take many)
  auto mode_solves = [&]() {
    const int C = (nr + 31) / 32;
    const int nw = G * (kSmallThreads / 32);
    for (int l = warp * G + b; l < nz; l += nw) {
      if (C <= 1) thomas_warp<1>(a, l, lane);
      else if (C <= 2) thomas_warp<2>(a, l, lane);
      else if (C <= 4) thomas_warp<4>(a, l, lane);
      else if (C <= 8) thomas_warp<8>(a, l, lane);
      else thomas_warp<16>(a, l, lane);
    }
  };

  // ---- A y at node (i, k) from a value function (0 outside the grid):
  // W y + CR_i (y - y_{i+1}) + CR_{i-1} (y - y_{i-1}) + CZ_{k+1} (y - y_{k+1})
  // + CZ_k (y - y_{k-1}), the operator of Eq. scheme_op_r_z
  auto apply_at = [&](int i, int k, auto val) {
    const size_t e = (size_t)i * P + k;
    const double y = val(i, k);
    double v = __ldg(a.W + e) * y;
    v = fma(__ldg(a.CR + e), y - val(i + 1, k), v);
    v = fma(i > 0 ? __ldg(a.CR + e - P) : 0.0, y - val(i - 1, k), v);
    v = fma(__ldg(a.CZ + (size_t)i * PZ + k + 1), y - val(i, k + 1), v);
    v = fma(__ldg(a.CZ + (size_t)i * PZ + k), y - val(i, k - 1), v);
    return v;
  };
  const int N = nr * nz;
  const int gstride = G * kSmallThreads;

  // true residual r = phi - A x into the current buffer, ||r||^2 partial
  auto true_residual = [&]() {
    double acc = 0.0;
    double *r = rbuf[rsel];
    auto xv = [&](int i, int k) {
      return (i < 0 || i >= nr || k < 0 || k >= nz) ? 0.0 : __ldcg(a.x + (size_t)i * P + k);
    };
    for (int n = b * kSmallThreads + tid; n < N; n += gstride) {
      const int i = n / nz, k = n % nz;
      const size_t e = (size_t)i * P + k;
      const double res = __ldg(a.phi + e) - apply_at(i, k, xv);
      r[e] = res;
      acc = fma(res, res, acc);
    }
    put(kPartRR, acc);
  };

  bool failed = false, done = false;
  int status = AX_OK;
  if (a.f != nullptr) {
    // phi = r f, r = phi, x = 0 (A x = 0), and the state of sc_start
    double acc = 0.0;
    for (int n = b * kSmallThreads + tid; n < N; n += gstride) {
      const int i = n / nz, k = n % nz;
      const size_t e = (size_t)i * P + k;
      const double v = __ldg(a.R + i) * __ldg(a.f + n);
      const_cast<double *>(a.phi)[e] = v;
      a.r[e] = v;
      a.x[e] = 0.0;
      acc = fma(v, v, acc);
    }
    put(kPartRR, acc);
    if (!sync()) return;
    const double bb = total(kPartRR);
    s.rr = bb;
    s.bb = bb;
    s.thresh2 = a.tol2 * bb;
    s.iters = 0;
    s.max_iter = a.max_iter;
    s.beta = 0.0;
    s.status = AX_OK;
    if (!isfinite(bb)) {
      failed = true;
      status = AX_ERR_BREAKDOWN;
    } else if (bb <= s.thresh2 || bb == 0.0) {
      done = true;
    }
  }
  double rho = 0.0, beta = 0.0, alpha = 0.0, rr = s.rr;
  // z = B^-1 r, rho = (r, z)
  if (!failed && !done) {
    double acc = 0.0;
    transform(1, 0.0, nullptr, acc);
    if (!sync()) return;
    mode_solves();
    if (!sync()) return;
    acc = 0.0;
    transform(2, 0.0, nullptr, acc);
    put(kPartRZ, acc);
    if (!sync()) return;
    rho = total(kPartRZ);
    if (!isfinite(rho)) {
      failed = true;
      status = AX_ERR_BREAKDOWN;
    }
  }
  int iters = s.iters;
  while (!failed && !done) {
    // 1. p = z + beta p_old, q = A p, (p, q)
    const double *pold = (iters & 1) ? a.pb : a.pa;
    double *pnew = (iters & 1) ? a.pa : a.pb;
    {
      auto pv = [&](int i, int k) {
        if (i < 0 || i >= nr || k < 0 || k >= nz) return 0.0;
        const size_t e = (size_t)i * P + k;
        return beta == 0.0 ? __ldcg(a.z + e) : fma(beta, __ldcg(pold + e), __ldcg(a.z + e));  // p_1 = z
      };
      double acc = 0.0;
      for (int n = b * kSmallThreads + tid; n < N; n += gstride) {
        const int i = n / nz, k = n % nz;
        const size_t e = (size_t)i * P + k;
        const double p = pv(i, k);
        const double q = apply_at(i, k, pv);
        pnew[e] = p;
        a.q[e] = q;
        acc = fma(p, q, acc);
      }
      put(kPartPQ, acc);
    }
    if (!sync()) return;
    const double pq = total(kPartPQ);
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rho)) {
      failed = true;
      status = AX_ERR_BREAKDOWN;
      break;
    }
    alpha = rho / pq;
    // 2. r_new = r - alpha q, x += alpha p, ||r_new||^2, t = F r_new
    {
      double acc = 0.0;
      transform(0, alpha, pnew, acc);
      put(kPartRR, acc);
    }
    if (!sync()) return;
    rr = total(kPartRR);
    rsel ^= 1;
    ++iters;
    if (!isfinite(rr)) {
      failed = true;
      status = AX_ERR_BREAKDOWN;
      break;
    }
    if (rr <= s.thresh2) {
      // the recursive residual passed: test the true one
      true_residual();
      if (!sync()) return;
      rr = total(kPartRR);
      if (rr <= s.thresh2) {
        done = true;
        break;
      }
      if (iters >= s.max_iter) {
        failed = true;
        status = AX_ERR_NO_CONVERGENCE;
        break;
      }
      double acc = 0.0;
      transform(1, 0.0, nullptr, acc);  // t = F r_true
      if (!sync()) return;
    } else if (iters >= s.max_iter) {
      failed = true;
      status = AX_ERR_NO_CONVERGENCE;
      break;
    }
    // 3. mode solves
    mode_solves();
    if (!sync()) return;
    // 4. z = F^T t, (r, z), beta
    {
      double acc = 0.0;
      transform(2, 0.0, nullptr, acc);
      put(kPartRZ, acc);
    }
    if (!sync()) return;
    const double rz = total(kPartRZ);
    if (!isfinite(rz) || rho == 0.0) {
      failed = true;
      status = AX_ERR_BREAKDOWN;
      break;
    }
    beta = rz / rho;
    rho = rz;
  }
  if (a.u != nullptr) {
    // u = x (x is final: its last update came before the last barrier)
    for (int n = b * kSmallThreads + tid; n < N; n += gstride) {
      const int i = n / nz, k = n % nz;
      a.u[n] = __ldcg(a.x + (size_t)i * P + k);
    }
  }
  if (b == 0 && tid == 0) {
    s.iters = iters;
    s.rr = rr;
    s.rho = rho;
    s.alpha = alpha;
    s.beta = beta;
    s.status = status;
    s.state = done ? kDone : kFailed;
    *a.st = s;
  }
}

struct SmallGeom {
  int device = -1, maxg = 0;
};
std::mutex g_small_mu;
std::vector<SmallGeom> g_small_geom;

int max_coresident(int device) {
  std::lock_guard<std::mutex> lock(g_small_mu);
  for (auto &g : g_small_geom)
    if (g.device == device) return g.maxg;
  SmallGeom g;
  g.device = device;
  int sms = 0, per = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_small_kernel, kSmallThreads, 0) == cudaSuccess)
    g.maxg = sms * per;
  g_small_geom.push_back(g);
  return g.maxg;
}

}  // namespace

int small_pcg_grid(int nr, int nz, int *nch) {
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return 0;
  const int maxg = max_coresident(device);
  if (maxg < 1) return 0;
  // enough (row, output chunk) items for the CTAs, chunks of >= 16 outputs,
  // at most one CTA per SM's worth of the co-resident limit
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int target = std::min(std::min(maxg, std::max(sms, 1)), 256);  // the partial sums take <= 256
  int c = std::max(1, std::min(target / std::max(nr, 1), nz / 16));
  *nch = c;
  return std::min(nr * c, target);
}

cudaError_t launch_small_pcg(const SmallPcgArgs &a0, int grid, cudaStream_t s) {
  SmallPcgArgs a = a0;
  // Each CTA's items share one output chunk (nch = 1, or grid = nr nch by
  // small_pcg_grid), so its transform rows go to shared memory where they fit.
  const int CH = (a.nz + a.nch - 1) / a.nch;
  const size_t smem = 2 * (size_t)CH * (a.nz + 1) * sizeof(double);
  a.msm = (a.nch == 1 || grid == a.nr * a.nch) && smem <= kSmallSmem ? 1 : 0;
  const size_t dyn = a.msm ? smem : 0;
  if (dyn > 48 * 1024) {
    cudaError_t e = ensure_smem_attr((const void *)pcg_small_kernel, dyn);
    if (e != cudaSuccess) return e;
  }
  note_launch();
  void *args[] = {&a};
  return cudaLaunchCooperativeKernel((const void *)pcg_small_kernel, dim3(grid), dim3(kSmallThreads), args, dyn, s);
}

}  // namespace ax
