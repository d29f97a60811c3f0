// Operator set-up, iteration drivers and the C ABI of libaxpcg.
//
// Iterations (Section 2.2): preconditioned conjugate gradients with the
// Laplace preconditioner B of Eq. coeff2 (A B^-1 A is self-adjoint, so CG
// applies), and the implicit three-layer Chebyshev scheme of Eq. main-scheme.
// The stop rule is the paper's (Section 4.2): the true residual
// ||A y - phi|| / ||phi|| <= tol.
//
// GPU organisation.  Scalars (alpha, beta, rho, norms) live on the device in
// one RhsState per right-hand side and are produced by tiny "scalar" kernels
// that reduce per-CTA FP64 partial sums in a fixed order (deterministic, no
// atomics).  Every iteration kernel reads its RHS's state and returns at once
// unless the state matches the kernel's mask, so converged right-hand sides
// stop costing bandwidth while the others continue.  A block of iterations is
// captured once into a CUDA graph and replayed; the host reads the states
// between replays.
//
// Mixed precision (AX_PCG_MIXED / AX_CHEB_MIXED): iterative refinement.  The
// outer loop forms the true residual r = phi - A x in FP64 (FP64 stencil,
// FP64 coefficients), the inner loop solves A d = r in FP32 to a relative
// tolerance eta_in (or a fixed number of steps), and x += d in FP64.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <chrono>
#include <map>
#include <string>
#include <vector>

#include "ax_common.cuh"

namespace ax {

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  int key = -1;
  size_t nodes = 0;
};

struct ProfEvent {
  int kind;
  cudaEvent_t a, b;
  double units;
};

struct Workspace {
  int m64 = 0, m32 = 0, mbase = 0;
  // FP64 vectors [m][nr][pitch]
  double *phi64 = nullptr, *x64 = nullptr;
  double *r64 = nullptr, *pa64 = nullptr, *pb64 = nullptr, *q64 = nullptr, *z64 = nullptr, *y64prev = nullptr;
  // FP32 vectors
  float *xh = nullptr, *xl = nullptr, *phh = nullptr, *phl = nullptr;  // double-float x and phi (mixed PCG)
  float *x32 = nullptr, *r32 = nullptr, *pa32 = nullptr, *pb32 = nullptr, *q32 = nullptr, *z32 = nullptr,
        *y32prev = nullptr;
  // partial sums [4][m][kPartialStride]
  double *part = nullptr;
  double *chp = nullptr;      // Chebyshev (tau, rho0^2) per right-hand side [m][2]
  double *rscale = nullptr;   // mixed methods: power-of-two scale of phi and x per right-hand side [m]
  RhsState *st = nullptr, *st_outer = nullptr;
  // [0] right-hand sides the residual-replacement step has put in kCheck (the
  // gate of its masked launches; reset at the end of the step), [1] the same
  // counted over the current solve (option "replace_checks")
  int *chk = nullptr;
  int replace_gate = 1;         // 0: the replacement step's launches are not gated
  RhsState *h_st = nullptr;   // pinned host mirror [2 m]
  // dense FP64 staging for host buffers and single-step entry points
  double *stage_a = nullptr, *stage_b = nullptr;
  size_t stage_elems = 0;
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  unsigned char *split = nullptr;  // BF16 split operand of the tensor-core transform
  size_t split_bytes = 0;
  cudaStream_t cap = nullptr;
  GraphCache g64, g32, gc64, gc32;
  // options
  double inner_tol = 1e-4;
  int inner_max = 400;
  int graph_iters = 16;
  int max_outer = 30;
  int mixed_restart = 0;        // 1: AX_PCG_MIXED uses restarted refinement instead of replacement
  int tc_stall_test = 0;        // 1: the next tensor-core transform lets one bounded wait run out
  int tc_unfused = 0;           // 1: mixed PCG forms p in the stencil, not in the inverse transform
  double replace_delta = 0.1;   // residual reduction between FP64 replacements
  int cheb_bounds = -1;         // Chebyshev bounds: 0 face-wise, 1 Lanczos estimate, -1 Lanczos
                                // where the face-wise gamma_1 degenerates (q_min = 0 < q_max)
  int cheb_steps = 20;          // PCG steps of the Lanczos estimate
  double cheb_widen = 0.05;     // relative widening of the estimated bounds
  int cheb_check = 1;           // Chebyshev: residual norm (a reduction) every cheb_check-th step
  int host_chunks = 1;          // host-buffer solves: right-hand-side chunks whose copies overlap the solve
                                // (1: none; at 1024^2 x 64, 4 chunks of 16 took 73 ms against 63 ms for one
                                // 64-RHS solve with its copies in series)
  int small_path = 1;           // FP64 PCG of one right-hand side on a small grid: one persistent launch
  int small_stall_test = 0;     // 1: the next persistent launch lets its barrier waits run out
  double *small_buf = nullptr;  // its second residual buffer and transformed field [2][nr][pitch]
  unsigned *small_bar = nullptr;  // its grid-barrier words [2]
  int *h_flag = nullptr;          // pinned host copy of the expiry flag
  cudaStream_t copy = nullptr;  // copy stream of those chunks
  cudaEvent_t cev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // per right-hand-side completion times (ms since lat_t0) of the current
  // solve, taken when the host reads the states after each graph replay
  // (resolution: one replay); set by the batched solve, -1 = not finished
  bool lat_track = false;
  std::chrono::steady_clock::time_point lat_t0;
  std::vector<double> lat_ms;
  // per-launch profiler (off by default; graphs are not used while it is on)
  bool profile = false;
  std::vector<ProfEvent> prof_events;
  double prof_ms[kProfKinds] = {0}, prof_launches[kProfKinds] = {0}, prof_units[kProfKinds] = {0};
};

static long long g_launches = 0;
// Serialises workspace allocation and graph capture across host threads (the
// batched solve runs one thread per group): an allocation, which may
// synchronise the device, must never overlap another thread's capture.
static std::recursive_mutex g_alloc_capture_mutex;
static char g_last_error[256] = "no error";
static thread_local bool g_capturing = false;
void note_launch() {
  if (!g_capturing) __atomic_add_fetch(&g_launches, 1, __ATOMIC_RELAXED);
}

cudaError_t ensure_smem_attr(const void *func, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void *, size_t>> limits;
  std::lock_guard<std::mutex> lock(mu);
  for (auto &e : limits)
    if (e.first == func) {
      if (e.second >= bytes) return cudaSuccess;
      cudaError_t r = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (r == cudaSuccess) e.second = bytes;
      return r;
    }
  cudaError_t r = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (r == cudaSuccess) limits.push_back({func, bytes});
  return r;
}

namespace {

int status_from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return AX_OK;
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return AX_ERR_OOM;
  return AX_ERR_CUDA;
}

#define AX_TRY(expr)                                  \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) return status_from_cuda(_e); \
  } while (0)

#define AX_CHECK_LAUNCH() AX_TRY(cudaGetLastError())

template <typename P>
cudaError_t dalloc(P **p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(P));
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  // cudaMemset is queued on the legacy stream, which does not order itself
  // with the non-blocking streams the batched groups run on: wait for the
  // fill here so that no later launch on any stream can see it in flight.
  e = cudaMemset(*p, 0, count * sizeof(P));
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  return e;
}

template <typename P>
void dfree(P *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

void free_graph(GraphCache &g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  g.key = -1;
}

void free_vectors64(Workspace *w) {
  dfree(w->r64); dfree(w->pa64); dfree(w->pb64); dfree(w->q64); dfree(w->z64); dfree(w->y64prev);
  w->m64 = 0;
  free_graph(w->g64);
  free_graph(w->gc64);
}
void free_vectors32(Workspace *w) {
  dfree(w->x32); dfree(w->r32); dfree(w->pa32); dfree(w->pb32); dfree(w->q32); dfree(w->z32); dfree(w->y32prev);
  dfree(w->xh); dfree(w->xl); dfree(w->phh); dfree(w->phl);
  w->m32 = 0;
  free_graph(w->g32);
  free_graph(w->gc32);
}
void free_base(Workspace *w) {
  dfree(w->phi64); dfree(w->x64); dfree(w->part); dfree(w->chp); dfree(w->rscale); dfree(w->st);
  dfree(w->st_outer); dfree(w->chk);
  if (w->h_st) cudaFreeHost(w->h_st);
  w->h_st = nullptr;
  w->mbase = 0;
  free_graph(w->g64); free_graph(w->g32); free_graph(w->gc64); free_graph(w->gc32);
}

size_t field_elems(const ax_operator *op) { return (size_t)op->nr * op->pitch; }

int ensure_base(ax_operator *op, int m) {
  std::lock_guard<std::recursive_mutex> lock(g_alloc_capture_mutex);
  Workspace *w = op->ws;
  if (w->mbase >= m) return AX_OK;
  free_base(w);
  const size_t f = field_elems(op) * m;
  AX_TRY(dalloc(&w->phi64, f));
  AX_TRY(dalloc(&w->x64, f));
  AX_TRY(dalloc(&w->part, (size_t)4 * m * kPartialStride));
  AX_TRY(dalloc(&w->chp, (size_t)2 * m));
  AX_TRY(dalloc(&w->rscale, (size_t)m));
  AX_TRY(dalloc(&w->st, (size_t)m));
  AX_TRY(dalloc(&w->st_outer, (size_t)m));
  AX_TRY(dalloc(&w->chk, 2));
  AX_TRY(cudaMemset(w->chk, 0, 2 * sizeof(int)));
  AX_TRY(cudaMallocHost((void **)&w->h_st, sizeof(RhsState) * 2 * m));
  w->mbase = m;
  return AX_OK;
}

int ensure_vec64(ax_operator *op, int m, bool cheb) {
  std::lock_guard<std::recursive_mutex> lock(g_alloc_capture_mutex);
  Workspace *w = op->ws;
  if (w->m64 >= m && (!cheb || w->y64prev)) return AX_OK;
  free_vectors64(w);
  const size_t f = field_elems(op) * m;
  AX_TRY(dalloc(&w->r64, f));
  AX_TRY(dalloc(&w->pa64, f));
  AX_TRY(dalloc(&w->pb64, f));
  AX_TRY(dalloc(&w->q64, f));
  AX_TRY(dalloc(&w->z64, f));
  if (cheb) AX_TRY(dalloc(&w->y64prev, f));
  w->m64 = m;
  return AX_OK;
}

int ensure_vec32(ax_operator *op, int m, bool cheb) {
  std::lock_guard<std::recursive_mutex> lock(g_alloc_capture_mutex);
  Workspace *w = op->ws;
  if (w->m32 >= m && (!cheb || w->y32prev)) return AX_OK;
  free_vectors32(w);
  const size_t f = field_elems(op) * m;
  AX_TRY(dalloc(&w->x32, f));
  AX_TRY(dalloc(&w->r32, f));
  AX_TRY(dalloc(&w->pa32, f));
  AX_TRY(dalloc(&w->pb32, f));
  AX_TRY(dalloc(&w->q32, f));
  AX_TRY(dalloc(&w->z32, f));
  AX_TRY(dalloc(&w->xh, f));
  AX_TRY(dalloc(&w->xl, f));
  AX_TRY(dalloc(&w->phh, f));
  AX_TRY(dalloc(&w->phl, f));
  if (cheb) AX_TRY(dalloc(&w->y32prev, f));
  w->m32 = m;
  return AX_OK;
}

int ensure_stage(ax_operator *op, size_t elems) {
  std::lock_guard<std::recursive_mutex> lock(g_alloc_capture_mutex);
  Workspace *w = op->ws;
  if (w->stage_elems >= elems) return AX_OK;
  dfree(w->stage_a);
  dfree(w->stage_b);
  w->stage_elems = 0;
  AX_TRY(dalloc(&w->stage_a, elems));
  AX_TRY(dalloc(&w->stage_b, elems));
  w->stage_elems = elems;
  return AX_OK;
}

int ensure_split(ax_operator *op, size_t bytes) {
  std::lock_guard<std::recursive_mutex> lock(g_alloc_capture_mutex);
  Workspace *w = op->ws;
  if (w->split_bytes >= bytes) return AX_OK;
  dfree(w->split);
  w->split_bytes = 0;
  AX_TRY(dalloc(&w->split, bytes));  // zero: padding rows and columns stay zero
  w->split_bytes = bytes;
  return AX_OK;
}

int ensure_scratch(ax_operator *op, size_t bytes) {
  std::lock_guard<std::recursive_mutex> lock(g_alloc_capture_mutex);
  Workspace *w = op->ws;
  if (w->scratch_bytes >= bytes) return AX_OK;
  if (w->scratch) cudaFree(w->scratch);
  w->scratch = nullptr;
  w->scratch_bytes = 0;
  unsigned char *p = nullptr;
  AX_TRY(dalloc(&p, bytes));
  w->scratch = p;
  w->scratch_bytes = bytes;
  return AX_OK;
}

// Records a pair of events around the launches in its lifetime when the
// operator's profiler is on.
struct ProfScope {
  Workspace *w;
  int kind;
  double units;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(Workspace *w_, int kind_, double units_, cudaStream_t s_) : w(w_), kind(kind_), units(units_), s(s_) {
    if (w && w->profile && !g_capturing && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, s);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) != cudaSuccess) return;
    cudaEventRecord(b, s);
    w->prof_events.push_back({kind, a, b, units});
  }
};

void prof_collect(Workspace *w) {
  for (auto &e : w->prof_events) {
    float ms = 0.f;
    cudaEventSynchronize(e.b);
    cudaEventElapsedTime(&ms, e.a, e.b);
    w->prof_ms[e.kind] += ms;
    w->prof_launches[e.kind] += 1;
    w->prof_units[e.kind] += e.units;
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  w->prof_events.clear();
}

double *part_ptr(Workspace *w, int kind) { return w->part + (size_t)kind * w->mbase * kPartialStride; }
enum { kPartA = 0, kPartB = 1, kPartC = 2, kPartD = 3 };

// ---------------------------------------------------------------------------
// Conversion kernels (dense caller layout <-> padded device layout)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void dense_to_padded(const double *__restrict__ src, T *__restrict__ dst, long long rows, int nz,
                                int pitch) {
  for (long long row = blockIdx.x; row < rows; row += gridDim.x)
    for (int k = threadIdx.x; k < nz; k += blockDim.x) dst[row * pitch + k] = (T)src[row * nz + k];
}

template <typename T>
__global__ void padded_to_dense(const T *__restrict__ src, double *__restrict__ dst, long long rows, int nz,
                                int pitch) {
  for (long long row = blockIdx.x; row < rows; row += gridDim.x)
    for (int k = threadIdx.x; k < nz; k += blockDim.x) dst[row * nz + k] = (double)src[row * pitch + k];
}

// Mixed methods: sigma_m = 2^-round(log2(rms(phi_m))) (1 for phi_m = 0), from
// the ||phi||^2 partials, so that the FP32 inner iteration works on values of
// order one whatever the units of f (FP32 squares of residuals near 1e-20
// would underflow).  A power of two scales FP64 values exactly.
// sigma = 2^-e with max |phi| = f 2^e, 1/2 <= f < 1 (frexp): the scaled
// right-hand side has its largest magnitude in [1/2, 1) for any finite
// nonzero phi of FP64 (no square is formed, so nothing overflows or
// underflows on the way); 1 for phi = 0 or non-finite phi.  pmax holds the
// per-CTA maxima of |phi| (nb per right-hand side).
__global__ void rhs_scale(double *scale, const double *pmax, int nb, int m) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double mx = 0.0;
  for (int b = 0; b < nb; ++b) mx = fmax(mx, pmax[(size_t)j * kPartialStride + b]);
  double sc = 1.0;
  if (mx > 0.0 && isfinite(mx)) {
    int e = 0;
    frexp(mx, &e);
    sc = ldexp(1.0, -e);
  }
  scale[j] = sc;
}

// Per-CTA partials of ||phi||^2 in the block structure of prep_rhs (grid
// (m, ceil(nr / 16)), 256 threads), for the scaled right-hand side.
__global__ void phi_norm2(const double *__restrict__ phi, int nr, int nz, int pitch, double *__restrict__ part) {
  __shared__ double red[8];
  const int m = blockIdx.x;
  const int i0 = blockIdx.y * 16, i1 = min(i0 + 16, nr);
  double acc = 0.0;
  for (int i = i0; i < i1; ++i) {
    const double *pr = phi + ((size_t)m * nr + i) * pitch;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) acc = fma(pr[k], pr[k], acc);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[(size_t)m * kPartialStride + blockIdx.y] = s;
}

// phi *= sigma and x *= sigma (x may be null) with the ||phi||^2 partials *=
// sigma^2 (inverse = false), or x /= sigma (inverse = true).  grid (., m).
__global__ void apply_rhs_scale(double *phi, double *x, const double *scale, double *part, int nb, size_t field,
                                bool inverse) {
  const int m = blockIdx.y;
  const double sc = inverse ? 1.0 / scale[m] : scale[m];
  const size_t b = (size_t)m * field;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < field; e += (size_t)gridDim.x * blockDim.x) {
    if (phi) phi[b + e] *= sc;
    if (x) x[b + e] *= sc;
  }
  if (part && blockIdx.x == 0)
    for (int k = threadIdx.x; k < nb; k += blockDim.x) part[(size_t)m * kPartialStride + k] *= sc * sc;
}

// phi = r_i f (Eq. diff_approx1), FP64, plus per-CTA partials of ||phi||^2
// (part) and of max |phi| (pmax).  grid (m, ceil(nr / 16)), 256 threads.
__global__ void prep_rhs(const double *__restrict__ f, double *__restrict__ phi, const double *__restrict__ R,
                         int nr, int nz, int pitch, double *__restrict__ part, double *__restrict__ pmax) {
  __shared__ double red[8];
  __shared__ double redm[8];
  const int m = blockIdx.x;
  const int i0 = blockIdx.y * 16, i1 = min(i0 + 16, nr);
  double acc = 0.0, mx = 0.0;
  for (int i = i0; i < i1; ++i) {
    const double ri = R[i];
    const double *fr = f + ((size_t)m * nr + i) * nz;
    double *pr = phi + ((size_t)m * nr + i) * pitch;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
      const double v = ri * fr[k];
      pr[k] = v;
      acc = fma(v, v, acc);
      mx = fmax(mx, fabs(v));
    }
  }
  const double s = block_sum(acc, red);
  // block maximum (fixed order as block_sum)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) redm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, redm[w]);
    part[(size_t)m * kPartialStride + blockIdx.y] = s;
    pmax[(size_t)m * kPartialStride + blockIdx.y] = b;
  }
}

template <typename T>
__global__ void to_precision(const double *__restrict__ src, T *__restrict__ dst, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (T)src[e];
}

// x64 += d32 for right-hand sides whose outer state matches `mask`.
__global__ void add_correction(double *__restrict__ x, const float *__restrict__ d, size_t field,
                               const RhsState *st, int mask) {
  const int m = blockIdx.y;
  if (!rhs_selected(st, mask, m)) return;
  const size_t b = (size_t)m * field;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < field; e += (size_t)gridDim.x * blockDim.x)
    x[b + e] += (double)d[b + e];
}

// Task t of a right-hand side: the 8 consecutive columns 8 (t % nch) ..
// of row t / nch (nch = chunks of 8 columns per row): consecutive threads walk
// along a row, so every warp reads 1 KB of contiguous row data per field.
__device__ __forceinline__ void split_task(int t, int nch, int &row, int &col) {
  row = t / nch;
  col = (t - row * nch) * 8;
}

// FP64 field -> double-float pair (hi = fl(x), lo = fl(x - hi)) and back.
// n is a multiple of 32 (whole rows of pitch elements): pairs of elements.
__global__ void to_df(const double *__restrict__ x, float *__restrict__ h, float *__restrict__ l, size_t n) {
  const double2 *x2 = reinterpret_cast<const double2 *>(x);
  float2 *h2 = reinterpret_cast<float2 *>(h), *l2 = reinterpret_cast<float2 *>(l);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n / 2; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = x2[i];
    const float hx = (float)v.x, hy = (float)v.y;
    h2[i] = make_float2(hx, hy);
    l2[i] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
  }
}
__global__ void from_df(const float *__restrict__ h, const float *__restrict__ l, double *__restrict__ x, size_t n) {
  const float2 *h2 = reinterpret_cast<const float2 *>(h), *l2 = reinterpret_cast<const float2 *>(l);
  double2 *x2 = reinterpret_cast<double2 *>(x);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n / 2; i += (size_t)gridDim.x * blockDim.x) {
    const float2 a = h2[i], b = l2[i];
    x2[i] = make_double2((double)a.x + (double)b.x, (double)a.y + (double)b.y);
  }
}
// Replacement of the selected right-hand sides in double-float: (xh, xl) +=
// x32 (two-sum, then renormalised) and x32 = 0 in one pass.  Launched with
// many CTAs per right-hand side, since only the few that are due at a step
// do work (the others return at once).
__global__ void fold_df(float *__restrict__ xh, float *__restrict__ xl, float *__restrict__ d, size_t field,
                        const RhsState *st, int mask) {
  const int m = blockIdx.y;
  if (!rhs_selected(st, mask, m)) return;
  // field is a multiple of 32 (rows of pitch elements): whole float4 groups
  float4 *h4 = reinterpret_cast<float4 *>(xh + (size_t)m * field);
  float4 *l4 = reinterpret_cast<float4 *>(xl + (size_t)m * field);
  float4 *d4 = reinterpret_cast<float4 *>(d + (size_t)m * field);
  const size_t n4 = field / 4;
  auto fold = [](float a, float c, float lo, float &h, float &l) {
    const float s = a + c, bb = s - a;
    const float err = ((a - (s - bb)) + (c - bb)) + lo;
    h = s + err;
    l = err - (h - s);
  };
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n4; e += (size_t)gridDim.x * blockDim.x) {
    const float4 a = h4[e], c = d4[e], lo = l4[e];
    float4 h, l;
    fold(a.x, c.x, lo.x, h.x, l.x);
    fold(a.y, c.y, lo.y, h.y, l.y);
    fold(a.z, c.z, lo.z, h.z, l.z);
    fold(a.w, c.w, lo.w, h.w, l.w);
    h4[e] = h;
    l4[e] = l;
    d4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// x += alpha p, r -= alpha q for the selected right-hand sides, with per-block
// partials of ||r||^2 and the new r written split into BF16 halves for the
// tensor-core transform: the update that the FFT forward transform fuses into
// its load phase.  p is pb for an even iteration count, pa for an odd one (as
// in the stencil).  x == nullptr: r only (the iterate update then happens in
// the inverse transform's epilogue, with the next direction).
// CTAs per right-hand side of the update and split passes: about four
// 8-column tasks per thread (at least 64, at most 4096 CTAs), so that large
// fields keep enough loads in flight.
int update_blocks(int rows, int nz) {
  const long long tasks = (long long)rows * ((nz + 7) / 8);
  const long long b = (tasks + 4 * 256 - 1) / (4 * 256);
  return (int)std::max(64LL, std::min(4096LL, b));
}
__global__ void __launch_bounds__(256) pcg_update(float *__restrict__ x, float *__restrict__ r,
                                                  const float *__restrict__ q, const float *__restrict__ pa,
                                                  const float *__restrict__ pb, int nr, int n, int pitch,
                                                  size_t field, int mtiles, int ktiles, int kbe,
                                                  unsigned char *__restrict__ split,
                                                  const RhsState *st, int mask, double *__restrict__ partial,
                                                  int cosine) {
  __shared__ double red[8];
  const int m = blockIdx.y;
  if (!rhs_selected(st, mask, m)) return;
  const float alpha = (float)st[m].alpha;
  const float *p = (st[m].iters & 1) ? pa : pb;
  const int nch = (n + 7) >> 3;
  const int tasks = nr * nch;
  float acc = 0.f;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tasks; t += gridDim.x * blockDim.x) {
    int row, col;
    split_task(t, nch, row, col);  // row < nr, col < n, col + 8 <= n rounded up to 8 <= pitch
    const size_t e = (size_t)m * field + (size_t)row * pitch + col;
    float rv[8], qv[8];
    *reinterpret_cast<float4 *>(rv) = *reinterpret_cast<const float4 *>(r + e);
    *reinterpret_cast<float4 *>(rv + 4) = *reinterpret_cast<const float4 *>(r + e + 4);
    *reinterpret_cast<float4 *>(qv) = *reinterpret_cast<const float4 *>(q + e);
    *reinterpret_cast<float4 *>(qv + 4) = *reinterpret_cast<const float4 *>(q + e + 4);
    if (x != nullptr) {
      float xv[8], pv[8];
      *reinterpret_cast<float4 *>(xv) = *reinterpret_cast<const float4 *>(x + e);
      *reinterpret_cast<float4 *>(xv + 4) = *reinterpret_cast<const float4 *>(x + e + 4);
      *reinterpret_cast<float4 *>(pv) = *reinterpret_cast<const float4 *>(p + e);
      *reinterpret_cast<float4 *>(pv + 4) = *reinterpret_cast<const float4 *>(p + e + 4);
#pragma unroll
      for (int i = 0; i < 8; ++i) xv[i] = fmaf(alpha, pv[i], xv[i]);
      *reinterpret_cast<float4 *>(x + e) = *reinterpret_cast<const float4 *>(xv);
      *reinterpret_cast<float4 *>(x + e + 4) = *reinterpret_cast<const float4 *>(xv + 4);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      rv[i] = fmaf(-alpha, qv[i], rv[i]);
      acc = fmaf(rv[i], rv[i], acc);
    }
    *reinterpret_cast<float4 *>(r + e) = *reinterpret_cast<const float4 *>(rv);
    *reinterpret_cast<float4 *>(r + e + 4) = *reinterpret_cast<const float4 *>(rv + 4);
    // the cosine transform folds mirrored columns, which other threads update:
    // its split input is written by a separate pass (split_field)
    if (!cosine) split_store8(split, m, row, col, mtiles, ktiles, kbe, rv);
  }
  const double sum = block_sum((double)acc, red);
  if (threadIdx.x == 0) partial[(size_t)m * kPartialStride + blockIdx.x] = sum;
}

// The rows of a field written split into BF16 halves (tensor-core transform input).
// cosine: the folded input of the cosine forward transform instead (fold_store8).
__global__ void __launch_bounds__(256) split_field(const float *__restrict__ in, int nr, int n, int pitch,
                                                   size_t field, int mtiles, int ktiles, int kbe,
                                                   unsigned char *__restrict__ split,
                                                   const RhsState *st, int mask, int cosine,
                                                   const int *gate) {
  if (gate != nullptr && *gate == 0) return;  // nothing selected (see GemmDstArgs::gate)
  const int m = blockIdx.y;
  if (!rhs_selected(st, mask, m)) return;
  const int nch = (n + 7) >> 3;
  const int tasks = nr * nch;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tasks; t += gridDim.x * blockDim.x) {
    int row, col;
    split_task(t, nch, row, col);  // row < nr, col < n, col + 8 <= n rounded up to 8 <= pitch
    const size_t e = (size_t)m * field + (size_t)row * pitch + col;
    float v[8];
    *reinterpret_cast<float4 *>(v) = *reinterpret_cast<const float4 *>(in + e);
    *reinterpret_cast<float4 *>(v + 4) = *reinterpret_cast<const float4 *>(in + e + 4);
    if (!cosine) {
      split_store8(split, m, row, col, mtiles, ktiles, kbe, v);
    } else if (2 * col < n) {  // chunks of the first half: u and w of columns col .. col + 7
      const float *rowp = in + (size_t)m * field + (size_t)row * pitch;
      float vm[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) vm[i] = (col + i < n) ? rowp[n - 1 - col - i] : 0.f;
      fold_store8(split, m, row, col, n, mtiles, ktiles, kbe, v, vm);
    }
  }
}

// ---------------------------------------------------------------------------
// Scalar kernels: one warp per right-hand side, fixed-order reductions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double reduce_part(const double *p, int nb) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) s += p[i];
  return warp_sum(s);
}

// rr = ||phi - A x||^2, bb = ||phi||^2 (or given), start the iteration.
__global__ void sc_start(RhsState *st, const double *prr, int nbr, const double *pbb, int nbb, double tol2,
                         int max_iter, int mask, int use_rr_as_bb) {
  const int m = blockIdx.x;
  if (!rhs_selected(st, mask, m)) return;
  const double rr = reduce_part(prr + (size_t)m * kPartialStride, nbr);
  const double bb = use_rr_as_bb ? rr : reduce_part(pbb + (size_t)m * kPartialStride, nbb);
  if (threadIdx.x == 0) {
    RhsState s = st[m];
    s.rr = rr;
    s.bb = bb;
    s.thresh2 = tol2 * bb;
    s.iters = 0;
    s.max_iter = max_iter;
    s.beta = 0.0;
    s.cheb_a = 2.0;
    s.status = AX_OK;
    s.due = 0;
    if (!isfinite(rr) || !isfinite(bb)) {
      s.state = kFailed;
      s.status = AX_ERR_BREAKDOWN;
    } else {
      s.state = (rr <= s.thresh2 || bb == 0.0) ? kDone : kActive;
    }
    st[m] = s;
  }
}

__global__ void sc_rho_init(RhsState *st, const double *p, int nb, int mask) {
  const int m = blockIdx.x;
  if (!rhs_selected(st, mask, m)) return;
  const double rz = reduce_part(p + (size_t)m * kPartialStride, nb);
  if (threadIdx.x == 0) {
    st[m].rho = rz;
    st[m].beta = 0.0;
    if (!isfinite(rz)) {
      st[m].state = kFailed;
      st[m].status = AX_ERR_BREAKDOWN;
    }
  }
}

__global__ void sc_alpha(RhsState *st, const double *p, int nb) {
  const int m = blockIdx.x;
  if (st[m].state != kActive) return;
  const double pq = reduce_part(p + (size_t)m * kPartialStride, nb);
  if (threadIdx.x == 0) {
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(st[m].rho)) {
      st[m].state = kFailed;
      st[m].status = AX_ERR_BREAKDOWN;
    } else {
      st[m].alpha = st[m].rho / pq;
    }
  }
}

// After x, r update: count the iteration and test the recursive residual.
// on_converge == kDue: a right-hand side that passes its threshold stays
// active for the rest of the iteration and is marked due for the replacement
// step at its end (mixed PCG).
__global__ void sc_after_update(RhsState *st, const double *p, int nb, int on_converge) {
  const int m = blockIdx.x;
  if (st[m].state != kActive) return;
  const double rr = reduce_part(p + (size_t)m * kPartialStride, nb);
  if (threadIdx.x == 0) {
    RhsState s = st[m];
    s.rr = rr;
    s.iters += 1;
    if (!isfinite(rr)) {
      s.state = kFailed;
      s.status = AX_ERR_BREAKDOWN;
    } else if (rr <= s.thresh2) {
      if (on_converge == kDue) s.due = 1;
      else s.state = on_converge;
    } else if (s.iters >= s.max_iter) {
      s.state = (on_converge == kDone) ? kDone : kFailed;
      if (on_converge != kDone) s.status = AX_ERR_NO_CONVERGENCE;
    }
    st[m] = s;
  }
}

// use_prev: the right-hand side already took this iteration's direction
// update from its recursive residual; the new beta refers to the rho before
// that update (mixed PCG residual replacement).
__global__ void sc_beta(RhsState *st, const double *p, int nb, int mask, int next_state, int use_prev = 0) {
  const int m = blockIdx.x;
  if (st[m].state != mask) return;
  const double rz = reduce_part(p + (size_t)m * kPartialStride, nb);
  if (threadIdx.x == 0) {
    const double rho = use_prev ? st[m].rho_prev : st[m].rho;
    if (!isfinite(rz) || rho == 0.0) {
      st[m].state = kFailed;
      st[m].status = AX_ERR_BREAKDOWN;
    } else {
      if (!use_prev) st[m].rho_prev = rho;
      st[m].beta = rz / rho;
      st[m].rho = rz;
      st[m].state = next_state;
    }
  }
}

// Right-hand sides (of n) in state `from` move to `to`.
__global__ void sc_promote(RhsState *st, int n, int from, int to, int *reset) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n && st[m].state == from) st[m].state = to;
  if (reset != nullptr && m == 0) *reset = 0;
}

// True-residual test of right-hand sides in kCheck.
__global__ void sc_true_check(RhsState *st, const double *p, int nb) {
  const int m = blockIdx.x;
  if (st[m].state != kCheck) return;
  const double rr = reduce_part(p + (size_t)m * kPartialStride, nb);
  if (threadIdx.x == 0) {
    st[m].rr = rr;
    if (rr <= st[m].thresh2) st[m].state = kDone;
    else if (st[m].iters >= st[m].max_iter) {
      st[m].state = kFailed;
      st[m].status = AX_ERR_NO_CONVERGENCE;
    }
  }
}

// Chebyshev: rr = ||A y - phi||^2 of the current iterate; stop or continue and
// advance alpha_{k+1} = 4 / (4 - rho0^2 alpha_k) (alpha for the first step is 1).
// check = 0: a step without the residual norm (no reduction): only the
// recurrence advances.
__global__ void sc_cheb(RhsState *st, const double *p, int nb, const double *chp, int on_converge, int check = 1) {
  const int m = blockIdx.x;
  if (st[m].state != kActive) return;
  const double rho0sq = chp[2 * m + 1];
  const double rr = check ? reduce_part(p + (size_t)m * kPartialStride, nb) : st[m].rr;
  if (threadIdx.x == 0) {
    RhsState s = st[m];
    s.rr = rr;
    if (!isfinite(rr)) {
      s.state = kFailed;
      s.status = AX_ERR_BREAKDOWN;
    } else if (check && rr <= s.thresh2) {
      s.state = on_converge;
    } else if (s.iters >= s.max_iter) {
      s.state = (on_converge == kDone) ? kDone : kFailed;
      if (on_converge != kDone) s.status = AX_ERR_NO_CONVERGENCE;
    } else {
      if (s.iters == 0) {
        s.cheb_a = 1.0;  // y_1 = y_0 - tau B^-1 (A y_0 - phi) (the y_{-1} term drops out)
      } else {
        const double prev = (s.iters == 1) ? 2.0 : s.cheb_a;
        s.cheb_a = 4.0 / (4.0 - rho0sq * prev);
      }
      s.iters += 1;
    }
    st[m] = s;
  }
}

// Mixed PCG with residual replacement: start.  rr = ||phi - A x||^2 (FP64),
// bb = ||phi||^2; the FP32 iteration runs until its recursive residual falls
// below thresh2 = max(delta^2 rr_true, (tol/2)^2 bb), then the true residual
// replaces it.
__global__ void sc_mixed_start(RhsState *st, const double *prr, int nbr, const double *pbb, int nbb, double tol2,
                               double delta2, int max_iter) {
  const int m = blockIdx.x;
  const double rr = reduce_part(prr + (size_t)m * kPartialStride, nbr);
  const double bb = reduce_part(pbb + (size_t)m * kPartialStride, nbb);
  if (threadIdx.x == 0) {
    RhsState s;
    memset(&s, 0, sizeof(s));
    s.rr = rr;
    s.bb = bb;
    s.max_iter = max_iter;
    s.status = AX_OK;
    if (!isfinite(rr) || !isfinite(bb)) {
      s.state = kFailed;
      s.status = AX_ERR_BREAKDOWN;
    } else if (rr <= tol2 * bb || bb == 0.0) {
      s.state = kDone;
    } else {
      s.state = kActive;
      s.thresh2 = fmax(delta2 * rr, 0.25 * tol2 * bb);
    }
    st[m] = s;
  }
}

// Residual replacement: rr = ||phi - A x64||^2 just computed in FP64 for the
// right-hand sides in kCheck.  Done, failed, or a new threshold (the caller
// then recomputes z = B^-1 r and resumes with sc_beta).
__global__ void sc_mixed_replace(RhsState *st, const double *prr, int nbr, double tol2, double delta2, int *chk) {
  const int m = blockIdx.x;
  if (!rhs_selected(st, kDue, m)) return;
  const double rr = reduce_part(prr + (size_t)m * kPartialStride, nbr);
  if (threadIdx.x == 0) {
    RhsState s = st[m];
    // the iteration's z and rho came from the recursive residual: when the
    // true one differs noticeably (||r||^2 by more than 1%: typically once the
    // recursion has run below the FP32 accuracy of x), the right-hand side goes
    // to kCheck for z = B^-1 r and beta from the new (r, z)
    const bool consistent = fabs(rr - s.rr) <= 1e-2 * rr;
    s.rr = rr;
    s.due = 0;
    s.tmp += 1.0;  // replacements
    if (!isfinite(rr)) {
      s.state = kFailed;
      s.status = AX_ERR_BREAKDOWN;
    } else if (rr <= tol2 * s.bb) {
      s.state = kDone;
    } else if (s.iters >= s.max_iter) {
      s.state = kFailed;
      s.status = AX_ERR_NO_CONVERGENCE;
    } else {
      s.thresh2 = fmax(delta2 * rr, 0.25 * tol2 * s.bb);
      if (!consistent) {
        s.state = kCheck;
        atomicAdd(chk, 1);  // opens the gate of the step's masked launches
        atomicAdd(chk + 1, 1);
      }
    }
    st[m] = s;
  }
}

template <typename T>
__global__ void zero_masked(T *x, size_t field, const RhsState *st, int mask) {
  const int m = blockIdx.y;
  if (!rhs_selected(st, mask, m)) return;
  const size_t b = (size_t)m * field;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < field; e += (size_t)gridDim.x * blockDim.x)
    x[b + e] = T(0);
}

// Outer refinement step: rr = ||phi - A x||^2 (FP64).  Converged RHS -> done;
// the others get an inner solve with reference ||r||^2.
__global__ void sc_outer(RhsState *so, RhsState *si, const double *prr, int nbr, const double *pbb, int nbb,
                         double tol2, double eta2, int inner_max, int first) {
  const int m = blockIdx.x;
  if (so[m].state != kActive) {
    if (threadIdx.x == 0) si[m].state = kIdle;
    return;
  }
  const double rr = reduce_part(prr + (size_t)m * kPartialStride, nbr);
  double bb = 0.0;
  if (first) bb = reduce_part(pbb + (size_t)m * kPartialStride, nbb);
  if (threadIdx.x == 0) {
    RhsState s = so[m];
    if (first) {
      s.bb = bb;
      s.thresh2 = tol2 * bb;
      s.iters = 0;
      s.status = AX_OK;
      s.tmp = 0.0;  // outer steps
    } else {
      s.iters += si[m].iters;  // inner iterations of the step just finished
      if (si[m].state == kFailed) {
        s.state = kFailed;
        s.status = si[m].status;
      }
    }
    s.rr = rr;
    RhsState in = si[m];
    in.state = kIdle;
    if (s.state == kActive) {
      if (!isfinite(rr)) {
        s.state = kFailed;
        s.status = AX_ERR_BREAKDOWN;
      } else if (rr <= s.thresh2 || s.bb == 0.0) {
        s.state = kDone;
      } else if (s.iters >= s.max_iter) {
        s.state = kFailed;
        s.status = AX_ERR_NO_CONVERGENCE;
      } else {
        s.tmp += 1.0;
        in.state = kActive;
        in.bb = rr;
        in.rr = rr;
        in.thresh2 = eta2 * rr;
        in.iters = 0;
        in.max_iter = inner_max;
        in.beta = 0.0;
        in.cheb_a = 2.0;
        in.status = AX_OK;
      }
    }
    so[m] = s;
    si[m] = in;
  }
}

// ---------------------------------------------------------------------------
// Host-side plan and coefficient construction
// ---------------------------------------------------------------------------
FftPlan make_plan(int L) {
  FftPlan p;
  p.L = L;
  std::vector<int> odd_big, fives, threes;
  int twos = 0, m = L;
  while (m % 2 == 0) { m /= 2; ++twos; }
  for (int d = 3; (long long)d * d <= m; d += 2) {
    while (m % d == 0) {
      if (d == 3) threes.push_back(3);
      else if (d == 5) fives.push_back(5);
      else odd_big.push_back(d);
      m /= d;
    }
  }
  if (m > 1) {
    if (m == 3) threes.push_back(3);
    else if (m == 5) fives.push_back(5);
    else odd_big.push_back(m);
  }
  std::sort(odd_big.rbegin(), odd_big.rend());
  std::vector<int> r;
  for (int x : odd_big) r.push_back(x);
  for (int x : fives) r.push_back(x);
  for (int x : threes) r.push_back(x);
  while (twos >= 3) { r.push_back(8); twos -= 3; }
  if (twos == 2) r.push_back(4);
  if (twos == 1) r.push_back(2);
  p.nstages = (int)r.size();
  int ns = 1;
  for (int i = 0; i < p.nstages && i < kMaxStages; ++i) {
    p.radix[i] = r[i];
    p.ns_div[i] = make_fastdiv(ns);
    p.tn_div[i] = make_fastdiv(L / r[i]);
    ns *= r[i];
  }
  // Rader's algorithm for a first radix that is a prime above the unrolled
  // set, when R - 1 has only the factors 2, 3, 5.
  if (p.nstages > 0 && p.radix[0] > 47) {
    const int P = p.radix[0] - 1;
    int m = P, t2 = 0;
    std::vector<int> sub;
    while (m % 2 == 0) { m /= 2; ++t2; }
    while (m % 5 == 0) { m /= 5; sub.push_back(5); }
    while (m % 3 == 0) { m /= 3; sub.push_back(3); }
    while (t2 >= 3) { sub.push_back(8); t2 -= 3; }
    if (t2 == 2) sub.push_back(4);
    if (t2 == 1) sub.push_back(2);
    if (m == 1 && sub.size() <= 8) {
      p.rader = 1;
      p.sub_n = (int)sub.size();
      int sns = 1;
      for (int i = 0; i < p.sub_n; ++i) {
        p.sub_radix[i] = sub[i];
        p.sub_ns[i] = make_fastdiv(sns);
        p.sub_tn[i] = make_fastdiv(P / sub[i]);
        sns *= sub[i];
      }
      p.p_div = make_fastdiv(P);
    }
  }
  return p;
}

// Tables of Rader's algorithm for prime R (P = R - 1): permutations by a
// primitive root g, the DFT of the permuted kernel c'_m = exp(-2 pi i g^-m / R)
// (FP64, direct sum) and the twiddles of length P.
void rader_tables(int R, std::vector<int> &perm, std::vector<double> &rk, std::vector<double> &rt) {
  const int P = R - 1;
  auto powmod = [R](long long b, long long e) {
    long long x = 1;
    b %= R;
    while (e > 0) {
      if (e & 1) x = x * b % R;
      b = b * b % R;
      e >>= 1;
    }
    return (int)x;
  };
  std::vector<int> fs;
  for (int m = P, d = 2; m > 1; ++d) {
    if (m % d == 0) {
      fs.push_back(d);
      while (m % d == 0) m /= d;
    }
  }
  int g = 2;
  for (;; ++g) {
    bool ok = true;
    for (int f : fs) ok = ok && powmod(g, P / f) != 1;
    if (ok) break;
  }
  const int ginv = powmod(g, R - 2);
  perm.assign(2 * P, 0);
  for (int q = 0; q < P; ++q) {
    perm[q] = powmod(g, q);
    perm[P + q] = powmod(ginv, q);
  }
  std::vector<double> cr(P), ci(P);
  for (int mm = 0; mm < P; ++mm) {
    const double ang = -2.0 * M_PI * perm[P + mm] / R;
    cr[mm] = std::cos(ang);
    ci[mm] = std::sin(ang);
  }
  rk.assign(2 * P, 0.0);
  for (int k = 0; k < P; ++k) {
    double sr = 0.0, si = 0.0;
    for (int mm = 0; mm < P; ++mm) {
      const long long e = ((long long)mm * k) % P;
      const double c = std::cos(2.0 * M_PI * e / P), sn = -std::sin(2.0 * M_PI * e / P);
      sr += cr[mm] * c - ci[mm] * sn;
      si += cr[mm] * sn + ci[mm] * c;
    }
    rk[2 * k] = sr;
    rk[2 * k + 1] = si;
  }
  rt.assign(2 * P, 0.0);
  for (int j = 0; j < P; ++j) {
    rt[2 * j] = std::cos(2.0 * M_PI * j / P);
    rt[2 * j + 1] = std::sin(2.0 * M_PI * j / P);
  }
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<double> &src) {
  std::vector<T> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = (T)src[i];
  cudaError_t e = dalloc(dst, src.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T>
void free_coef(Coef<T> &c) {
  dfree(c.CR); dfree(c.CZ); dfree(c.W); dfree(c.IP); dfree(c.E); dfree(c.R); dfree(c.TW); dfree(c.HW); dfree(c.CW);
  dfree(c.RK); dfree(c.RT);
  dfree(c.CRl); dfree(c.CZl); dfree(c.Wl);
  dfree(c.IPS); dfree(c.RS); dfree(c.IPST);
}

// ---------------------------------------------------------------------------
// One preconditioner application on the rows of `v` (already in rhat layout):
// forward transform, mode solves, inverse transform.
// ---------------------------------------------------------------------------
template <typename T>
const Coef<T> &coef(const ax_operator *op);
template <>
const Coef<double> &coef<double>(const ax_operator *op) { return op->c64; }
template <>
const Coef<float> &coef<float>(const ax_operator *op) { return op->c32; }

template <typename T>
DstArgs<T> dst_args(const ax_operator *op, int m, int rows, const RhsState *st, int mask) {
  DstArgs<T> a{};
  const Coef<T> &c = coef<T>(op);
  a.TW = c.TW;
  a.HW = c.HW;
  a.CW = c.CW;
  a.cosine = op->bc_z == 1;
  a.RK = c.RK;
  a.RT = c.RT;
  a.RP = op->rader_perm;
  a.plan = op->plan;
  a.n = op->nz;
  a.rows = rows;
  a.pitch = op->pitch;
  a.field = (long long)rows * op->pitch;
  a.m = m;
  a.scale = op->bc_z == 1 ? 1.0 / std::sqrt(2.0 * op->nz) : 0.5 / std::sqrt(2.0 * op->plan.L);
  a.st = st;
  a.mask = mask;
  return a;
}

template <typename T>
StencilArgs<T> stencil_args(const ax_operator *op, int m, const RhsState *st, int mask) {
  StencilArgs<T> a{};
  const Coef<T> &c = coef<T>(op);
  a.CR = c.CR;
  a.CZ = c.CZ;
  a.W = c.W;
  a.cstride = op->cstride;
  a.czstride = op->czstride;
  a.nr = op->nr;
  a.nz = op->nz;
  a.pitch = op->pitch;
  a.pitchz = op->pitchz;
  a.field = (long long)field_elems(op);
  a.m = m;
  a.st = st;
  a.mask = mask;
  return a;
}

template <typename T>
TriArgs<T> tri_args(const ax_operator *op, int m, const T *in, T *out, const RhsState *st, int mask) {
  TriArgs<T> a{};
  const Coef<T> &c = coef<T>(op);
  a.IP = c.IP;
  a.E = c.E;
  a.IPS = c.IPS;
  a.RS = c.RS;
  a.cstride = op->cstride;
  a.estride = op->estride;
  a.nr = op->nr;
  a.nz = op->nz;
  a.pitch = op->pitch;
  a.field = (long long)field_elems(op);
  a.m = m;
  a.in = in;
  a.out = out;
  a.st = st;
  a.mask = mask;
  a.variant = op->tri_variant;
  return a;
}

int dst_blocks(const ax_operator *op, int rows, int bytes) {
  const int rpb = dst_rows_per_block(dst_buffer_len(op->plan.L, op->nz), bytes);
  return (rows + rpb - 1) / rpb;
}

// ---- tensor-core transform (FP32 path, nz <= kMaxTcN) ----------------------
constexpr int kMaxTcN = 4096;

// BF16 DST-matrix tiles per (device, nz), built on first use and kept for the
// life of the process (shared by every operator with that nz); and one device
// flag per device for expired waits of the GEMM kernel.
struct TcCache {
  std::mutex mu;
  std::vector<std::pair<long long, uint16_t *>> tables;
  std::vector<std::pair<int, int *>> flags;
};
TcCache &tc_cache() {
  static TcCache c;
  return c;
}
const uint16_t *tc_table(int device, int n, int kind = kTableSine) {
  TcCache &c = tc_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  const long long key = (long long)device << 32 | (unsigned)n | (long long)kind << 24;
  for (auto &e : c.tables)
    if (e.first == key) return e.second;
  std::vector<uint16_t> t = dst_gemm_table(n, kind);
  uint16_t *d = nullptr;
  std::lock_guard<std::recursive_mutex> lock2(g_alloc_capture_mutex);
  if (dalloc(&d, t.size()) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, t.data(), t.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  c.tables.push_back({key, d});
  return d;
}
int *tc_flag(int device) {
  TcCache &c = tc_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  for (auto &e : c.flags)
    if (e.first == device) return e.second;
  int *d = nullptr;
  std::lock_guard<std::recursive_mutex> lock2(g_alloc_capture_mutex);
  if (dalloc(&d, 1) != cudaSuccess) return nullptr;
  c.flags.push_back({device, d});
  return d;
}

// Dense FP64 matrices of the z-transform for the persistent small-grid PCG,
// per (device, nz, boundary condition), kept for the life of the process:
// F[l][k] (forward) followed by F^T.  Sine (bc_z = 0): the orthonormal DST-I,
// F[l][k] = sqrt(2 / (nz + 1)) sin(pi (l + 1)(k + 1) / (nz + 1)), symmetric.
// Cosine (bc_z = 1): the orthonormal pair of the cell-centred grid,
// F[l][k] = sqrt(2 / nz) w_l cos(pi l (k + 1/2) / nz), w_0 = 1 / sqrt 2, w_l = 1
// otherwise (mode l + 1 of Eq. eq_trid).  The angles are reduced exactly in
// integers before the sine / cosine.
struct DenseCache {
  std::mutex mu;
  std::vector<std::pair<long long, double *>> tables;
};
const double *dense_table(int device, int n, int cosine) {
  static DenseCache c;
  std::lock_guard<std::mutex> lock(c.mu);
  const long long key = (long long)device << 32 | (unsigned)n | (long long)cosine << 24;
  for (auto &e : c.tables)
    if (e.first == key) return e.second;
  std::vector<double> t(2 * (size_t)n * n);
  for (int l = 0; l < n; ++l)
    for (int k = 0; k < n; ++k) {
      double v;
      if (!cosine) {
        const long long j = (long long)(l + 1) * (k + 1) % (2LL * (n + 1));  // angle pi j / (n + 1)
        v = std::sqrt(2.0 / (n + 1)) * std::sin(M_PI * (double)j / (n + 1));
      } else {
        const long long j = (long long)l * (2 * k + 1) % (4LL * n);  // angle pi j / (2 n)
        v = std::sqrt(2.0 / n) * (l == 0 ? std::sqrt(0.5) : 1.0) * std::cos(M_PI * (double)j / (2.0 * n));
      }
      t[(size_t)l * n + k] = v;
      t[(size_t)n * n + (size_t)k * n + l] = v;
    }
  double *d = nullptr;
  std::lock_guard<std::recursive_mutex> lock2(g_alloc_capture_mutex);
  if (dalloc(&d, t.size()) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  c.tables.push_back({key, d});
  return d;
}

// The persistent FP64 PCG applies to one right-hand side on a grid whose
// transform fits its dense tables and whose mode solves fit one warp per
// column (16 rows per lane).
bool small_applies(const ax_operator *op, int m) {
  return op->ws->small_path && m == 1 && op->nr <= kSmallMaxNr && op->nz <= kSmallMaxNz &&
         (long long)op->nr * op->nz <= kSmallMaxN && op->cstride == 0;
}

// Runs it from the state sc_start left (r = phi - A x in r64); or, with f
// (dense, device), the whole solve: phi, r, x = 0 and the state are formed in
// the launch, u (dense, device) is written at its end, and info is filled.
int small_pcg_run(ax_operator *op, cudaStream_t s, const double *f = nullptr, double *u = nullptr,
                  double tol = 0.0, int max_iter = 0, ax_solve_info *info = nullptr) {
  Workspace *w = op->ws;
  int nch = 1;
  const int grid = small_pcg_grid(op->nr, op->nz, &nch);
  if (grid < 1) return AX_ERR_UNSUPPORTED;
  const double *F = dense_table(op->device, op->nz, op->bc_z);
  int *flag = tc_flag(op->device);
  if (!F || !flag) return AX_ERR_OOM;
  const size_t fe = field_elems(op);
  {
    std::lock_guard<std::recursive_mutex> lock(g_alloc_capture_mutex);
    if (!w->small_buf) AX_TRY(dalloc(&w->small_buf, 2 * fe));
    if (!w->small_bar) AX_TRY(dalloc(&w->small_bar, 2));
    if (!w->h_flag) AX_TRY(cudaMallocHost(&w->h_flag, sizeof(int)));
  }
  AX_TRY(cudaMemsetAsync(w->small_bar, 0, 2 * sizeof(unsigned), s));
  SmallPcgArgs a{};
  a.f = f;
  a.u = u;
  a.R = op->c64.R;
  a.tol2 = tol * tol;
  a.max_iter = max_iter;
  const Coef<double> &c = op->c64;
  a.CR = c.CR;
  a.CZ = c.CZ;
  a.W = c.W;
  a.IP = c.IP;
  a.E = c.E;
  a.F = F;
  a.Ft = F + (size_t)op->nz * op->nz;
  a.phi = w->phi64;
  a.x = w->x64;
  a.r = w->r64;
  a.r2 = w->small_buf;
  a.z = w->z64;
  a.pa = w->pa64;
  a.pb = w->pb64;
  a.q = w->q64;
  a.t = w->small_buf + fe;
  a.part = part_ptr(w, kPartA);
  a.bar = w->small_bar;
  a.st = w->st;
  a.nr = op->nr;
  a.nz = op->nz;
  a.pitch = op->pitch;
  a.pitchz = op->pitchz;
  a.nch = nch;
  a.err = flag;
  if (w->small_stall_test) {  // test of the expiry path (option "small_stall_test"), once
    a.stall = 1;
    a.polls = 1u << 12;
    w->small_stall_test = 0;
  }
  AX_TRY(launch_small_pcg(a, grid, s));
  // one synchronisation for the expiry flag and (whole solve) the state
  AX_TRY(cudaMemcpyAsync(w->h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (f) AX_TRY(cudaMemcpyAsync(w->h_st, w->st, sizeof(RhsState), cudaMemcpyDeviceToHost, s));
  AX_TRY(cudaStreamSynchronize(s));
  if (*w->h_flag) {
    AX_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    snprintf(g_last_error, sizeof(g_last_error), "a grid-barrier wait of the persistent small-grid solve expired");
    return AX_ERR_TIMEOUT;
  }
  if (!f) return AX_OK;
  const RhsState &h = w->h_st[0];
  int st = h.status;
  if (st == AX_OK && h.state != kDone) st = AX_ERR_NO_CONVERGENCE;
  if (info) {
    info[0].iters = h.iters;
    info[0].outer = 0;
    info[0].rel_res = h.bb > 0.0 ? std::sqrt(h.rr / h.bb) : 0.0;
    info[0].guess_accepted = 0;
    info[0].status = st;
  }
  return st;
}

template <typename T>
bool use_tc(const ax_operator *op) {
  return sizeof(T) == 4 && op->dst_tc != 0;
}

// Geometry of the split operand for `rows` rows per RHS.
struct SplitGeom {
  int mtiles, ktiles, kbe;
  size_t bytes_per_rhs;
};
SplitGeom split_geom(const ax_operator *op, int rows) {
  SplitGeom g;
  g.mtiles = dst_gemm_mtiles(rows);
  g.ktiles = dst_gemm_ktiles(op->nz);
  g.kbe = dst_gemm_kbe(op->nz);
  g.bytes_per_rhs = (size_t)g.mtiles * g.ktiles * kSplitTileBytes;
  return g;
}

// Tensor-core transform of `rows` rows per RHS: out = A S for the selected
// right-hand sides (A in the split layout; S the sine matrix, or for the
// zero-flux z boundary the forward cosine matrix on folded input or its
// inverse); with r, the (r, out) partials into `partial`.  With pa, pb the result is not stored but forms the next
// search direction p_new = out + beta p_old (and, with x, x += alpha p_old);
// see GemmDstArgs.
// FP32 mode-solve variant of the tensor-core path for m right-hand sides, and
// whether it is a pipelined one, which works on the row-scaled systems: the
// transforms around it then take the scaling D in their epilogues.
int tc_mode_variant(const ax_operator *op, int m) {
  return tridiag_effective(op->nr, op->tri_variant, m, op->c32.IPS != nullptr && op->c32.RS != nullptr);
}
bool tc_scaled(const ax_operator *op, int m) { return tc_mode_variant(op, m) >= 2; }
// The forward transform of a preconditioner application writes mode-major
// for the mode-solve kernel 14, when that layout fits the buffer it writes
// (m nr pitch floats: nz tpitch <= nr pitch) and its factor table exists.
bool tc_tr_mode(const ax_operator *op, int m) {
  return tc_mode_variant(op, m) == 14 && op->c32.IPST != nullptr && op->tpitch > 0 &&
         (long long)op->nz * op->tpitch <= (long long)op->nr * op->pitch;
}

// scaled: multiply every output row by D (the row scale of the pipelined mode
// solves); set for the two transforms of a preconditioner application
// exactly when tc_scaled(op, m).
void tc_transform(const ax_operator *op, int m, int rows, const unsigned char *A, bool inverse, float *out,
                  const RhsState *st, int mask, const float *r, double *partial, cudaStream_t s, int three = -1,
                  float *pa = nullptr, float *pb = nullptr, float *x = nullptr, bool scaled = false,
                  bool tout = false, const int *gate = nullptr) {
  GemmDstArgs g{};
  g.gate = gate;
  if (tout) {  // mode-major output for the mode-solve kernel 14 (forward only)
    g.tout = 1;
    g.tpitch = op->tpitch;
  }
  if (scaled) {
    g.rowscale = op->c32.RS;
    g.rsstride = op->estride;
  }
  g.pa = pa;
  g.pb = pb;
  g.x = x;
  g.polls = 0;
  g.stall_at = -1;
  if (op->ws->tc_stall_test) {  // test of the expiry path (option "tc_stall_test"), once
    g.polls = 1u << 14;
    g.stall_at = 0;
    op->ws->tc_stall_test = 0;
  }
  const int kind = op->bc_z == 1 ? (inverse ? kTableCosInverse : kTableCosForward) : kTableSine;
  g.cosfwd = kind == kTableCosForward;
  g.A = A;
  g.out = out;
  g.SB = tc_table(op->device, op->nz, kind);
  g.n = op->nz;
  g.nr = rows;
  g.pitch = op->pitch;
  g.field = (long long)rows * op->pitch;
  g.m = m;
  g.mtiles = dst_gemm_mtiles(rows);
  g.ntiles = dst_gemm_ntiles(op->nz);
  g.ktiles = dst_gemm_ktiles(op->nz);
  g.kbe = dst_gemm_kbe(op->nz);
  g.three = three >= 0 ? three : (op->dst_tc == 1 ? 1 : 0);
  g.r = r;
  g.partial = partial;
  g.st = st;
  g.mask = mask;
  g.err = tc_flag(op->device);
  launch_dst_gemm(g, s);
}

// FP32 field -> split operand (rows per RHS `rows`).
void tc_split(const ax_operator *op, int m, int rows, const float *in, unsigned char *split, const RhsState *st,
              int mask, cudaStream_t s, const int *gate = nullptr) {
  const SplitGeom g = split_geom(op, rows);
  // kCheck (the replacement step's recomputation of z) selects a right-hand
  // side rarely: fewer CTAs per right-hand side, so that the usual launch in
  // which none is selected ends soon (the CTAs loop over the rows)
  const int bx = mask == kCheck ? std::min(update_blocks(rows, op->nz), 8) : update_blocks(rows, op->nz);
  note_launch();
  split_field<<<dim3(bx, m), 256, 0, s>>>(in, rows, op->nz, op->pitch,
                                                                   (size_t)rows * op->pitch,
                                                      g.mtiles, g.ktiles, g.kbe, split, st, mask, op->bc_z == 1,
                                                      gate);
}

// Mode solves z -> split operand (the tile kernel writes it directly; otherwise
// through the FP32 buffer tmp).
// With `prz` (tile kernel only), the mode solves also form the partials of
// (rhat, yhat), equal to (r, z) up to the rounding of the split input: S is
// symmetric, so (r, S yhat) = (S r, yhat).
void tc_mode_solve(const ax_operator *op, int m, const float *z, float *tmp, unsigned char *split,
                   const RhsState *st, int mask, cudaStream_t s, double *prz = nullptr, const int *gate = nullptr) {
  const SplitGeom g = split_geom(op, op->nr);
  TriArgs<float> t = tri_args<float>(op, m, z, tmp, st, mask);
  t.variant = tc_mode_variant(op, m);
  t.prescaled = tc_scaled(op, m);
  if (tc_tr_mode(op, m)) {  // z is mode-major (the forward transform wrote it so)
    t.IPST = op->c32.IPST;
    t.tcstride = op->cstride != 0 ? (long long)op->nz * op->tpitch : 0;
    t.tpitch = op->tpitch;
    if (mask == kCheck) {  // rarely selected: a short grid, gated where the caller keeps the count
      t.short_grid = 1;
      t.gate = gate;
    }
  } else if (t.variant == 14) {
    t.variant = 9;
  }
  if (tridiag_split_ok(op->nr)) {
    t.split = split;
    t.split_mtiles = g.mtiles;
    t.split_ktiles = g.ktiles;
    t.split_kbe = g.kbe;
    t.partial = prz;
    launch_tridiag<float>(t, s);
  } else {
    launch_tridiag<float>(t, s);
    tc_split(op, m, op->nr, tmp, split, st, mask, s, gate);
  }
}

// Where the (r, z) partials of the tensor-core path come from: the mode solves
// (one per column group of the FP32 tile kernel) when it runs, else the
// inverse transform.
bool tc_dot_in_modes(const ax_operator *op) { return tridiag_split_ok(op->nr); }

// Number of (r, z) partial slots per RHS that precond_apply writes for m
// right-hand sides.
template <typename T>
int precond_partials(const ax_operator *op, int m) {
  if (use_tc<T>(op)) {
    if (!tc_dot_in_modes(op)) return dst_gemm_mtiles(op->nr) * dst_gemm_ntiles(op->nz);
    const int cols = tridiag_reg_cols(op->nr, tc_mode_variant(op, m));
    return (op->nz + cols - 1) / cols;
  }
  return dst_blocks(op, op->nr, (int)sizeof(T));
}

// z = B^-1 r for selected RHS, with (r, z) partials into `prz`.  The
// tensor-core path goes through the workspace's split operand (and tmp when
// the mode solves cannot write it directly); the FFT path works in place in z.
template <typename T>
void precond_apply(const ax_operator *op, int m, const T *r, T *z, const RhsState *st, int mask, double *prz,
                   cudaStream_t s, T *tmp = nullptr) {
  if constexpr (sizeof(T) == 4) {
    if (use_tc<T>(op) && tmp != nullptr) {
      unsigned char *sp = op->ws->split;
      const bool dm = tc_dot_in_modes(op);
      tc_split(op, m, op->nr, r, sp, st, mask, s);
      const bool sc = tc_scaled(op, m);
      tc_transform(op, m, op->nr, sp, false, z, st, mask, nullptr, nullptr, s, -1, nullptr, nullptr, nullptr, sc,
                   tc_tr_mode(op, m));
      tc_mode_solve(op, m, z, tmp, sp, st, mask, s, dm ? prz : nullptr);
      tc_transform(op, m, op->nr, sp, true, z, st, mask, dm ? nullptr : r, dm ? nullptr : prz, s, -1, nullptr, nullptr,
                   nullptr, sc);
      return;
    }
  }
  DstArgs<T> f = dst_args<T>(op, m, op->nr, st, mask);
  f.in = r;
  f.out = z;
  launch_dst<T>(kDstPlain, f, s);
  launch_tridiag<T>(tri_args<T>(op, m, z, z, st, mask), s);
  DstArgs<T> b = dst_args<T>(op, m, op->nr, st, mask);
  b.in = z;
  b.out = z;
  b.r = const_cast<T *>(r);
  b.partial = prz;
  launch_dst<T>(kDstPcgInverse, b, s);
}

// ---------------------------------------------------------------------------
// PCG (generic over the working precision T)
// ---------------------------------------------------------------------------
template <typename T>
struct PcgVecs {
  T *x, *r, *pa, *pb, *q, *z;
};

// Whether the mixed PCG loop runs the fused tensor-core iteration: the inverse
// transform's epilogue forms the next direction p = z + beta p and updates x
// (beta is known before it because the mode solves give the (r, z) partials),
// so z is never stored, the stencil reads p alone and the update pass only r.
bool tc_fused(const ax_operator *op) { return use_tc<float>(op) && tc_dot_in_modes(op) && !op->ws->tc_unfused; }

// One PCG iteration for the right-hand sides in kActive.  fused (FP32
// tensor-core path with tc_fused only): p was formed by the previous
// iteration's inverse transform (or the start), see tc_fused.
template <typename T>
void pcg_iteration(const ax_operator *op, int m, const PcgVecs<T> &v, RhsState *st, Workspace *w,
                   int on_converge, cudaStream_t s, double units = 0.0, bool fused = false) {
  const int V = VecT<T>::n;
  const int nbs = stencil_blocks_per_rhs(op->nr, op->nz, V);
  const int nbd = dst_blocks(op, op->nr, (int)sizeof(T));
  double *pq = part_ptr(w, kPartA), *prr = part_ptr(w, kPartB), *prz = part_ptr(w, kPartC);
  StencilArgs<T> sa = stencil_args<T>(op, m, st, kActive);
  sa.in = v.z;
  sa.pa = v.pa;
  sa.pb = v.pb;
  sa.out = v.q;
  sa.partial = pq;
  {
    ProfScope ps(w, kProfStencil, units, s);
    launch_stencil<T>(fused ? kStencilPcgP : kStencilPcg, sa, s);
  }
  {
    ProfScope ps(w, kProfScalar, 0.0, s);
    note_launch();
    sc_alpha<<<m, 32, 0, s>>>(st, pq, nbs);
  }
  if constexpr (sizeof(T) == 4) {
    if (use_tc<T>(op)) {
      // update pass (r written split too), transform r -> z, mode solves
      // z -> split, inverse transform split -> z with the (r, z) partials
      const SplitGeom g = split_geom(op, op->nr);
      unsigned char *sp = w->split;
      {
        ProfScope ps(w, kProfUpdate, units, s);
        note_launch();
        pcg_update<<<dim3(update_blocks(op->nr, op->nz), m), 256, 0, s>>>(fused ? nullptr : v.x, v.r, v.q, v.pa,
                                                                           v.pb, op->nr,
                                                          op->nz, op->pitch, field_elems(op), g.mtiles, g.ktiles,
                                                          g.kbe, sp, st, kActive, prr, op->bc_z == 1);
        if (op->bc_z == 1) tc_split(op, m, op->nr, v.r, sp, st, kActive, s);
      }
      const bool sc = tc_scaled(op, m);
      {
        ProfScope ps(w, kProfDstFwd, units, s);
        tc_transform(op, m, op->nr, sp, false, v.z, st, kActive, nullptr, nullptr, s, -1, nullptr, nullptr, nullptr, sc,
                     tc_tr_mode(op, m));
      }
      {
        ProfScope ps(w, kProfScalar, 0.0, s);
        note_launch();
        sc_after_update<<<m, 32, 0, s>>>(st, prr, update_blocks(op->nr, op->nz), on_converge);
      }
      const bool dm = tc_dot_in_modes(op);
      {
        ProfScope ps(w, kProfTridiag, units, s);
        tc_mode_solve(op, m, v.z, v.q, sp, st, kActive, s, dm ? prz : nullptr);
      }
      if (fused) {
        {
          ProfScope ps(w, kProfScalar, 0.0, s);
          note_launch();
          sc_beta<<<m, 32, 0, s>>>(st, prz, precond_partials<T>(op, m), kActive, kActive);
        }
        ProfScope ps(w, kProfDstInv, units, s);
        tc_transform(op, m, op->nr, sp, true, v.z, st, kActive, nullptr, nullptr, s, -1, v.pa, v.pb, v.x, sc);
        return;
      }
      {
        ProfScope ps(w, kProfDstInv, units, s);
        tc_transform(op, m, op->nr, sp, true, v.z, st, kActive, dm ? nullptr : v.r, dm ? nullptr : prz, s, -1, nullptr,
                     nullptr, nullptr, sc);
      }
      {
        ProfScope ps(w, kProfScalar, 0.0, s);
        note_launch();
        sc_beta<<<m, 32, 0, s>>>(st, prz, precond_partials<T>(op, m), kActive, kActive);
      }
      return;
    }
  }
  DstArgs<T> f = dst_args<T>(op, m, op->nr, st, kActive);
  f.in = v.q;
  f.out = v.z;
  f.x = v.x;
  f.r = v.r;
  f.pa = v.pa;
  f.pb = v.pb;
  f.partial = prr;
  { ProfScope ps(w, kProfDstFwd, units, s); launch_dst<T>(kDstPcgForward, f, s); }
  {
    ProfScope ps(w, kProfScalar, 0.0, s);
    note_launch();
    sc_after_update<<<m, 32, 0, s>>>(st, prr, nbd, on_converge);
  }
  { ProfScope ps(w, kProfTridiag, units, s); launch_tridiag<T>(tri_args<T>(op, m, v.z, v.z, st, kActive), s); }
  DstArgs<T> b = dst_args<T>(op, m, op->nr, st, kActive);
  b.in = v.z;
  b.out = v.z;
  b.r = v.r;
  b.partial = prz;
  { ProfScope ps(w, kProfDstInv, units, s); launch_dst<T>(kDstPcgInverse, b, s); }
  {
    ProfScope ps(w, kProfScalar, 0.0, s);
    note_launch();
    sc_beta<<<m, 32, 0, s>>>(st, prz, nbd, kActive, kActive);
  }
}

// Chebyshev step for RHS in kActive: res = A y - phi, test, ybar = y - tau
// B^-1 res, y_{k+1} = a ybar + (1 - a) y_{k-1} (written over y_{k-1}; the
// caller swaps the two buffers by parity).
template <typename T>
struct ChebVecs {
  T *ya, *yb, *res, *phi;
};

template <typename T>
void cheb_iteration(const ax_operator *op, int m, const ChebVecs<T> &v, RhsState *st, Workspace *w,
                    int on_converge, int parity, cudaStream_t s, bool check = true) {
  const int V = VecT<T>::n;
  const int nbs = stencil_blocks_per_rhs(op->nr, op->nz, V);
  double *prr = part_ptr(w, kPartB);
  T *y = parity ? v.yb : v.ya;
  T *yprev = parity ? v.ya : v.yb;
  StencilArgs<T> sa = stencil_args<T>(op, m, st, kActive);
  sa.in = y;
  sa.out = v.res;
  sa.phi = v.phi;
  sa.partial = check ? prr : nullptr;  // no reduction on the steps between checks
  launch_stencil<T>(kStencilCheb, sa, s);
  note_launch();
  sc_cheb<<<m, 32, 0, s>>>(st, prr, nbs, w->chp, on_converge, check ? 1 : 0);
  DstArgs<T> f = dst_args<T>(op, m, op->nr, st, kActive);
  f.in = v.res;
  f.out = v.res;
  launch_dst<T>(kDstPlain, f, s);
  launch_tridiag<T>(tri_args<T>(op, m, v.res, v.res, st, kActive), s);
  DstArgs<T> b = dst_args<T>(op, m, op->nr, st, kActive);
  b.in = v.res;
  b.y = y;
  b.yprev = yprev;
  b.chp = w->chp;
  launch_dst<T>(kDstChebInverse, b, s);
}

int read_states(Workspace *w, const RhsState *dev, int m, cudaStream_t s, RhsState *host) {
  AX_TRY(cudaMemcpyAsync(host, dev, sizeof(RhsState) * m, cudaMemcpyDeviceToHost, s));
  AX_TRY(cudaStreamSynchronize(s));
  return AX_OK;
}

// Completion times: right-hand sides whose top-level state (just read into h)
// is final get the current time, once.
void lat_mark(Workspace *w, const RhsState *h, int m) {
  if (!w->lat_track) return;
  if ((int)w->lat_ms.size() < m) w->lat_ms.resize(m, -1.0);
  const double now = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - w->lat_t0).count();
  for (int i = 0; i < m; ++i)
    if (w->lat_ms[i] < 0.0 && (h[i].state == kDone || h[i].state == kFailed)) w->lat_ms[i] = now;
}

// Runs `iters` captured iterations of `body` on stream s (graph cached by key).
template <typename F>
int run_graph(Workspace *w, GraphCache &g, int key, cudaStream_t s, F body) {
  if (g.exec == nullptr || g.key != key) {
    std::lock_guard<std::recursive_mutex> lock(g_alloc_capture_mutex);
    free_graph(g);
    cudaGraph_t graph = nullptr;
    AX_TRY(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeRelaxed));
    g_capturing = true;
    body(w->cap);
    g_capturing = false;
    cudaError_t e = cudaStreamEndCapture(w->cap, &graph);
    if (e != cudaSuccess) return status_from_cuda(e);
    g.nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &g.nodes);
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g.exec = nullptr;
      return status_from_cuda(e);
    }
    g.key = key;
  }
  AX_TRY(cudaGraphLaunch(g.exec, s));
  __atomic_add_fetch(&g_launches, (long long)g.nodes, __ATOMIC_RELAXED);
  return AX_OK;
}

int count_state(const RhsState *h, int m, int state) {
  int c = 0;
  for (int i = 0; i < m; ++i) c += (h[i].state == state);
  return c;
}

bool any_state(const RhsState *h, int m, int state) {
  for (int i = 0; i < m; ++i)
    if (h[i].state == state) return true;
  return false;
}

// PCG for the vectors v with right-hand side phi (in v.r on entry as the
// residual).  Assumes st has been started (sc_start) and x holds the start.
// If `true_check`, right-hand sides whose recursive residual passes get an
// FP64-exact test with the true residual phi - A x (plain method); otherwise
// they finish at once (inner solves).
template <typename T>
int pcg_loop(ax_operator *op, int m, const PcgVecs<T> &v, const T *phi, RhsState *st, GraphCache &g, bool true_check,
             cudaStream_t s) {
  Workspace *w = op->ws;
  const int V = VecT<T>::n;
  const int nbs = stencil_blocks_per_rhs(op->nr, op->nz, V);
  const int nbd = precond_partials<T>(op, m);
  // z = B^-1 r, rho = (r, z), p = 0 so that p_1 = z
  precond_apply<T>(op, m, v.r, v.z, st, kActive, part_ptr(w, kPartC), s, v.q);
  note_launch();
  sc_rho_init<<<m, 32, 0, s>>>(st, part_ptr(w, kPartC), nbd, kActive);
  AX_TRY(cudaMemsetAsync(v.pa, 0, sizeof(T) * field_elems(op) * m, s));
  AX_CHECK_LAUNCH();
  const int on_conv = true_check ? kCheck : kDone;
  const int K = w->graph_iters;
  const int key = m * 4 + (true_check ? 1 : 0);
  // True-residual test of the right-hand sides in kCheck, inside the graph
  // after every iteration (the kernels return at once for the others).
  auto check_step = [&](cudaStream_t ss) {
    if (!true_check) return;
    StencilArgs<T> ra = stencil_args<T>(op, m, st, kCheck);
    ra.in = v.x;
    ra.phi = phi;
    ra.out_res = v.r;
    ra.partial = part_ptr(w, kPartB);
    launch_stencil<T>(kStencilResidual, ra, ss);
    note_launch();
    sc_true_check<<<m, 32, 0, ss>>>(st, part_ptr(w, kPartB), nbs);
    precond_apply<T>(op, m, v.r, v.z, st, kCheck, part_ptr(w, kPartC), ss, v.q);
    note_launch();
    sc_beta<<<m, 32, 0, ss>>>(st, part_ptr(w, kPartC), nbd, kCheck, kActive);
  };
  const double per_rhs = (double)op->nr * op->nz;
  for (int guard = 0; guard < 1000000; ++guard) {
    int rc = AX_OK;
    RhsState *h = w->h_st;
    if (w->profile) {
      // one iteration at a time, so every launch is timed with the true
      // number of right-hand sides it works on
      if ((rc = read_states(w, st, m, s, h)) != AX_OK) return rc;
      pcg_iteration<T>(op, m, v, st, w, on_conv, s, per_rhs * count_state(h, m, kActive));
      check_step(s);
      AX_CHECK_LAUNCH();
    } else {
      rc = run_graph(w, g, key, s, [&](cudaStream_t cs) {
        for (int k = 0; k < K; ++k) {
          pcg_iteration<T>(op, m, v, st, w, on_conv, cs);
          check_step(cs);
        }
      });
    }
    if (rc != AX_OK) return rc;
    if ((rc = read_states(w, st, m, s, h)) != AX_OK) return rc;
    if (true_check) lat_mark(w, h, m);
    if (!any_state(h, m, kActive) && !any_state(h, m, kCheck)) break;
  }
  return AX_OK;
}

// ---------------------------------------------------------------------------
// Lanczos estimate of the Chebyshev bounds (Eq. energy_rel).  The face-wise
// bounds min / max of kappa / kappa~ and q / q~ are rigorous, but with
// q_min = 0 < q_max the lower one is 0, which leaves the Chebyshev iteration
// without a spectral interval.  There the bounds come from `cheb_steps` PCG
// steps (FP32 kernels, every right-hand side at once, from zero): the
// coefficients alpha_j, beta_j are the Lanczos process of B^-1 A in the
// B-inner product, with the tridiagonal matrix (Saad, "Iterative methods for
// sparse linear systems", 2nd ed., Section 6.7.3)
//   T[j][j] = 1 / alpha_j + beta_{j-1} / alpha_{j-1},  T[j][j+1] = sqrt(beta_j) / alpha_j,
// whose extreme eigenvalues (Ritz values) approach those of B^-1 A from
// inside; they are widened by `cheb_widen` (gamma_1 = (1 - w) theta_min,
// gamma_2 = (1 + w) theta_max).  Cached per operator and right-hand side.
// ---------------------------------------------------------------------------
bool cheb_uses_lanczos(const ax_operator *op, double face_gamma1) {
  const int mode = op->ws->cheb_bounds;
  return mode == 1 || (mode == -1 && !(face_gamma1 > 0.0));
}

// The estimate's steps of a right-hand side stop once its residual has fallen
// to 1e-6 of ||phi|| (thresh2 = rel2 ||phi||^2; pbb: the ||phi||^2 partials):
// the FP32 steps reach their rounding floor near 1e-7, the coefficients of
// later steps come from rounding noise, and their Ritz values need not lie in
// the spectrum of B^-1 A (with 40 steps one batched instance that PCG solves
// in 9 iterations got bounds on which Chebyshev diverged).
__global__ void sc_lanczos_stop(RhsState *st, const double *pbb, int nbb, double rel2) {
  const int m = blockIdx.x;
  const double bb = reduce_part(pbb + (size_t)m * kPartialStride, nbb);
  if (threadIdx.x == 0) st[m].thresh2 = rel2 * bb;
}

// hist[m][2 k]: (alpha_j, beta_j) of step j of right-hand side m; an alpha of
// 0 marks the end (the step did not run, or broke down).
__global__ void sc_record_lanczos(const RhsState *st, double *hist, int m, int j, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const RhsState s = st[i];
  double *h = hist + (size_t)i * 2 * k;
  const bool ran = (s.state == kActive || s.state == kDone) && s.iters == j + 1 && isfinite(s.alpha);
  h[2 * j] = ran ? s.alpha : 0.0;
  h[2 * j + 1] = (ran && s.state == kActive && isfinite(s.beta)) ? s.beta : 0.0;
}

// Number of eigenvalues below x of the symmetric tridiagonal (d, e) (Sturm
// count of the LDL^T pivots; Golub and Van Loan, Section 8.4).
static int sturm_count(const std::vector<double> &d, const std::vector<double> &e, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t j = 0; j < d.size(); ++j) {
    const double e2 = j ? e[j - 1] * e[j - 1] : 0.0;
    q = d[j] - x - (j ? e2 / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Smallest and largest eigenvalue of the symmetric tridiagonal (d, e) by
// bisection on the Gershgorin interval.
static void tridiag_extremes(const std::vector<double> &d, const std::vector<double> &e, double &lo, double &hi) {
  const size_t n = d.size();
  double a = d[0], b = d[0];
  for (size_t j = 0; j < n; ++j) {
    const double r = (j ? std::fabs(e[j - 1]) : 0.0) + (j + 1 < n ? std::fabs(e[j]) : 0.0);
    a = std::min(a, d[j] - r);
    b = std::max(b, d[j] + r);
  }
  double x0 = a, x1 = b;  // smallest: count(x) >= 1
  for (int it = 0; it < 200 && x1 - x0 > 1e-15 * std::max(std::fabs(x0), std::fabs(x1)); ++it) {
    const double mid = 0.5 * (x0 + x1);
    if (sturm_count(d, e, mid) >= 1) x1 = mid; else x0 = mid;
  }
  lo = 0.5 * (x0 + x1);
  x0 = a, x1 = b;  // largest: count(x) >= n
  for (int it = 0; it < 200 && x1 - x0 > 1e-15 * std::max(std::fabs(x0), std::fabs(x1)); ++it) {
    const double mid = 0.5 * (x0 + x1);
    if (sturm_count(d, e, mid) >= (int)n) x1 = mid; else x0 = mid;
  }
  hi = 0.5 * (x0 + x1);
}

// Runs the PCG steps of the estimate on phi64 (already formed) and caches the
// bounds of every right-hand side in op->lz_g1 / lz_g2; `steps` (host
// vector, may be null) receives the steps each right-hand side ran.  Uses
// the FP32 vectors and the right-hand-side states (before the solve sets them).
int cheb_estimate(ax_operator *op, int m, cudaStream_t s, std::vector<int> *steps) {
  Workspace *w = op->ws;
  const int k = w->cheb_steps;
  const size_t field = field_elems(op);
  int rc;
  if ((rc = ensure_vec32(op, m, false)) != AX_OK) return rc;
  if (op->dst_tc) {
    if ((rc = ensure_split(op, (size_t)m * split_geom(op, op->nr).bytes_per_rhs)) != AX_OK) return rc;
    const bool cz = op->bc_z == 1;
    if (!tc_table(op->device, op->nz, cz ? kTableCosForward : kTableSine) ||
        !tc_table(op->device, op->nz, cz ? kTableCosInverse : kTableSine) || !tc_flag(op->device))
      return AX_ERR_OOM;
  }
  double *hist = nullptr;
  AX_TRY(dalloc(&hist, (size_t)m * 2 * k));
  struct Free { double *p; ~Free() { dfree(p); } } hold{hist};
  AX_TRY(cudaMemsetAsync(hist, 0, sizeof(double) * m * 2 * k, s));
  const size_t n = field * m;
  const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 65535);
  note_launch();
  to_precision<float><<<blocks, 256, 0, s>>>(w->phi64, w->r32, n);
  AX_TRY(cudaMemsetAsync(w->x32, 0, sizeof(float) * n, s));
  // states: every right-hand side active, max_iter = k, the threshold set
  // below (sc_lanczos_stop)
  {
    std::vector<RhsState> init(m);
    for (int i = 0; i < m; ++i) {
      std::memset(&init[i], 0, sizeof(RhsState));
      init[i].state = kActive;
      init[i].max_iter = k;
      init[i].thresh2 = 0.0;
      init[i].bb = 1.0;
    }
    AX_TRY(cudaMemcpyAsync(w->st, init.data(), sizeof(RhsState) * m, cudaMemcpyHostToDevice, s));
  }
  // ||phi||^2 partials of ax_solve (prep_rhs / phi_norm2; r starts as phi)
  note_launch();
  sc_lanczos_stop<<<m, 32, 0, s>>>(w->st, part_ptr(w, kPartD), (op->nr + 15) / 16, 1e-12);
  PcgVecs<float> v{w->x32, w->r32, w->pa32, w->pb32, w->q32, w->z32};
  const int nbd = precond_partials<float>(op, m);
  precond_apply<float>(op, m, v.r, v.z, w->st, kActive, part_ptr(w, kPartC), s, v.q);
  note_launch();
  sc_rho_init<<<m, 32, 0, s>>>(w->st, part_ptr(w, kPartC), nbd, kActive);
  AX_TRY(cudaMemsetAsync(v.pa, 0, sizeof(float) * n, s));
  for (int j = 0; j < k; ++j) {
    pcg_iteration<float>(op, m, v, w->st, w, kDone, s);
    note_launch();
    sc_record_lanczos<<<(m + 31) / 32, 32, 0, s>>>(w->st, hist, m, j, k);
  }
  AX_CHECK_LAUNCH();
  std::vector<double> h((size_t)m * 2 * k);
  AX_TRY(cudaMemcpyAsync(h.data(), hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  AX_TRY(cudaStreamSynchronize(s));
  op->lz_g1.assign(m, 0.0);
  op->lz_g2.assign(m, 0.0);
  if (steps) steps->assign(m, 0);
  const double wd = w->cheb_widen;
  for (int i = 0; i < m; ++i) {
    const double *hi = &h[(size_t)i * 2 * k];
    int cnt = 0;
    while (cnt < k && hi[2 * cnt] > 0.0) ++cnt;
    // the last beta is only needed when a further step follows
    std::vector<double> d(cnt), e(cnt > 0 ? cnt - 1 : 0);
    bool ok = cnt > 0;
    for (int j = 0; j < cnt && ok; ++j) {
      d[j] = 1.0 / hi[2 * j] + (j ? hi[2 * j - 1] / hi[2 * j - 2] : 0.0);
      if (j + 1 < cnt) {
        ok = hi[2 * j + 1] > 0.0;
        e[j] = std::sqrt(std::max(hi[2 * j + 1], 0.0)) / hi[2 * j];
      }
    }
    const bool mem = (size_t)i < op->mgamma1.size();
    double g1 = mem ? op->mgamma1[i] : op->gamma1, g2 = mem ? op->mgamma2[i] : op->gamma2;
    if (ok) {
      double lo, hi2;
      tridiag_extremes(d, e, lo, hi2);
      if (lo > 0.0 && std::isfinite(hi2) && hi2 >= lo) {
        g1 = (1.0 - wd) * lo;
        g2 = (1.0 + wd) * hi2;
      }
    }
    if (!(g1 > 0.0)) g1 = 1e-3 * g2;  // no usable estimate: a wide interval
    op->lz_g1[i] = g1;
    op->lz_g2[i] = g2;
    if (steps) (*steps)[i] = cnt;
  }
  if (op->mgamma1.empty()) {
    // one operator: the spectrum is that of every right-hand side, so all of
    // them take the widest interval found
    const double g1 = *std::min_element(op->lz_g1.begin(), op->lz_g1.end());
    const double g2 = *std::max_element(op->lz_g2.begin(), op->lz_g2.end());
    op->lz_g1.assign(m, g1);
    op->lz_g2.assign(m, g2);
  }
  op->lz_m = m;
  return AX_OK;
}

// Inner Chebyshev solves of known length: right-hand side i runs exactly
// n[i] steps (the residual test is off; the FP64 outer residual decides).
__global__ void sc_cheb_fixed(RhsState *st, const int *n, int m) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m || st[i].state != kActive) return;
  st[i].max_iter = n[i];
  st[i].thresh2 = -1.0;
}

// Smallest n >= 1 with the Chebyshev bound 2 rho1^n / (1 + rho1^(2n)) <= eta
// on the A-norm error (rho1 = (1 - sqrt xi) / (1 + sqrt xi), xi =
// gamma1 / gamma2), at most cap.
static int cheb_steps_for(double xi, double eta, int cap) {
  const double sx = std::sqrt(std::max(xi, 0.0)), rho1 = (1.0 - sx) / (1.0 + sx);
  double pn = 1.0;
  for (int n = 1; n <= cap; ++n) {
    pn *= rho1;
    if (2.0 * pn / (1.0 + pn * pn) <= eta) return n;
  }
  return cap;
}

// apriori_eta > 0 (the inner solves of AX_CHEB_MIXED): every active
// right-hand side runs the number of steps whose Chebyshev bound reaches
// apriori_eta, with no residual test on the way (the residual norm is formed
// on the last step of each graph replay only): no inner products at all.
// The residual an FP32 iteration recomputes as A y - phi stops falling at its
// rounding level (far above the inner tolerance for ill-conditioned A), so a
// residual test there never passes.
template <typename T>
int cheb_loop(ax_operator *op, int m, const ChebVecs<T> &v, RhsState *st, GraphCache &g, int on_conv, int *parity,
              cudaStream_t s, double apriori_eta = 0.0) {
  Workspace *w = op->ws;
  // tau_0 = 2 / (gamma1 + gamma2), rho_0 = (1 - xi) / (1 + xi), xi = gamma1 / gamma2,
  // per right-hand side: the members of a batched group have their own bounds
  {
    std::vector<double> par(2 * (size_t)m);
    for (int i = 0; i < m; ++i) {
      const bool mem = (size_t)i < op->mgamma1.size();
      double g1 = mem ? op->mgamma1[i] : op->gamma1, g2 = mem ? op->mgamma2[i] : op->gamma2;
      if (op->lz_m >= m && cheb_uses_lanczos(op, g1)) {
        g1 = op->lz_g1[i];
        g2 = op->lz_g2[i];
      }
      const double xi = g1 / g2, rho0 = (1.0 - xi) / (1.0 + xi);
      par[2 * i] = 2.0 / (g1 + g2);
      par[2 * i + 1] = rho0 * rho0;
    }
    AX_TRY(cudaMemcpyAsync(w->chp, par.data(), sizeof(double) * par.size(), cudaMemcpyHostToDevice, s));
    if (apriori_eta > 0.0) {
      std::vector<int> n(m);
      for (int i = 0; i < m; ++i) {
        const double rho0 = std::sqrt(par[2 * i + 1]), xi = (1.0 - rho0) / (1.0 + rho0);
        n[i] = cheb_steps_for(xi, apriori_eta, w->inner_max);
      }
      int *dn = reinterpret_cast<int *>(part_ptr(w, kPartD));  // free at this point of the solve
      AX_TRY(cudaMemcpyAsync(dn, n.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
      note_launch();
      sc_cheb_fixed<<<(m + 31) / 32, 32, 0, s>>>(st, dn, m);
    }
    AX_TRY(cudaStreamSynchronize(s));
  }
  const int K = 2 * std::max(1, w->graph_iters / 2);  // even: the buffer roles repeat
  const int key = m * 4 + 2 + (on_conv == kDone ? 1 : 0) + (*parity << 20) + (apriori_eta > 0.0 ? 1 << 21 : 0);
  for (int guard = 0; guard < 1000000; ++guard) {
    // the residual norm every cheb_check-th step, and on the last step of
    // each replay (where the host reads the states)
    const int ck = apriori_eta > 0.0 ? K : w->cheb_check;
    int rc = run_graph(w, g, key, s, [&](cudaStream_t cs) {
      for (int k = 0; k < K; ++k)
        cheb_iteration<T>(op, m, v, st, w, on_conv, (*parity + k) & 1, cs, (k + 1) % ck == 0 || k == K - 1);
    });
    if (rc != AX_OK) return rc;
    RhsState *h = w->h_st;
    if ((rc = read_states(w, st, m, s, h)) != AX_OK) return rc;
    if (apriori_eta == 0.0) lat_mark(w, h, m);  // the top-level Chebyshev (not an inner solve)
    if (!any_state(h, m, kActive)) break;
  }
  return AX_OK;
}

// Stores sum(partials) of each right-hand side into gate_phi (which = 0) or
// gate_res (which = 1).
__global__ void sc_store_gate(RhsState *st, const double *p, int nb, int which) {
  const int m = blockIdx.x;
  const double v = reduce_part(p + (size_t)m * kPartialStride, nb);
  if (threadIdx.x == 0) {
    if (which == 0) st[m].gate_phi = v;
    else st[m].gate_res = v;
  }
}

// Initial-guess gate.  CG reduces the error in the energy norm, and a learned
// guess is typically close to the solution in that norm while its small
// high-frequency errors make the plain residual norm large; so the guess of a
// right-hand side is kept only if its preconditioned residual norm
// (r0, B^-1 r0) is below that of the zero start, (phi, B^-1 phi) (both the
// energy norm of the start error in the metric of B^-1 A).  Rejected ones
// restart from zero; `restart` re-runs the residual and start kernels for all
// right-hand sides.  phiT and r0T hold phi and the guess residual in the
// working precision; zbuf and tmp are scratch.  accepted[i] = 1 if kept.
template <typename T, typename F>
int gate_guess(ax_operator *op, int m, RhsState *st, const T *phiT, const T *r0T, T *zbuf, T *tmp,
               std::vector<int> &accepted, cudaStream_t s, F restart) {
  Workspace *w = op->ws;
  const int nbd = precond_partials<T>(op, m);
  precond_apply<T>(op, m, phiT, zbuf, st, -1, part_ptr(w, kPartC), s, tmp);
  note_launch();
  sc_store_gate<<<m, 32, 0, s>>>(st, part_ptr(w, kPartC), nbd, 0);
  precond_apply<T>(op, m, r0T, zbuf, st, -1, part_ptr(w, kPartC), s, tmp);
  note_launch();
  sc_store_gate<<<m, 32, 0, s>>>(st, part_ptr(w, kPartC), nbd, 1);
  AX_CHECK_LAUNCH();
  int rc = read_states(w, st, m, s, w->h_st);
  if (rc != AX_OK) return rc;
  const size_t field = field_elems(op);
  bool any = false;
  for (int i = 0; i < m; ++i) {
    const RhsState &h = w->h_st[i];
    const bool ok = std::isfinite(h.gate_res) && std::isfinite(h.rr) && h.gate_res < h.gate_phi;
    accepted[i] = ok ? 1 : 0;
    if (!ok) {
      any = true;
      AX_TRY(cudaMemsetAsync(w->x64 + (size_t)i * field, 0, field * sizeof(double), s));
    }
  }
  if (any) restart();
  AX_CHECK_LAUNCH();
  return AX_OK;
}

// Mixed precision PCG with residual replacement.  The iteration runs in FP32
// (x32 holds the correction accumulated since the last replacement); the
// iterate lives in double-float (xh + xl).  When a right-hand side's recursive
// residual passes its threshold it finishes the iteration (z and beta from the
// recursive residual), then x += x32 and the true residual phi - A x
// (double-float) replaces r; the next iteration continues from it with the
// same search direction.  It stops when the true residual meets tol.
int pcg_mixed_loop(ax_operator *op, int m, double tol, double delta, int max_iter, bool check_guess,
                   std::vector<int> &accepted, cudaStream_t s) {
  Workspace *w = op->ws;
  RhsState *st = w->st;
  const size_t field = field_elems(op);
  const int nbdf = residual_df_blocks(op->nr, op->nz);
  const int nbf = (op->nr + 15) / 16;
  const int nbd = precond_partials<float>(op, m);
  PcgVecs<float> v{w->x32, w->r32, w->pa32, w->pb32, w->q32, w->z32};
  const size_t nall = field * m;
  const unsigned cblocks = (unsigned)std::min<size_t>((nall + 255) / 256, 65535);
  // up to ~8k CTAs in all for the replacement fold (see fold_df): many per
  // right-hand side, since only the few that are due at a step do work
  const unsigned fold_x = (unsigned)std::max<size_t>(
      1, std::min<size_t>((field / 4 + 255) / 256, (size_t)std::max(16, 8192 / std::max(1, m))));
  const dim3 zg(fold_x, m);
  // The true residual phi - A x in double-float (x and phi as FP32 pairs, the
  // FP64 coefficients as FP32 + low part): FP32 arithmetic throughout.
  auto residual64 = [&](int mask, cudaStream_t ss) {
    DfResidualArgs ra{};
    ra.CRh = op->c32.CR; ra.CRl = op->c32.CRl;
    ra.CZh = op->c32.CZ; ra.CZl = op->c32.CZl;
    ra.Wh = op->c32.W; ra.Wl = op->c32.Wl;
    ra.cstride = op->cstride;
    ra.czstride = op->czstride;
    ra.nr = op->nr; ra.nz = op->nz; ra.pitch = op->pitch; ra.pitchz = op->pitchz;
    ra.field = (long long)field;
    ra.m = m;
    ra.xh = w->xh; ra.xl = w->xl; ra.ph = w->phh; ra.pl = w->phl;
    ra.r32 = w->r32;
    ra.st = st;
    ra.mask = mask;
    ra.partial = part_ptr(w, kPartB);
    ProfScope ps(w, kProfOuter, (double)op->nr * op->nz * m, ss);
    launch_residual_df(ra, ss);
  };
  auto start = [&]() {
    note_launch();
    to_df<<<cblocks, 256, 0, s>>>(w->x64, w->xh, w->xl, nall);
    residual64(-1, s);
    note_launch();
    sc_mixed_start<<<m, 32, 0, s>>>(st, part_ptr(w, kPartB), nbdf, part_ptr(w, kPartD), nbf, tol * tol,
                                    delta * delta, max_iter);
  };
  note_launch();
  to_df<<<cblocks, 256, 0, s>>>(w->phi64, w->phh, w->phl, nall);
  AX_TRY(cudaMemsetAsync(w->chk, 0, 2 * sizeof(int), s));
  // Residual replacement, inside the captured graph after every iteration: the
  // right-hand sides marked due went through the whole iteration (z and beta
  // from their recursive residual); x32 is folded into the double-float x and
  // r is replaced by the true residual, which the next iteration's update
  // continues from.  Where the true residual differs from the recursive one
  // (kCheck), z and beta are recomputed from it.  Every kernel returns at once
  // for the others; no right-hand side waits for the host.
  const bool fused = tc_fused(op);
  auto replace_step = [&](cudaStream_t ss) {
    note_launch();
    fold_df<<<zg, 256, 0, ss>>>(w->xh, w->xl, w->x32, field, st, kDue);
    residual64(kDue, ss);
    note_launch();
    sc_mixed_replace<<<m, 32, 0, ss>>>(st, part_ptr(w, kPartB), nbdf, tol * tol, delta * delta, w->chk);
    if (fused) {
      // z = B^-1 r and beta from the true residual, then the direction of this
      // step again, p_new = z + beta p_old (x already holds alpha p_old).  The
      // launches are gated by the count of right-hand sides in kCheck, which
      // is usually 0: they then return at once, where they would otherwise
      // walk their tile lists or grids (sc_promote resets the count); the mode
      // solves run on a short grid of CTAs looping over the tiles
      unsigned char *sp = w->split;
      const int *gate = w->replace_gate ? w->chk : nullptr;
      tc_split(op, m, op->nr, v.r, sp, st, kCheck, ss, gate);
      const bool sc = tc_scaled(op, m);
      tc_transform(op, m, op->nr, sp, false, v.z, st, kCheck, nullptr, nullptr, ss, -1, nullptr, nullptr, nullptr, sc,
                   tc_tr_mode(op, m), gate);
      tc_mode_solve(op, m, v.z, v.q, sp, st, kCheck, ss, part_ptr(w, kPartC), gate);
      note_launch();
      sc_beta<<<m, 32, 0, ss>>>(st, part_ptr(w, kPartC), nbd, kCheck, kCheck, 1);
      tc_transform(op, m, op->nr, sp, true, v.z, st, kCheck, nullptr, nullptr, ss, -1, v.pa, v.pb, nullptr, sc, false,
                   gate);
      note_launch();
      sc_promote<<<(m + 31) / 32, 32, 0, ss>>>(st, m, kCheck, kActive, w->chk);
      return;
    }
    precond_apply<float>(op, m, v.r, v.z, st, kCheck, part_ptr(w, kPartC), ss, v.q);
    note_launch();
    sc_beta<<<m, 32, 0, ss>>>(st, part_ptr(w, kPartC), nbd, kCheck, kActive, 1);
  };
  start();
  if (check_guess) {
    const size_t n = field * m;
    note_launch();
    to_precision<float><<<(unsigned)std::min<size_t>((n + 255) / 256, 65535), 256, 0, s>>>(w->phi64, w->pa32, n);
    int grc = gate_guess<float>(op, m, st, w->pa32, w->r32, w->z32, w->q32, accepted, s, start);
    if (grc != AX_OK) return grc;
  }
  AX_TRY(cudaMemsetAsync(w->x32, 0, sizeof(float) * field * m, s));
  AX_CHECK_LAUNCH();
  precond_apply<float>(op, m, v.r, v.z, st, kActive, part_ptr(w, kPartC), s, v.q);
  note_launch();
  sc_rho_init<<<m, 32, 0, s>>>(st, part_ptr(w, kPartC), nbd, kActive);
  AX_TRY(cudaMemsetAsync(v.pa, 0, sizeof(float) * field * m, s));
  // fused iteration: the first direction p_0 = z_0, where an even iteration
  // count finds it (pb)
  if (fused) AX_TRY(cudaMemcpyAsync(v.pb, v.z, sizeof(float) * field * m, cudaMemcpyDeviceToDevice, s));
  AX_CHECK_LAUNCH();
  const int K = w->graph_iters;
  const int key = m * 4 + 3;
  const double per_rhs = (double)op->nr * op->nz;
  for (int guard = 0; guard < 1000000; ++guard) {
    int rc = AX_OK;
    RhsState *h = w->h_st;
    if (w->profile) {
      if ((rc = read_states(w, st, m, s, h)) != AX_OK) return rc;
      pcg_iteration<float>(op, m, v, st, w, kDue, s, per_rhs * count_state(h, m, kActive), fused);
      replace_step(s);
      AX_CHECK_LAUNCH();
    } else {
      rc = run_graph(w, w->g32, key, s, [&](cudaStream_t cs) {
        for (int k = 0; k < K; ++k) {
          pcg_iteration<float>(op, m, v, st, w, kDue, cs, 0.0, fused);
          replace_step(cs);
        }
      });
    }
    if (rc != AX_OK) return rc;
    if ((rc = read_states(w, st, m, s, h)) != AX_OK) return rc;
    lat_mark(w, h, m);
    if (!any_state(h, m, kActive) && !any_state(h, m, kCheck)) break;
  }
  // the iterate back in FP64
  note_launch();
  from_df<<<cblocks, 256, 0, s>>>(w->xh, w->xl, w->x64, nall);
  AX_CHECK_LAUNCH();
  return AX_OK;
}

}  // namespace
}  // namespace ax

using namespace ax;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *ax_status_string(int status) {
  switch (status) {
    case AX_OK: return "ok";
    case AX_ERR_INVALID_ARG: return "invalid argument";
    case AX_ERR_NO_CONVERGENCE: return "no convergence within max_iter";
    case AX_ERR_BREAKDOWN: return "breakdown (non-positive curvature or non-finite scalar)";
    case AX_ERR_TIMEOUT: return "bounded device wait expired";
    case AX_ERR_OOM: return "device out of memory";
    case AX_ERR_CUDA: return "CUDA runtime error";
    case AX_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

const char *ax_version(void) { return "axpcg 0.1 sm_103a"; }

const char *ax_last_error(void) { return g_last_error; }

int64_t ax_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

// Host-buffer solve in right-hand-side chunks: the copies of one chunk
// overlap the solve of another.  With nch = host_chunks chunks of mc right-hand
// sides, chunk k's f (and guess u) goes host -> device on the copy stream
// while chunk k - 1 solves, and its u goes back while chunk k + 1 solves; the
// device staging holds two chunks (slots k mod 2).  Events order the slots:
// a chunk solves after its inputs arrived and after the copy-back of the chunk
// that used its slot two steps earlier.  Each chunk is an ordinary
// device-buffer solve of mc right-hand sides (every right-hand side iterates
// on its own, so the results and iteration counts are those of one call).
static int solve_host_chunked(ax_operator *op, const double *f, double *u, int m, double tol, int max_iter,
                              int method, int flags, ax_solve_info *info, cudaStream_t s) {
  Workspace *w = op->ws;
  const int nch = w->host_chunks;
  const int mc = (m + nch - 1) / nch;
  const size_t per = (size_t)op->nr * op->nz;
  const bool guess = (flags & AX_FLAG_USE_GUESS) != 0;
  int rc = ensure_stage(op, 2 * (size_t)mc * per);
  if (rc != AX_OK) return rc;
  {
    std::lock_guard<std::recursive_mutex> lock(g_alloc_capture_mutex);
    if (!w->copy) AX_TRY(cudaStreamCreateWithFlags(&w->copy, cudaStreamNonBlocking));
    for (cudaEvent_t &e : w->cev)
      if (!e) AX_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  cudaEvent_t *h2d = w->cev, *solved = w->cev + 2, *d2h = w->cev + 4;
  auto slot_f = [&](int k) { return w->stage_a + (size_t)(k & 1) * mc * per; };
  auto slot_u = [&](int k) { return w->stage_b + (size_t)(k & 1) * mc * per; };
  auto rows = [&](int k) { return std::min(mc, m - k * mc); };
  auto upload = [&](int k) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(slot_f(k), f + (size_t)k * mc * per, rows(k) * per * sizeof(double),
                                    cudaMemcpyHostToDevice, w->copy);
    if (e == cudaSuccess && guess)
      e = cudaMemcpyAsync(slot_u(k), u + (size_t)k * mc * per, rows(k) * per * sizeof(double), cudaMemcpyHostToDevice,
                          w->copy);
    if (e == cudaSuccess) e = cudaEventRecord(h2d[k & 1], w->copy);
    return e;
  };
  // the copy stream starts after the caller's earlier work on s
  AX_TRY(cudaEventRecord(solved[1], s));
  AX_TRY(cudaStreamWaitEvent(w->copy, solved[1], 0));
  AX_TRY(upload(0));
  int worst = AX_OK;
  const int last = (m - 1) / mc;
  for (int k = 0; k <= last; ++k) {
    if (k + 1 <= last) AX_TRY(upload(k + 1));  // the slot's previous chunk k - 1 is solved and copied back first
    AX_TRY(cudaStreamWaitEvent(s, h2d[k & 1], 0));
    if (k >= 2) AX_TRY(cudaStreamWaitEvent(s, d2h[k & 1], 0));
    const int st = ax_solve(op, slot_f(k), slot_u(k), rows(k), tol, max_iter, method, flags & ~AX_FLAG_HOST_BUFFERS,
                            info ? info + (size_t)k * mc : nullptr, s);
    if (st != AX_OK && st != AX_ERR_NO_CONVERGENCE && st != AX_ERR_BREAKDOWN) {
      cudaStreamSynchronize(w->copy);
      return st;
    }
    if (st != AX_OK && (worst == AX_OK || st > worst)) worst = st;
    AX_TRY(cudaEventRecord(solved[k & 1], s));
    AX_TRY(cudaStreamWaitEvent(w->copy, solved[k & 1], 0));
    AX_TRY(cudaMemcpyAsync(u + (size_t)k * mc * per, slot_u(k), rows(k) * per * sizeof(double), cudaMemcpyDeviceToHost,
                           w->copy));
    AX_TRY(cudaEventRecord(d2h[k & 1], w->copy));
  }
  AX_TRY(cudaStreamSynchronize(w->copy));
  AX_TRY(cudaStreamSynchronize(s));
  return worst;
}

int ax_profile_read(ax_operator *op, int32_t kind, double *ms, double *launches, double *units) {
  if (!op || kind < 0 || kind >= kProfKinds) return AX_ERR_INVALID_ARG;
  prof_collect(op->ws);
  if (ms) *ms = op->ws->prof_ms[kind];
  if (launches) *launches = op->ws->prof_launches[kind];
  if (units) *units = op->ws->prof_units[kind];
  return AX_OK;
}

int ax_destroy_operator(ax_operator *op) {
  if (!op) return AX_OK;
  free_coef(op->c64);
  free_coef(op->c32);
  dfree(op->rader_perm);
  if (op->ws) {
    Workspace *w = op->ws;
    free_vectors64(w);
    free_vectors32(w);
    free_base(w);
    dfree(w->stage_a);
    dfree(w->stage_b);
    dfree(w->split);
    dfree(w->small_buf);
    dfree(w->small_bar);
    if (w->h_flag) cudaFreeHost(w->h_flag);
    if (w->scratch) cudaFree(w->scratch);
    if (w->cap) cudaStreamDestroy(w->cap);
    if (w->copy) cudaStreamDestroy(w->copy);
    for (cudaEvent_t e : w->cev)
      if (e) cudaEventDestroy(e);
    delete w;
  }
  delete op;
  return AX_OK;
}

int ax_operator_info(const ax_operator *op, double *kappa_t, double *q_t, double *gamma1, double *gamma2) {
  if (!op) return AX_ERR_INVALID_ARG;
  if (kappa_t) *kappa_t = op->kappa_t;
  if (q_t) *q_t = op->q_t;
  if (gamma1) *gamma1 = op->gamma1;
  if (gamma2) *gamma2 = op->gamma2;
  return AX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner.  For an operator's grid shape and a number of right-hand sides
// it times FP32 PCG iterations (those of the mixed method: stencil, vector
// updates, z-transforms, mode solves, scalars) for every candidate
// configuration, on the operator's own tables, and keeps the fastest: the FFT transform (dst_tensor 0), or the tensor-core transform
// (dst_tensor 1, nz <= 4096) with each FP32 mode-solve kernel that covers nr
// (mode_kernel: the staged register kernel or a pipelined column-tile
// kernel of its tile width and CTA size).  Choices are cached per process by
// (device name, nr, nz, bc_z, right-hand sides rounded up to a power of two)
// and, if the environment variable AX_TUNE_CACHE names a file, kept there
// across processes (one line per entry: the key fields, the transform and the
// kernel, the time in ms).
// ---------------------------------------------------------------------------
namespace {
struct TuneChoice { int dst = 0, variant = 0; double ms = 0.0; };
std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const ax_operator *op, int m) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, op->device);
  int mb = 1;
  while (mb < m) mb <<= 1;
  std::string name = prop.name;
  for (char &c : name)
    if (c == ' ' || c == '|') c = '_';
  char buf[256];
  snprintf(buf, sizeof(buf), "%s|%d|%d|%d|%d", name.c_str(), op->nr, op->nz, op->bc_z, mb);
  return buf;
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = std::getenv("AX_TUNE_CACHE");
  if (!path) return;
  FILE *fp = fopen(path, "r");
  if (!fp) return;
  char key[200];
  TuneChoice c;
  while (fscanf(fp, "%199s %d %d %lf", key, &c.dst, &c.variant, &c.ms) == 4) g_tune[key] = c;
  fclose(fp);
}

void tune_save() {
  const char *path = std::getenv("AX_TUNE_CACHE");
  if (!path) return;
  FILE *fp = fopen(path, "w");
  if (!fp) return;
  for (auto &e : g_tune) fprintf(fp, "%s %d %d %.6f\n", e.first.c_str(), e.second.dst, e.second.variant, e.second.ms);
  fclose(fp);
}

void apply_choice(ax_operator *op, const TuneChoice &c) {
  op->dst_tc = c.dst;
  op->tri_variant = c.variant;
  Workspace *w = op->ws;
  free_graph(w->g64); free_graph(w->g32); free_graph(w->gc64); free_graph(w->gc32);
}
}  // namespace

extern "C" {

int ax_autotune(ax_operator *op, int32_t m, int32_t reps, void *stream) {
  if (!op || m < 1 || reps < 1 || reps > 1000) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const std::string key = tune_key(op, m);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      apply_choice(op, it->second);
      return AX_OK;
    }
  }
  Workspace *w = op->ws;
  int rc;
  if ((rc = ensure_base(op, m)) != AX_OK) return rc;
  if ((rc = ensure_vec32(op, m, false)) != AX_OK) return rc;
  std::vector<TuneChoice> cand;
  cand.push_back({0, 0});
  if (op->nz <= kMaxTcN) {
    int ids[16];
    const int n = tridiag_variants(op->nr, ids);
    if (n == 0) cand.push_back({1, 0});
    for (int i = 0; i < n; ++i) cand.push_back({1, ids[i]});
    if ((rc = ensure_split(op, (size_t)m * split_geom(op, op->nr).bytes_per_rhs)) != AX_OK) return rc;
    const bool cz = op->bc_z == 1;
    if (!tc_table(op->device, op->nz, cz ? kTableCosForward : kTableSine) ||
        !tc_table(op->device, op->nz, cz ? kTableCosInverse : kTableSine) || !tc_flag(op->device))
      return AX_ERR_OOM;
  }
  const TuneChoice saved{op->dst_tc, op->tri_variant, 0.0};
  const size_t n = field_elems(op) * m;
  cudaEvent_t e0, e1;
  AX_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return AX_ERR_CUDA;
  }
  // Each candidate runs 2 + reps FP32 PCG iterations (the mixed method's
  // iteration, fused as the solve would run it) on A x = r from x = 0 with
  // r = 0.747 in every element; the last reps are timed.
  PcgVecs<float> v{w->x32, w->r32, w->pa32, w->pb32, w->q32, w->z32};
  std::vector<RhsState> init(m);
  for (int i = 0; i < m; ++i) {
    std::memset(&init[i], 0, sizeof(RhsState));
    init[i].state = kActive;
    init[i].max_iter = 1 << 30;
    init[i].thresh2 = -1.0;
    init[i].bb = 1.0;
  }
  TuneChoice best;
  best.ms = -1.0;
  for (TuneChoice &c : cand) {
    apply_choice(op, c);
    const bool fused = tc_fused(op);
    AX_TRY(cudaMemsetAsync(w->r32, 0x3f, sizeof(float) * n, s));  // 0x3f3f3f3f: 0.747
    AX_TRY(cudaMemsetAsync(w->x32, 0, sizeof(float) * n, s));
    AX_TRY(cudaMemsetAsync(v.pa, 0, sizeof(float) * n, s));
    AX_TRY(cudaMemcpyAsync(w->st, init.data(), sizeof(RhsState) * m, cudaMemcpyHostToDevice, s));
    precond_apply<float>(op, m, v.r, v.z, w->st, kActive, part_ptr(w, kPartC), s, v.q);
    note_launch();
    sc_rho_init<<<m, 32, 0, s>>>(w->st, part_ptr(w, kPartC), precond_partials<float>(op, m), kActive);
    if (fused) AX_TRY(cudaMemcpyAsync(v.pb, v.z, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < 2; ++i) pcg_iteration<float>(op, m, v, w->st, w, kDone, s, 0.0, fused);
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; ++i) pcg_iteration<float>(op, m, v, w->st, w, kDone, s, 0.0, fused);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c.ms = ms / reps;
    if (best.ms < 0.0 || c.ms < best.ms) best = c;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || best.ms < 0.0) {
    apply_choice(op, saved);
    return e != cudaSuccess ? status_from_cuda(e) : AX_ERR_CUDA;
  }
  int *flag = tc_flag(op->device), hf = 0;
  if (flag) {  // a bounded wait of a tensor-core transform expired while timing
    AX_TRY(cudaMemcpy(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (hf) {
      cudaMemset(flag, 0, sizeof(int));
      apply_choice(op, saved);
      return AX_ERR_TIMEOUT;
    }
  }
  apply_choice(op, best);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best;
  tune_save();
  return AX_OK;
}

int ax_get_option(const ax_operator *op, const char *name, double *value) {
  if (!op || !name || !value) return AX_ERR_INVALID_ARG;
  const Workspace *w = op->ws;
  if (!strcmp(name, "dst_tensor")) *value = op->dst_tc;
  else if (!strcmp(name, "mode_kernel")) *value = op->tri_variant;
  else if (!strcmp(name, "small_path")) *value = op->ws->small_path;
  else if (!strcmp(name, "mode_kernel_effective"))  // the FP32 mode-solve kernel a solve runs (0: none of the tile kernels)
    *value = tridiag_effective(op->nr, op->tri_variant, 1, op->c32.IPS != nullptr && op->c32.RS != nullptr);
  else if (!strcmp(name, "inner_tol")) *value = w->inner_tol;
  else if (!strcmp(name, "inner_max_iter")) *value = w->inner_max;
  else if (!strcmp(name, "graph_iters")) *value = w->graph_iters;
  else if (!strcmp(name, "max_outer")) *value = w->max_outer;
  else if (!strcmp(name, "replace_delta")) *value = w->replace_delta;
  else if (!strcmp(name, "mixed_restart")) *value = w->mixed_restart;
  else if (!strcmp(name, "tc_fused")) *value = w->tc_unfused ? 0 : 1;
  else if (!strcmp(name, "replace_gate")) *value = w->replace_gate;
  else if (!strcmp(name, "replace_checks")) {  // read-only: synchronises the device
    int h = 0;
    if (w->chk != nullptr && cudaMemcpy(&h, w->chk + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return AX_ERR_CUDA;
    *value = h;
  }
  else if (!strcmp(name, "cheb_bounds")) *value = w->cheb_bounds;
  else if (!strcmp(name, "cheb_steps")) *value = w->cheb_steps;
  else if (!strcmp(name, "cheb_widen")) *value = w->cheb_widen;
  else if (!strcmp(name, "cheb_check")) *value = w->cheb_check;
  else if (!strcmp(name, "profile")) *value = w->profile ? 1 : 0;
  else if (!strcmp(name, "host_chunks")) *value = w->host_chunks;
  else return AX_ERR_INVALID_ARG;
  return AX_OK;
}

int ax_chebyshev_bounds(const ax_operator *op, int32_t m, double *gamma1, double *gamma2, int32_t *estimated) {
  if (!op || m < 1 || !gamma1 || !gamma2) return AX_ERR_INVALID_ARG;
  int any = 0;
  for (int i = 0; i < m; ++i) {
    const bool mem = (size_t)i < op->mgamma1.size();
    double g1 = mem ? op->mgamma1[i] : op->gamma1, g2 = mem ? op->mgamma2[i] : op->gamma2;
    if (op->lz_m >= m && cheb_uses_lanczos(op, g1)) {
      g1 = op->lz_g1[i];
      g2 = op->lz_g2[i];
      any = 1;
    }
    gamma1[i] = g1;
    gamma2[i] = g2;
  }
  if (estimated) *estimated = any;
  return AX_OK;
}

int ax_set_option(ax_operator *op, const char *name, double value) {
  if (!op || !name) return AX_ERR_INVALID_ARG;
  Workspace *w = op->ws;
  if (!strcmp(name, "inner_tol")) {
    if (!(value > 0.0 && value < 1.0)) return AX_ERR_INVALID_ARG;
    w->inner_tol = value;
  } else if (!strcmp(name, "inner_max_iter")) {
    if (!(value >= 1)) return AX_ERR_INVALID_ARG;
    w->inner_max = (int)value;
  } else if (!strcmp(name, "graph_iters")) {
    if (!(value >= 1 && value <= 256)) return AX_ERR_INVALID_ARG;
    w->graph_iters = (int)value;
    free_graph(w->g64); free_graph(w->g32); free_graph(w->gc64); free_graph(w->gc32);
  } else if (!strcmp(name, "profile")) {
    prof_collect(w);
    w->profile = value != 0.0;
    for (int k = 0; k < kProfKinds; ++k) w->prof_ms[k] = w->prof_launches[k] = w->prof_units[k] = 0.0;
  } else if (!strcmp(name, "mixed_restart")) {
    w->mixed_restart = value != 0.0;
  } else if (!strcmp(name, "replace_delta")) {
    if (!(value > 0.0 && value < 1.0)) return AX_ERR_INVALID_ARG;
    w->replace_delta = value;
  } else if (!strcmp(name, "tc_fused")) {
    w->tc_unfused = value == 0.0;
    free_graph(w->g32);
  } else if (!strcmp(name, "replace_gate")) {
    // 1 (default): the z recomputation of the residual-replacement step
    // (tensor-core path) returns at once when no right-hand side needs it; 0:
    // its launches walk their grids regardless.  Results are the same
    if (value != 0.0 && value != 1.0) return AX_ERR_INVALID_ARG;
    w->replace_gate = (int)value;
    free_graph(w->g32);
  } else if (!strcmp(name, "small_path")) {
    // AX_PCG_FP64 of one right-hand side on a small grid as one persistent
    // launch (1, default) or through the graph-replayed kernels (0)
    if (value != 0.0 && value != 1.0) return AX_ERR_INVALID_ARG;
    w->small_path = (int)value;
  } else if (!strcmp(name, "small_stall_test")) {
    // The next persistent small-grid solve has one CTA leave before its first
    // grid barrier, so that the others' bounded waits run out: the call
    // returns AX_ERR_TIMEOUT and the context stays usable.  For tests.
    w->small_stall_test = value != 0.0;
  } else if (!strcmp(name, "tc_stall_test")) {
    // The next tensor-core transform stops its copies before the first stage,
    // so that the MMA warp's bounded wait runs out (short limit): the call
    // returns AX_ERR_TIMEOUT and the context stays usable.  For tests.
    w->tc_stall_test = value != 0.0;
  } else if (!strcmp(name, "dst_tensor")) {
    if (value != 0.0 && value != 1.0 && value != 2.0) return AX_ERR_INVALID_ARG;
    if (value != 0.0 && op->nz > kMaxTcN) return AX_ERR_UNSUPPORTED;
    op->dst_tc = (int)value;
    free_graph(w->g64); free_graph(w->g32); free_graph(w->gc64); free_graph(w->gc32);
  } else if (!strcmp(name, "mode_kernel")) {
    // FP32 mode-solve kernel: 0 the default for nr, else a variant id of
    // tridiag_variants (1 the staged register kernel, 2..8 the pipelined
    // column-tile kernels, 9..12 and 14 the row-scaled staged kernels); ids
    // that do not cover nr are refused
    const int v = (int)value;
    if ((double)v != value || v < 0) return AX_ERR_INVALID_ARG;
    if (v != 0) {
      int ids[16];
      const int n = tridiag_variants(op->nr, ids);
      bool ok = false;
      for (int i = 0; i < n; ++i) ok = ok || ids[i] == v;
      if (!ok) return AX_ERR_INVALID_ARG;
    }
    op->tri_variant = v;
    free_graph(w->g64); free_graph(w->g32); free_graph(w->gc64); free_graph(w->gc32);
  } else if (!strcmp(name, "cheb_bounds")) {
    if (value != -1.0 && value != 0.0 && value != 1.0) return AX_ERR_INVALID_ARG;
    w->cheb_bounds = (int)value;
    op->lz_m = 0;
  } else if (!strcmp(name, "cheb_steps")) {
    if (!(value >= 2 && value <= 200) || value != (int)value) return AX_ERR_INVALID_ARG;
    w->cheb_steps = (int)value;
    op->lz_m = 0;
  } else if (!strcmp(name, "cheb_widen")) {
    if (!(value >= 0.0 && value < 1.0)) return AX_ERR_INVALID_ARG;
    w->cheb_widen = value;
    op->lz_m = 0;
  } else if (!strcmp(name, "host_chunks")) {
    if (!(value >= 1 && value <= 64) || value != (int)value) return AX_ERR_INVALID_ARG;
    w->host_chunks = (int)value;
  } else if (!strcmp(name, "cheb_check")) {
    if (!(value >= 1 && value <= 256) || value != (int)value) return AX_ERR_INVALID_ARG;
    w->cheb_check = (int)value;
    free_graph(w->gc64); free_graph(w->gc32);
  } else if (!strcmp(name, "max_outer")) {
    if (!(value >= 1)) return AX_ERR_INVALID_ARG;
    w->max_outer = (int)value;
  } else {
    return AX_ERR_INVALID_ARG;
  }
  return AX_OK;
}

int ax_setup_operator(const double *kappa_r, const double *kappa_z, const double *q, const ax_grid *g, void *stream,
                      ax_operator **out) {
  if (!out) return AX_ERR_INVALID_ARG;
  *out = nullptr;
  if (!kappa_r || !kappa_z || !q || !g) return AX_ERR_INVALID_ARG;
  if (g->bc_z != 0 && g->bc_z != 1) return AX_ERR_INVALID_ARG;
  const int cosine = g->bc_z == 1;
  const int nr = g->nr, nz = g->nz;
  if (nr < 1 || nz < 1 || nr > kMaxNr || nz > kMaxNz) return AX_ERR_INVALID_ARG;
  if (!(g->lr > 0.0) || !(g->lz > 0.0) || !std::isfinite(g->lr) || !std::isfinite(g->lz)) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  {
    const int prc = dst_prepare_device();
    if (prc != AX_OK) return prc;
  }
  const size_t nrz = (size_t)nr * nz, nrz1 = (size_t)nr * (nz + 1);
  std::vector<double> kr(nrz), kz(nrz1), qq(nrz);
  AX_TRY(cudaMemcpyAsync(kr.data(), kappa_r, nrz * sizeof(double), cudaMemcpyDeviceToHost, s));
  AX_TRY(cudaMemcpyAsync(kz.data(), kappa_z, nrz1 * sizeof(double), cudaMemcpyDeviceToHost, s));
  AX_TRY(cudaMemcpyAsync(qq.data(), q, nrz * sizeof(double), cudaMemcpyDeviceToHost, s));
  AX_TRY(cudaStreamSynchronize(s));
  double kmin = INFINITY, kmax = -INFINITY, qmin = INFINITY, qmax = -INFINITY;
  for (double v : kr) {
    if (!std::isfinite(v) || !(v > 0.0)) return AX_ERR_INVALID_ARG;
    kmin = std::min(kmin, v); kmax = std::max(kmax, v);
  }
  for (double v : kz) {
    if (!std::isfinite(v) || !(v > 0.0)) return AX_ERR_INVALID_ARG;
    kmin = std::min(kmin, v); kmax = std::max(kmax, v);
  }
  for (double v : qq) {
    if (!std::isfinite(v) || v < 0.0) return AX_ERR_INVALID_ARG;
    qmin = std::min(qmin, v); qmax = std::max(qmax, v);
  }

  ax_operator *op = new ax_operator();
  op->ws = new Workspace();
  op->nr = nr;
  op->nz = nz;
  op->pitch = (nz + 31) / 32 * 32;
  op->pitchz = (nz + 1 + 31) / 32 * 32;
  op->lr = g->lr;
  op->lz = g->lz;
  op->bc_z = g->bc_z;
  op->hr = g->lr / (nr + 0.5);
  // zero-flux z: cell-centred nodes, the boundary faces on z = 0 and z = lz
  op->hz = cosine ? g->lz / nz : g->lz / (nz + 1.0);
  cudaGetDevice(&op->device);
  // Eq. coeff2 with the footnote of Eq. diff_approx2: mean of the extremes.
  op->kappa_t = 0.5 * (kmin + kmax);
  op->q_t = 0.5 * (qmin + qmax);
  // gamma_1, gamma_2 (Eq. energy_rel): face-wise ratios bound the Rayleigh quotient.
  op->gamma1 = kmin / op->kappa_t;
  op->gamma2 = kmax / op->kappa_t;
  if (op->q_t > 0.0) {
    op->gamma1 = std::min(op->gamma1, qmin / op->q_t);
    op->gamma2 = std::max(op->gamma2, qmax / op->q_t);
  }
  // FFT length: the sine transform packs its odd extension of length 2(nz+1),
  // the cosine pair its even extension of length 2 nz
  const int L = cosine ? nz : nz + 1;
  op->plan = make_plan(L);
  if (op->plan.nstages > kMaxStages) {
    ax_destroy_operator(op);
    return AX_ERR_UNSUPPORTED;
  }
  // Transform of the FP32 path: the tensor-core GEMM when nz is within its
  // range and either the sine FFT of length L needs a prime radix above 8
  // (paired direct DFT or Rader stages, several times the work of the small
  // radices) or the transform is the cosine pair (its FFT form reads and
  // writes each row twice around the packing; at 1024^2 the GEMM pair solves
  // in 2/3 of the time).
  op->dst_tc = 0;
  if (nz <= kMaxTcN) {
    if (cosine) op->dst_tc = 1;
    for (int i = 0; i < op->plan.nstages; ++i)
      if (op->plan.radix[i] > 8) op->dst_tc = 1;
  }

  const double hr = op->hr, hz = op->hz, hr2 = hr * hr, hz2 = hz * hz;
  const int P = op->pitch, PZ = op->pitchz;
  std::vector<double> ri(nr), CR((size_t)nr * P, 0.0), CZ((size_t)nr * PZ, 0.0), W((size_t)nr * P, 0.0);
  for (int a = 0; a < nr; ++a) ri[a] = (a + 0.5) * hr;
  for (int a = 0; a < nr; ++a) {
    const double rbar = (a + 1) * hr;  // face between r-nodes a+1 and a+2 (1-based)
    for (int b = 0; b < nz; ++b) {
      CR[(size_t)a * P + b] = rbar * kr[(size_t)a * nz + b] / hr2;
      W[(size_t)a * P + b] = ri[a] * qq[(size_t)a * nz + b];
    }
    for (int c = 0; c <= nz; ++c) CZ[(size_t)a * PZ + c] = ri[a] * kz[(size_t)a * (nz + 1) + c] / hz2;
    if (cosine) {  // no flux through z = 0 and z = lz (one-sided rows of Eq. scheme_op_r_z)
      CZ[(size_t)a * PZ] = 0.0;
      CZ[(size_t)a * PZ + nz] = 0.0;
    }
  }
  // Per-mode Thomas factors of T_l (Eq. eq_trid), computed in FP64.
  std::vector<double> E(nr, 0.0), IP((size_t)nr * P, 0.0);
  const double kt = op->kappa_t, qt = op->q_t;
  for (int a = 0; a + 1 < nr; ++a) E[a] = -kt * (a + 1) * hr / hr2;
  for (int l = 1; l <= nz; ++l) {
    // mode eigenvalue of the z second difference: sine modes l = 1..nz, or the
    // cosine modes of Eq. eq_trid, 4/h^2 sin^2(pi (l - 1) / (2 nz)) (0 for l = 1)
    const double sn = cosine ? std::sin(M_PI * (l - 1) / (2.0 * nz)) : std::sin(M_PI * l / (2.0 * (nz + 1)));
    const double lam = 4.0 / hz2 * sn * sn;
    double delta = 0.0;
    for (int a = 0; a < nr; ++a) {
      const double rbar_hi = (a + 1) * hr, rbar_lo = a * hr;
      const double d = kt * (rbar_hi + rbar_lo) / hr2 + ri[a] * (kt * lam + qt);
      delta = (a == 0) ? d : d - E[a - 1] * E[a - 1] / delta;
      IP[(size_t)a * P + (l - 1)] = 1.0 / delta;
    }
  }
  // The same systems scaled to unit couplings for the FP32 pipelined mode
  // solves: T' = D T D, D = diag(rs), rs_a rs_{a+1} |E_a| = 1 (rs_0 =
  // |E_0|^-1/2, so the scale stays near |E_a|^-1/2); pivots of the scaled
  // diagonal rs_a^2 d_a(l) with off-diagonal -1.
  std::vector<double> RS(nr, 1.0), IPS((size_t)nr * P, 0.0);
  if (nr > 1) {
    RS[0] = 1.0 / std::sqrt(std::fabs(E[0]));
    for (int a = 0; a + 1 < nr; ++a) RS[a + 1] = 1.0 / (std::fabs(E[a]) * RS[a]);
  }
  for (int l = 1; l <= nz; ++l) {
    const double sn = cosine ? std::sin(M_PI * (l - 1) / (2.0 * nz)) : std::sin(M_PI * l / (2.0 * (nz + 1)));
    const double lam = 4.0 / hz2 * sn * sn;
    double delta = 0.0;
    for (int a = 0; a < nr; ++a) {
      const double rbar_hi = (a + 1) * hr, rbar_lo = a * hr;
      const double d = (kt * (rbar_hi + rbar_lo) / hr2 + ri[a] * (kt * lam + qt)) * RS[a] * RS[a];
      delta = (a == 0) ? d : d - 1.0 / delta;
      IPS[(size_t)a * P + (l - 1)] = 1.0 / delta;
    }
  }
  std::vector<double> TW(2 * (size_t)L), HW(2 * (size_t)L);
  for (int j = 0; j < L; ++j) {
    TW[2 * j] = std::cos(2.0 * M_PI * j / L);
    TW[2 * j + 1] = std::sin(2.0 * M_PI * j / L);
    HW[2 * j] = std::cos(M_PI * j / L);
    HW[2 * j + 1] = std::sin(M_PI * j / L);
  }
  // Cosine pair, per mode l = 0..nz-1 with phi = pi l / (2 nz): forward
  // factors s_l / 4 * (cos phi, sin phi, cos 3 phi, sin 3 phi), s_l the
  // orthonormal scale (sqrt(1/nz) for l = 0, sqrt(2/nz) otherwise); inverse
  // factors (cos phi, sin phi) (times sqrt 2 for l = 0: X_0 = sqrt(nz) Xhat_0
  // against sqrt(nz / 2) for the others, which the store scale holds) and
  // (cos 2 phi, sin 2 phi).
  std::vector<double> CWt;
  if (cosine) {
    CWt.assign(8 * (size_t)nz, 0.0);
    for (int l = 0; l < nz; ++l) {
      const double phi = M_PI * l / (2.0 * nz);
      const double f = 0.25 * std::sqrt(2.0 / nz) * (l == 0 ? std::sqrt(0.5) : 1.0);
      const double g0 = l == 0 ? std::sqrt(2.0) : 1.0;
      double *t = &CWt[8 * (size_t)l];
      t[0] = f * std::cos(phi); t[1] = f * std::sin(phi);
      t[2] = f * std::cos(3 * phi); t[3] = f * std::sin(3 * phi);
      t[4] = g0 * std::cos(phi); t[5] = g0 * std::sin(phi);
      t[6] = std::cos(2 * phi); t[7] = std::sin(2 * phi);
    }
  }
  cudaError_t e = cudaSuccess;
  if (cosine) {
    e = upload<double>(&op->c64.CW, CWt);
    if (e == cudaSuccess) e = upload<float>(&op->c32.CW, CWt);
  }
#define AX_UP(T, field, vec) \
  if (e == cudaSuccess) e = upload<T>(&op->field, vec);
  AX_UP(double, c64.CR, CR) AX_UP(double, c64.CZ, CZ) AX_UP(double, c64.W, W) AX_UP(double, c64.IP, IP)
  AX_UP(double, c64.E, E) AX_UP(double, c64.R, ri) AX_UP(double, c64.TW, TW) AX_UP(double, c64.HW, HW)
  AX_UP(float, c32.CR, CR) AX_UP(float, c32.CZ, CZ) AX_UP(float, c32.W, W) AX_UP(float, c32.IP, IP)
  AX_UP(float, c32.E, E) AX_UP(float, c32.R, ri) AX_UP(float, c32.TW, TW) AX_UP(float, c32.HW, HW)
  AX_UP(float, c32.IPS, IPS) AX_UP(float, c32.RS, RS)
#undef AX_UP
  {
    // IPS mode-major for the mode-solve kernel 14: column l is the run of its
    // nr factors, padded to tpitch with zeros
    op->tpitch = (nr + 31) / 32 * 32;
    std::vector<double> ipst((size_t)nz * op->tpitch, 0.0);
    for (int a2 = 0; a2 < nr; ++a2)
      for (int l = 0; l < nz; ++l) ipst[(size_t)l * op->tpitch + a2] = IPS[(size_t)a2 * P + l];
    if (e == cudaSuccess) e = upload<float>(&op->c32.IPST, ipst);
  }
  {
    // low parts for the double-float residual: v64 = (float)v64 + lo
    auto lo_of = [](const std::vector<double> &v) {
      std::vector<double> lo(v.size());
      for (size_t i = 0; i < v.size(); ++i) lo[i] = v[i] - (double)(float)v[i];
      return lo;
    };
    if (e == cudaSuccess) e = upload<float>(&op->c32.CRl, lo_of(CR));
    if (e == cudaSuccess) e = upload<float>(&op->c32.CZl, lo_of(CZ));
    if (e == cudaSuccess) e = upload<float>(&op->c32.Wl, lo_of(W));
  }
  if (e == cudaSuccess && op->plan.rader) {
    std::vector<int> perm;
    std::vector<double> rk, rt;
    rader_tables(op->plan.radix[0], perm, rk, rt);
    e = upload<double>(&op->c64.RK, rk);
    if (e == cudaSuccess) e = upload<double>(&op->c64.RT, rt);
    if (e == cudaSuccess) e = upload<float>(&op->c32.RK, rk);
    if (e == cudaSuccess) e = upload<float>(&op->c32.RT, rt);
    if (e == cudaSuccess) e = dalloc(&op->rader_perm, perm.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(op->rader_perm, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&op->ws->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    ax_destroy_operator(op);
    return status_from_cuda(e);
  }
  *out = op;
  return AX_OK;
}

}  // extern "C"

// out[m][i][k] = r_i f[m][i][k], r_i = (i + 1/2) h_r (dense rows): the
// right-hand side phi = r f of the r-weighted form.
__global__ void scale_rows_by_r(const double *__restrict__ f, double *__restrict__ out, long long rows, int nr, int nz,
                                double hr) {
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const double r = ((double)(row % nr) + 0.5) * hr;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) out[row * nz + k] = r * f[row * nz + k];
  }
}

// x[m][i][k] *= rs[m rsstride + i] for the rows i < rows of each right-hand
// side (the row scaling D of the pipelined mode solves), in place.
__global__ void scale_rows(float *__restrict__ x, const float *__restrict__ rs, long long rsstride, int rows,
                           int pitch, size_t field) {
  const int m = blockIdx.y;
  const int per_row = pitch / 4;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)rows * per_row;
       t += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(t / per_row), c4 = (int)(t % per_row);
    const float sv = rs[m * rsstride + row];
    float4 *p = reinterpret_cast<float4 *>(x + m * field + (size_t)row * pitch) + c4;
    float4 v = *p;
    v.x *= sv; v.y *= sv; v.z *= sv; v.w *= sv;
    *p = v;
  }
}

// ---- single-step entry points --------------------------------------------
template <typename T>
static int apply_step(ax_operator *op, const double *in, double *out, int m, int rows_per, int which,
                      cudaStream_t s, bool tc = false, int tc_three = 0) {
  Workspace *w = op->ws;
  const size_t field = (size_t)rows_per * op->pitch;
  int rc = ensure_scratch(op, 2 * field * m * sizeof(T));
  if (rc != AX_OK) return rc;
  if (tc && (rc = ensure_split(op, (size_t)m * split_geom(op, rows_per).bytes_per_rhs)) != AX_OK) return rc;
  T *a = reinterpret_cast<T *>(w->scratch);
  T *b = a + field * m;
  AX_TRY(cudaMemsetAsync(w->scratch, 0, 2 * field * m * sizeof(T), s));
  const long long rows = (long long)rows_per * m;
  const int blocks = (int)std::min<long long>(rows, 65535);
  note_launch();
  dense_to_padded<T><<<blocks, 256, 0, s>>>(in, a, rows, op->nz, op->pitch);
  if (which == 0) {
    StencilArgs<T> sa = stencil_args<T>(op, m, nullptr, -1);
    sa.in = a;
    sa.out = b;
    launch_stencil<T>(kStencilApply, sa, s);
  } else if (which == 1) {
    if constexpr (sizeof(T) == 4) {
      if (tc) {
        unsigned char *sp = w->split;
        tc_split(op, m, rows_per, a, sp, nullptr, -1, s);
        tc_transform(op, m, rows_per, sp, false, b, nullptr, -1, nullptr, nullptr, s, tc_three);
      }
    }
    if (!tc) {
      DstArgs<T> d = dst_args<T>(op, m, rows_per, nullptr, -1);
      d.in = a;
      d.out = b;
      launch_dst<T>(kDstPlain, d, s);
    }
  } else if (which == 4) {  // inverse transform (the sine transform is its own)
    DstArgs<T> d = dst_args<T>(op, m, rows_per, nullptr, -1);
    d.in = a;
    d.out = b;
    d.inverse = 1;
    launch_dst<T>(kDstPlain, d, s);
  } else if (which == 2) {
    TriArgs<T> t = tri_args<T>(op, m, a, b, nullptr, -1);
    if constexpr (sizeof(T) == 4) {
      // the pipelined kernels solve the row-scaled systems: b' = D b, y = D y'
      t.variant = tc_mode_variant(op, m);
      t.prescaled = t.variant >= 2;
      if (t.prescaled) {
        note_launch();
        scale_rows<<<dim3(update_blocks(rows_per, op->nz), m), 256, 0, s>>>(a, op->c32.RS, op->estride, rows_per,
                                                                           op->pitch, field);
      }
      launch_tridiag<T>(t, s);
      if (t.prescaled) {
        note_launch();
        scale_rows<<<dim3(update_blocks(rows_per, op->nz), m), 256, 0, s>>>(b, op->c32.RS, op->estride, rows_per,
                                                                           op->pitch, field);
      }
    } else {
      launch_tridiag<T>(t, s);
    }
  } else if (tc) {
    if constexpr (sizeof(T) == 4) {
      unsigned char *sp = w->split;
      tc_split(op, m, rows_per, a, sp, nullptr, -1, s);
      const bool sc = tc_scaled(op, m);
      tc_transform(op, m, rows_per, sp, false, b, nullptr, -1, nullptr, nullptr, s, tc_three, nullptr, nullptr, nullptr,
                   sc, rows_per == op->nr && tc_tr_mode(op, m));
      tc_mode_solve(op, m, b, a, sp, nullptr, -1, s);
      tc_transform(op, m, rows_per, sp, true, b, nullptr, -1, nullptr, nullptr, s, tc_three, nullptr, nullptr, nullptr,
                   sc);
    }
  } else {
    DstArgs<T> d = dst_args<T>(op, m, rows_per, nullptr, -1);
    d.in = a;
    d.out = b;
    launch_dst<T>(kDstPlain, d, s);
    launch_tridiag<T>(tri_args<T>(op, m, b, b, nullptr, -1), s);
    DstArgs<T> d2 = dst_args<T>(op, m, rows_per, nullptr, -1);
    d2.in = b;
    d2.out = b;
    d2.inverse = 1;
    launch_dst<T>(kDstPlain, d2, s);
  }
  note_launch();
  padded_to_dense<T><<<blocks, 256, 0, s>>>(b, out, rows, op->nz, op->pitch);
  AX_CHECK_LAUNCH();
  if (tc) {
    int *flag = tc_flag(op->device), hf = 0;
    if (flag) {
      AX_TRY(cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      AX_TRY(cudaStreamSynchronize(s));
      if (hf) {
        AX_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
        snprintf(g_last_error, sizeof(g_last_error), "tensor-core transform: a bounded wait expired");
        return AX_ERR_TIMEOUT;
      }
    }
  }
  return AX_OK;
}

static int apply_dispatch(ax_operator *op, const double *in, double *out, int m, int rows_per, int precision,
                          int which, void *stream) {
  if (!op || !in || !out || m < 1 || rows_per < 1) return AX_ERR_INVALID_ARG;
  const bool tc = precision == AX_PREC_FP32_TC || precision == AX_PREC_FP32_TC3;
  if (precision != AX_PREC_FP64 && precision != AX_PREC_FP32 && !tc) return AX_ERR_INVALID_ARG;
  if ((long long)rows_per * m > 2147483647LL / 2) return AX_ERR_INVALID_ARG;
  if (tc) {
    if (which != 1 && which != 3) return AX_ERR_INVALID_ARG;
    if (op->nz > kMaxTcN) return AX_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return precision == AX_PREC_FP64 ? apply_step<double>(op, in, out, m, rows_per, which, s)
                                   : apply_step<float>(op, in, out, m, rows_per, which, s, tc,
                                                       precision == AX_PREC_FP32_TC3 ? 1 : 0);
}

extern "C" {

int ax_apply_operator(ax_operator *op, const double *in, double *out, int32_t m, int32_t precision, void *stream) {
  return apply_dispatch(op, in, out, m, op ? op->nr : 0, precision, 0, stream);
}
int ax_apply_dst(ax_operator *op, const double *in, double *out, int32_t rows, int32_t precision, void *stream) {
  if (op && rows > 65535 * 16) return AX_ERR_INVALID_ARG;
  return apply_dispatch(op, in, out, 1, rows, precision, 1, stream);
}
int ax_apply_dst_inverse(ax_operator *op, const double *in, double *out, int32_t rows, int32_t precision,
                         void *stream) {
  if (op && rows > 65535 * 16) return AX_ERR_INVALID_ARG;
  if (precision != AX_PREC_FP64 && precision != AX_PREC_FP32) return AX_ERR_INVALID_ARG;
  return apply_dispatch(op, in, out, 1, rows, precision, 4, stream);
}
int ax_apply_mode_solve(ax_operator *op, const double *in, double *out, int32_t m, int32_t precision,
                        void *stream) {
  return apply_dispatch(op, in, out, m, op ? op->nr : 0, precision, 2, stream);
}
int ax_apply_preconditioner(ax_operator *op, const double *in, double *out, int32_t m, int32_t precision,
                            void *stream) {
  return apply_dispatch(op, in, out, m, op ? op->nr : 0, precision, 3, stream);
}

int ax_guessnet_features_pre(ax_operator *op, const double *kappa, const double *q, const double *f, int32_t m,
                             int32_t hw, float *x, double *scale, void *stream) {
  if (!op || !kappa || !q || !f || !x || !scale || m < 1 || hw < 1) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long rows = (long long)op->nr * m;
  const size_t dense = (size_t)rows * op->nz;
  int rc = ensure_stage(op, dense);
  if (rc != AX_OK) return rc;
  Workspace *w = op->ws;
  note_launch();
  scale_rows_by_r<<<(unsigned)std::min<long long>(rows, 65535), 256, 0, s>>>(f, w->stage_a, rows, op->nr, op->nz,
                                                                           op->hr);
  AX_CHECK_LAUNCH();
  rc = apply_dispatch(op, w->stage_a, w->stage_b, m, op->nr, AX_PREC_FP32, 3, stream);
  if (rc != AX_OK) return rc;
  return ax_guessnet_features(kappa, q, w->stage_b, m, op->nr, op->nz, hw, x, scale, stream);
}

// ---- solve ------------------------------------------------------------------
static int finish_info(ax_operator *op, int m, const RhsState *dev, ax_solve_info *info, int outer_kind,
                       const std::vector<int> &accepted, cudaStream_t s) {
  Workspace *w = op->ws;
  int rc = read_states(w, dev, m, s, w->h_st);
  if (rc != AX_OK) return rc;
  int worst = AX_OK;
  for (int i = 0; i < m; ++i) {
    const RhsState &h = w->h_st[i];
    int st = h.status;
    if (st == AX_OK && h.state != kDone) st = AX_ERR_NO_CONVERGENCE;
    if (info) {
      info[i].iters = h.iters;
      info[i].outer = outer_kind ? (int)h.tmp : 0;
      info[i].rel_res = h.bb > 0.0 ? std::sqrt(h.rr / h.bb) : 0.0;
      info[i].guess_accepted = accepted[i];
      info[i].status = st;
    }
    if (st != AX_OK && (worst == AX_OK || st > worst)) worst = st;
  }
  return worst;
}

static int solve_host_chunked(ax_operator *op, const double *f, double *u, int m, double tol, int max_iter,
                              int method, int flags, ax_solve_info *info, cudaStream_t s);

int ax_solve(ax_operator *op, const double *f, double *u, int32_t m, double tol, int32_t max_iter, int32_t method,
             int32_t flags, ax_solve_info *info, void *stream) {
  if (!op || !f || !u || m < 1) return AX_ERR_INVALID_ARG;
  if (!(tol > 0.0) || !std::isfinite(tol) || max_iter < 1) return AX_ERR_INVALID_ARG;
  if (method < AX_PCG_FP64 || method > AX_CHEB_MIXED) return AX_ERR_INVALID_ARG;
  if ((size_t)m * kPartialStride * 4 > ((size_t)1 << 40)) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace *w = op->ws;
  if ((flags & AX_FLAG_HOST_BUFFERS) && w->host_chunks > 1 && m >= 2 * w->host_chunks)
    return solve_host_chunked(op, f, u, m, tol, max_iter, method, flags, info, s);
  const int nr = op->nr, nz = op->nz, P = op->pitch;
  const size_t field = field_elems(op), dense = (size_t)nr * nz * m;
  int rc;
  if ((rc = ensure_base(op, m)) != AX_OK) return rc;
  if (method == AX_PCG_FP64 && !(flags & (AX_FLAG_HOST_BUFFERS | AX_FLAG_USE_GUESS)) && small_applies(op, m)) {
    // the whole solve as one persistent launch
    if ((rc = ensure_vec64(op, m, false)) != AX_OK) return rc;
    return small_pcg_run(op, s, f, u, tol, max_iter, info);
  }
  const bool host = (flags & AX_FLAG_HOST_BUFFERS) != 0;
  const bool guess = (flags & AX_FLAG_USE_GUESS) != 0;
  const bool check_guess = guess && (flags & AX_FLAG_CHECK_GUESS) != 0;
  std::vector<int> accepted(m, guess ? 1 : 0);
  const double *fd = f;
  double *ud = u;
  if (host) {
    if ((rc = ensure_stage(op, dense)) != AX_OK) return rc;
    AX_TRY(cudaMemcpyAsync(w->stage_a, f, dense * sizeof(double), cudaMemcpyHostToDevice, s));
    if (guess) AX_TRY(cudaMemcpyAsync(w->stage_b, u, dense * sizeof(double), cudaMemcpyHostToDevice, s));
    fd = w->stage_a;
    ud = w->stage_b;
  }
  const long long rows = (long long)nr * m;
  const int cblocks = (int)std::min<long long>(rows, 65535);
  // phi = r f (FP64) and ||phi||^2 partials
  note_launch();
  prep_rhs<<<dim3(m, (nr + 15) / 16), 256, 0, s>>>(fd, w->phi64, op->c64.R, nr, nz, P, part_ptr(w, kPartD),
                                                   part_ptr(w, kPartC));
  const int nbf = (nr + 15) / 16;
  // x64: guess or zero
  if (guess) {
    note_launch();
    dense_to_padded<double><<<cblocks, 256, 0, s>>>(ud, w->x64, rows, nz, P);
  } else {
    AX_TRY(cudaMemsetAsync(w->x64, 0, field * m * sizeof(double), s));
  }
  // the mixed methods solve A (sigma u) = sigma phi (see rhs_scale)
  const bool scaled = (method == AX_PCG_MIXED || method == AX_CHEB_MIXED);
  const unsigned sblocks =
      (unsigned)std::max<size_t>(1, std::min<size_t>((field + 1023) / 1024, (8192 + (size_t)m - 1) / (size_t)m));
  if (scaled) {
    note_launch();
    rhs_scale<<<(m + 31) / 32, 32, 0, s>>>(w->rscale, part_ptr(w, kPartC), nbf, m);
    note_launch();
    apply_rhs_scale<<<dim3(sblocks, m), 256, 0, s>>>(w->phi64, guess ? w->x64 : nullptr, w->rscale, nullptr, 0,
                                                     field, false);
    // ||phi||^2 of the scaled right-hand side, formed anew (the unscaled
    // squares may have overflowed or underflowed)
    note_launch();
    phi_norm2<<<dim3(m, nbf), 256, 0, s>>>(w->phi64, nr, nz, P, part_ptr(w, kPartD));
  }
  AX_CHECK_LAUNCH();
  const int nbs64 = stencil_blocks_per_rhs(nr, nz, 2);
  const bool cheb = (method == AX_CHEB_FP64 || method == AX_CHEB_MIXED);
  // Chebyshev bounds from a Lanczos estimate where they are needed (see
  // cheb_estimate); its PCG steps count as iterations of this solve
  std::vector<int> lz_steps;
  if (cheb && op->lz_m < m) {
    bool need = false;
    for (int i = 0; i < m && !need; ++i)
      need = cheb_uses_lanczos(op, (size_t)i < op->mgamma1.size() ? op->mgamma1[i] : op->gamma1);
    if (need && (rc = cheb_estimate(op, m, s, &lz_steps)) != AX_OK) return rc;
  }

  if (method == AX_PCG_FP64 || method == AX_CHEB_FP64) {
    if ((rc = ensure_vec64(op, m, cheb)) != AX_OK) return rc;
    // r = phi - A x, start
    StencilArgs<double> ra = stencil_args<double>(op, m, w->st, -1);
    ra.in = w->x64;
    ra.phi = w->phi64;
    ra.out_res = w->r64;
    ra.partial = part_ptr(w, kPartB);
    auto start = [&]() {
      launch_stencil<double>(kStencilResidual, ra, s);
      note_launch();
      sc_start<<<m, 32, 0, s>>>(w->st, part_ptr(w, kPartB), nbs64, part_ptr(w, kPartD), nbf, tol * tol, max_iter,
                                -1, 0);
    };
    start();
    AX_CHECK_LAUNCH();
    if (check_guess &&
        (rc = gate_guess<double>(op, m, w->st, w->phi64, w->r64, w->z64, w->q64, accepted, s, start)) != AX_OK)
      return rc;
    if (!cheb && small_applies(op, m)) {
      if ((rc = small_pcg_run(op, s)) != AX_OK) return rc;
    } else if (!cheb) {
      PcgVecs<double> v{w->x64, w->r64, w->pa64, w->pb64, w->q64, w->z64};
      if ((rc = pcg_loop<double>(op, m, v, w->phi64, w->st, w->g64, true, s)) != AX_OK) return rc;
    } else {
      // y_{-1} = y_0 (so that the first step, with alpha = 1, is plain)
      AX_TRY(cudaMemcpyAsync(w->y64prev, w->x64, field * m * sizeof(double), cudaMemcpyDeviceToDevice, s));
      ChebVecs<double> v{w->x64, w->y64prev, w->r64, w->phi64};
      int parity = 0;
      if ((rc = cheb_loop<double>(op, m, v, w->st, w->gc64, kDone, &parity, s)) != AX_OK) return rc;
      // The iterate that passed the test is y (the buffer read by the last
      // residual); with parity flipping every step it is x64 when iters is even.
      // Copy the odd ones back into x64.
      // (handled per RHS below)
      RhsState *h = w->h_st;
      if ((rc = read_states(w, w->st, m, s, h)) != AX_OK) return rc;
      for (int i = 0; i < m; ++i)
        if (h[i].iters & 1)
          AX_TRY(cudaMemcpyAsync(w->x64 + (size_t)i * field, w->y64prev + (size_t)i * field,
                                 field * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    rc = finish_info(op, m, w->st, info, 0, accepted, s);
  } else {
    // ---- mixed precision
    if ((rc = ensure_vec32(op, m, cheb)) != AX_OK) return rc;
    if (op->dst_tc) {
      // buffers and tables before any graph capture
      if ((rc = ensure_split(op, (size_t)m * split_geom(op, nr).bytes_per_rhs)) != AX_OK) return rc;
      const bool cz = op->bc_z == 1;
      if (!tc_table(op->device, nz, cz ? kTableCosForward : kTableSine) ||
          !tc_table(op->device, nz, cz ? kTableCosInverse : kTableSine) || !tc_flag(op->device))
        return AX_ERR_OOM;
    }
    if (!cheb && !w->mixed_restart) {
      // FP32 PCG with FP64 residual replacement
      if ((rc = pcg_mixed_loop(op, m, tol, w->replace_delta, max_iter, check_guess, accepted, s)) != AX_OK)
        return rc;
      rc = finish_info(op, m, w->st, info, 1, accepted, s);
    } else {
    // FP64 iterative refinement around restarted FP32 inner solves
    RhsState *so = w->st_outer, *si = w->st;
    // outer states start active
    {
      std::vector<RhsState> init(m);
      for (int i = 0; i < m; ++i) {
        std::memset(&init[i], 0, sizeof(RhsState));
        init[i].state = kActive;
        init[i].max_iter = max_iter;
      }
      AX_TRY(cudaMemcpyAsync(so, init.data(), sizeof(RhsState) * m, cudaMemcpyHostToDevice, s));
      AX_TRY(cudaStreamSynchronize(s));
    }
    const double eta2 = w->inner_tol * w->inner_tol;
    for (int outer = 0; outer <= w->max_outer; ++outer) {
      if (outer > 0) {
        dim3 g((unsigned)std::min<size_t>((field + 255) / 256, 4096), m);
        note_launch();
        add_correction<<<g, 256, 0, s>>>(w->x64, w->x32, field, so, kActive);
      }
      StencilArgs<double> ra = stencil_args<double>(op, m, so, kActive);
      ra.in = w->x64;
      ra.phi = w->phi64;
      ra.out32 = w->r32;
      ra.partial = part_ptr(w, kPartB);
      {
        ProfScope ps(w, kProfOuter, (double)nr * nz * m, s);
        launch_stencil<double>(kStencilResidual, ra, s);
      }
      note_launch();
      sc_outer<<<m, 32, 0, s>>>(so, si, part_ptr(w, kPartB), nbs64, part_ptr(w, kPartD), nbf, tol * tol, eta2,
                                w->inner_max, outer == 0);
      AX_CHECK_LAUNCH();
      RhsState *h = w->h_st;
      if ((rc = read_states(w, so, m, s, h)) != AX_OK) return rc;
      lat_mark(w, h, m);
      if (!any_state(h, m, kActive) || outer == w->max_outer) break;
      AX_TRY(cudaMemsetAsync(w->x32, 0, field * m * sizeof(float), s));
      if (!cheb) {
        PcgVecs<float> v{w->x32, w->r32, w->pa32, w->pb32, w->q32, w->z32};
        if ((rc = pcg_loop<float>(op, m, v, nullptr, si, w->g32, false, s)) != AX_OK) return rc;
      } else {
        // inner Chebyshev on A d = r from d = 0: phi_inner = r32, iterate in x32/y32prev
        AX_TRY(cudaMemsetAsync(w->y32prev, 0, field * m * sizeof(float), s));
        ChebVecs<float> v{w->x32, w->y32prev, w->z32, w->r32};
        int parity = 0;
        if ((rc = cheb_loop<float>(op, m, v, si, w->gc32, kDone, &parity, s, w->inner_tol)) != AX_OK) return rc;
        RhsState *hh = w->h_st + m;
        if ((rc = read_states(w, si, m, s, hh)) != AX_OK) return rc;
        for (int i = 0; i < m; ++i)
          if (hh[i].state != kIdle && (hh[i].iters & 1))
            AX_TRY(cudaMemcpyAsync(w->x32 + (size_t)i * field, w->y32prev + (size_t)i * field,
                                   field * sizeof(float), cudaMemcpyDeviceToDevice, s));
      }
    }
    rc = finish_info(op, m, so, info, 1, accepted, s);
    }
  }
  if (info && !lz_steps.empty())
    for (int i = 0; i < m; ++i) info[i].iters += lz_steps[i];
  if (scaled) {
    note_launch();
    apply_rhs_scale<<<dim3(sblocks, m), 256, 0, s>>>(nullptr, w->x64, w->rscale, nullptr, 0, field, true);
  }
  note_launch();
  padded_to_dense<double><<<cblocks, 256, 0, s>>>(w->x64, ud, rows, nz, P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return status_from_cuda(e);
  if (host) {
    AX_TRY(cudaMemcpyAsync(u, ud, dense * sizeof(double), cudaMemcpyDeviceToHost, s));
    AX_TRY(cudaStreamSynchronize(s));
  }
  if (op->dst_tc) {
    // a bounded wait of the tensor-core transform expired: report and re-arm
    int *flag = tc_flag(op->device), hf = 0;
    if (flag) {
      AX_TRY(cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
      AX_TRY(cudaStreamSynchronize(s));
      if (hf) {
        AX_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
        snprintf(g_last_error, sizeof(g_last_error), "tensor-core transform: a bounded wait expired");
        return AX_ERR_TIMEOUT;
      }
    }
  }
  return rc;
}

}  // extern "C"

// ===========================================================================
// Batched solve of many independent operators (uneven grids)
// ===========================================================================
// Operators with the same grid shape form a group: their coefficient tables
// and mode-solve factors are stacked into one group operator whose right-hand
// side m uses table m (per-RHS strides in the kernel arguments), so a single
// launch of every kernel serves the whole group, with per-instance
// convergence masks, graph-replayed iterations and deterministic reductions
// exactly as for one operator with many right-hand sides.  Each group runs
// its own iteration loop on its own stream and host thread, so groups
// execute concurrently on the GPU.
#include <chrono>
#include <thread>

namespace ax {
namespace {

struct BatchGroup {
  ax_operator *gop = nullptr;
  std::vector<int> members;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  double *f_stack = nullptr, *u_stack = nullptr;  // dense [m][nr][nz]
};

template <typename T>
cudaError_t stack_table(T **dst, size_t per, const std::vector<const T *> &src, cudaStream_t s) {
  cudaError_t e = dalloc(dst, per * src.size());
  for (size_t i = 0; e == cudaSuccess && i < src.size(); ++i)
    e = cudaMemcpyAsync(*dst + i * per, src[i], per * sizeof(T), cudaMemcpyDeviceToDevice, s);
  return e;
}

template <typename T>
cudaError_t copy_table(T **dst, const T *src, size_t n, cudaStream_t s) {
  cudaError_t e = dalloc(dst, n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyDeviceToDevice, s);
  return e;
}

template <typename T>
cudaError_t build_group_coef(Coef<T> &g, const std::vector<const ax_operator *> &ops, const Coef<T> &(*pick)(const ax_operator *),
                             cudaStream_t s) {
  const ax_operator *o = ops[0];
  const size_t f = (size_t)o->nr * o->pitch, fz = (size_t)o->nr * o->pitchz;
  std::vector<const T *> cr, cz, w, ip, e;
  for (auto *op : ops) {
    const Coef<T> &c = pick(op);
    cr.push_back(c.CR); cz.push_back(c.CZ); w.push_back(c.W); ip.push_back(c.IP); e.push_back(c.E);
  }
  cudaError_t err = stack_table(&g.CR, f, cr, s);
  if (err == cudaSuccess) err = stack_table(&g.CZ, fz, cz, s);
  if (err == cudaSuccess) err = stack_table(&g.W, f, w, s);
  if (err == cudaSuccess) err = stack_table(&g.IP, f, ip, s);
  if (err == cudaSuccess) err = stack_table(&g.E, (size_t)o->nr, e, s);
  if (pick(o).IPS != nullptr) {
    std::vector<const T *> ips, rs;
    for (auto *op : ops) {
      ips.push_back(pick(op).IPS);
      rs.push_back(pick(op).RS);
    }
    if (err == cudaSuccess) err = stack_table(&g.IPS, f, ips, s);
    if (err == cudaSuccess) err = stack_table(&g.RS, (size_t)o->nr, rs, s);
  }
  if (pick(o).IPST != nullptr) {
    std::vector<const T *> ipst;
    for (auto *op : ops) ipst.push_back(pick(op).IPST);
    if (err == cudaSuccess) err = stack_table(&g.IPST, (size_t)o->nz * o->tpitch, ipst, s);
  }
  if (pick(o).CRl != nullptr) {
    std::vector<const T *> crl, czl, wl;
    for (auto *op : ops) {
      const Coef<T> &c = pick(op);
      crl.push_back(c.CRl); czl.push_back(c.CZl); wl.push_back(c.Wl);
    }
    if (err == cudaSuccess) err = stack_table(&g.CRl, f, crl, s);
    if (err == cudaSuccess) err = stack_table(&g.CZl, fz, czl, s);
    if (err == cudaSuccess) err = stack_table(&g.Wl, f, wl, s);
  }
  const Coef<T> &c0 = pick(o);
  if (err == cudaSuccess) err = copy_table(&g.R, c0.R, (size_t)o->nr, s);
  if (err == cudaSuccess) err = copy_table(&g.TW, c0.TW, 2 * (size_t)o->plan.L, s);
  if (err == cudaSuccess) err = copy_table(&g.HW, c0.HW, 2 * (size_t)o->plan.L, s);
  if (err == cudaSuccess && c0.CW != nullptr) err = copy_table(&g.CW, c0.CW, 8 * (size_t)o->nz, s);
  if (err == cudaSuccess && o->plan.rader) {
    const size_t P = (size_t)o->plan.radix[0] - 1;
    err = copy_table(&g.RK, c0.RK, 2 * P, s);
    if (err == cudaSuccess) err = copy_table(&g.RT, c0.RT, 2 * P, s);
  }
  return err;
}

const Coef<double> &pick64(const ax_operator *op) { return op->c64; }
const Coef<float> &pick32(const ax_operator *op) { return op->c32; }

}  // namespace
}  // namespace ax

struct ax_batch {
  std::vector<ax::BatchGroup> groups;
  int n = 0;
  std::vector<int> nr, nz;
  std::vector<double> latency_ms;  // per instance, from the last solve
};

extern "C" {

int ax_batch_destroy(ax_batch *b) {
  if (!b) return AX_OK;
  for (auto &g : b->groups) {
    if (g.gop) ax_destroy_operator(g.gop);
    dfree(g.f_stack);
    dfree(g.u_stack);
    if (g.done) cudaEventDestroy(g.done);
    if (g.stream) cudaStreamDestroy(g.stream);
  }
  delete b;
  return AX_OK;
}

int ax_batch_create(ax_operator *const *ops, int32_t n, void *stream, ax_batch **out) {
  if (!out) return AX_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ops || n < 1) return AX_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!ops[i] || ops[i]->cstride != 0) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  ax_batch *b = new ax_batch();
  b->n = n;
  for (int i = 0; i < n; ++i) {
    b->nr.push_back(ops[i]->nr);
    b->nz.push_back(ops[i]->nz);
  }
  // group by grid shape, domain and z boundary, in order of first appearance
  std::vector<int> key_of(n, -1);
  for (int i = 0; i < n; ++i) {
    if (key_of[i] >= 0) continue;
    BatchGroup g;
    for (int j = i; j < n; ++j) {
      if (key_of[j] >= 0) continue;
      const ax_operator *a = ops[i], *c = ops[j];
      if (a->nr == c->nr && a->nz == c->nz && a->lr == c->lr && a->lz == c->lz && a->bc_z == c->bc_z) {
        key_of[j] = (int)b->groups.size();
        g.members.push_back(j);
      }
    }
    b->groups.push_back(g);
  }
  int rc = AX_OK;
  for (auto &g : b->groups) {
    std::vector<const ax_operator *> mops;
    for (int j : g.members) mops.push_back(ops[j]);
    const ax_operator *o = mops[0];
    ax_operator *gop = new ax_operator();
    gop->ws = new Workspace();
    {  // solver options of the group: those of its first member
      Workspace *gw = gop->ws;
      const Workspace *ow = o->ws;
      gw->inner_tol = ow->inner_tol;
      gw->inner_max = ow->inner_max;
      gw->graph_iters = ow->graph_iters;
      gw->max_outer = ow->max_outer;
      gw->mixed_restart = ow->mixed_restart;
      gw->tc_unfused = ow->tc_unfused;
      gw->replace_gate = ow->replace_gate;
      gw->replace_delta = ow->replace_delta;
      gw->cheb_bounds = ow->cheb_bounds;
      gw->cheb_steps = ow->cheb_steps;
      gw->cheb_widen = ow->cheb_widen;
      gw->cheb_check = ow->cheb_check;
      gw->small_path = ow->small_path;
    }
    gop->nr = o->nr; gop->nz = o->nz; gop->pitch = o->pitch; gop->pitchz = o->pitchz; gop->bc_z = o->bc_z;
    gop->tpitch = o->tpitch;
    gop->lr = o->lr; gop->lz = o->lz; gop->hr = o->hr; gop->hz = o->hz;
    gop->kappa_t = o->kappa_t; gop->q_t = o->q_t; gop->gamma1 = o->gamma1; gop->gamma2 = o->gamma2;
    for (const ax_operator *mo : mops) {  // Chebyshev bounds of each member
      gop->mgamma1.push_back(mo->gamma1);
      gop->mgamma2.push_back(mo->gamma2);
    }
    gop->device = o->device;
    gop->plan = o->plan;
    gop->dst_tc = o->dst_tc;
    gop->tri_variant = o->tri_variant;
    gop->cstride = (long long)o->nr * o->pitch;
    gop->czstride = (long long)o->nr * o->pitchz;
    gop->estride = o->nr;
    g.gop = gop;
    cudaError_t e = build_group_coef<double>(gop->c64, mops, pick64, s);
    if (e == cudaSuccess) e = build_group_coef<float>(gop->c32, mops, pick32, s);
    if (e == cudaSuccess && o->plan.rader)
      e = copy_table(&gop->rader_perm, o->rader_perm, 2 * (size_t)(o->plan.radix[0] - 1), s);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&gop->ws->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    const size_t dense = (size_t)o->nr * o->nz * g.members.size();
    if (e == cudaSuccess) e = dalloc(&g.f_stack, dense);
    if (e == cudaSuccess) e = dalloc(&g.u_stack, dense);
    if (e != cudaSuccess) {
      rc = status_from_cuda(e);
      break;
    }
  }
  if (rc == AX_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = AX_ERR_CUDA;
  if (rc != AX_OK) {
    ax_batch_destroy(b);
    return rc;
  }
  *out = b;
  return AX_OK;
}

int ax_batch_solve(ax_batch *b, const double *const *f, double *const *u, double tol, int32_t max_iter,
                   int32_t method, int32_t flags, ax_solve_info *info, void *stream) {
  if (!b || !f || !u) return AX_ERR_INVALID_ARG;
  if (method < AX_PCG_FP64 || method > AX_CHEB_MIXED) return AX_ERR_INVALID_ARG;
  if (flags & AX_FLAG_HOST_BUFFERS) return AX_ERR_UNSUPPORTED;
  for (int i = 0; i < b->n; ++i)
    if (!f[i] || !u[i]) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t start;
  if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess) return AX_ERR_CUDA;
  cudaEventRecord(start, s);
  b->latency_ms.assign(b->n, 0.0);
  std::vector<int> status(b->groups.size(), AX_OK);
  std::vector<std::vector<ax_solve_info>> ginfo(b->groups.size());
  const auto t0 = std::chrono::steady_clock::now();
  int dev = 0;
  cudaGetDevice(&dev);
  auto run = [&](size_t gi) {
    cudaSetDevice(dev);
    BatchGroup &g = b->groups[gi];
    const ax_operator *o = g.gop;
    const size_t per = (size_t)o->nr * o->nz;
    const int m = (int)g.members.size();
    cudaStreamWaitEvent(g.stream, start, 0);
    for (int k = 0; k < m; ++k) {
      cudaMemcpyAsync(g.f_stack + k * per, f[g.members[k]], per * sizeof(double), cudaMemcpyDeviceToDevice, g.stream);
      if (flags & AX_FLAG_USE_GUESS)
        cudaMemcpyAsync(g.u_stack + k * per, u[g.members[k]], per * sizeof(double), cudaMemcpyDeviceToDevice,
                        g.stream);
    }
    ginfo[gi].resize(m);
    Workspace *gw = g.gop->ws;
    gw->lat_track = true;
    gw->lat_t0 = t0;
    gw->lat_ms.assign(m, -1.0);
    status[gi] = ax_solve(g.gop, g.f_stack, g.u_stack, m, tol, max_iter, method, flags & ~AX_FLAG_SERIAL_GROUPS,
                          ginfo[gi].data(), g.stream);
    gw->lat_track = false;
    for (int k = 0; k < m; ++k)
      cudaMemcpyAsync(u[g.members[k]], g.u_stack + k * per, per * sizeof(double), cudaMemcpyDeviceToDevice, g.stream);
    cudaEventRecord(g.done, g.stream);
    cudaStreamSynchronize(g.stream);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < m; ++k) {
      const double own = k < (int)gw->lat_ms.size() ? gw->lat_ms[k] : -1.0;
      b->latency_ms[g.members[k]] = own >= 0.0 ? own : ms;
    }
  };
  if (flags & AX_FLAG_SERIAL_GROUPS) {
    for (size_t gi = 0; gi < b->groups.size(); ++gi) run(gi);
  } else {
    std::vector<std::thread> th;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) th.emplace_back(run, gi);
    for (auto &t : th) t.join();
  }
  for (auto &g : b->groups) cudaStreamWaitEvent(s, g.done, 0);
  cudaEventDestroy(start);
  int worst = AX_OK;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const int st = status[gi];
    if (st != AX_OK && (worst == AX_OK || st > worst)) worst = st;
    if (info)
      for (size_t k = 0; k < b->groups[gi].members.size(); ++k) info[b->groups[gi].members[k]] = ginfo[gi][k];
  }
  if (cudaGetLastError() != cudaSuccess) return AX_ERR_CUDA;
  return worst;
}

int ax_batch_autotune(ax_batch *b, int32_t reps, void *stream) {
  if (!b) return AX_ERR_INVALID_ARG;
  for (auto &g : b->groups) {
    const int rc = ax_autotune(g.gop, (int)g.members.size(), reps, stream);
    if (rc != AX_OK) return rc;
  }
  return AX_OK;
}

int ax_batch_config(const ax_batch *b, int32_t group, int32_t *nr, int32_t *nz, int32_t *members, int32_t *dst_tensor,
                    int32_t *mode_kernel) {
  if (!b || group < 0 || group >= (int)b->groups.size()) return AX_ERR_INVALID_ARG;
  const ax::BatchGroup &g = b->groups[group];
  if (nr) *nr = g.gop->nr;
  if (nz) *nz = g.gop->nz;
  if (members) *members = (int32_t)g.members.size();
  if (dst_tensor) *dst_tensor = g.gop->dst_tc;
  if (mode_kernel) *mode_kernel = ax::tridiag_effective(g.gop->nr, g.gop->tri_variant, (int)g.members.size(),
                                                         g.gop->c32.IPS != nullptr);
  return AX_OK;
}

int ax_batch_latency(const ax_batch *b, double *ms, int32_t *groups) {
  if (!b) return AX_ERR_INVALID_ARG;
  if (groups) *groups = (int32_t)b->groups.size();
  if (ms)
    for (int i = 0; i < b->n; ++i) ms[i] = i < (int)b->latency_ms.size() ? b->latency_ms[i] : 0.0;
  return AX_OK;
}

int ax_solve_batched(ax_operator *const *ops, const double *const *f, double *const *u, int32_t n, double tol,
                     int32_t max_iter, int32_t method, int32_t flags, ax_solve_info *info, void *stream) {
  ax_batch *b = nullptr;
  int rc = ax_batch_create(ops, n, stream, &b);
  if (rc != AX_OK) return rc;
  rc = ax_batch_solve(b, f, u, tol, max_iter, method, flags, info, stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  ax_batch_destroy(b);
  return rc;
}

}  // extern "C"
