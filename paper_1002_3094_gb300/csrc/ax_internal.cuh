// Internal declarations shared by the CUDA translation units of libaxpcg.
//
// Device data layout (all grid functions): [m][nr][pitch], z fastest, pitch =
// nz rounded up to a multiple of 32 elements, so every row starts on a
// 128-byte (FP32) or 256-byte (FP64) boundary.  Padding columns are kept zero
// and never read as data.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <cstddef>
#include <vector>

#include "../../include/axpcg.h"

namespace ax {

constexpr int kMaxStages = 24;

// Radix plan of the complex FFT of length L = nz + 1 used by the sine
// transform.  Odd radices larger than 8 use the generic paired kernel.
// Division by a runtime constant d (1 <= d < 2^31) for 0 <= n < 2^31:
// q = (umulhi(n, mul) + n) >> shift, with mul = floor(2^32 (2^shift - d) / d) + 1
// and shift = ceil(log2 d) (the round-up multiplier method of Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994).
struct FastDiv {
  unsigned mul = 0;
  int shift = 0;
  int d = 1;
};
inline FastDiv make_fastdiv(int d) {
  FastDiv f;
  f.d = d;
  if (d <= 1) return f;
  int l = 0;
  while ((1ll << l) < d) ++l;
  f.shift = l;
  f.mul = (unsigned)((((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d) + 1);
  return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ FastDiv make_fastdiv_dev(int d) {
  FastDiv f;
  f.d = d;
  if (d <= 1) return f;
  const int l = 32 - __clz(d - 1);  // ceil(log2 d)
  f.shift = l;
  f.mul = (unsigned)((((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d) + 1);
  return f;
}
__device__ __forceinline__ int fdiv(int n, const FastDiv &f) {
  return (int)((__umulhi((unsigned)n, f.mul) + (unsigned)n) >> f.shift);
}
#endif

struct FftPlan {
  int L = 0;
  int nstages = 0;
  int radix[kMaxStages] = {0};
  FastDiv ns_div[kMaxStages];  // Ns of stage s (product of the earlier radices)
  FastDiv tn_div[kMaxStages];  // L / radix[s]
  // Rader's algorithm for a large prime first radix R: the length-R DFT becomes
  // a cyclic convolution of length P = R - 1 done with these sub-stages.
  int rader = 0;
  int sub_n = 0;
  int sub_radix[8] = {0};
  FastDiv sub_ns[8], sub_tn[8];
  FastDiv p_div;               // P
};

// Per-precision device tables of one operator.
template <typename T>
struct Coef {
  T *CR = nullptr;   // [nr][pitch]   KR_i / h_r^2   (face rbar_i, between r-nodes i and i+1)
  T *CZ = nullptr;   // [nr][pitchz]  KZ_{i,c} / h_z^2, c = 0..nz (face zbar_c)
  T *W = nullptr;    // [nr][pitch]   r_i q
  T *IP = nullptr;   // [nr][pitch]   1 / delta_i(l): inverse Thomas pivots of T_l (column l)
  T *E = nullptr;    // [nr]          off-diagonal of T_l between rows i and i+1 (0 at i = nr)
  T *R = nullptr;    // [nr]          r_i
  T *TW = nullptr;   // [2 L]         (cos, sin)(2 pi j / L), j < L
  T *HW = nullptr;   // [2 L]         (cos, sin)(pi j / L),   j < L
  T *CW = nullptr;   // [8 nz]        zero-flux z only: cosine-transform factors of mode l
                     //               (forward: scaled cos/sin of phi_l, 3 phi_l; inverse:
                     //               cos/sin of phi_l, 2 phi_l; phi_l = pi l / (2 nz))
  T *IPST = nullptr; // [nz][tpitch]  IPS mode-major (FP32 mode-solve kernel 14)
  T *RK = nullptr;   // [2 P]         Rader: DFT of the permuted kernel W^(g^-m)
  T *RT = nullptr;   // [2 P]         Rader: (cos, sin)(2 pi j / P)
  // FP32 only: the mode systems scaled to unit couplings, T'_l = D T_l D with
  // D = diag(RS), RS_i RS_{i+1} |E_i| = 1: IPS [nr][pitch] the inverse pivots
  // 1 / delta'_i(l) of T'_l (column l), RS [nr]
  T *IPS = nullptr, *RS = nullptr;
  // FP32 only: low parts of the FP64 stencil coefficients, CR64 = CR + CRl (CR the
  // FP32 rounding), for the double-float residual of the mixed method
  T *CRl = nullptr, *CZl = nullptr, *Wl = nullptr;
};

// Scalar state of one right-hand side during an iteration.  Lives in device
// memory; written only by the scalar kernels.
struct RhsState {
  double rho;      // (r, z)
  double alpha;    // step length
  double beta;     // direction update
  double rr;       // ||r||^2 of the recursive residual
  double bb;       // reference norm^2 (||phi||^2, or ||r_outer||^2 for inner solves)
  double thresh2;  // stop when rr <= thresh2
  double cheb_a;   // Chebyshev alpha_k
  double tmp;
  double gate_phi; // (phi, B^-1 phi): preconditioned norm^2 of the zero-start residual
  double gate_res; // (r0, B^-1 r0) of the residual of a supplied initial guess
  double rho_prev; // rho before the last direction update (residual replacement)
  int state;       // kActive / kCheck / kDone / kFailed
  int iters;
  int status;      // AX_* status
  int max_iter;
  int due;         // mixed PCG: residual replacement due at the end of this iteration
  int pad_;
};

enum { kActive = 0, kCheck = 1, kDone = 2, kFailed = 3, kIdle = 4 };
// Selection mask of the replacement step: active right-hand sides marked due.
constexpr int kDue = 8;

// Launch geometry shared by producers and consumers of per-CTA partial sums.
constexpr int kStencilRows = 16;     // rows per stencil CTA
constexpr int kStencilWarps = 8;     // warps per stencil CTA (along z)
constexpr int kPartialStride = 8192; // max partials per RHS per kind
constexpr int kMaxNr = 8192, kMaxNz = 7000;

struct Workspace;

// Host-side count of kernels issued (direct launches, plus the kernel nodes of
// every replayed CUDA graph).  Launchers call note_launch(); while a graph is
// being captured nothing is counted (the replay counts the nodes).
void note_launch();

// Raises (never lowers) a kernel's dynamic shared-memory limit to `bytes`.
// Thread-safe: host threads of a batched solve launch the same kernels with
// different shared-memory sizes concurrently.
cudaError_t ensure_smem_attr(const void *func, size_t bytes);

// Kernel classes of the per-launch profiler (ax_profile_read).
enum { kProfStencil = 0, kProfDstFwd = 1, kProfTridiag = 2, kProfDstInv = 3, kProfScalar = 4,
       kProfOuter = 5, kProfUpdate = 6, kProfOther = 7, kProfKinds = 8 };

}  // namespace ax

struct ax_operator {
  int nr = 0, nz = 0, pitch = 0, pitchz = 0;
  int tpitch = 0;  // rows per mode column of the mode-major layout (nr rounded up to 32)
  int bc_z = 0;  // 0: u = 0 at z = 0, lz (sine transform); 1: zero flux there (cosine pair)
  // A group operator stacks the coefficient tables of several operators of one
  // grid shape; right-hand side m then uses table m (strides in elements).
  long long cstride = 0, czstride = 0, estride = 0;
  double lr = 1, lz = 1, hr = 0, hz = 0;
  double kappa_t = 0, q_t = 0, gamma1 = 0, gamma2 = 0;
  // group operator of a batch: the Chebyshev bounds of each member (by RHS)
  std::vector<double> mgamma1, mgamma2;
  // Lanczos estimates of the Chebyshev bounds per right-hand side (option
  // "cheb_bounds"), valid for lz_m right-hand sides (0: none)
  std::vector<double> lz_g1, lz_g2;
  int lz_m = 0;
  int device = 0;
  ax::FftPlan plan;
  int *rader_perm = nullptr;  // [2 P] device
  int dst_tc = 0;             // 1: the FP32 PCG path transforms with the tensor-core GEMM
  int tri_variant = 0;        // FP32 mode-solve kernel (0: default for nr; option "mode_kernel")
  int *tc_err = nullptr;      // device flag: a bounded wait of the GEMM expired
  ax::Coef<double> c64;
  ax::Coef<float> c32;
  ax::Workspace *ws = nullptr;
};

namespace ax {

// ---------------------------------------------------------------------------
// Kernel launchers (implemented in the .cu files).  `mask` selects the right-
// hand sides whose RhsState.state equals it; mask < 0 runs every RHS.
// ---------------------------------------------------------------------------

// Stencil modes
enum { kStencilApply = 0, kStencilPcg = 1, kStencilResidual = 2, kStencilCheb = 3, kStencilPcgP = 4 };

template <typename T>
struct StencilArgs {
  const T *CR, *CZ, *W;
  long long cstride, czstride;  // coefficient elements per RHS (0: one operator for all RHS)
  int nr, nz, pitch, pitchz;
  long long field;       // elements per RHS (nr * pitch)
  int m;
  const T *in;           // Apply: y.  Pcg: z.  Residual: x.  Cheb: y.  PcgP: unused (p by parity)
  T *pa, *pb;            // Pcg: the two search-direction buffers; an RHS with an even
                         // iteration count reads pa and writes pb, an odd one the reverse.
                         // PcgP: p is already formed (by the inverse transform); q = A p
                         // from pb (even count) or pa (odd)
  T *out;                // Apply: A y.  Pcg: q = A p_new.  Cheb: res = A y - phi
  const T *phi;          // Residual, Cheb: phi
  float *out32;          // Residual: phi - A x rounded to FP32 (may be null)
  T *out_res;            // Residual: phi - A x (may be null)
  const RhsState *st;    // per RHS state (Pcg reads beta)
  int mask;
  double *partial;       // [m][kPartialStride] per-CTA sums: Pcg (p,q); Residual, Cheb ||res||^2
};

template <typename T>
void launch_stencil(int mode, const StencilArgs<T> &a, cudaStream_t s);
// CTAs (and partial sums) per right-hand side of a stencil launch
int stencil_blocks_per_rhs(int nr, int nz, int vec);

// Double-float true residual r = phi - A x of the mixed method: x, phi and the
// coefficients as pairs of FP32 numbers (hi + lo), all arithmetic in FP32 with
// error-free transformations; r is returned rounded to FP32 with per-CTA
// partials of ||r||^2.
struct DfResidualArgs {
  const float *CRh, *CRl, *CZh, *CZl, *Wh, *Wl;
  long long cstride, czstride;  // coefficient elements per RHS (0: one operator for all RHS)
  int nr, nz, pitch, pitchz;
  long long field;
  int m;
  const float *xh, *xl, *ph, *pl;
  float *r32;
  const RhsState *st;
  int mask;
  double *partial;  // [m][kPartialStride], slot blockIdx.y * gridDim.x + blockIdx.x
};
void launch_residual_df(const DfResidualArgs &a, cudaStream_t s);
int residual_df_blocks(int nr, int nz);

// Persistent FP64 PCG of one right-hand side on a small grid (ax_small.cu):
// the whole iteration in one cooperative launch, phases separated by bounded
// grid barriers.  Inputs are the state after sc_start (r = phi - A x, rr, bb,
// thresh2); on return x, r and the state hold the result.
struct SmallPcgArgs {
  const double *CR, *CZ, *W, *IP, *E;  // operator and Thomas tables (FP64)
  const double *F, *Ft;                // dense forward transform F[l][k] and its transpose
  const double *phi;                   // [nr][pitch]
  double *x, *r, *r2, *z, *pa, *pb, *q, *t; // [nr][pitch]; r, r2 the double-buffered
                                           // residual; t the transformed field
  double *part;                        // [4][G] per-CTA partial sums
  unsigned *bar;                       // [2] barrier count and generation (zero at launch)
  RhsState *st;
  int nr, nz, pitch, pitchz;
  int nch;                             // output chunks per row of the dense transforms
  int msm;                             // set by the launcher: transform rows in shared memory
  // Whole solve in the launch (f non-null): phi = r f, x = 0, r = phi and the
  // stop threshold tol2 ||phi||^2 are formed first (the state is initialised
  // as sc_start does), and u = x is written at the end.
  const double *f;                     // dense [nr][nz] right-hand side, or null
  double *u;                           // dense [nr][nz] solution (with f)
  const double *R;                     // r_i [nr]
  double tol2;
  int max_iter;
  int *err;                            // set when a bounded wait expired
  unsigned polls;                      // wait limit (0: the default)
  int stall;                           // test of the expiry path: CTA 0 skips its first barrier
};
constexpr int kSmallMaxNr = 512, kSmallMaxNz = 256, kSmallMaxN = 65536;
// Grid size for a launch (0 if the device cannot hold enough co-resident CTAs).
int small_pcg_grid(int nr, int nz, int *nch);
cudaError_t launch_small_pcg(const SmallPcgArgs &a, int grid, cudaStream_t s);

// Sine-transform modes
enum { kDstPlain = 0, kDstPcgForward = 1, kDstPcgInverse = 2, kDstChebInverse = 3 };

template <typename T>
struct DstArgs {
  const T *TW, *HW;
  const T *CW;             // cosine: per-mode factors (Coef::CW)
  int cosine;              // 0: sine transform (DST-I, its own inverse); 1: cosine pair
  int inverse;             // cosine, plain mode: 1 = inverse (DCT-III), 0 = forward (DCT-II)
  const T *RK, *RT;        // Rader tables (plan.rader)
  const int *RP;           // Rader permutations: g^p mod R (p < P), then g^-q mod R
  FftPlan plan;
  int n, rows, pitch;      // n = nz; rows per RHS
  long long field;         // elements per RHS
  int m;
  const T *in;             // Plain: input rows.  PcgForward: q.  PcgInverse/Cheb: yhat rows
  T *out;                  // Plain: output rows.  PcgForward: rhat.  PcgInverse: z (in place ok)
  T *x, *r;                // PcgForward: x += alpha p, r -= alpha q.  PcgInverse: r for (r,z)
  T *pa, *pb;              // PcgForward: p is pb for an even iteration count, pa for odd
  T *y, *yprev;            // Cheb: y_{k+1} = a (y - tau res^) + (1 - a) y_{k-1}, written to yprev
  const double *chp;      // Cheb: (tau_0, rho_0^2) per right-hand side
  double scale;           // sine: 0.5 / sqrt(2 L), the orthonormal scaling folded with the
                          // real-FFT split; cosine inverse: 1 / sqrt(2 nz)
  int rpb;                // rows per CTA (set by the launcher)
  const RhsState *st;
  int mask;
  double *partial;        // [m][kPartialStride]: PcgForward ||r||^2, PcgInverse (r, z)
};

template <typename T>
void launch_dst(int mode, const DstArgs<T> &a, cudaStream_t s);
template <>
void launch_dst<float>(int mode, const DstArgs<float> &a, cudaStream_t s);
template <>
void launch_dst<double>(int mode, const DstArgs<double> &a, cudaStream_t s);
int dst_rows_per_block(int L, int elem_bytes);
int dst_prepare_device();  // constant tables of the unrolled prime radices (once per device)
int dst_prepare_f64();
size_t dst_smem_bytes(int L, int elem_bytes);
// Row length (complex values) of the transform's shared buffers: the FFT
// length L, or more when the staging copy of a row (n rounded up to 4 reals)
// needs it (the cosine transform of n = 1, whose L is 1).
__host__ __device__ inline int dst_buffer_len(int L, int n) {
  const int need = ((n + 3) & ~3) / 2;
  return L > need ? L : need;
}

// Tensor-core sine transform (input split into BF16 halves in the tile layout
// of ax_common.cuh, BF16 DST matrix, FP32 accumulation).
struct GemmDstArgs {
  const unsigned char *A;  // split input, tiles (m, mtiles, ktiles), even columns first
  float *out;              // rows of the output field (columns < n written)
  const uint16_t *SB;      // S_hi / S_lo tiles (dst_gemm_table)
  int n, nr, pitch;        // n = nz; rows per RHS
  long long field;         // elements per RHS of out
  int m, mtiles, ntiles, ktiles, kbe;  // kbe: K tiles of even input columns
  int three;               // 1: add hi S_lo (the transform is S to ~2^-16)
  const float *r;          // non-null: per-CTA partials of (r, out) into partial
  double *partial;         // [m][kPartialStride], slot mt * ntiles + nt
  const RhsState *st;
  int mask;
  int *err;                // set to 1 when a bounded wait expired
  // PCG direction update in the epilogue (out is then not written): with
  // p_old / p_new the two direction buffers by the parity of st[m].iters
  // (odd: pb -> pa, even: pa -> pb), p_new = out + beta p_old, and with x
  // also x += alpha p_old (the iterate update of the step that produced
  // p_old); alpha and beta from st[m]
  float *pa, *pb;
  float *x;
  // cosine forward (table kTableCosForward): the two accumulators hold the
  // even and the odd output columns (out[2l] = P, out[2l+1] = Q) instead of
  // the mirrored pair
  int cosfwd;
  // Bounded waits: tries per mbarrier wait (0: the default, ~2^22).  Test of
  // the expiry path: with stall_at >= 0 the copy warp stops before issuing
  // stage stall_at, so that the MMA warp's wait for it runs out (the kernel
  // then sets err, waits for its own copies in flight, frees TMEM and returns);
  // -1 in normal use.
  unsigned polls;
  int stall_at;
  // non-null: every output row (grid row i < nr of right-hand side m) is
  // multiplied by rowscale[m rsstride + i] before it is stored or combined
  // (the row scaling D of the pipelined mode solves)
  const float *rowscale;
  long long rsstride;
  // tout: the output is written mode-major, column l of right-hand side m as
  // the run out[(m n + l) tpitch + i], i < nr (no p update, no partials); the
  // input of the mode-solve kernel 14
  int tout, tpitch;
  // non-null: the launch returns at once while *gate == 0 (a count, kept by
  // the scalar kernels, of the right-hand sides its mask can select; for the
  // masked launches of the residual-replacement step)
  const int *gate;
};
void launch_dst_gemm(const GemmDstArgs &a, cudaStream_t s);
size_t dst_gemm_smem_bytes(int three);
int dst_gemm_ktiles(int n);
int dst_gemm_kbe(int n);
int dst_gemm_ntiles(int n);
int dst_gemm_mtiles(int rows);
// B tables of the tensor-core transform: the sine matrix (its own inverse),
// or the orthonormal cosine pair of the zero-flux z boundary: the forward
// DCT-II on folded input (u = r_k + r_{n-1-k} first, w = r_k - r_{n-1-k}
// second; output columns 2l and 2l + 1) and the inverse DCT-III (even modes
// first, outputs l and n - 1 - l as for the sine matrix).
enum { kTableSine = 0, kTableCosForward = 1, kTableCosInverse = 2 };
std::vector<uint16_t> dst_gemm_table(int n, int kind);

template <typename T>
struct TriArgs {
  const T *IP, *E;
  // FP32 pipelined kernels: the factors of the row-scaled systems (Coef::IPS,
  // Coef::RS), with the strides of IP and E; null: those kernels are not used
  const T *IPS, *RS;
  long long cstride, estride;   // factor elements per RHS (0: one operator for all RHS)
  int nr, nz, pitch;
  long long field;
  int m;
  const T *in;
  T *out;                  // may alias in
  const RhsState *st;
  int mask;
  // FP32 tile kernel only: if set, the solution is written split into BF16
  // halves (layout of ax_common.cuh, tiles mtiles x ktiles) instead of to out
  unsigned char *split;
  int split_mtiles, split_ktiles, split_kbe;
  // FP32 tile kernels only: if set, per-CTA partials of (in, out) into
  // partial[m][g], one slot g per group of tridiag_reg_cols(nr, variant) columns
  // (variant = tridiag_effective(...))
  double *partial;
  // FP32 kernel choice (0: the tuned or default choice for nr; see
  // tridiag_variants); set from the operator's "mode_kernel" option
  int variant;
  // 1: in and out hold the row-scaled systems of IPS / RS (b' = D b, y' =
  // T'^-1 b'; the pipelined kernels); 0: the plain systems of IP / E.  Set
  // exactly when tridiag_effective(...) >= 2.
  int prescaled;
  // kernel 14: `in` is mode-major (column l of right-hand side m at
  // in[(m nz + l) tpitch + i]) and IPST the factors IPS in the same layout
  // ([nz][tpitch], tcstride elements per right-hand side for stacked groups)
  const T *IPST;
  long long tcstride;
  int tpitch;
  // kernel 14, for a mask that rarely selects a right-hand side: short_grid =
  // 1 runs a few CTAs per SM that loop over the tiles (instead of one CTA per
  // tile), returning at once while *gate == 0 if gate is set (see
  // GemmDstArgs::gate)
  int short_grid;
  const int *gate;
};

template <typename T>
void launch_tridiag(const TriArgs<T> &a, cudaStream_t s);
// whether launch_tridiag<float> can write the split layout for these sizes
bool tridiag_split_ok(int nr);
// Mode columns per partial slot of the FP32 kernel `variant` for nr rows (0:
// no FP32 tile kernel covers nr); its (in, out) partials come in
// ceil(nz / cols) slots per right-hand side
int tridiag_reg_cols(int nr, int variant = 0);
// FP32 mode-solve kernels that cover nr rows: fills ids (at most 8) and
// returns their number; ids[0] is the default.  1: the staged register
// kernel; 2..: the pipelined column-tile kernels (see ax_tridiag.cu).
int tridiag_variants(int nr, int *ids);
// The FP32 kernel variant that runs for nr rows, option `variant`, m
// right-hand sides, and whether the scaled tables exist (0: none covers nr).
// The pipelined variants (>= 2) run on row-scaled data only.
int tridiag_effective(int nr, int variant, int m, bool scaled_tables);

}  // namespace ax
