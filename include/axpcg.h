/*
 * axpcg.h — C ABI of the GB300 (sm_103a) solver for the axisymmetric elliptic
 * equation of Terekhov, "High performance parallel algorithm for solving
 * elliptic equations with non-separable variables" (arXiv 1002.3094):
 *
 *     (1/r) d_r(r kappa d_r u) + d_z(kappa d_z u) - q u = -f     on [0,lr] x [0,lz]
 *
 * (Section 2.1, Eq. main_eq), r kappa u_r = 0 on the axis r = 0, u = 0 on r = lr,
 * and on z = 0 and z = lz either u = 0 (bc_z = 0, the sine-transform variant)
 * or the paper's own zero-flux condition u_z = 0 (bc_z = 1, the cosine pair of
 * Eq. fft_phi); see the note on bc_z below.  Many right-hand sides share one
 * operator (Section 1, Eq. main_problem).
 *
 * Discretisation (Section 2.1, Eqs. poisson_diff_2, scheme_op_r_z,
 * diff_approx1): r_i = (i - 1/2) h_r, h_r = lr / (nr + 1/2), i = 1..nr, with
 * u = 0 at r_{nr+1} = lr; faces rbar_i = i h_r.  bc_z = 0: z_k = k h_z,
 * h_z = lz/(nz+1), k = 1..nz; faces zbar_k = (k + 1/2) h_z, k = 0..nz.  bc_z = 1:
 * z_k = (k - 1/2) h_z, h_z = lz/nz; faces zbar_k = k h_z, with KZ = 0 on the
 * two boundary faces k = 0 and k = nz.  The discrete operator is
 * the r-weighted conservative 5-point scheme, sign-reversed so that it is
 * symmetric positive definite (Section 2.2, Eq. a-eq):
 *   (A y)_{i,k} = [KR_i (y_{i,k}-y_{i+1,k}) + KR_{i-1} (y_{i,k}-y_{i-1,k})] / h_r^2
 *               + [KZ_{i,k} (y_{i,k}-y_{i,k+1}) + KZ_{i,k-1} (y_{i,k}-y_{i,k-1})] / h_z^2
 *               + W_{i,k} y_{i,k},
 * KR_i = rbar_i kappa(rbar_i, z_k), KZ_{i,k} = r_i kappa(r_i, zbar_k),
 * W = r_i q(r_i, z_k), right-hand side phi = r_i f(r_i, z_k), KR_0 = 0.
 *
 * Each iteration of the solver applies A once and the preconditioner
 * B = kappa~ Delta - q~ (Eq. coeff2, with f~ = (min f + max f)/2 as in the
 * footnote of Eq. diff_approx2) once, inverted by separation of variables
 * (Section 4.2, Eqs. fft_phi, eq_trid): an orthonormal sine transform (DST-I)
 * along z, one tridiagonal solve along r per z-mode l with the diagonal
 * shifted by r_i (kappa~ lambda_l + q~), lambda_l = (4/h_z^2) sin^2(pi l /
 * (2 (nz+1))), and the inverse transform.
 *
 * Conventions for every entry point:
 *  - Grid functions are FP64, row-major [m][nr][nz] (z fastest), index
 *    [m][i-1][k-1] for node (r_i, z_k), right-hand side m.
 *  - Array pointers are CALLER-OWNED device memory unless a flag says host;
 *    the library never frees them.  The operator owns its own workspace.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Work is queued on it; calls that must return host results
 *    (ax_solve's info, ax_setup_operator) synchronise that stream.
 *  - Every function returns an AX_* status; none aborts, traps or exits.
 */
#ifndef AXPCG_H
#define AXPCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
  AX_OK = 0,
  AX_ERR_INVALID_ARG = 1,   /* null pointer, bad size, kappa <= 0, q < 0, non-finite input  */
  AX_ERR_NO_CONVERGENCE = 2,/* max_iter reached; u holds the last iterate, info.rel_res set */
  AX_ERR_BREAKDOWN = 3,     /* (p, Ap) <= 0 or a NaN scalar in the iteration                */
  AX_ERR_TIMEOUT = 4,       /* a bounded device wait expired                                 */
  AX_ERR_OOM = 5,           /* device allocation failed                                      */
  AX_ERR_CUDA = 6,          /* any other CUDA runtime error                                  */
  AX_ERR_UNSUPPORTED = 7    /* option not built (e.g. the tensor-core transform for nz > 4096) */
};

/* ---- methods and flags -------------------------------------------------- */
enum {
  AX_PCG_FP64 = 0,    /* plain method: PCG, every kernel in FP64 (Section 2.2, Section 4.2)      */
  AX_CHEB_FP64 = 1,   /* three-layer Chebyshev iteration (Eq. main-scheme), FP64                  */
  AX_PCG_MIXED = 2,   /* FP32 PCG with FP64 residual replacement (x accumulated in FP64)          */
  AX_CHEB_MIXED = 3   /* FP32 Chebyshev inner solves inside FP64 iterative refinement             */
};
enum {
  AX_FLAG_USE_GUESS = 1,    /* u holds an initial guess on entry (else the start is zero)   */
  AX_FLAG_HOST_BUFFERS = 4, /* f and u are host pointers; copies are made inside the call   */
  AX_FLAG_SERIAL_GROUPS = 16, /* ax_batch_solve: run the shape groups one after another on the
                                 calling thread instead of concurrently                     */
  AX_FLAG_CHECK_GUESS = 8   /* with AX_FLAG_USE_GUESS: keep a right-hand side's guess only if
                               its preconditioned residual norm (r0, B^-1 r0), r0 = phi - A u0,
                               is below (phi, B^-1 phi), the zero start's (both measure the
                               start error in the energy norm that CG reduces); else start that
                               right-hand side from zero (AX_PCG_FP64, AX_PCG_MIXED;
                               info.guess_accepted tells which; costs two B^-1 applications)  */
};
/* AX_PREC_FP32_TC, AX_PREC_FP32_TC3 (single-step entry points, transform and
 * preconditioner only): FP32 data through the tensor-core sine transform.  The
 * input is split into BF16 halves, hi = bf16(x), lo = bf16(x - hi), and
 * multiplied in FP32 accumulation by S_hi = bf16(S) (TC: the products hi S_hi
 * + lo S_hi) or by S_hi + S_lo, S_lo = bf16(S - S_hi) (TC3: + hi S_lo, S to
 * about 2^-16).  See the option "dst_tensor". */
enum { AX_PREC_FP64 = 0, AX_PREC_FP32 = 1, AX_PREC_FP32_TC = 2, AX_PREC_FP32_TC3 = 3 };

typedef struct {
  int32_t nr, nz;   /* unknowns along r and z (>= 1)                                        */
  double lr, lz;    /* domain [0, lr] x [0, lz]                                             */
  int32_t bc_z;     /* 0: u = 0 at z = 0, lz; nodes z_k = k h_z, h_z = lz/(nz+1); sine
                          transform (DST-I).
                       1: the paper's zero-flux condition du/dz = 0 at z = 0, lz
                          (Eq. main_eq); cell-centred nodes z_k = (k - 1/2) h_z,
                          h_z = lz/nz, faces zbar_c = c h_z (c = 0..nz; kappa_z is still
                          sampled there, but the two boundary faces carry no flux: the
                          one-sided rows of Eq. scheme_op_r_z); the cosine pair of
                          Eq. fft_phi.
                       Other values: AX_ERR_INVALID_ARG                                    */
} ax_grid;

typedef struct ax_operator ax_operator; /* opaque, library-owned */

typedef struct {
  int32_t iters;          /* operator products A p (inner iterations for the mixed methods) */
  int32_t outer;          /* FP64 refinement steps (mixed methods), else 0                  */
  double rel_res;         /* final FP64 true residual ||phi - A u|| / ||phi||               */
  int32_t guess_accepted; /* 1 if the initial guess was kept                                 */
  int32_t status;         /* AX_* status of this right-hand side                              */
} ax_solve_info;

/* ---- operator set-up (Section 2.1, Eq. diff_approx1; Eq. coeff2) ---------
 * kappa_r : [nr][nz]   kappa(rbar_i, z_k), i = 1..nr          device pointer
 * kappa_z : [nr][nz+1] kappa(r_i, zbar_k), k = 0..nz          device pointer
 * q       : [nr][nz]   q(r_i, z_k) >= 0                        device pointer
 * Validates 0 < kappa, 0 <= q, all finite (Eq. elliptic_condition; q >= 0 as in
 * Eq. main_problem) and the sizes; builds the scaled coefficients in FP64 and
 * FP32, the per-mode tridiagonal factors (computed in FP64) and the transform
 * tables.  Synchronises `stream`.  On success *out owns device memory that
 * ax_destroy_operator frees.  Errors: AX_ERR_INVALID_ARG, AX_ERR_UNSUPPORTED,
 * AX_ERR_OOM, AX_ERR_CUDA (nothing is leaked). */
int ax_setup_operator(const double *kappa_r, const double *kappa_z, const double *q,
                      const ax_grid *g, void *stream, ax_operator **out);

/* Frees everything the operator owns.  NULL is accepted. */
int ax_destroy_operator(ax_operator *op);

/* Preconditioner constants kappa~, q~ (Eq. coeff2) and the Chebyshev bounds
 * gamma_1 <= (Ay,y)/(By,y) <= gamma_2 (Eq. energy_rel) of a set-up operator. */
int ax_operator_info(const ax_operator *op, double *kappa_t, double *q_t,
                     double *gamma1, double *gamma2);

/* Reads an option of ax_set_option (and the ones the autotuner sets:
 * "dst_tensor", "mode_kernel"), or the read-only
 * "mode_kernel_effective": the FP32 mode-solve kernel id that option
 * "mode_kernel" resolves to for this nr (0: nr above the tile kernels, the
 * register-chunk kernel runs), and the read-only "replace_checks": how many
 * times the last AX_PCG_MIXED solve recomputed z after a residual replacement
 * (synchronises the device; AX_ERR_CUDA if that read fails); unknown names:
 * AX_ERR_INVALID_ARG. */
int ax_get_option(const ax_operator *op, const char *name, double *value);

/* Autotuner (the paper has no counterpart; its workloads ran one fixed code).
 * Times `reps` FP32 PCG iterations (those of AX_PCG_MIXED) on m right-hand
 * sides of the operator's own grid for every candidate: the FFT
 * transform, or the tensor-core transform (nz <= 4096) with each FP32
 * mode-solve kernel covering nr, and sets "dst_tensor" and "mode_kernel" to
 * the fastest.  Choices are cached per process by (device name, nr, nz, bc_z,
 * m rounded up to a power of two) and, when the environment variable
 * AX_TUNE_CACHE names a file, in that file across processes.  Synchronises
 * `stream`; uses the operator's workspace (not concurrently with a solve on
 * it).  Errors: AX_ERR_INVALID_ARG (reps outside 1..1000), AX_ERR_OOM,
 * AX_ERR_CUDA, AX_ERR_TIMEOUT (a bounded wait of the tensor-core transform
 * expired; the previous configuration is kept). */
int ax_autotune(ax_operator *op, int32_t m, int32_t reps, void *stream);

/* The Chebyshev bounds (gamma_1, gamma_2 of Eq. energy_rel) that a solve of m
 * right-hand sides uses, per right-hand side (host arrays [m]): the Lanczos
 * estimate of option "cheb_bounds" where it applies and has been formed (by
 * an earlier Chebyshev solve of at least m right-hand sides), else the
 * face-wise bounds.  *estimated = 1 if any right-hand side takes the
 * estimate.  No device work. */
int ax_chebyshev_bounds(const ax_operator *op, int32_t m, double *gamma1, double *gamma2, int32_t *estimated);

/* Tuning options of an operator (host-side settings, no device work):
 *   "profile"        1: per-launch CUDA-event profiler on (see ax_profile_read)
 *   "inner_tol"      relative residual reduction of each FP32 inner solve of the
 *                    mixed methods (0 < v < 1, default 1e-4)
 *   "inner_max_iter" cap on the iterations of one inner solve (default 400)
 *   "graph_iters"    iterations captured per CUDA-graph replay (1..256, default 16)
 *   "max_outer"      cap on FP64 refinement steps (default 30)
 *   "replace_delta"  AX_PCG_MIXED: recursive-residual reduction (relative to the
 *                    last FP64 true residual) that triggers the next FP64
 *                    residual replacement (0 < v < 1, default 0.1; with 1e-2
 *                    the FP32 recursion of the tensor-core path can drift for
 *                    many iterations between replacements on ill-conditioned
 *                    media)
 *   "dst_tensor"     AX_PCG_MIXED's FP32 kernels transform along z with the
 *                    tcgen05 tensor-core GEMM: 1 by S_hi + S_lo (three BF16
 *                    products, S to about 2^-16), 2 by S_hi = bf16(S) alone
 *                    (two products; a fixed symmetric matrix within ~3e-3 of
 *                    S, so the preconditioner S_hi T^-1 S_hi stays SPD and
 *                    close to B^-1); 0: the FFT transform.  Default: 1 when
 *                    nz <= 4096 and the FFT length nz + 1 has a prime factor
 *                    above 7 (e.g. 1025 = 5^2 41), or bc_z = 1; else 0.
 *                    For bc_z = 1 the tensor-core transform multiplies by the
 *                    orthonormal cosine pair (the forward on folded input:
 *                    r_k + r_{n-1-k} against the even modes, r_k - r_{n-1-k}
 *                    against the odd ones).  Accepted for nz <= 4096, else
 *                    AX_ERR_UNSUPPORTED
 *   "mixed_restart"  1: AX_PCG_MIXED runs restarted iterative refinement (FP32
 *                    inner PCG to "inner_tol", x += d in FP64) instead
 *   "tc_fused"       1 (default): with the tensor-core transform, the mixed PCG
 *                    forms p = z + beta p and x += alpha p in the inverse
 *                    transform's epilogue; 0: in the stencil and update pass
 *   "replace_gate"   1 (default): with the fused tensor-core iteration, the
 *                    launches that recompute z for the right-hand sides whose
 *                    true residual departed from the recursive one (residual
 *                    replacement) return at once when there are none (a device
 *                    count kept by the scalar kernels); 0: they walk their
 *                    grids.  Results are the same bit for bit
 *   "mode_kernel"    FP32 mode solves (the per-mode tridiagonal systems of
 *                    Eq. eq_trid): 0 (default) the library's choice, 1 the
 *                    staged register kernel, 9 the same on the row-scaled
 *                    systems D T_l D (unit couplings; the transforms around
 *                    the mode solves then apply D; 12 on 16-column tiles,
 *                    nr <= 1024), 10 and 11 that kernel
 *                    with the factors of a column tile kept in registers
 *                    over 4 or 8 right-hand sides, 14 that kernel fed
 *                    mode-major by the forward tensor-core transform (the
 *                    factors in the same layout; no shared-memory staging of
 *                    the input; row-major inputs take 9), 2..8 pipelined
 *                    column-tile kernels on the row-scaled systems; an id
 *                    whose column does not fit nr is refused
 *   "cheb_bounds"    Chebyshev bounds gamma_1, gamma_2 (Eq. energy_rel): 0 the
 *                    face-wise bounds (min / max of kappa / kappa~ and q / q~),
 *                    1 a Lanczos estimate from "cheb_steps" PCG steps (the
 *                    extreme eigenvalues of the Lanczos tridiagonal of the PCG
 *                    coefficients, widened by "cheb_widen"), -1 (default) the
 *                    estimate only where the face-wise gamma_1 is 0 (q_min = 0 <
 *                    q_max).  The estimate runs once per operator (FP32 kernels,
 *                    all right-hand sides, cached); its steps count in
 *                    info.iters of the solve that ran it
 *   "cheb_steps"     PCG steps of that estimate (2..200, default 20)
 *   "cheb_widen"     relative widening of the estimate (0 <= v < 1, default 0.05)
 *   "host_chunks"    AX_FLAG_HOST_BUFFERS solves of m >= 2 v right-hand sides
 *                    run in v chunks (1..64, default 1: one copy in, one copy
 *                    out): the copies of one chunk overlap the solve of another
 *                    (a second stream; two chunks of device staging).  The
 *                    results equal a device-buffer solve's bit for bit.  Pays
 *                    where the copies outweigh the loss of solving fewer
 *                    right-hand sides per launch
 *   "cheb_check"     the Chebyshev methods form the residual norm (a reduction)
 *                    every v-th step only (1..256, default 1; always on the last
 *                    step of each graph replay); the steps between advance the
 *                    three-term recurrence without any inner product
 *   "tc_stall_test"  1: test of the failure path: the next tensor-core transform
 *                    stops its copies before the first stage, one of its bounded
 *                    waits (short limit) runs out, the kernel sets the device's
 *                    error flag, frees its tensor memory and returns; the call
 *                    returns AX_ERR_TIMEOUT and the context stays usable
 * Unknown names or out-of-range values: AX_ERR_INVALID_ARG. */
int ax_set_option(ax_operator *op, const char *name, double value);

/* ---- solve (Section 2.2, Eq. main-scheme and CG; stop rule of Section 4.2) --
 * f : [m][nr][nz] physical f (the library forms phi = r_i f), device pointer
 *     (host pointer with AX_FLAG_HOST_BUFFERS)
 * u : [m][nr][nz] out: solution; in: guess if AX_FLAG_USE_GUESS
 * Each right-hand side stops when its FP64 true residual satisfies
 * ||phi - A u||_2 <= tol ||phi||_2, or fails after max_iter iterations.
 * The mixed methods solve A (sigma u) = sigma phi with sigma = 2^-e per
 * right-hand side, max |phi| = f 2^e with 1/2 <= f < 1 (exact in FP64, and no
 * square of phi is formed before the scaling), so their FP32 inner iteration
 * does not depend on the units of f anywhere in the FP64 range.
 * info : host array [m] (may be NULL).  Returns the worst per-RHS status. */
int ax_solve(ax_operator *op, const double *f, double *u, int32_t m, double tol,
             int32_t max_iter, int32_t method, int32_t flags, ax_solve_info *info, void *stream);

/* ---- many independent operators (uneven grids) in one batched solve ---------
 * Operators with the same (nr, nz, lr, lz, bc_z) form a group whose coefficient
 * tables are stacked, so each kernel launch serves the whole group with
 * per-instance convergence masks; groups run concurrently on their own
 * streams.  The paper has no batched form; it solves one series of right-hand
 * sides per operator (Eq. main_problem).
 * ax_batch_create copies the tables of `ops` (the operators stay owned by the
 * caller and may be destroyed afterwards) and the solver options set with
 * ax_set_option (instances of one shape share those of the first of them).
 * Synchronises `stream`.
 * ax_batch_solve: f[i], u[i] are device arrays [nr_i][nz_i] of instance i;
 * every method of ax_solve (the Chebyshev methods with each instance's own
 * gamma bounds, hence its own tau_0 and rho_0); info is a host array [n]
 * (may be NULL).  Blocks until all groups are done.
 * ax_batch_latency: per-instance time (ms) from the start of the last
 * ax_batch_solve until the host saw that instance's solve finish (its group's
 * states are read after every graph replay of iterations, so the resolution
 * is one replay); *groups = count.
 * ax_batch_autotune: ax_autotune on every group (m = its instances).
 * ax_batch_config: grid, instance count and the transform / mode-solve
 * kernel (ax_get_option names) that group `group` (0 .. groups-1) uses (any
 * output pointer may be NULL).
 * ax_solve_batched = create + solve + destroy. */
typedef struct ax_batch ax_batch;
int ax_batch_create(ax_operator *const *ops, int32_t n, void *stream, ax_batch **out);
int ax_batch_solve(ax_batch *b, const double *const *f, double *const *u, double tol, int32_t max_iter,
                   int32_t method, int32_t flags, ax_solve_info *info, void *stream);
int ax_batch_latency(const ax_batch *b, double *ms, int32_t *groups);
int ax_batch_autotune(ax_batch *b, int32_t reps, void *stream);
int ax_batch_config(const ax_batch *b, int32_t group, int32_t *nr, int32_t *nz, int32_t *members, int32_t *dst_tensor,
                    int32_t *mode_kernel);
int ax_batch_destroy(ax_batch *b);
int ax_solve_batched(ax_operator *const *ops, const double *const *f, double *const *u, int32_t n, double tol,
                     int32_t max_iter, int32_t method, int32_t flags, ax_solve_info *info, void *stream);

/* ---- learned initial guess --------------------------------------------------
 * A convolutional encoder-decoder (4 levels, channels c1..c4, default 24, 48,
 * 96, 192: about 1.0 M parameters) mapping the features (log kappa, q, f / s)
 * on an hw x hw lattice to u0 / s; BF16 weights and activations, FP32
 * accumulation, FP32 master weights, Adam.  The paper has no counterpart; the
 * solver only keeps a proposed u0 if it lowers the initial residual
 * (AX_FLAG_CHECK_GUESS) and always iterates to the requested tolerance.
 * Arrays are device pointers: features x [B][3][hw][hw] FP32, outputs and
 * targets [B][hw][hw] FP32.  Flat parameter order: for each layer (e1a e1b e2a
 * e2b e3a e3b b1 b2 d3a d3b d2a d2b d1a d1b) weights [3][3][cin][cout] then
 * biases [cout]; the 1x1 head's weights [c1] then its bias.
 *   create: hw a multiple of 8; channels NULL for the default; batch_capacity
 *           the largest B; He-normal initialisation from `seed`.
 *   forward: y = net(x).
 *   gradients: loss = (1/n) [sum d^2 + h1 sum over lattice edges (d_p - d_q)^2],
 *           d = net(x) - target, n = B hw hw (h1 = 0 by default: the mean
 *           squared error), and its gradient (host copy in grad_host if not
 *           NULL, [num_params]).
 *   set_loss: the edge weight h1 >= 0 (a discrete H1 seminorm term, which
 *           penalises errors the way the operator's energy norm does).
 *   train_step: gradients + one Adam step (beta 0.9 / 0.999, eps 1e-8).
 *   save / load: header (magic "AXGN", version, hw, channels, count), FP32
 *           little-endian parameters, FNV-1a 64-bit checksum.
 *   features: per RHS m, s[m] = max |f_m| and the lattice features (cell
 *           averages when nr, nz are multiples of hw, else nearest samples) from
 *           kappa [nr][nz] (e.g. the kappa_r samples), q [nr][nz], f [m][nr][nz].
 *   features_pre: as features, with f_m replaced by g_m = B^-1 (r f_m), the
 *           right-hand side after one application of the operator's Laplace
 *           preconditioner (FP32 kernels; Section 4.2): the solution of the
 *           averaged-coefficient problem, which the network then corrects for
 *           the variable kappa.  s[m] = max |g_m|.  Uses the operator's
 *           staging buffers (not concurrently with a host-buffer solve on it).
 *   lift:   u[m] = s[m] * bilinear interpolation of y[m] onto the grid nodes. */
int ax_guessnet_create(int32_t hw, const int32_t *channels, int32_t batch_capacity, uint64_t seed, void **net);
int ax_guessnet_destroy(void *net);
int64_t ax_guessnet_num_params(void *net);
int ax_guessnet_get_params(void *net, float *host, int64_t n);
int ax_guessnet_set_params(void *net, const float *host, int64_t n);
int ax_guessnet_forward(void *net, const float *x, float *y, int32_t batch, void *stream);
int ax_guessnet_gradients(void *net, const float *x, const float *target, int32_t batch, float *grad_host,
                          double *loss, void *stream);
int ax_guessnet_train_step(void *net, const float *x, const float *target, int32_t batch, float lr,
                           double *loss, void *stream);
int ax_guessnet_save(void *net, const char *path);
int ax_guessnet_load(void *net, const char *path);
int ax_guessnet_features(const double *kappa, const double *q, const double *f, int32_t m, int32_t nr,
                         int32_t nz, int32_t hw, float *x, double *scale, void *stream);
int ax_guessnet_set_loss(void *net, double h1_weight);
int ax_guessnet_features_pre(ax_operator *op, const double *kappa, const double *q, const double *f, int32_t m,
                             int32_t hw, float *x, double *scale, void *stream);
int ax_guessnet_lift(const float *y, int32_t m, int32_t hw, const double *scale, int32_t nr, int32_t nz,
                     double *u, void *stream);

/* Solve from the network's guess, the learned-guess path in one call (the
 * pieces above, composed): the features of (kappa, q, f) on the network's
 * lattice (features_pre when pre != 0, else features; kappa, q [nr][nz] as
 * there), the forward pass (in batches of the network's capacity), the lift
 * u0 = (s / target_scale) * bilinear(y) (target_scale > 0: the factor the
 * training targets u / s were multiplied by, 1 if none) into u, then ax_solve
 * with AX_FLAG_USE_GUESS | AX_FLAG_CHECK_GUESS added to flags: a right-hand
 * side keeps its guess only if the gate accepts it (info.guess_accepted) and
 * always iterates to tol.  f, u: [m][nr][nz] device FP64 (host buffers:
 * AX_ERR_UNSUPPORTED).  Allocates and frees its scratch (features, outputs,
 * scales: (4 hw^2 + 2) m words) and, like ax_solve, returns after the solve. */
int ax_solve_learned(ax_operator *op, void *net, const double *kappa, const double *q, const double *f, double *u,
                     int32_t m, double tol, int32_t max_iter, int32_t method, int32_t flags, int32_t pre,
                     double target_scale, ax_solve_info *info, void *stream);

/* ---- single steps of the hot path, for testing each kernel -----------------
 * All take FP64 device arrays [m][nr][nz]; precision selects the kernel
 * (AX_PREC_FP64 or AX_PREC_FP32 — the FP32 kernels round the input to FP32
 * first and widen the output).  in and out must not overlap. */

/* out = A in (the 5-point stencil of Eqs. poisson_diff_2, scheme_op_r_z). */
int ax_apply_operator(ax_operator *op, const double *in, double *out, int32_t m,
                      int32_t precision, void *stream);

/* out[row] = S in[row] for every one of `rows` rows of length nz: the forward
 * z-transform of the preconditioner.  bc_z = 0: S[l][k] = sqrt(2/(nz+1))
 * sin(pi k l/(nz+1)) (orthonormal DST-I, the sine counterpart of Eq. fft_phi;
 * S = S^T = S^-1).  bc_z = 1: S[l][k] = c_l sqrt(2/nz) cos(pi (k - 1/2) l / nz),
 * l = 0..nz-1, c_0 = 1/sqrt 2, else 1 (orthonormal DCT-II: the forward sum of
 * Eq. fft_phi with its first mode divided by sqrt 2). */
int ax_apply_dst(ax_operator *op, const double *in, double *out, int32_t rows,
                 int32_t precision, void *stream);

/* out[row] = S^T in[row]: the inverse z-transform (bc_z = 0: the same DST-I;
 * bc_z = 1: the orthonormal DCT-III, the inverse sum of Eq. fft_phi with its
 * first mode times sqrt 2).  precision AX_PREC_FP64 or AX_PREC_FP32 only. */
int ax_apply_dst_inverse(ax_operator *op, const double *in, double *out, int32_t rows,
                         int32_t precision, void *stream);

/* For each right-hand side and each mode column l, solve T_l y[:, l] = in[:, l]
 * along r, T_l = Lr(kappa~) + diag(r_i (kappa~ lambda_l + q~)) (Eq. eq_trid). */
int ax_apply_mode_solve(ax_operator *op, const double *in, double *out, int32_t m,
                        int32_t precision, void *stream);

/* out = B^-1 in (sine transform, mode solves, inverse transform). */
int ax_apply_preconditioner(ax_operator *op, const double *in, double *out, int32_t m,
                            int32_t precision, void *stream);

/* out = B^-1 in like ax_apply_preconditioner, but without allocating device
 * memory.  The paper has no counterpart; this exists for callers that cannot
 * call cudaMalloc (code running under CUDA-graph stream capture, pools that
 * own all device memory, loops that must not enter the memory manager).
 * Staging goes through one 32 MiB array compiled into the library, held on
 * every GPU that loads it until the process exits.  Needs
 * 2 * m * nr * pitch * sizeof(T) bytes of it (pitch = nz rounded up to 32,
 * T = double for AX_PREC_FP64, float for AX_PREC_FP32); larger requests return
 * AX_ERR_INVALID_ARG and queue nothing.  The first call on a device looks up
 * the array's device address, so make it before any stream capture.  All calls
 * share the array: calls whose GPU work may overlap (unordered streams) race
 * and must be serialised by the caller.  Calls no cudaMalloc or cudaFree. */
int ax_apply_preconditioner_noalloc(ax_operator *op, const double *in, double *out, int32_t m,
                                    int32_t precision, void *stream);

/* ---- Laguerre-harmonic chain ---------------------------------------------
 * Section 4.1, Eq. laguerre_h: harmonic m of the Laguerre transform in time
 * solves the operator of ax_solve with kappa = V, q = h^2 / (4 rho^2) and the
 * physical right-hand side
 *   f_m src - c2 a_m S_m,   S_m = sum_{k<m} (m - k) w_k Q_k,
 *   a_m = sqrt(m! / (m + alpha)!),  w_k = sqrt((k + alpha)! / k!),  c2 = h^2 / rho^2,
 * where src approximates the point source delta(x - x_0) and f_m is the m-th
 * Laguerre coefficient of the source wavelet.  After Q_m is solved,
 * ax_laguerre_step advances the running fields
 *   T <- T + w_m Q_m   (T = sum_{k<=m} w_k Q_k),   S <- S + T   (S = S_{m+1})
 * and writes the right-hand side of harmonic m + 1:
 *   f_out = f_next src - c2 a_next S,   (w_m, a_next, f_next: host scalars).
 * T and S start at zero (harmonic 0 has f = f_0 src: call with Q = NULL and
 * w_m = 0).  Q, T, S, c2, src and f_out are dense FP64 device arrays [nr][nz]
 * of op's grid (caller-owned; T, S and f_out are written and must not overlap
 * each other or the inputs).  Errors: AX_ERR_INVALID_ARG for a null pointer
 * (Q only with w_m = 0), Q equal to T, S or f_out, or a non-finite scalar;
 * AX_ERR_CUDA if the launch fails. */
int ax_laguerre_step(ax_operator *op, const double *Q, double *T, double *S, const double *c2,
                     const double *src, double w_m, double a_next, double f_next, double *f_out,
                     void *stream);

/* ---- diagnostics ----------------------------------------------------------
 * Number of CUDA kernels this library has issued in this process (direct
 * launches plus the kernel nodes of replayed graphs). */
int64_t ax_kernel_launches(void);

/* Per-launch profiler.  ax_set_option(op, "profile", 1) turns it on (and
 * clears it); while it is on, solves launch iterations one by one (no graph)
 * and bracket each kernel with CUDA events on the solve's stream.  kind:
 * 0 stencil (p update + A p), 1 forward sine transform (the FFT form fuses
 * the x, r update), 2 mode solves, 3 inverse sine transform (fused (r, z)),
 * 4 scalar kernels, 5 true residual of the mixed method (double-float) or FP64
 * outer residual, 6 x, r update pass ahead of the tensor-core transform,
 * 7 other.  Returns the summed event time in ms, the number of launches and
 * the grid unknowns they processed (right-hand sides active at launch x nr x
 * nz). */
int ax_profile_read(ax_operator *op, int32_t kind, double *ms, double *launches, double *units);

/* Human-readable name of a status code (static storage). */
const char *ax_status_string(int status);

/* Name and description of the last CUDA runtime error the library turned into
 * AX_ERR_CUDA / AX_ERR_OOM (static storage, overwritten by later errors). */
const char *ax_last_error(void);

/* Library version string (static storage). */
const char *ax_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AXPCG_H */
