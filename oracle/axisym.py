"""FP64 oracle: discretisation, Laplace preconditioner by separation of
variables, textbook PCG and Chebyshev iteration.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain and slow on
purpose: an assembled sparse operator, an explicit O(N^2) sine-transform
matrix, a plain Thomas sweep, textbook PCG.

Array conventions: a grid function y is an array of shape (nr, nz) with
y[a, b] the value at r-node i = a + 1 and z-node k = b + 1 (z fastest).  The
flat unknown index is a * nz + b.

Readings of the paper taken here:
* z boundary, bc_z = 0: homogeneous Dirichlet at z = 0 and z = 1 on the
  vertex grid z_k = k h_z, h_z = 1 / (nz + 1), k = 1..nz, faces
  zbar_k = (k + 1/2) h_z, k = 0..nz; the sine transform diagonalises the
  z-part of B.
* z boundary, bc_z = 1 (the paper's own, Eq. main_eq): zero flux at z = 0 and
  z = lz.  Cell-centred nodes z_k = (k - 1/2) h_z, h_z = lz / nz, faces
  zbar_k = k h_z, k = 0..nz, so the two outer faces lie on the boundary and
  carry no flux: the one-sided rows of Eq. scheme_op_r_z at k = 1 and
  k = N_2.  The cosine pair of Eq. fft_phi diagonalises the z-part of B.
  (Section 2.1 prints h_2 = l_2 / (N_2 - 1/2), which puts the last node on
  z = l_2 and the zero-flux face half a cell outside the domain; the
  one-sided rows and the cosine basis are the same for either spacing, and
  h_z = lz / nz keeps the second order at z = lz.)
* r grid as in Section 2.1: r_i = (i - 1/2) h_r, h_r = 1 / (nr + 1/2),
  i = 1..nr + 1, with y = 0 at r_{nr+1} = 1; faces rbar_i = i h_r, i = 0..nr.
* Sign: the operator is the paper's Eq. poisson_diff_2 multiplied by -1, so
  that A is symmetric positive definite (Section 2.2, Eq. a-eq).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np
import scipy.sparse as sp


# ---------------------------------------------------------------------------
# Grid (Section 2.1, grid omega-bar) and coefficient sampling (Eq. diff_approx1)
# ---------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Grid:
    nr: int
    nz: int
    lr: float = 1.0
    lz: float = 1.0
    bc_z: int = 0  # 0: u = 0 at z = 0, lz; 1: zero flux there (Eq. main_eq)

    @property
    def hr(self) -> float:
        return self.lr / (self.nr + 0.5)

    @property
    def hz(self) -> float:
        return self.lz / (self.nz + 1.0) if self.bc_z == 0 else self.lz / self.nz

    @property
    def r(self) -> np.ndarray:
        """Nodes r_i = (i - 1/2) h_r, i = 1..nr."""
        return (np.arange(1, self.nr + 1) - 0.5) * self.hr

    @property
    def rbar(self) -> np.ndarray:
        """Faces rbar_i = r_i + h_r / 2 = i h_r, i = 0..nr."""
        return np.arange(0, self.nr + 1) * self.hr

    @property
    def z(self) -> np.ndarray:
        """Nodes z_k = k h_z (bc_z = 0) or (k - 1/2) h_z (bc_z = 1), k = 1..nz."""
        k = np.arange(1, self.nz + 1)
        return (k if self.bc_z == 0 else k - 0.5) * self.hz

    @property
    def zbar(self) -> np.ndarray:
        """Faces zbar_k = z_k + h_z / 2, k = 0..nz (z_0 = 0, resp. -h_z / 2)."""
        c = np.arange(0, self.nz + 1)
        return (c + 0.5 if self.bc_z == 0 else c) * self.hz


def sample_medium(medium, grid: Grid, rhs_index=None):
    """Point samples the paper's Eq. diff_approx1 needs:
    kappa_r[a, b] = kappa(rbar_{a+1}, z_{b+1})      shape (nr, nz)
    kappa_z[a, c] = kappa(r_{a+1}, zbar_c)          shape (nr, nz + 1)
    q[a, b]       = q(r_{a+1}, z_{b+1})             shape (nr, nz)
    f[m, a, b]    = f_m(r_{a+1}, z_{b+1})           shape (M, nr, nz)
    """
    r, rbar, z, zbar = grid.r, grid.rbar, grid.z, grid.zbar
    kappa_r = medium.kappa(rbar[1:, None], z[None, :])
    kappa_z = medium.kappa(r[:, None], zbar[None, :])
    q = medium.q(r[:, None], z[None, :])
    idx = range(medium.n_rhs) if rhs_index is None else rhs_index
    fs = [np.broadcast_to(medium.f(r[:, None], z[None, :], m), (grid.nr, grid.nz)) for m in idx]
    f = np.stack(fs) if fs else np.zeros((0, grid.nr, grid.nz))
    return (np.ascontiguousarray(kappa_r, dtype=np.float64),
            np.ascontiguousarray(kappa_z, dtype=np.float64),
            np.ascontiguousarray(q, dtype=np.float64),
            np.ascontiguousarray(f, dtype=np.float64))


def scheme_coefficients(kappa_r, kappa_z, q, grid: Grid):
    """Eq. diff_approx1: a1 = rbar_i kappa(rbar_i, z_k), a2 = r_i kappa(r_i, zbar_k),
    w = r_i q(r_i, z_k).  Returns (KR (nr, nz), KZ (nr, nz+1), W (nr, nz)).
    The face rbar_0 = 0 on the axis carries no flux (axis condition of
    Eq. main_eq), so it is not stored.  With the zero-flux z boundary
    (bc_z = 1) the faces zbar_0 = 0 and zbar_nz = lz carry no flux either (the
    one-sided rows of Eq. scheme_op_r_z at k = 1 and k = N_2): their KZ is 0."""
    KR = grid.rbar[1:, None] * kappa_r
    KZ = grid.r[:, None] * kappa_z
    if grid.bc_z == 1:
        KZ = KZ.copy()
        KZ[:, 0] = 0.0
        KZ[:, -1] = 0.0
    W = grid.r[:, None] * q
    return KR, KZ, W


def rhs_phi(f, grid: Grid):
    """Eq. diff_approx1: phi = r_i f(r_i, z_k)."""
    return grid.r[:, None] * f


# ---------------------------------------------------------------------------
# Operator A (Eqs. poisson_diff_2, scheme_op_r_z), assembled as CSR
# ---------------------------------------------------------------------------
def assemble(KR, KZ, W, grid: Grid) -> sp.csr_matrix:
    """A = -(Lambda_r + Lambda_z) + w, scaled by the cell widths h_r^2, h_z^2
    implied by the paper's difference quotients:

      (A y)_{i,k} = [KR_i (y_{i,k} - y_{i+1,k}) + KR_{i-1} (y_{i,k} - y_{i-1,k})] / h_r^2
                  + [KZ_{i,k} (y_{i,k} - y_{i,k+1}) + KZ_{i,k-1} (y_{i,k} - y_{i,k-1})] / h_z^2
                  + W_{i,k} y_{i,k}

    with KR_0 = 0 (one-sided axis row of Eq. scheme_op_r_z), y_{nr+1,k} = 0
    (exact Dirichlet at r = l1, Section 2.1) and y_{i,0} = y_{i,nz+1} = 0
    (for bc_z = 1 the boundary faces have KZ = 0, so those values drop out)."""
    nr, nz = grid.nr, grid.nz
    hr2, hz2 = grid.hr ** 2, grid.hz ** 2
    n = nr * nz
    idx = np.arange(n).reshape(nr, nz)
    KR_lo = np.vstack([np.zeros((1, nz)), KR[:-1]])  # KR_{i-1}
    diag = (KR + KR_lo) / hr2 + (KZ[:, 1:] + KZ[:, :-1]) / hz2 + W
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [diag.ravel()]
    if nr > 1:  # r-neighbours (i, k) - (i+1, k) through face rbar_i
        a, b = idx[:-1].ravel(), idx[1:].ravel()
        v = (-KR[:-1] / hr2).ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [v, v]
    if nz > 1:  # z-neighbours (i, k) - (i, k+1) through face zbar_k
        a, b = idx[:, :-1].ravel(), idx[:, 1:].ravel()
        v = (-KZ[:, 1:-1] / hz2).ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [v, v]
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return A.tocsr()


# ---------------------------------------------------------------------------
# Preconditioner B (Eq. coeff2; Section 4.2, Eqs. precond, diff_approx2)
# ---------------------------------------------------------------------------
def preconditioner_constants(kappa_r, kappa_z, q):
    """Eq. coeff2 with the footnote of Eq. diff_approx2: the mean of the
    extreme values, f~ = (min f + max f) / 2, taken over all sampled
    coefficient values."""
    kmin = min(float(kappa_r.min()), float(kappa_z.min()))
    kmax = max(float(kappa_r.max()), float(kappa_z.max()))
    return 0.5 * (kmin + kmax), 0.5 * (float(q.min()) + float(q.max()))


def assemble_preconditioner(kappa_t: float, q_t: float, grid: Grid) -> sp.csr_matrix:
    """B: the operator A with kappa -> kappa~ and q -> q~ (Eq. coeff2)."""
    nr, nz = grid.nr, grid.nz
    KR, KZ, W = scheme_coefficients(np.full((nr, nz), kappa_t), np.full((nr, nz + 1), kappa_t),
                                    np.full((nr, nz), q_t), grid)
    return assemble(KR, KZ, W, grid)  # bc_z = 1: boundary faces zeroed there too


def dst1_matrix(n: int) -> np.ndarray:
    """Orthonormal DST-I: S[l-1, k-1] = sqrt(2/(n+1)) sin(pi k l / (n+1)),
    k, l = 1..n.  The eigenvectors of the Dirichlet second difference along z
    (the sine counterpart of the cosine sums of Eq. fft_phi)."""
    k = np.arange(1, n + 1)
    # sin(pi k l / (n+1)) has period 2 (n+1) in the integer k l: reduce it
    # exactly before scaling, so large arguments lose no accuracy.
    kl = np.outer(k, k) % (2 * (n + 1))
    return math.sqrt(2.0 / (n + 1)) * np.sin(np.pi * kl / (n + 1))


def cosine_pair(n: int):
    """The two cosine sums of Eq. fft_phi for N_2 = n, as matrices acting on
    the index k (rows of F and G are the modes l = 1..n):
      forward  phi~(l) = sqrt(2/n) sum_k f_k cos(pi (k - 1/2)(l - 1) / n),
               F[l-1, k-1] = sqrt(2/n) cos(pi (k - 1/2)(l - 1) / n);
      inverse  y_k = sqrt(2/n) (y~(1) / 2 + sum_{l>=2} y~(l) cos(...)),
               G[l-1, k-1] = w_l F[l-1, k-1], w_1 = 1/2, w_l = 1 otherwise."""
    k = np.arange(1, n + 1)
    l = np.arange(0, n)
    # cos(pi (k - 1/2)(l - 1) / n) = cos(pi m / (2n)) with the integer
    # m = (2k - 1)(l - 1), of period 4n: reduce it exactly before scaling, so
    # large arguments lose no accuracy.
    m = np.outer(l, 2 * k - 1) % (4 * n)
    F = math.sqrt(2.0 / n) * np.cos(np.pi * m / (2.0 * n))
    w = np.ones(n)
    w[0] = 0.5
    return F, w[:, None] * F


def mode_eigenvalues(nz: int, hz: float, bc_z: int = 0) -> np.ndarray:
    """bc_z = 0: lambda_l = (4 / h_z^2) sin^2(pi l / (2 (nz + 1))), l = 1..nz,
    the eigenvalues of (2 y_k - y_{k-1} - y_{k+1}) / h_z^2 with
    y_0 = y_{nz+1} = 0 (the Dirichlet counterpart of the shift in Eq. eq_trid).
    bc_z = 1: lambda_l = (4 / h_z^2) sin^2(pi (l - 1) / (2 nz)), l = 1..nz, the
    shift of Eq. eq_trid (the zero-flux second difference; lambda_1 = 0)."""
    l = np.arange(1, nz + 1)
    if bc_z == 1:
        return (4.0 / hz ** 2) * np.sin(np.pi * (l - 1) / (2.0 * nz)) ** 2
    return (4.0 / hz ** 2) * np.sin(np.pi * l / (2.0 * (nz + 1))) ** 2


def mode_tridiagonal(kappa_t: float, q_t: float, lam, grid: Grid):
    """Eq. eq_trid in SPD form: the r-operator of B for z-mode l,
      T_l = Lr(kappa~) + diag(r_i (kappa~ lambda_l + q~)),
    returned as (sub, diag, sup); sub[j] couples rows j and j+1.  lam may be an
    array of eigenvalues, in which case diag has shape (nr, len(lam))."""
    rbar, r = grid.rbar, grid.r
    hr2 = grid.hr ** 2
    lam = np.asarray(lam, dtype=np.float64)
    lr_diag = kappa_t * (rbar[1:] + rbar[:-1]) / hr2
    shift = np.multiply.outer(r, kappa_t * lam + q_t)
    diag = (lr_diag.reshape((-1,) + (1,) * lam.ndim) + shift)
    off = (-kappa_t * rbar[1:-1] / hr2).reshape((-1,) + (1,) * lam.ndim)
    return off, diag, off


def thomas(sub, diag, sup, b):
    """Plain Thomas algorithm (forward elimination, back substitution) for
    tridiagonal systems along the first axis.  diag has shape (n, ...),
    sub and sup shape (n-1, ...), b shape (n, ...); the trailing axes index
    independent systems (a series of tridiagonal systems, Eq. main_eq3), each
    eliminated in the textbook order."""
    diag = np.asarray(diag, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = diag.shape[0]
    extra = (1,) * max(0, b.ndim - diag.ndim)  # same matrix for every trailing rhs
    diag = diag.reshape(diag.shape + extra)
    sub = np.asarray(sub, dtype=np.float64)
    sup = np.asarray(sup, dtype=np.float64)
    sub = sub.reshape(sub.shape + (1,) * (diag.ndim - sub.ndim))
    sup = sup.reshape(sup.shape + (1,) * (diag.ndim - sup.ndim))
    shape = np.broadcast(diag, b).shape
    c = np.zeros(shape)
    d = np.zeros(shape)
    denom = diag[0]
    if n > 1:
        c[0] = sup[0] / denom
    d[0] = b[0] / denom
    for i in range(1, n):
        denom = diag[i] - sub[i - 1] * c[i - 1]
        if i < n - 1:
            c[i] = sup[i] / denom
        d[i] = (b[i] - sub[i - 1] * d[i - 1]) / denom
    x = np.zeros(shape)
    x[n - 1] = d[n - 1]
    for i in range(n - 2, -1, -1):
        x[i] = d[i] - c[i] * x[i + 1]
    return x


def z_transforms(grid: Grid):
    """(forward, inverse) matrices M with vt = v @ M along z: the sine matrix
    (its own inverse) for bc_z = 0, the cosine pair of Eq. fft_phi for
    bc_z = 1."""
    if grid.bc_z == 1:
        F, G = cosine_pair(grid.nz)
        return F.T, G
    S = dst1_matrix(grid.nz)
    return S, S


def precond_solve(v, kappa_t: float, q_t: float, grid: Grid, S=None):
    """y = B^{-1} v by separation of variables (Section 4.2, Eqs. fft_phi,
    eq_trid): transform every r-row along z (sine matrix for bc_z = 0, the
    cosine sums of Eq. fft_phi for bc_z = 1), solve one tridiagonal system
    along r per z-mode l, transform back.  v has shape (nr, nz); S, if given,
    is the (forward, inverse) pair of z_transforms."""
    fwd, inv = z_transforms(grid) if S is None else S
    vt = v @ fwd  # vt[:, l] = sum_k v[:, k] fwd[k, l]
    lam = mode_eigenvalues(grid.nz, grid.hz, grid.bc_z)
    sub, diag, sup = mode_tridiagonal(kappa_t, q_t, lam, grid)
    yt = thomas(sub, diag, sup, vt)  # one system per column l
    return yt @ inv


# ---------------------------------------------------------------------------
# Iterations (Section 2.2, Eq. main-scheme; stop rule of Section 4.2)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class SolveInfo:
    iters: int
    rel_res: float
    converged: bool
    history: list


def pcg(apply_A: Callable, apply_Binv: Callable, phi, tol: float, y0=None, max_iter: int = 10000):
    """Textbook preconditioned conjugate gradients (Section 2.2: B = B* > 0
    and A B^-1 A self-adjoint, so CG applies).  Stops when the true residual
    satisfies ||A y - phi|| <= tol ||phi|| (Section 4.2 stop rule): once the
    recursive residual passes, it is replaced by the true residual and the test
    is repeated on that.  "iters" counts products A p."""
    phi = np.asarray(phi, dtype=np.float64)
    y = np.zeros_like(phi) if y0 is None else np.array(y0, dtype=np.float64, copy=True)
    nphi = float(np.linalg.norm(phi))
    r = phi - apply_A(y)
    hist = [float(np.linalg.norm(r)) / nphi]
    if hist[-1] <= tol:
        return y, SolveInfo(0, hist[-1], True, hist)
    z = apply_Binv(r)
    p = z.copy()
    rho = float(np.vdot(r, z))
    it = 0
    while it < max_iter:
        q = apply_A(p)
        it += 1
        pq = float(np.vdot(p, q))
        if not (pq > 0.0) or not math.isfinite(pq):
            raise FloatingPointError(f"PCG breakdown: (p, Ap) = {pq}")
        alpha = rho / pq
        y = y + alpha * p
        r = r - alpha * q
        rel = float(np.linalg.norm(r)) / nphi
        if rel <= tol:
            r = phi - apply_A(y)
            rel = float(np.linalg.norm(r)) / nphi
            if rel <= tol:
                hist.append(rel)
                return y, SolveInfo(it, rel, True, hist)
        hist.append(rel)
        z = apply_Binv(r)
        rho_new = float(np.vdot(r, z))
        beta = rho_new / rho
        rho = rho_new
        p = z + beta * p
    return y, SolveInfo(it, hist[-1], False, hist)


def chebyshev_bounds(kappa_r, kappa_z, q, kappa_t: float, q_t: float):
    """gamma_1, gamma_2 of Eq. energy_rel for B of Eq. coeff2.  (A y, y) and
    (B y, y) are sums over faces of kappa-weighted squared differences plus a
    q-weighted sum of squares with the same non-negative geometric weights, so
    the ratio lies between the smallest and largest face-wise ratio."""
    kmin = min(float(kappa_r.min()), float(kappa_z.min()))
    kmax = max(float(kappa_r.max()), float(kappa_z.max()))
    lo, hi = kmin / kappa_t, kmax / kappa_t
    if q_t > 0.0:
        lo = min(lo, float(q.min()) / q_t)
        hi = max(hi, float(q.max()) / q_t)
    return lo, hi


def lanczos_bounds(apply_A: Callable, apply_Binv: Callable, phi, steps: int = 20, widen: float = 0.05):
    """Estimates of gamma_1, gamma_2 (Eq. energy_rel) for the Chebyshev
    iteration where the face-wise bounds are loose or degenerate (q_min = 0 <
    q_max).  `steps` textbook PCG steps (the iteration of pcg() without its
    stop test) on A y = phi from y = 0 give the coefficients alpha_j, beta_j;
    they are the Lanczos process of B^-1 A in the B-inner product, whose
    tridiagonal matrix T has (Saad, "Iterative methods for sparse linear
    systems", 2nd ed., Section 6.7.3)
      T[j, j] = 1 / alpha_j + beta_{j-1} / alpha_{j-1}   (beta_{-1} = 0),
      T[j, j+1] = T[j+1, j] = sqrt(beta_j) / alpha_j.
    Its extreme eigenvalues (Ritz values) approach lambda_min and lambda_max of
    B^-1 A from inside; the estimates are widened: gamma_1 = (1 - widen)
    theta_min, gamma_2 = (1 + widen) theta_max.  Stops early when the
    residual vanishes.  Returns (gamma1, gamma2, alphas, betas)."""
    phi = np.asarray(phi, dtype=np.float64)
    r = phi.copy()
    z = apply_Binv(r)
    p = z.copy()
    rho = float(np.vdot(r, z))
    alphas, betas = [], []
    for _ in range(steps):
        if rho == 0.0:
            break
        q = apply_A(p)
        alpha = rho / float(np.vdot(p, q))
        alphas.append(alpha)
        r = r - alpha * q
        z = apply_Binv(r)
        rho_new = float(np.vdot(r, z))
        beta = rho_new / rho
        betas.append(beta)
        rho = rho_new
        p = z + beta * p
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    theta = np.linalg.eigvalsh(T)
    return (1.0 - widen) * theta[0], (1.0 + widen) * theta[-1], alphas, betas


def chebyshev(apply_A: Callable, apply_Binv: Callable, phi, gamma1: float, gamma2: float,
              tol: float, y0=None, max_iter: int = 100000):
    """Implicit three-layer Chebyshev iteration (Eq. main-scheme) with the
    constant step tau_0 = 2 / (gamma1 + gamma2):
      y_1     = y_0 - tau_0 B^{-1}(A y_0 - phi),
      ybar    = y_k - tau_0 B^{-1}(A y_k - phi),
      y_{k+1} = alpha_{k+1} ybar + (1 - alpha_{k+1}) y_{k-1},   k >= 1,
      alpha_1 = 2,  alpha_{k+1} = 4 / (4 - rho_0^2 alpha_k),
    rho_0 = (1 - xi) / (1 + xi), xi = gamma1 / gamma2 (the parameters are the
    Chebyshev-polynomial ones of the cited Samarskii-Nikolaev book; the paper
    does not print them).  Stops on the true residual (computed every step
    anyway).  "iters" counts preconditioner applications."""
    phi = np.asarray(phi, dtype=np.float64)
    y = np.zeros_like(phi) if y0 is None else np.array(y0, dtype=np.float64, copy=True)
    nphi = float(np.linalg.norm(phi))
    tau0 = 2.0 / (gamma1 + gamma2)
    xi = gamma1 / gamma2
    rho0 = (1.0 - xi) / (1.0 + xi)
    res = apply_A(y) - phi
    rel = float(np.linalg.norm(res)) / nphi
    hist = [rel]
    if rel <= tol:
        return y, SolveInfo(0, rel, True, hist)
    y_prev = y
    y = y - tau0 * apply_Binv(res)
    it = 1
    alpha = 2.0
    while True:
        res = apply_A(y) - phi
        rel = float(np.linalg.norm(res)) / nphi
        hist.append(rel)
        if rel <= tol:
            return y, SolveInfo(it, rel, True, hist)
        if it >= max_iter or not math.isfinite(rel):
            return y, SolveInfo(it, rel, False, hist)
        alpha = 4.0 / (4.0 - rho0 * rho0 * alpha)
        ybar = y - tau0 * apply_Binv(res)
        y, y_prev = alpha * ybar + (1.0 - alpha) * y_prev, y
        it += 1


# ---------------------------------------------------------------------------
# Convenience: one operator, many right-hand sides (Eq. main_problem)
# ---------------------------------------------------------------------------
class Operator:
    """The discrete operator A, the preconditioner constants and B^{-1} for
    one (kappa, q, grid); solves any number of right-hand sides."""

    def __init__(self, kappa_r, kappa_z, q, grid: Grid):
        self.grid = grid
        self.kappa_r, self.kappa_z, self.q = kappa_r, kappa_z, q
        self.KR, self.KZ, self.W = scheme_coefficients(kappa_r, kappa_z, q, grid)
        self.A = assemble(self.KR, self.KZ, self.W, grid)
        self.kappa_t, self.q_t = preconditioner_constants(kappa_r, kappa_z, q)
        self.S = z_transforms(grid)
        self.gamma = chebyshev_bounds(kappa_r, kappa_z, q, self.kappa_t, self.q_t)

    @classmethod
    def from_medium(cls, medium, grid: Grid):
        kr, kz, q, _ = sample_medium(medium, grid, rhs_index=[])
        return cls(kr, kz, q, grid)

    def apply_A(self, y):
        return (self.A @ y.reshape(-1)).reshape(y.shape)

    def apply_Binv(self, v):
        return precond_solve(v, self.kappa_t, self.q_t, self.grid, self.S)

    def phi(self, f):
        return rhs_phi(f, self.grid)

    def solve(self, f, tol: float, method: str = "pcg", y0=None, max_iter: int = 10000):
        phi = self.phi(f)
        if method == "pcg":
            return pcg(self.apply_A, self.apply_Binv, phi, tol, y0, max_iter)
        return chebyshev(self.apply_A, self.apply_Binv, phi, self.gamma[0], self.gamma[1],
                         tol, y0, max_iter)
