"""Pins for the FP64 oracle, each tied to something other than the oracle itself:
closed forms, library routines (scipy), brute force on tiny grids, a
manufactured solution and the textbook Chebyshev error bound."""
import math
import os

import numpy as np
import pytest
import scipy.fft
import scipy.linalg
import scipy.sparse.linalg as spl

import oracle as O
from workloads import bumps_medium, manufactured_medium, manufactured_medium_neumann, Medium

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_medium(seed):
    rng = np.random.default_rng(seed)
    a, b, c = rng.uniform(0.5, 2.0, 3)

    def kappa(r, z):
        return 1.0 + a * np.sin(3 * r + b) ** 2 + c * z * z

    def q(r, z):
        return 0.3 + 0.2 * np.cos(2 * r * z) ** 2

    return Medium("rand", kappa, q, [lambda r, z: np.exp(r - z)])


def _op(nr, nz, seed=0):
    g = O.Grid(nr, nz)
    kr, kz, q, f = O.sample_medium(_random_medium(seed), g)
    return O.Operator(kr, kz, q, g), f


# --------------------------------------------------------------------------- A
@pytest.mark.parametrize("nr,nz", [(1, 1), (1, 4), (3, 1), (3, 5), (6, 4), (9, 7)])
def test_operator_symmetric_positive_definite(nr, nz):
    op, _ = _op(nr, nz)
    A = op.A.toarray()
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0.0


def test_operator_tiny_by_hand():
    line = [l for l in open(os.path.join(GOLDEN, "tiny_operator.txt")) if l.startswith("A ")][0]
    vals = [float(x) for x in line.split()[1:]]
    g = O.Grid(2, 1)
    kr, kz, q, _ = O.sample_medium(Medium("one", lambda r, z: np.ones(np.broadcast(r, z).shape),
                                          lambda r, z: np.zeros(np.broadcast(r, z).shape),
                                          [lambda r, z: r * 0]), g)
    A = O.assemble(*O.scheme_coefficients(kr, kz, q, g), g).toarray()
    np.testing.assert_allclose(A.ravel(), vals, rtol=1e-14)


def test_operator_row_sums_conservative():
    """Flux form: away from Dirichlet neighbours a constant has zero flux
    divergence, so (A 1) = W there, including the one-sided axis row."""
    nr, nz = 7, 9
    op, _ = _op(nr, nz, seed=3)
    s = op.apply_A(np.ones((nr, nz)))
    inner = (slice(0, nr - 1), slice(1, nz - 1))
    np.testing.assert_allclose(s[inner], op.W[inner], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("variable_kappa", [False, True])
def test_manufactured_solution_second_order(variable_kappa):
    """Section 2.1 states second-order accuracy (Table 2 prints error ratios
    4.09 and 5 per halving).  With u* = cos(pi r/2) sin(pi z) the max-norm
    nodal error must fall about 4x per halving of h."""
    med, u = manufactured_medium(q0=1.0, variable_kappa=variable_kappa)
    errs = []
    for n in (16, 32, 64, 128):
        g = O.Grid(n, n)
        kr, kz, q, f = O.sample_medium(med, g)
        op = O.Operator(kr, kz, q, g)
        y = spl.spsolve(op.A.tocsc(), op.phi(f[0]).ravel()).reshape(n, n)
        errs.append(np.abs(y - u(g.r[:, None], g.z[None, :])).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.5 < x < 5.1 for x in ratios), ratios
    assert errs[-1] < 1e-4


# ------------------------------------------------------------- sine transform
def test_dst1_golden_and_closed_forms():
    lines = [l for l in open(os.path.join(GOLDEN, "dst1_n3.txt")) if not l.startswith("#")]
    S3 = np.array([[float(x) for x in l.split()] for l in lines[:3]])
    np.testing.assert_allclose(O.dst1_matrix(3), S3, atol=1e-15)
    eig = [float(x) for x in lines[3].split()[1:]]
    np.testing.assert_allclose(O.mode_eigenvalues(3, 0.25), eig, rtol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 7, 64, 127])
def test_dst1_orthogonal_and_matches_scipy(n):
    S = O.dst1_matrix(n)
    np.testing.assert_allclose(S @ S, np.eye(n), atol=1e-13)
    ref = scipy.fft.dst(np.eye(n), type=1, norm="ortho", axis=0)
    np.testing.assert_allclose(S, ref, atol=1e-14)


@pytest.mark.parametrize("n", [1, 5, 33])
def test_dst1_diagonalises_dirichlet_second_difference(n):
    h = 1.0 / (n + 1)
    L = (2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)) / h ** 2
    S = O.dst1_matrix(n)
    np.testing.assert_allclose(S @ L @ S, np.diag(O.mode_eigenvalues(n, h)), atol=1e-9 * (n + 1) ** 2)


# ------------------------------------------------------------------- Thomas
@pytest.mark.parametrize("n,k", [(1, 1), (2, 3), (3, 1), (17, 4), (100, 2)])
def test_thomas_matches_banded_solver(n, k):
    rng = np.random.default_rng(n)
    sub = rng.uniform(-1, 1, n - 1)
    sup = rng.uniform(-1, 1, n - 1)
    diag = 2.5 + rng.uniform(0, 1, n)
    b = rng.normal(size=(n, k))
    ab = np.zeros((3, n))
    ab[0, 1:], ab[1], ab[2, :-1] = sup, diag, sub
    ref = scipy.linalg.solve_banded((1, 1), ab, b)
    np.testing.assert_allclose(O.thomas(sub, diag, sup, b), ref, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------ preconditioner
@pytest.mark.parametrize("nr,nz", [(1, 1), (2, 3), (5, 2), (8, 8), (13, 6)])
def test_precond_solve_matches_dense_solve_of_B(nr, nz):
    g = O.Grid(nr, nz)
    kt, qt = 1.7, 0.35
    B = O.assemble_preconditioner(kt, qt, g).toarray()
    v = np.random.default_rng(nr * 31 + nz).normal(size=(nr, nz))
    ref = np.linalg.solve(B, v.ravel()).reshape(nr, nz)
    np.testing.assert_allclose(O.precond_solve(v, kt, qt, g), ref, rtol=1e-11, atol=1e-13)


def test_preconditioner_constants_mean_of_extremes():
    kr = np.array([[1.0, 4.0]])
    kz = np.array([[2.0, 3.0, 9.0]])
    q = np.array([[0.5, 1.5]])
    assert O.preconditioner_constants(kr, kz, q) == (5.0, 1.0)


def test_pcg_one_iteration_when_coefficients_constant():
    """kappa and q constant => B = A exactly (Eq. coeff2), so PCG converges in
    one step."""
    g = O.Grid(24, 20)
    med = Medium("const", lambda r, z: np.full(np.broadcast(r, z).shape, 2.3),
                 lambda r, z: np.full(np.broadcast(r, z).shape, 0.7),
                 [lambda r, z: np.exp(-((r - .3) ** 2 + (z - .6) ** 2) * 20)])
    kr, kz, q, f = O.sample_medium(med, g)
    op = O.Operator(kr, kz, q, g)
    assert (abs(op.A - O.assemble_preconditioner(op.kappa_t, op.q_t, g)).max()) < 1e-10
    y, info = op.solve(f[0], tol=1e-13)
    assert info.iters == 1 and info.rel_res <= 1e-13


# ------------------------------------------------------------------------ PCG
@pytest.mark.parametrize("nr,nz", [(3, 4), (16, 9), (33, 20)])
def test_pcg_matches_direct_solve(nr, nz):
    op, f = _op(nr, nz, seed=nr)
    y, info = op.solve(f[0], tol=1e-13)
    ref = spl.spsolve(op.A.tocsc(), op.phi(f[0]).ravel()).reshape(nr, nz)
    assert info.converged
    assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)


def test_pcg_bumps_64_matches_direct_solve():
    g = O.Grid(64, 64)
    kr, kz, q, f = O.sample_medium(bumps_medium(), g)
    op = O.Operator(kr, kz, q, g)
    y, info = op.solve(f[0], tol=1e-10)
    assert info.converged and info.rel_res <= 1e-10
    ref = spl.spsolve(op.A.tocsc(), op.phi(f[0]).ravel()).reshape(64, 64)
    assert np.linalg.norm(y - ref) <= 1e-8 * np.linalg.norm(ref)
    assert 5 <= info.iters <= 60


def test_pcg_iterations_independent_of_grid():
    """The condition number of B^-1 A does not depend on h (Section 2.2), and
    Table 2 prints nearly equal counts for three grids."""
    its = []
    for n in (32, 64, 128):
        g = O.Grid(n, n)
        kr, kz, q, f = O.sample_medium(bumps_medium(), g)
        _, info = O.Operator(kr, kz, q, g).solve(f[0], tol=1e-10)
        its.append(info.iters)
    assert max(its) <= 1.15 * min(its) + 1, its


# ------------------------------------------------------------------ Chebyshev
def test_chebyshev_bounds_contain_generalised_spectrum():
    op, _ = _op(6, 5, seed=7)
    A = op.A.toarray()
    B = O.assemble_preconditioner(op.kappa_t, op.q_t, op.grid).toarray()
    ev = scipy.linalg.eigh(A, B, eigvals_only=True)
    g1, g2 = op.gamma
    assert g1 <= ev.min() * (1 + 1e-12) and ev.max() <= g2 * (1 + 1e-12)


def test_chebyshev_error_bound_each_step():
    """A-norm error after n steps <= 2 rho1^n / (1 + rho1^(2n)) ||e0||_A,
    rho1 = (1 - sqrt(xi)) / (1 + sqrt(xi)): the Chebyshev-polynomial bound."""
    op, f = _op(10, 12, seed=11)
    phi = op.phi(f[0])
    u = spl.spsolve(op.A.tocsc(), phi.ravel()).reshape(phi.shape)
    A = op.A

    def anorm(e):
        return math.sqrt(float(e.ravel() @ (A @ e.ravel())))

    g1, g2 = op.gamma
    xi = g1 / g2
    rho1 = (1 - math.sqrt(xi)) / (1 + math.sqrt(xi))
    e0 = anorm(u)
    for n in range(1, 12):
        y, info = O.chebyshev(op.apply_A, op.apply_Binv, phi, g1, g2, tol=0.0, max_iter=n)
        assert info.iters == n
        bound = 2 * rho1 ** n / (1 + rho1 ** (2 * n))
        assert anorm(u - y) <= bound * e0 * (1 + 1e-9) + 1e-14


def test_lanczos_ritz_values_interlace_and_converge():
    """The Lanczos tridiagonal of the PCG coefficients: its Ritz values lie
    inside the spectrum of B^-1 A (the generalised eigenvalues of (A, B),
    scipy.linalg.eigh) and its extreme ones reach the extreme eigenvalues."""
    op, f = _op(6, 5, seed=3)
    A = op.A.toarray()
    B = O.assemble_preconditioner(op.kappa_t, op.q_t, op.grid).toarray()
    ev = scipy.linalg.eigh(A, B, eigvals_only=True)
    phi = op.phi(f[0])
    for steps in (3, 6, 12, 24):
        g1, g2, al, be = O.lanczos_bounds(op.apply_A, op.apply_Binv, phi, steps=steps, widen=0.0)
        assert len(al) == steps and len(be) == steps
        assert g1 >= ev.min() * (1 - 1e-10) and g2 <= ev.max() * (1 + 1e-10), steps
    assert g1 <= ev.min() * (1 + 1e-6) and g2 >= ev.max() * (1 - 1e-6)


@pytest.mark.parametrize("q_zero", [False, True])
def test_lanczos_bounds_contain_spectrum_and_drive_chebyshev(q_zero):
    """20 PCG steps, widened 5%, enclose the spectrum of B^-1 A on a 16 x 14
    grid (10 steps leave the smallest Ritz value 6% above lambda_min here);
    with q = 0 on part of the domain (q_min = 0 < q_max) the face-wise
    gamma_1 is 0 (degenerate) while the estimate is not, and the Chebyshev
    iteration with the estimate converges in at most 1.5 times the PCG
    iterations (plus 4)."""
    g = O.Grid(16, 14)
    med = _random_medium(5)
    if q_zero:
        med = Medium("qzero", med.kappa, lambda r, z: np.where(z < 0.5, 0.0, 0.8) + 0 * r, med.sources)
    kr, kz, q, f = O.sample_medium(med, g)
    op = O.Operator(kr, kz, q, g)
    A = op.A.toarray()
    B = O.assemble_preconditioner(op.kappa_t, op.q_t, g).toarray()
    ev = scipy.linalg.eigh(A, B, eigvals_only=True)
    phi = op.phi(f[0])
    g1, g2, _, _ = O.lanczos_bounds(op.apply_A, op.apply_Binv, phi, steps=20, widen=0.05)
    assert 0.0 < g1 <= ev.min() and ev.max() <= g2
    if q_zero:
        assert op.gamma[0] == 0.0
    _, ipcg = op.solve(f[0], tol=1e-10)
    _, icheb = O.chebyshev(op.apply_A, op.apply_Binv, phi, g1, g2, tol=1e-10)
    assert icheb.converged and icheb.iters <= 1.5 * ipcg.iters + 4, (icheb.iters, ipcg.iters)


def test_chebyshev_agrees_with_pcg():
    g = O.Grid(64, 64)
    kr, kz, q, f = O.sample_medium(bumps_medium(), g)
    op = O.Operator(kr, kz, q, g)
    y1, i1 = op.solve(f[0], tol=1e-11)
    y2, i2 = op.solve(f[0], tol=1e-11, method="cheb")
    assert i1.converged and i2.converged
    assert np.linalg.norm(y1 - y2) <= 1e-8 * np.linalg.norm(y1)


# ---------------------------------------------- zero-flux z boundary (bc_z = 1)
def _op_n(nr, nz, seed=0, q_zero=False):
    g = O.Grid(nr, nz, bc_z=1)
    med = _random_medium(seed)
    if q_zero:
        med = Medium("rand0", med.kappa, lambda r, z: np.zeros(np.broadcast(r, z).shape), med.sources)
    kr, kz, q, f = O.sample_medium(med, g)
    return O.Operator(kr, kz, q, g), f


@pytest.mark.parametrize("nr,nz", [(1, 1), (1, 4), (3, 1), (3, 5), (6, 4), (9, 7)])
@pytest.mark.parametrize("q_zero", [False, True])
def test_neumann_operator_symmetric_positive_definite(nr, nz, q_zero):
    """With zero flux at z = 0, lz and q = 0 the only Dirichlet part is r = 1,
    which still makes A definite (Eq. main_eq with Eq. elliptic_condition)."""
    op, _ = _op_n(nr, nz, q_zero=q_zero)
    A = op.A.toarray()
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0.0


def test_neumann_row_sums_conservative():
    """Every z-row is interior once the boundary faces carry no flux: (A 1) = W
    on all rows but the last r-row (a non-zero boundary flux fails this)."""
    nr, nz = 7, 9
    op, _ = _op_n(nr, nz, seed=3)
    s = op.apply_A(np.ones((nr, nz)))
    np.testing.assert_allclose(s[:-1], op.W[:-1], rtol=1e-12, atol=1e-12)


def test_neumann_grid_nodes_and_faces():
    g = O.Grid(3, 4, lz=2.0, bc_z=1)
    np.testing.assert_allclose(g.z, [0.25, 0.75, 1.25, 1.75], rtol=1e-15)
    np.testing.assert_allclose(g.zbar, [0.0, 0.5, 1.0, 1.5, 2.0], rtol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 7, 64, 127])
def test_cosine_pair_matches_scipy_and_inverts(n):
    """Eq. fft_phi's sums are scipy's unnormalised DCT-II (forward) and DCT-III
    (inverse) times sqrt(2/n) / 2; the pair inverts exactly."""
    F, G = O.cosine_pair(n)
    I = np.eye(n)
    np.testing.assert_allclose(F, 0.5 * math.sqrt(2.0 / n) * scipy.fft.dct(I, type=2, axis=0), atol=1e-14)
    np.testing.assert_allclose(G.T, 0.5 * math.sqrt(2.0 / n) * scipy.fft.dct(I, type=3, axis=0), atol=1e-14)
    np.testing.assert_allclose(F.T @ G, I, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 5, 33])
def test_cosine_diagonalises_zero_flux_second_difference(n):
    """Eq. eq_trid's shift: the rows of F are eigenvectors of the second
    difference with one-sided end rows, eigenvalues 4/h^2 sin^2(pi(l-1)/(2n))."""
    h = 1.0 / n
    L = (2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))
    L[0, 0] -= 1.0  # no flux through the face z = 0
    L[-1, -1] -= 1.0  # nor through z = lz
    L /= h ** 2
    F, _ = O.cosine_pair(n)
    lam = O.mode_eigenvalues(n, h, bc_z=1)
    assert lam[0] == 0.0
    np.testing.assert_allclose(L @ F.T, F.T * lam[None, :], atol=1e-9 * n ** 2)


@pytest.mark.parametrize("nr,nz", [(1, 1), (2, 3), (5, 2), (8, 8), (13, 6)])
@pytest.mark.parametrize("qt", [0.35, 0.0])
def test_neumann_precond_solve_matches_dense_solve_of_B(nr, nz, qt):
    g = O.Grid(nr, nz, bc_z=1)
    kt = 1.7
    B = O.assemble_preconditioner(kt, qt, g).toarray()
    v = np.random.default_rng(nr * 31 + nz).normal(size=(nr, nz))
    ref = np.linalg.solve(B, v.ravel()).reshape(nr, nz)
    np.testing.assert_allclose(O.precond_solve(v, kt, qt, g), ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("variable_kappa", [False, True])
def test_neumann_manufactured_solution_second_order(variable_kappa):
    """u* = cos(pi r/2) cos(pi z) has zero z-flux at z = 0, 1: the max-norm
    nodal error must fall about 4x per halving of h (Section 2.1)."""
    med, u = manufactured_medium_neumann(q0=1.0, variable_kappa=variable_kappa)
    errs = []
    for n in (16, 32, 64, 128):
        g = O.Grid(n, n, bc_z=1)
        kr, kz, q, f = O.sample_medium(med, g)
        op = O.Operator(kr, kz, q, g)
        y = spl.spsolve(op.A.tocsc(), op.phi(f[0]).ravel()).reshape(n, n)
        errs.append(np.abs(y - u(g.r[:, None], g.z[None, :])).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.5 < x < 5.1 for x in ratios), ratios
    assert errs[-1] < 1e-3


@pytest.mark.parametrize("q0", [0.7, 0.0])
def test_neumann_pcg_one_iteration_when_coefficients_constant(q0):
    g = O.Grid(24, 20, bc_z=1)
    med = Medium("const", lambda r, z: np.full(np.broadcast(r, z).shape, 2.3),
                 lambda r, z: np.full(np.broadcast(r, z).shape, q0),
                 [lambda r, z: np.exp(-((r - .3) ** 2 + (z - .6) ** 2) * 20)])
    kr, kz, q, f = O.sample_medium(med, g)
    op = O.Operator(kr, kz, q, g)
    assert (abs(op.A - O.assemble_preconditioner(op.kappa_t, op.q_t, g)).max()) < 1e-10
    y, info = op.solve(f[0], tol=1e-12)
    assert info.iters == 1 and info.rel_res <= 1e-12


@pytest.mark.parametrize("nr,nz", [(3, 4), (16, 9), (33, 20)])
def test_neumann_pcg_and_chebyshev_match_direct_solve(nr, nz):
    op, f = _op_n(nr, nz, seed=nr)
    ref = spl.spsolve(op.A.tocsc(), op.phi(f[0]).ravel()).reshape(nr, nz)
    for method in ("pcg", "cheb"):
        y, info = op.solve(f[0], tol=1e-13, method=method)
        assert info.converged
        assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)


def test_neumann_chebyshev_bounds_contain_generalised_spectrum():
    op, _ = _op_n(6, 5, seed=7)
    A = op.A.toarray()
    B = O.assemble_preconditioner(op.kappa_t, op.q_t, op.grid).toarray()
    ev = scipy.linalg.eigh(A, B, eigvals_only=True)
    g1, g2 = op.gamma
    assert g1 <= ev.min() * (1 + 1e-12) and ev.max() <= g2 * (1 + 1e-12)
