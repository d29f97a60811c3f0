"""The persistent small-grid FP64 PCG (one cooperative launch per solve)
against the oracle and the graph-replayed FP64 path, through the C ABI.

AX_PCG_FP64 of one right-hand side on a grid with nr <= 512, nz <= 256,
nr nz <= 65536 runs the whole iteration (Section 2.2, Eq. main-scheme, with
the preconditioner of Section 4.2) in one launch, phases separated by bounded
grid barriers, the z-transform as dense FP64 products and the mode solves as
warp-cooperative chunked Thomas (Section 3's dichotomy observation).  It must
  - meet the tolerance in the oracle's FP64 true residual, and agree with the
    graph-replayed path (option small_path = 0) in iterations (within 1) and
    solution (1e-9 relative, both stop on the same true-residual test);
  - cover sine and cosine z-transforms, one-row and one-column grids, the
    largest sizes it takes, warm starts (AX_FLAG_USE_GUESS) including an
    exact guess (no iteration), and max_iter (AX_ERR_NO_CONVERGENCE);
  - take host buffers (set-up on the host side, then the persistent launch)
    and a zero right-hand side (converged at the start, u = 0);
  - on the expiry path (option small_stall_test: one CTA leaves before the
    first barrier, so the others' bounded waits run out) return
    AX_ERR_TIMEOUT, with the next solve on the same context correct.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_1002_3094_gb300 as P  # noqa: E402
from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs  # noqa: E402
from workloads import bumps_medium, layered_inclusion_medium  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.load_library()
    return torch.device("cuda:0")


def _setup(med, nr, nz, dev, bc_z=0):
    kr, kz, q = sample_operator_inputs(med, nr, nz, bc_z=bc_z)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(dev) for x in (kr, kz, q)], nr, nz, bc_z=bc_z)
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz, bc_z=bc_z))
    f = sample_rhs(med, nr, nz, bc_z=bc_z)[:1]
    return op, ora, f


def _solve(op, f, dev, small, tol, max_iter=5000, u0=None, raise_on_error=True):
    P.ax_set_option(op, "small_path", 1 if small else 0)
    fd = torch.from_numpy(f).to(dev)
    u = torch.from_numpy(u0).to(dev) if u0 is not None else torch.zeros_like(fd)
    flags = P.AX_FLAG_USE_GUESS if u0 is not None else 0
    st, info = P.ax_solve(op, fd, u, 1, tol, max_iter, P.AX_PCG_FP64, flags, raise_on_error=raise_on_error)
    torch.cuda.synchronize()
    return st, info[0], u.cpu().numpy()[0]


def _true_res(ora, f, u):
    phi = ora.phi(f)
    return np.linalg.norm(phi - ora.apply_A(u)) / np.linalg.norm(phi)


SHAPES = [(64, 64, 0), (1, 1, 0), (1, 7, 0), (5, 3, 0), (33, 17, 0), (100, 50, 0), (512, 64, 0), (200, 256, 0),
          (64, 1, 0), (128, 128, 1), (37, 90, 1), (256, 256, 0)]


@pytest.mark.parametrize("nr,nz,bc", SHAPES)
def test_small_path_matches_oracle_and_graph_path(cuda, nr, nz, bc):
    med = bumps_medium(0) if (nr, nz) == (64, 64) else layered_inclusion_medium(n_rhs=1, nominal_n=max(nr, nz),
                                                                                 instance=nr + nz)
    op, ora, f = _setup(med, nr, nz, cuda, bc)
    tol = 1e-10
    st, i1, u1 = _solve(op, f[0:1], cuda, True, tol)
    assert st == P.AX_OK and i1["status"] == P.AX_OK
    st, i0, u0 = _solve(op, f[0:1], cuda, False, tol)
    assert st == P.AX_OK
    assert _true_res(ora, f[0], u1) <= tol
    assert abs(i1["iters"] - i0["iters"]) <= 1, (i1, i0)
    assert np.linalg.norm(u1 - u0) <= 1e-9 * np.linalg.norm(u0)
    P.ax_destroy_operator(op)


def test_warm_starts_and_max_iter(cuda):
    nr, nz = 96, 80
    med = layered_inclusion_medium(n_rhs=1, nominal_n=96, instance=11)
    op, ora, f = _setup(med, nr, nz, cuda)
    st, i_ref, u_ref = _solve(op, f, cuda, True, 1e-10)
    assert st == P.AX_OK
    # the exact answer as the guess: converged at the start
    st, i_ex, u_ex = _solve(op, f, cuda, True, 1e-8, u0=u_ref[None])
    assert st == P.AX_OK and i_ex["iters"] == 0
    # a perturbed guess: fewer iterations than from zero, same tolerance
    g = u_ref * (1.0 + 1e-3 * np.random.default_rng(2).normal(size=u_ref.shape))
    st, i_g, u_g = _solve(op, f, cuda, True, 1e-10, u0=g[None])
    assert st == P.AX_OK and i_g["iters"] < i_ref["iters"]
    assert _true_res(ora, f[0], u_g) <= 1e-10
    # max_iter: no convergence after exactly that many iterations
    st, i_m, _ = _solve(op, f, cuda, True, 1e-14, max_iter=3, raise_on_error=False)
    assert st == P.AX_ERR_NO_CONVERGENCE and i_m["iters"] == 3
    st0, i_m0, _ = _solve(op, f, cuda, False, 1e-14, max_iter=3, raise_on_error=False)
    assert st0 == P.AX_ERR_NO_CONVERGENCE and i_m0["iters"] == 3
    P.ax_destroy_operator(op)


def test_option_and_fallbacks(cuda):
    med = layered_inclusion_medium(n_rhs=2, nominal_n=64, instance=3)
    op, ora, f2 = _setup(med, 64, 48, cuda)
    assert int(P.ax_get_option(op, "small_path")) == 1
    assert P.ax_set_option(op, "small_path", 2, raise_on_error=False) == P.AX_ERR_INVALID_ARG
    # two right-hand sides take the graph-replayed path
    f = sample_rhs(med, 64, 48)
    fd = torch.from_numpy(f).to(cuda)
    u = torch.zeros_like(fd)
    st, info = P.ax_solve(op, fd, u, 2, 1e-10, 5000, P.AX_PCG_FP64)
    assert st == P.AX_OK
    for j in range(2):
        assert _true_res(ora, f[j], u.cpu().numpy()[j]) <= 1e-10
    # host buffers: the set-up runs on the host side, then the persistent launch
    fh = np.ascontiguousarray(f[:1])
    uh = np.zeros_like(fh)
    st, info = P.ax_solve(op, fh, uh, 1, 1e-10, 5000, P.AX_PCG_FP64, P.AX_FLAG_HOST_BUFFERS)
    assert st == P.AX_OK and _true_res(ora, f[0], uh[0]) <= 1e-10
    # a zero right-hand side: converged at the start, u = 0
    z = torch.zeros((1, 64, 48), dtype=torch.float64, device=cuda)
    uz = torch.ones_like(z)
    st, info = P.ax_solve(op, z, uz, 1, 1e-10, 5000, P.AX_PCG_FP64)
    assert st == P.AX_OK and info[0]["iters"] == 0 and float(uz.abs().max()) == 0.0
    P.ax_destroy_operator(op)


def test_bounded_wait_expiry_returns_timeout(cuda):
    med = bumps_medium(0)
    op, ora, f = _setup(med, 64, 64, cuda)
    P.ax_set_option(op, "small_stall_test", 1)
    st, _, _ = _solve(op, f, cuda, True, 1e-10, raise_on_error=False)
    assert st == P.AX_ERR_TIMEOUT
    st, i1, u1 = _solve(op, f, cuda, True, 1e-10)
    assert st == P.AX_OK
    assert _true_res(ora, f[0], u1) <= 1e-10
    P.ax_destroy_operator(op)
