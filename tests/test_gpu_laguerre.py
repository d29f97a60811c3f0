"""The Laguerre-harmonic chain (Section 4.1, Eq. laguerre_h) on the GPU
against the oracle's direct sums: the running-field step element by element,
and whole chains of sequential solves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle import laguerre as L  # noqa: E402
import paper_1002_3094_gb300 as P  # noqa: E402
from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs  # noqa: E402
from paper_1002_3094_gb300.laguerre import solve_chain  # noqa: E402
from workloads.laguerre import ALPHA, H_LAG, fault_medium  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.load_library()
    return torch.device("cuda:0")


def _setup(nr, nz, lr, dev):
    med = fault_medium(lr, lr, sigma=2.5 * lr / nr)
    kr, kz, q = sample_operator_inputs(med, nr, nz, lr, lr, bc_z=1)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(dev) for x in (kr, kz, q)], nr, nz, lr, lr, bc_z=1)
    src = sample_rhs(med, nr, nz, lr, lr, bc_z=1)[0]
    src = src / np.abs(src).max()
    c2 = 4.0 * q
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz, lr, lr, bc_z=1))
    return op, ora, c2, src


@pytest.mark.parametrize("nr,nz", [(40, 24), (33, 65)])
def test_step_matches_the_direct_sum(cuda, nr, nz):
    op, _, c2, src = _setup(nr, nz, 512.0, cuda)
    rng = np.random.default_rng(nr + nz)
    Q = [rng.normal(size=(nr, nz)) for _ in range(7)]
    fm = rng.normal(size=8)
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda)
    T, S, f = (torch.zeros((nr, nz), dtype=torch.float64, device=cuda) for _ in range(3))
    c2d, srcd = d(c2), d(src)
    P.ax_laguerre_step(op, None, T, S, c2d, srcd, 0.0, L.weights(0, ALPHA)[0], fm[0], f)
    assert np.array_equal(f.cpu().numpy(), fm[0] * src)
    for m in range(7):
        P.ax_laguerre_step(op, d(Q[m]), T, S, c2d, srcd, L.weights(m, ALPHA)[1], L.weights(m + 1, ALPHA)[0],
                           fm[m + 1], f)
        want = L.harmonic_rhs(m + 1, Q[:m + 1], c2, src, fm[m + 1], ALPHA)
        got = f.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), m
    with pytest.raises(P.AxError):
        P.ax_laguerre_step(op, d(Q[0]), T, S, c2d, srcd, float("nan"), 1.0, 1.0, f)
    with pytest.raises(P.AxError):  # no field to add, but a weight
        P.ax_laguerre_step(op, None, T, S, c2d, srcd, 0.5, 1.0, 1.0, f)
    with pytest.raises(P.AxError):  # Q is read while T is written
        P.ax_laguerre_step(op, T, T, S, c2d, srcd, 0.5, 1.0, 1.0, f)
    P.ax_destroy_operator(op)


@pytest.mark.parametrize("method,tol", [(P.AX_PCG_FP64, 1e-12), (P.AX_PCG_MIXED, 1e-9)])
def test_chain_matches_the_oracle_chain(cuda, method, tol):
    nr, nz, n = 48, 40, 6
    op, ora, c2, src = _setup(nr, nz, 256.0, cuda)
    fm = np.array([1.0, -0.6, 0.35, 0.2, -0.1, 0.05])
    want = L.chain(lambda rhs, prev: ora.solve(rhs, 1e-13)[0], c2, src, fm, ALPHA)
    got = []
    q = torch.zeros((1, nr, nz), dtype=torch.float64, device=cuda)
    work = torch.zeros((3, nr, nz), dtype=torch.float64, device=cuda)
    infos = solve_chain(op, torch.from_numpy(c2).to(cuda), torch.from_numpy(src).to(cuda), fm, ALPHA, tol, q, work,
                        method=method, on_harmonic=lambda m, u, info: got.append(u[0].cpu().numpy().copy()))
    assert len(infos) == n
    for m in range(n):
        # each GPU harmonic meets the tolerance for the right-hand side its own
        # earlier harmonics define, and the chain stays within the tolerance's
        # propagation of the oracle chain
        phi = ora.phi(L.harmonic_rhs(m, got[:m], c2, src, fm[m], ALPHA))
        assert np.linalg.norm(phi - ora.apply_A(got[m])) <= tol * np.linalg.norm(phi), m
        assert np.linalg.norm(got[m] - want[m]) <= 1e3 * tol * np.linalg.norm(want[m]), m
    P.ax_destroy_operator(op)
