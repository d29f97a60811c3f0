"""Every FP32 mode-solve kernel variant (option "mode_kernel") against the
oracle, through the C ABI.

The per-mode systems T_l y = b (Section 4.2, Eq. eq_trid; one fixed matrix
per mode, Section 3, Eq. main_eq3) are solved by whichever kernel the
option selects: 1 the staged register kernel, 9 the same on the row-scaled
systems (12 on 16-column tiles), 10 and 11 that one with the factors kept
over 4 or 8 right-hand sides, 14 the staged kernel fed mode-major by the
forward tensor-core transform (through the preconditioner and the solves; a
row-major input, as in ax_apply_mode_solve, takes 9), 2..8 the pipelined column-tile kernels (persistent CTAs, lanes along
the mode index, chunk carries composed by a shared-memory scan).  Each variant that covers nr must give
  - the backward error ||T_l y - b|| <= 2e-6 ||T_l|| ||y|| of every column
    (FP32), and the forward error against the oracle's Thomas <= 1e-3;
  - through the tensor-core preconditioner (split BF16 output of the mode
    solves, AX_PREC_FP32_TC3) the same B^-1 as the register kernel to 1e-4
    (two FP32 eliminations of systems with cond ~ nr^2 differ by their
    rounding) and the FP64 B^-1 to 1e-3;
  - a mixed PCG solve (the split output plus its (rhat, yhat) partials, masks
    of converged right-hand sides) whose oracle FP64 true residual is <= 1e-8.
Shapes span partial column tiles (nz not a multiple of the tile width),
ragged chunks (nr not a multiple of 16) and both CTA sizes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_1002_3094_gb300 as P  # noqa: E402
from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs  # noqa: E402
from workloads import layered_inclusion_medium  # noqa: E402

pytestmark = pytest.mark.gpu

VARIANTS = range(1, 15)


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.load_library()
    return torch.device("cuda:0")


def _setup(nr, nz, dev, n_rhs=3, seed=4):
    med = layered_inclusion_medium(n_rhs=n_rhs, nominal_n=max(nr, nz), instance=seed)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(dev) for x in (kr, kz, q)], nr, nz)
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz))
    return op, ora, med


def _covering(op):
    """Variant ids the library accepts for this operator's nr."""
    ok = [v for v in VARIANTS if P.ax_set_option(op, "mode_kernel", v, raise_on_error=False) == P.AX_OK]
    P.ax_set_option(op, "mode_kernel", 0)
    return ok


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SHAPES = [(300, 37), (511, 64), (513, 100), (700, 130), (1024, 96), (1300, 45), (2047, 40), (2500, 24),
          (4096, 20)]


def test_variant_lists(cuda):
    """Each nr is covered by the register kernel and by the pipelined kernels
    whose column fits it with at most half idle; unknown ids are refused."""
    reg = {1, 9, 10, 11, 14}
    for nr, want in [(64, reg | {12}), (300, reg | {2, 3, 12}), (1024, reg | {4, 5, 12}), (2047, reg | {6, 7}),
                     (4096, reg | {8}), (5000, set())]:
        op, _, _ = _setup(nr, 8, cuda)
        assert set(_covering(op)) == want, nr
        assert P.ax_set_option(op, "mode_kernel", 13, raise_on_error=False) == P.AX_ERR_INVALID_ARG
        assert P.ax_set_option(op, "mode_kernel", 15, raise_on_error=False) == P.AX_ERR_INVALID_ARG
        assert P.ax_set_option(op, "mode_kernel", 1.5, raise_on_error=False) == P.AX_ERR_INVALID_ARG
        P.ax_destroy_operator(op)


@pytest.mark.parametrize("nr,nz", SHAPES)
def test_mode_solves_every_variant(cuda, nr, nz):
    op, ora, _ = _setup(nr, nz, cuda)
    m = 3
    b = np.random.default_rng(nr + nz).normal(size=(m, nr, nz))
    g = ora.grid
    lam = O.mode_eigenvalues(nz, g.hz)
    sub, diag, sup = O.mode_tridiagonal(ora.kappa_t, ora.q_t, lam, g)
    tnorm = np.abs(diag).max() + 2 * np.abs(sub).max()
    ref = [O.thomas(sub, diag, sup, b[j]) for j in range(m)]
    bd = torch.from_numpy(b).to(cuda)
    for v in _covering(op):
        P.ax_set_option(op, "mode_kernel", v)
        out = torch.zeros((m, nr, nz), dtype=torch.float64, device=cuda)
        P.ax_apply_mode_solve(op, bd, out, m, P.AX_PREC_FP32)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for j in range(m):
            y = got[j]
            Ty = diag * y
            Ty[:-1] += sup * y[1:]
            Ty[1:] += sub * y[:-1]
            res = np.linalg.norm(Ty - b[j], axis=0)
            assert (res <= 2e-6 * tnorm * np.linalg.norm(y, axis=0)).all(), (v, j)
            assert _rel(y, ref[j]) <= 1e-3, (v, j)
    P.ax_destroy_operator(op)


@pytest.mark.parametrize("nr,nz", [(511, 200), (1024, 130), (2047, 72), (4096, 40)])
def test_tensor_preconditioner_every_variant(cuda, nr, nz):
    op, _, _ = _setup(nr, nz, cuda)
    m = 2
    x = torch.from_numpy(np.random.default_rng(7).normal(size=(m, nr, nz))).to(cuda)
    outs = {}
    for v in _covering(op):
        P.ax_set_option(op, "mode_kernel", v)
        out = torch.zeros((m, nr, nz), dtype=torch.float64, device=cuda)
        P.ax_apply_preconditioner(op, x, out, m, P.AX_PREC_FP32_TC3)
        torch.cuda.synchronize()
        outs[v] = out.cpu().numpy()
    ex = torch.zeros((m, nr, nz), dtype=torch.float64, device=cuda)
    P.ax_apply_preconditioner(op, x, ex, m, P.AX_PREC_FP64)
    ex = ex.cpu().numpy()
    for v, got in outs.items():
        assert _rel(got, outs[1]) <= 1e-4, v
        assert _rel(got, ex) <= 1e-3, v
    P.ax_destroy_operator(op)


@pytest.mark.parametrize("nr,nz", [(700, 96), (1024, 64), (2047, 33)])
def test_mixed_pcg_every_variant(cuda, nr, nz):
    op, ora, med = _setup(nr, nz, cuda, n_rhs=3)
    f = sample_rhs(med, nr, nz)
    fd = torch.from_numpy(f).to(cuda)
    for v in _covering(op):
        P.ax_set_option(op, "mode_kernel", v)
        u = torch.zeros_like(fd)
        st, info = P.ax_solve(op, fd, u, 3, 1e-8, 5000, P.AX_PCG_MIXED)
        torch.cuda.synchronize()
        assert st == P.AX_OK, (v, info)
        un = u.cpu().numpy()
        for j in range(3):
            phi = ora.phi(f[j])
            assert np.linalg.norm(phi - ora.apply_A(un[j])) <= 1e-8 * np.linalg.norm(phi), (v, j)
    P.ax_destroy_operator(op)
