"""The stencil variants (option "stencil_kernel") against the oracle, through
the C ABI.

The operator of Eq. scheme_op_r_z (Section 2.1) is applied by the register-
window kernel (0) or by the kernel whose producer warp streams p and the
coefficient rows through a ring of shared-memory slots with bulk copies (1).
Each must give
  - y -> A y in FP32 within 2e-6 of the oracle's FP64 A y, and bit for bit
    the register kernel's result (the same FMAs in the same order per node);
  - in the fused mixed PCG iteration (q = A p with the (p, q) partials, summed
    over other CTA tiles by variant 1), an oracle FP64 true residual <= 1e-8
    within 2 iterations of variant 0;
  - on the expiry path (option "stencil_stall_test": no copy is issued, every
    bounded wait runs out) AX_ERR_TIMEOUT, and a correct result from the next
    call on the same context.
Shapes span one and several column strips of 1024 (nz > 1024, ragged last
strip), nz a multiple of 128 (the range tests compiled out) and not, nz not a
multiple of 4, nr not a multiple of the rows per CTA, and a single row.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_1002_3094_gb300 as P  # noqa: E402
from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs  # noqa: E402
from workloads import layered_inclusion_medium  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.load_library()
    return torch.device("cuda:0")


def _setup(nr, nz, dev, n_rhs=3, seed=5):
    med = layered_inclusion_medium(n_rhs=n_rhs, nominal_n=max(nr, nz), instance=seed)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(dev) for x in (kr, kz, q)], nr, nz)
    return op, O.Operator(kr, kz, q, O.Grid(nr, nz)), med


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _apply(op, y, dev):
    m = y.shape[0]
    out = torch.zeros(y.shape, dtype=torch.float64, device=dev)
    P.ax_apply_operator(op, torch.from_numpy(y).to(dev), out, m, P.AX_PREC_FP32)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("nr,nz,m", [(1, 7, 2), (5, 3, 3), (17, 130, 2), (40, 1024, 1), (33, 1030, 3), (100, 2051, 2),
                                     (250, 4096, 2), (1031, 96, 3), (1, 128, 1), (19, 384, 2), (64, 2048, 1),
                                     (65, 1000, 1)])
def test_apply_matches_oracle_and_register_kernel(cuda, nr, nz, m):
    op, ora, _ = _setup(nr, nz, cuda)
    y = np.random.default_rng(nr * 7 + nz).normal(size=(m, nr, nz))
    ref = _apply(op, y, cuda)
    P.ax_set_option(op, "stencil_kernel", 1)
    assert int(P.ax_get_option(op, "stencil_kernel")) == 1
    got = _apply(op, y, cuda)
    assert np.array_equal(got, ref), np.abs(got - ref).max()
    for j in range(m):
        assert _rel(got[j], ora.apply_A(y[j])) <= 2e-6
    P.ax_destroy_operator(op)


@pytest.mark.parametrize("nr,nz", [(600, 200), (1024, 96), (129, 1300), (200, 1024), (301, 256)])
def test_fused_mixed_pcg(cuda, nr, nz):
    op, ora, med = _setup(nr, nz, cuda)
    f = sample_rhs(med, nr, nz)
    fd = torch.from_numpy(f).to(cuda)
    P.ax_set_option(op, "dst_tensor", 1)
    iters = {}
    for v in (0, 1):
        P.ax_set_option(op, "stencil_kernel", v)
        u = torch.zeros_like(fd)
        st, info = P.ax_solve(op, fd, u, 3, 1e-8, 5000, P.AX_PCG_MIXED)
        torch.cuda.synchronize()
        assert st == P.AX_OK
        iters[v] = [i["iters"] for i in info]
        un = u.cpu().numpy()
        for j in range(3):
            phi = ora.phi(f[j])
            assert np.linalg.norm(phi - ora.apply_A(un[j])) <= 1e-8 * np.linalg.norm(phi), (v, j)
    assert all(abs(a - b) <= 2 for a, b in zip(iters[1], iters[0])), iters
    P.ax_destroy_operator(op)


def test_option_values(cuda):
    op, _, _ = _setup(64, 64, cuda)
    assert P.ax_set_option(op, "stencil_kernel", 2, raise_on_error=False) == P.AX_ERR_INVALID_ARG
    assert P.ax_set_option(op, "stencil_kernel", 0.5, raise_on_error=False) == P.AX_ERR_INVALID_ARG
    assert int(P.ax_get_option(op, "stencil_kernel")) == 0
    P.ax_destroy_operator(op)


def test_bounded_wait_expiry_returns_timeout(cuda):
    """No copy is issued, so every wait of the launch runs out: the kernel
    flags the error and returns, the call reports AX_ERR_TIMEOUT, and the
    next call on the same context computes A y."""
    nr, nz = 48, 300
    op, ora, med = _setup(nr, nz, cuda)
    P.ax_set_option(op, "stencil_kernel", 1)
    y = np.random.default_rng(3).normal(size=(1, nr, nz))
    P.ax_set_option(op, "stencil_stall_test", 1)
    with pytest.raises(P.AxError) as e:
        _apply(op, y, cuda)
    assert e.value.status == P.AX_ERR_TIMEOUT
    assert _rel(_apply(op, y, cuda)[0], ora.apply_A(y[0])) <= 2e-6
    # the same through a solve (the fused iteration's stencil)
    P.ax_set_option(op, "dst_tensor", 1)
    f = sample_rhs(med, nr, nz)
    fd = torch.from_numpy(f).to(cuda)
    u = torch.zeros_like(fd)
    P.ax_set_option(op, "stencil_stall_test", 1)
    st, _ = P.ax_solve(op, fd, u, 3, 1e-8, 40, P.AX_PCG_MIXED, raise_on_error=False)
    assert st == P.AX_ERR_TIMEOUT
    u.zero_()
    st, _ = P.ax_solve(op, fd, u, 3, 1e-8, 5000, P.AX_PCG_MIXED)
    assert st == P.AX_OK
    un = u.cpu().numpy()
    for j in range(3):
        phi = ora.phi(f[j])
        assert np.linalg.norm(phi - ora.apply_A(un[j])) <= 1e-8 * np.linalg.norm(phi)
    P.ax_destroy_operator(op)
