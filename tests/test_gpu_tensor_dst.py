"""The tensor-core sine transform (tcgen05 GEMM by the BF16-split DST-I
matrix) against the oracle, through the C ABI.

What it computes is fixed by its definition, with x32 = fp32(in),
hi = bf16(x32), lo = bf16(x32 - hi), S the oracle's orthonormal DST-I matrix,
S_hi = bf16(S), S_lo = bf16(S - S_hi):
  AX_PREC_FP32_TC   out = (hi + lo) S_hi
  AX_PREC_FP32_TC3  out = (hi + lo) S_hi + hi S_lo
The reference evaluates these products in FP64 (the kernel accumulates up to
3 nz products in FP32: tolerance 1e-5 relative per row).  Against the exact
transform S x, TC differs by the BF16 rounding of S (about 3e-3 in the
spectral norm: tolerance 1e-2) and TC3 by the dropped lo S_lo and the
rounding of S_lo (tolerance 1e-4).  The preconditioner built from the TC
transform, S_hi T^-1 S_hi, must stay symmetric (tolerance 1e-5 on
(u, B^ v) - (B^ u, v), the input splitting being the only asymmetry) and close
to B^-1 (2e-2), and the mixed PCG that uses either form must meet 1e-8 in the
oracle's FP64 true residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle import guessnet as G  # noqa: E402
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


def _op(nr, nz, dev, seed=3):
    med = layered_inclusion_medium(n_rhs=2, nominal_n=max(nr, nz), instance=seed)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    t = [torch.from_numpy(x).to(dev) for x in (kr, kz, q)]
    return P.ax_setup_operator(*t, nr, nz), med, t


def _split_reference(x, n, three):
    x32 = x.astype(np.float32).astype(np.float64)
    hi = G.round_bf16(x32)
    lo = G.round_bf16(x32 - hi)
    S = O.dst1_matrix(n)
    Sh = G.round_bf16(S)
    out = (hi + lo) @ Sh
    if three:
        out = out + hi @ G.round_bf16(S - Sh)
    return out


@pytest.mark.parametrize("rows,nz", [(300, 1024), (129, 200), (7, 31), (128, 256), (1, 1), (5, 2), (3, 9),
                                     (130, 65), (64, 127), (260, 2048), (40, 4096), (9, 3001)])
@pytest.mark.parametrize("prec", [P.AX_PREC_FP32_TC, P.AX_PREC_FP32_TC3])
def test_tensor_transform_matches_split_products(cuda, rows, nz, prec):
    op, _, _ = _op(max(rows, 2), nz, cuda)
    x = np.random.default_rng(rows + nz).normal(size=(rows, nz))
    y = torch.zeros((rows, nz), dtype=torch.float64, device=cuda)
    P.ax_apply_dst(op, torch.from_numpy(x).to(cuda), y, rows, prec)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    three = prec == P.AX_PREC_FP32_TC3
    ref = _split_reference(x, nz, three)
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-5, err.max()
    exact = x @ O.dst1_matrix(nz)
    assert np.linalg.norm(got - exact) <= (1e-4 if three else 1e-2) * np.linalg.norm(exact)
    P.ax_destroy_operator(op)


def test_tensor_preconditioner_symmetric_and_close(cuda):
    nr, nz = 160, 300
    op, _, _ = _op(nr, nz, cuda)
    rng = np.random.default_rng(5)
    u, v = rng.normal(size=(1, nr, nz)), rng.normal(size=(1, nr, nz))

    def apply(x, prec):
        out = torch.zeros((1, nr, nz), dtype=torch.float64, device=cuda)
        P.ax_apply_preconditioner(op, torch.from_numpy(x).to(cuda), out, 1, prec)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    bu, bv = apply(u, P.AX_PREC_FP32_TC), apply(v, P.AX_PREC_FP32_TC)
    a, b = np.sum(u * bv), np.sum(bu * v)
    assert abs(a - b) <= 1e-5 * np.sqrt(np.sum(u * bu) * np.sum(v * bv))
    ex = apply(v, P.AX_PREC_FP64)
    assert np.linalg.norm(bv - ex) <= 2e-2 * np.linalg.norm(ex)
    P.ax_destroy_operator(op)


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("nr,nz", [(160, 144), (1500, 130), (3000, 72)])
def test_mixed_pcg_with_tensor_transform_meets_tolerance(cuda, form, nr, nz):
    """Also for tall grids, whose mode solves run 4 or 8 warps per column
    (nr > 1024) and still write the split operand and the (r, z) partials."""
    med = layered_inclusion_medium(n_rhs=4, nominal_n=max(nr, nz))
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(cuda) for x in (kr, kz, q)], nr, nz)
    g = O.Grid(nr, nz)
    ora = O.Operator(kr, kz, q, g)
    f = sample_rhs(med, nr, nz)
    fd = torch.from_numpy(f).to(cuda)
    u64 = torch.zeros_like(fd)
    _, i64 = P.ax_solve(op, fd, u64, 4, 1e-8, 5000, P.AX_PCG_FP64)
    P.ax_set_option(op, "dst_tensor", form)
    u = torch.zeros_like(fd)
    st, imx = P.ax_solve(op, fd, u, 4, 1e-8, 5000, P.AX_PCG_MIXED)
    torch.cuda.synchronize()
    assert st == P.AX_OK
    un = u.cpu().numpy()
    for j in range(4):
        phi = ora.phi(f[j])
        assert np.linalg.norm(phi - ora.apply_A(un[j])) <= 1e-8 * np.linalg.norm(phi)
        assert imx[j]["iters"] <= 1.2 * i64[j]["iters"] + 4, (imx[j], i64[j])
    # back to the FFT transform: same answer to the tolerance
    P.ax_set_option(op, "dst_tensor", 0)
    u2 = torch.zeros_like(fd)
    st, _ = P.ax_solve(op, fd, u2, 4, 1e-8, 5000, P.AX_PCG_MIXED)
    assert st == P.AX_OK
    P.ax_destroy_operator(op)


@pytest.mark.parametrize("j,nr,nz,bc", [(66, 2047, 255, 0), (66, 2047, 1024, 0), (3, 1024, 4096, 0),
                                         (186, 2047, 1023, 1)])
def test_mixed_pcg_tensor_transform_ill_conditioned_media(cuda, j, nr, nz, bc):
    """Random-field media of the batched workload whose FP32 recursion, with
    the split-BF16 transform, drifted for up to 50 times the iterations when
    the FP64 residual replacement came only every 100-fold residual reduction:
    with the default (every 10-fold reduction) the tensor-core path needs
    about the FFT path's iterations, and both meet the tolerance in the
    oracle's FP64 residual (bc = 1: the cosine pair of the zero-flux
    boundary)."""
    from workloads import batched_instances
    _, _, med = batched_instances(256)[j]
    kr, kz, q = sample_operator_inputs(med, nr, nz, bc_z=bc)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(cuda) for x in (kr, kz, q)], nr, nz, bc_z=bc)
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz, bc_z=bc))
    f = sample_rhs(med, nr, nz, bc_z=bc)[:1]
    fd = torch.from_numpy(f).to(cuda)
    iters = {}
    for form in (0, 1):
        P.ax_set_option(op, "dst_tensor", form)
        u = torch.zeros_like(fd)
        st, info = P.ax_solve(op, fd, u, 1, 1e-8, 2000, P.AX_PCG_MIXED)
        torch.cuda.synchronize()
        assert st == P.AX_OK
        phi = ora.phi(f[0])
        assert np.linalg.norm(phi - ora.apply_A(u.cpu().numpy()[0])) <= 1e-8 * np.linalg.norm(phi)
        iters[form] = info[0]["iters"]
    assert iters[1] <= 1.3 * iters[0] + 4, iters
    P.ax_destroy_operator(op)


def test_tensor_option_rejects_long_columns(cuda):
    op, _, _ = _op(4, 4100, cuda)
    with pytest.raises(P.AxError):
        P.ax_set_option(op, "dst_tensor", 1)
    P.ax_destroy_operator(op)


def test_bounded_wait_expiry_returns_timeout_and_context_stays_usable(cuda):
    """The failure path of the tensor-core transform without a fault: the
    copy warp stops before its first stage, the MMA warp's bounded wait runs
    out, the kernel flags the error, frees its tensor memory and returns; the
    call reports AX_ERR_TIMEOUT, and the next call computes the transform."""
    rows, nz = 64, 256
    op, _, _ = _op(rows, nz, cuda)
    x = np.random.default_rng(1).normal(size=(rows, nz))
    xd = torch.from_numpy(x).to(cuda)
    y = torch.zeros((rows, nz), dtype=torch.float64, device=cuda)
    P.ax_set_option(op, "tc_stall_test", 1)
    with pytest.raises(P.AxError) as e:
        P.ax_apply_dst(op, xd, y, rows, P.AX_PREC_FP32_TC3)
    assert e.value.status == P.AX_ERR_TIMEOUT
    y.zero_()
    P.ax_apply_dst(op, xd, y, rows, P.AX_PREC_FP32_TC3)
    torch.cuda.synchronize()
    ref = _split_reference(x, nz, True)
    err = np.linalg.norm(y.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-5
    P.ax_destroy_operator(op)


@pytest.mark.parametrize("j,nr,nz,m,tol,checks", [(66, 2047, 255, 1, 1e-8, True), (None, 600, 700, 3, 1e-11, False)])
def test_replacement_gate_keeps_results(cuda, j, nr, nz, m, tol, checks):
    """The split and transform launches that recompute z after a residual
    replacement are gated by a device count of the right-hand sides that need
    it (option replace_gate): with and without the gate the solve is the same
    bit for bit, on a case where the recomputation does happen
    (replace_checks > 0: an ill-conditioned random-field medium) and on one
    where it does not (the gate stays closed)."""
    from workloads import batched_instances
    med = batched_instances(256)[j][2] if j is not None else layered_inclusion_medium(n_rhs=m, nominal_n=nr,
                                                                                       instance=9)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    op = P.ax_setup_operator(*[torch.from_numpy(x).to(cuda) for x in (kr, kz, q)], nr, nz)
    P.ax_set_option(op, "dst_tensor", 1)  # the fused tensor-core iteration, whose replacement step is gated
    assert int(P.ax_get_option(op, "replace_gate")) == 1
    assert P.ax_set_option(op, "replace_gate", 2, raise_on_error=False) == P.AX_ERR_INVALID_ARG
    f = sample_rhs(med, nr, nz)[:m]
    fd = torch.from_numpy(f).to(cuda)
    out = {}
    for gate in (1, 0):
        P.ax_set_option(op, "replace_gate", gate)
        u = torch.zeros_like(fd)
        st, info = P.ax_solve(op, fd, u, m, tol, 5000, P.AX_PCG_MIXED)
        torch.cuda.synchronize()
        assert st == P.AX_OK
        out[gate] = ([i["iters"] for i in info], u.cpu().numpy(), int(P.ax_get_option(op, "replace_checks")))
    assert (out[1][2] > 0) == checks and out[1][2] == out[0][2], (out[1][2], out[0][2])
    assert out[1][0] == out[0][0]
    assert np.array_equal(out[1][1], out[0][1])
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz))
    for k in range(m):
        phi = ora.phi(f[k])
        assert np.linalg.norm(phi - ora.apply_A(out[1][1][k])) <= tol * np.linalg.norm(phi)
    P.ax_destroy_operator(op)
