"""CUDA path vs the FP64 oracle, through the C ABI.

Tolerances (relative, 2-norm over the compared array unless stated):
  stencil      FP64 1e-14   FP32 2e-6
  sine transf. FP64 1e-13   FP32 2e-6
  mode solves  backward error FP64 1e-14, FP32 2e-6; forward error vs oracle 1e-9 / 1e-3
  B^-1         FP64 1e-12   FP32 1e-5
  FP64 PCG     |iters - oracle| <= 1, oracle true residual of the GPU answer <= tol;
               solved to 1e-13 both sides: ||u_gpu - u_oracle|| <= 1e-10 ||u_oracle||
  mixed forms  oracle FP64 true residual of the GPU answer <= tol = 1e-8
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_1002_3094_gb300 as P  # noqa: E402
from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs  # noqa: E402
from workloads import Medium, bumps_medium, layered_inclusion_medium, batched_instances  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.load_library()
    return torch.device("cuda:0")


def _rand_medium(seed):
    rng = np.random.default_rng(seed)
    a, b = rng.uniform(0.5, 3.0, 2)

    def kappa(r, z):
        return 1.0 + a * np.sin(5 * r + 2 * z) ** 2 + b * (z > 0.4)

    def q(r, z):
        return 0.2 + 0.3 * np.cos(3 * r * z) ** 2

    return Medium("rand", kappa, q, [lambda r, z: np.exp(-((r - .4) ** 2 + (z - .5) ** 2) * 30)])


class Pair:
    """The same operator set up in the library and in the oracle."""

    def __init__(self, medium, nr, nz, dev):
        kr, kz, q = sample_operator_inputs(medium, nr, nz)
        g = O.Grid(nr, nz)
        okr, okz, oq, _ = O.sample_medium(medium, g, rhs_index=[])
        assert np.array_equal(kr, okr) and np.array_equal(kz, okz) and np.array_equal(q, oq)
        self.t = [torch.from_numpy(x).to(dev) for x in (kr, kz, q)]
        self.op = P.ax_setup_operator(*self.t, nr, nz)
        self.ora = O.Operator(okr, okz, oq, g)
        self.nr, self.nz, self.dev, self.medium = nr, nz, dev, medium

    def close(self):
        P.ax_destroy_operator(self.op)

    def dev_array(self, x):
        return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(self.dev)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


SHAPES = [(1, 1), (2, 3), (5, 7), (16, 33), (33, 64), (64, 64), (40, 127), (17, 300), (9, 1024), (3, 1025)]


@pytest.mark.parametrize("nr,nz", SHAPES)
@pytest.mark.parametrize("prec,tol", [(P.AX_PREC_FP64, 1e-14), (P.AX_PREC_FP32, 2e-6)])
def test_stencil(cuda, nr, nz, prec, tol):
    pr = Pair(_rand_medium(nr + nz), nr, nz, cuda)
    m = 2
    y = np.random.default_rng(1).normal(size=(m, nr, nz))
    out = torch.zeros((m, nr, nz), dtype=torch.float64, device=cuda)
    P.ax_apply_operator(pr.op, pr.dev_array(y), out, m, prec)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for j in range(m):
        assert _rel(got[j], pr.ora.apply_A(y[j])) <= tol
    pr.close()


DST_N = [1, 2, 3, 4, 5, 6, 7, 8, 12, 15, 16, 40, 63, 64, 100, 127, 240, 255, 256, 1023, 1024, 2047, 4096]


@pytest.mark.parametrize("nz", DST_N)
@pytest.mark.parametrize("prec,tol", [(P.AX_PREC_FP64, 1e-13), (P.AX_PREC_FP32, 2e-6)])
def test_sine_transform(cuda, nz, prec, tol):
    pr = Pair(_rand_medium(3), 2, nz, cuda)
    rows = 7
    x = np.random.default_rng(nz).normal(size=(rows, nz))
    out = torch.zeros((rows, nz), dtype=torch.float64, device=cuda)
    P.ax_apply_dst(pr.op, pr.dev_array(x), out, rows, prec)
    torch.cuda.synchronize()
    ref = x @ O.dst1_matrix(nz)
    assert _rel(out.cpu().numpy(), ref) <= tol
    pr.close()


@pytest.mark.parametrize("nr,nz", [(1, 1), (2, 5), (31, 17), (32, 33), (33, 64), (100, 40), (513, 20), (1024, 9),
                                   (2047, 3), (4096, 2)])
@pytest.mark.parametrize("prec,bwd,fwd", [(P.AX_PREC_FP64, 1e-14, 1e-9), (P.AX_PREC_FP32, 2e-6, 1e-3)])
def test_mode_solves(cuda, nr, nz, prec, bwd, fwd):
    """Backward error ||T_l y - b|| / (||T_l|| ||y||) of every mode system
    (a backward-stable solver's guarantee), and the forward error against the
    oracle's Thomas, which cond(T_l) ~ nr^2 may amplify."""
    pr = Pair(_rand_medium(nr), nr, nz, cuda)
    m = 2
    b = np.random.default_rng(5).normal(size=(m, nr, nz))
    out = torch.zeros((m, nr, nz), dtype=torch.float64, device=cuda)
    P.ax_apply_mode_solve(pr.op, pr.dev_array(b), out, m, prec)
    torch.cuda.synchronize()
    g = pr.ora.grid
    lam = O.mode_eigenvalues(nz, g.hz)
    sub, diag, sup = O.mode_tridiagonal(pr.ora.kappa_t, pr.ora.q_t, lam, g)
    got = out.cpu().numpy()
    for j in range(m):
        y = got[j]
        Ty = diag * y
        Ty[:-1] += sup * y[1:]
        Ty[1:] += sub * y[:-1]
        tnorm = np.abs(diag).max() + 2 * np.abs(sub).max() if nr > 1 else np.abs(diag).max()
        for l in range(nz):
            assert np.linalg.norm(Ty[:, l] - b[j][:, l]) <= bwd * tnorm * np.linalg.norm(y[:, l])
        assert _rel(y, O.thomas(sub, diag, sup, b[j])) <= fwd
    pr.close()


@pytest.mark.parametrize("nr,nz", [(1, 1), (3, 4), (20, 31), (64, 64), (65, 100), (128, 255)])
@pytest.mark.parametrize("prec,tol", [(P.AX_PREC_FP64, 1e-12), (P.AX_PREC_FP32, 1e-5)])
def test_preconditioner(cuda, nr, nz, prec, tol):
    pr = Pair(_rand_medium(nz), nr, nz, cuda)
    m = 3
    v = np.random.default_rng(9).normal(size=(m, nr, nz))
    out = torch.zeros((m, nr, nz), dtype=torch.float64, device=cuda)
    P.ax_apply_preconditioner(pr.op, pr.dev_array(v), out, m, prec)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for j in range(m):
        assert _rel(got[j], pr.ora.apply_Binv(v[j])) <= tol
    pr.close()


def _solve(pr, f, method, tol, max_iter=5000, flags=0, u0=None):
    m = f.shape[0]
    u = pr.dev_array(u0) if u0 is not None else torch.zeros(f.shape, dtype=torch.float64, device=pr.dev)
    st, info = P.ax_solve(pr.op, pr.dev_array(f), u, m, tol, max_iter, method, flags)
    torch.cuda.synchronize()
    return st, info, u.cpu().numpy()


def _oracle_rel_res(pr, f, u):
    phi = pr.ora.phi(f)
    return np.linalg.norm(phi - pr.ora.apply_A(u)) / np.linalg.norm(phi)


def test_pcg_fp64_bumps_64(cuda):
    """Workload bumps_64: iteration count and residual against the oracle."""
    pr = Pair(bumps_medium(), 64, 64, cuda)
    f = sample_rhs(pr.medium, 64, 64)
    st, info, u = _solve(pr, f, P.AX_PCG_FP64, 1e-10)
    assert st == P.AX_OK
    _, oinfo = pr.ora.solve(f[0], 1e-10)
    assert abs(info[0]["iters"] - oinfo.iters) <= 1
    assert _oracle_rel_res(pr, f[0], u[0]) <= 1e-10
    # tight solves on both sides agree on the solution itself
    st, info, u = _solve(pr, f, P.AX_PCG_FP64, 1e-13)
    y, _ = pr.ora.solve(f[0], 1e-13)
    assert _rel(u[0], y) <= 1e-10
    pr.close()


@pytest.mark.parametrize("method", [P.AX_PCG_MIXED, P.AX_CHEB_FP64, P.AX_CHEB_MIXED])
def test_other_methods_bumps_64(cuda, method):
    pr = Pair(bumps_medium(), 64, 64, cuda)
    f = sample_rhs(pr.medium, 64, 64)
    tol = 1e-10 if method == P.AX_CHEB_FP64 else 1e-8
    st, info, u = _solve(pr, f, method, tol)
    assert st == P.AX_OK, info
    assert _oracle_rel_res(pr, f[0], u[0]) <= tol
    pr.close()


@pytest.mark.parametrize("method", [P.AX_PCG_FP64, P.AX_PCG_MIXED, P.AX_CHEB_MIXED])
def test_layered_inclusion_multi_rhs(cuda, method):
    """Shape of the 1024^2 x 64 workload at 128^2 x 5 (several tiles, ragged
    nothing): every right-hand side meets the tolerance in the oracle's norm."""
    med = layered_inclusion_medium(n_rhs=5, nominal_n=128)
    pr = Pair(med, 128, 128, cuda)
    f = sample_rhs(med, 128, 128)
    st, info, u = _solve(pr, f, method, 1e-8)
    assert st == P.AX_OK, info
    for j in range(f.shape[0]):
        assert _oracle_rel_res(pr, f[j], u[j]) <= 1e-8
    pr.close()


def test_batched_rhs_equal_single(cuda):
    """Deterministic reductions: each RHS of a batch gets bit-identical results
    to solving it alone."""
    med = layered_inclusion_medium(n_rhs=3, nominal_n=96)
    pr = Pair(med, 96, 80, cuda)
    # single right-hand sides through the same graph-replayed kernels as the
    # batch (the persistent small-grid path sums in another order)
    P.ax_set_option(pr.op, "small_path", 0)
    f = sample_rhs(med, 96, 80)
    _, info_b, ub = _solve(pr, f, P.AX_PCG_FP64, 1e-9)
    for j in range(3):
        _, info_s, us = _solve(pr, f[j:j + 1], P.AX_PCG_FP64, 1e-9)
        assert info_s[0]["iters"] == info_b[j]["iters"]
        assert np.array_equal(us[0], ub[j])
    pr.close()


def test_ragged_uneven_instance(cuda):
    """One instance of the uneven-size workload (odd sizes, non power of two)."""
    nr, nz, med = batched_instances(4)[1]
    nr, nz = min(nr, 255), min(nz, 255)
    pr = Pair(med, nr, nz, cuda)
    f = sample_rhs(med, nr, nz)
    for method in (P.AX_PCG_FP64, P.AX_PCG_MIXED):
        st, info, u = _solve(pr, f, method, 1e-8)
        assert st == P.AX_OK
        assert _oracle_rel_res(pr, f[0], u[0]) <= 1e-8
    pr.close()


def test_host_buffers_and_guess(cuda):
    pr = Pair(bumps_medium(), 64, 64, cuda)
    f = sample_rhs(pr.medium, 64, 64)
    _, info_d, ud = _solve(pr, f, P.AX_PCG_FP64, 1e-10)
    uh = np.zeros_like(f)
    st, info_h = P.ax_solve(pr.op, f, uh, 1, 1e-10, 5000, P.AX_PCG_FP64, P.AX_FLAG_HOST_BUFFERS)
    assert st == P.AX_OK and np.array_equal(uh, ud)
    # exact guess: zero iterations
    st, info, _ = _solve(pr, f, P.AX_PCG_FP64, 1e-10, flags=P.AX_FLAG_USE_GUESS, u0=ud)
    assert st == P.AX_OK and info[0]["iters"] == 0
    pr.close()


def test_invalid_arguments(cuda):
    nr, nz = 4, 5
    good = [torch.ones((nr, nz), dtype=torch.float64, device=cuda),
            torch.linspace(1, 3, nr * (nz + 1), dtype=torch.float64, device=cuda).reshape(nr, nz + 1),
            torch.zeros((nr, nz), dtype=torch.float64, device=cuda)]
    bad_k = good[0].clone()
    bad_k[1, 2] = 0.0
    with pytest.raises(P.AxError) as e:
        P.ax_setup_operator(bad_k, good[1], good[2], nr, nz)
    assert e.value.status == P.AX_ERR_INVALID_ARG
    bad_q = good[2].clone()
    bad_q[0, 0] = -1.0
    with pytest.raises(P.AxError):
        P.ax_setup_operator(good[0], good[1], bad_q, nr, nz)
    nan_k = good[1].clone()
    nan_k[0, 0] = float("nan")
    with pytest.raises(P.AxError):
        P.ax_setup_operator(good[0], nan_k, good[2], nr, nz)
    with pytest.raises(P.AxError) as e:
        P.ax_setup_operator(*good, nr, nz, bc_z=2)
    assert e.value.status == P.AX_ERR_INVALID_ARG
    with pytest.raises(P.AxError):
        P.ax_setup_operator(*good, 0, nz)
    op = P.ax_setup_operator(*good, nr, nz)
    f = torch.ones((1, nr, nz), dtype=torch.float64, device=cuda)
    u = torch.zeros_like(f)
    with pytest.raises(P.AxError):
        P.ax_solve(op, f, u, 1, -1.0)
    st, info = P.ax_solve(op, f, u, 1, 1e-14, 1, P.AX_PCG_FP64, raise_on_error=False)
    assert st == P.AX_ERR_NO_CONVERGENCE and info[0]["status"] == P.AX_ERR_NO_CONVERGENCE
    P.ax_destroy_operator(op)


def test_full_size_layered_1024_m64_sampled(cuda):
    """The benchmark's workload (1024 x 1024, 64 right-hand sides, mixed PCG,
    tol 1e-8): the oracle's FP64 true residual of sampled right-hand sides."""
    nr = nz = 1024
    med = layered_inclusion_medium(64, 1024)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    t = [torch.from_numpy(x).cuda() for x in (kr, kz, q)]
    op = P.ax_setup_operator(*t, nr, nz)
    f = torch.from_numpy(sample_rhs(med, nr, nz)).cuda()
    u = torch.zeros_like(f)
    st, info = P.ax_solve(op, f, u, 64, 1e-8, 5000, P.AX_PCG_MIXED)
    assert st == P.AX_OK
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz))
    fh, uh = f.cpu().numpy(), u.cpu().numpy()
    for j in (0, 17, 63):
        phi = ora.phi(fh[j])
        assert np.linalg.norm(phi - ora.apply_A(uh[j])) <= 1e-8 * np.linalg.norm(phi)
    P.ax_destroy_operator(op)


def test_full_size_large_4096_m16_sampled(cuda):
    """The 4096 x 4096 workload with 16 right-hand sides in the benchmark's
    launch configuration (mixed PCG, tensor-core transform of length 4097,
    tol 1e-8): the oracle's FP64 true residual of two sampled right-hand
    sides, and the (rhat, yhat)-based iteration count within a few of the
    FP64 method's on the first one."""
    from workloads import large_medium
    nr = nz = 4096
    med = large_medium(16, 4096)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    t = [torch.from_numpy(x).cuda() for x in (kr, kz, q)]
    op = P.ax_setup_operator(*t, nr, nz)
    fh = sample_rhs(med, nr, nz)
    f = torch.from_numpy(fh).cuda()
    u = torch.zeros_like(f)
    st, info = P.ax_solve(op, f, u, 16, 1e-8, 5000, P.AX_PCG_MIXED)
    assert st == P.AX_OK
    uh = u.cpu().numpy()
    del u
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz))
    for j in (0, 11):
        phi = ora.phi(fh[j])
        assert np.linalg.norm(phi - ora.apply_A(uh[j])) <= 1e-8 * np.linalg.norm(phi)
    u64 = torch.zeros_like(f[:1])
    _, i64 = P.ax_solve(op, f[:1], u64, 1, 1e-8, 5000, P.AX_PCG_FP64)
    assert info[0]["iters"] <= 1.2 * i64[0]["iters"] + 4, (info[0], i64[0])
    P.ax_destroy_operator(op)


def test_full_size_layered_1024_m64_zero_flux_sampled(cuda):
    """The benchmark's workload with the paper's zero-flux z boundary
    (tensor-core cosine pair): the oracle's FP64 true residual of sampled
    right-hand sides."""
    nr = nz = 1024
    med = layered_inclusion_medium(64, 1024)
    kr, kz, q = sample_operator_inputs(med, nr, nz, bc_z=1)
    t = [torch.from_numpy(x).cuda() for x in (kr, kz, q)]
    op = P.ax_setup_operator(*t, nr, nz, bc_z=1)
    fh = sample_rhs(med, nr, nz, bc_z=1)
    f = torch.from_numpy(fh).cuda()
    u = torch.zeros_like(f)
    st, info = P.ax_solve(op, f, u, 64, 1e-8, 5000, P.AX_PCG_MIXED)
    assert st == P.AX_OK
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz, bc_z=1))
    uh = u.cpu().numpy()
    for j in (0, 40, 63):
        phi = ora.phi(fh[j])
        assert np.linalg.norm(phi - ora.apply_A(uh[j])) <= 1e-8 * np.linalg.norm(phi)
    P.ax_destroy_operator(op)


@pytest.mark.parametrize("method", [P.AX_PCG_MIXED, P.AX_CHEB_MIXED])
@pytest.mark.parametrize("scale", [1e-200, 1e-30, 1e-12, 1e25, 1e200])
def test_mixed_methods_are_scale_invariant(cuda, method, scale):
    """f scaled by 1e-200 .. 1e200: the mixed methods (FP32 inner iteration)
    return scale times the unscaled solution to the tolerance, with the same
    iteration count (their right-hand side is scaled by the power of two that
    brings max |phi| into [1/2, 1) inside the solve).  The residual is
    checked on u / scale against the unscaled phi (squares of 1e200 overflow)."""
    nr, nz = 96, 80
    med = layered_inclusion_medium(2, 96)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    op = P.ax_setup_operator(*[torch.from_numpy(x).cuda() for x in (kr, kz, q)], nr, nz)
    f = torch.from_numpy(sample_rhs(med, nr, nz)).cuda()
    u1, u2 = torch.zeros_like(f), torch.zeros_like(f)
    st1, i1 = P.ax_solve(op, f, u1, 2, 1e-8, 5000, method)
    st2, i2 = P.ax_solve(op, f * scale, u2, 2, 1e-8, 5000, method)
    assert st1 == P.AX_OK and st2 == P.AX_OK
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz))
    fh, uh = f.cpu().numpy(), u2.cpu().numpy() / scale
    assert np.isfinite(uh).all()
    for j in range(2):
        phi = ora.phi(fh[j])
        assert np.linalg.norm(phi - ora.apply_A(uh[j])) <= 1.001e-8 * np.linalg.norm(phi)
        assert abs(i1[j]["iters"] - i2[j]["iters"]) <= 2, (i1[j], i2[j])
    P.ax_destroy_operator(op)


def test_mixed_replacement_keeps_fp64_iteration_count(cuda):
    """FP32 PCG with FP64 residual replacement keeps the search direction, so
    its iteration count stays close to the FP64 method's; the restarted
    refinement (option mixed_restart) also meets the tolerance."""
    med = layered_inclusion_medium(n_rhs=4, nominal_n=160)
    pr = Pair(med, 160, 144, cuda)
    f = sample_rhs(med, 160, 144)
    _, i64, _ = _solve(pr, f, P.AX_PCG_FP64, 1e-8)
    st, imx, u = _solve(pr, f, P.AX_PCG_MIXED, 1e-8)
    assert st == P.AX_OK
    for j in range(4):
        assert imx[j]["iters"] <= 1.2 * i64[j]["iters"] + 4, (imx[j], i64[j])
        assert imx[j]["outer"] >= 1
        assert _oracle_rel_res(pr, f[j], u[j]) <= 1e-8
    P.ax_set_option(pr.op, "mixed_restart", 1)
    st, irs, u = _solve(pr, f, P.AX_PCG_MIXED, 1e-8)
    assert st == P.AX_OK
    for j in range(4):
        assert _oracle_rel_res(pr, f[j], u[j]) <= 1e-8
    P.ax_set_option(pr.op, "mixed_restart", 0)
    pr.close()


@pytest.mark.parametrize("method", [P.AX_PCG_FP64, P.AX_PCG_MIXED, P.AX_CHEB_FP64, P.AX_CHEB_MIXED])
def test_batched_uneven_instances_equal_single_solves(cuda, method):
    """Instances of the uneven-size workload (sizes reduced to keep the test
    short; shapes repeat so groups hold several instances): the batched solve
    gives each instance bit-identical results to solving it alone, and the
    oracle's true residual meets the tolerance."""
    insts = batched_instances(7, sizes=(31, 64, 97))
    pairs, fs, us = [], [], []
    for nr, nz, med in insts:
        pr = Pair(med, nr, nz, cuda)
        P.ax_set_option(pr.op, "small_path", 0)  # the batch's kernels for the single solves too
        pairs.append(pr)
        fs.append(pr.dev_array(sample_rhs(med, nr, nz)[0]))
        us.append(torch.zeros((nr, nz), dtype=torch.float64, device=cuda))
    batch = P.ax_batch_create([p.op for p in pairs])
    st, info = P.ax_batch_solve(batch, fs, us, 1e-8, 5000, method)
    torch.cuda.synchronize()
    assert st == P.AX_OK
    lat, groups = P.ax_batch_latency(batch, len(pairs))
    assert groups < len(pairs) and all(x > 0 for x in lat)
    for j, pr in enumerate(pairs):
        f = fs[j].cpu().numpy()[None]
        st1, info1, u1 = _solve(pr, f, method, 1e-8)
        assert info1[0]["iters"] == info[j]["iters"]
        assert np.array_equal(u1[0], us[j].cpu().numpy())
        assert _oracle_rel_res(pr, f[0], u1[0]) <= 1e-8
    P.ax_batch_destroy(batch)
    for pr in pairs:
        pr.close()


@pytest.mark.parametrize("method", [P.AX_PCG_FP64, P.AX_PCG_MIXED])
def test_guess_gate_rejects_bad_and_keeps_good_guesses(cuda, method):
    """AX_FLAG_CHECK_GUESS: a garbage starting iterate (residual above ||phi||)
    is replaced by zero, a good one is kept and saves iterations; both reach
    the tolerance in the oracle's norm."""
    med = layered_inclusion_medium(n_rhs=2, nominal_n=96)
    pr = Pair(med, 96, 80, cuda)
    f = sample_rhs(med, 96, 80)
    _, i0, u_ref = _solve(pr, f, method, 1e-9)
    rng = np.random.default_rng(0)
    u0 = np.stack([1e3 * rng.normal(size=u_ref[0].shape),             # garbage
                   u_ref[1] * (1 + 1e-4 * rng.normal(size=u_ref[1].shape))])  # near solution
    flags = P.AX_FLAG_USE_GUESS | P.AX_FLAG_CHECK_GUESS
    st, info, u = _solve(pr, f, method, 1e-9, flags=flags, u0=u0)
    assert st == P.AX_OK
    assert info[0]["guess_accepted"] == 0 and info[1]["guess_accepted"] == 1
    assert info[0]["iters"] == i0[0]["iters"]
    assert info[1]["iters"] < i0[1]["iters"]
    for j in range(2):
        assert _oracle_rel_res(pr, f[j], u[j]) <= 1e-9
    pr.close()


def test_mixed_iterations_track_fp64_on_fast_instances(cuda):
    """Fast-converging instances of the uneven-size workload: the mixed
    method's residual replacement (true residual swapped in at the end of an
    iteration, z and beta recomputed only where it differs from the recursive
    one) must not stall CG once the recursion runs below the FP32 accuracy of
    the iterate: iterations within 1.5x + 8 of the FP64 method's."""
    insts = batched_instances(16, sizes=(63, 127))
    for nr, nz, med in insts:
        pr = Pair(med, nr, nz, cuda)
        f = sample_rhs(med, nr, nz)[:1]
        st64, i64, _ = _solve(pr, f, P.AX_PCG_FP64, 1e-8)
        st, imx, u = _solve(pr, f, P.AX_PCG_MIXED, 1e-8)
        assert st == P.AX_OK and st64 == P.AX_OK
        assert imx[0]["iters"] <= 1.5 * i64[0]["iters"] + 8, (nr, nz, imx[0], i64[0])
        assert _oracle_rel_res(pr, f[0], u[0]) <= 1e-8
        pr.close()
