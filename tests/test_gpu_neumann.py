"""The paper's zero-flux z boundary (bc_z = 1: cell-centred z, the cosine
pair of Eq. fft_phi) on the CUDA path against the FP64 oracle, through the
C ABI.

The library's cosine transforms are orthonormal: C = diag(c) F with F the
forward sum of Eq. fft_phi (oracle cosine_pair) and c_1 = 1/sqrt 2, c_l = 1
otherwise; the inverse is C^T (the paper's inverse sum G, whose 1/2 weight is
c_1^2, gives the same B^-1 = F^T T^-1 G = C^T T^-1 C).

Tolerances (relative, 2-norm), as for the sine variant:
  stencil      FP64 1e-14   FP32 2e-6
  cosine pair  FP64 1e-13   FP32 2e-6
  mode solves  backward error FP64 1e-14, FP32 2e-6
  B^-1         FP64 1e-12   FP32 1e-5
  solves       oracle FP64 true residual of the GPU answer <= tol; FP64 PCG
               iterations within 1 of the oracle's; solved to 1e-12:
               ||u_gpu - u_direct|| <= 1e-9 ||u_direct||
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle import guessnet as G  # noqa: E402
import scipy.sparse.linalg as spl  # noqa: E402
import paper_1002_3094_gb300 as P  # noqa: E402
from paper_1002_3094_gb300.inputs import sample_operator_inputs, sample_rhs  # noqa: E402
from workloads import Medium, layered_inclusion_medium, batched_instances  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.load_library()
    return torch.device("cuda:0")


def _rand_medium(seed, q_zero=False):
    rng = np.random.default_rng(seed)
    a, b = rng.uniform(0.5, 3.0, 2)

    def kappa(r, z):
        return 1.0 + a * np.sin(5 * r + 2 * z) ** 2 + b * (z > 0.4)

    def q(r, z):
        if q_zero:
            return np.zeros(np.broadcast(r, z).shape)
        return 0.2 + 0.3 * np.cos(3 * r * z) ** 2

    return Medium("rand", kappa, q, [lambda r, z: np.exp(-((r - .4) ** 2 + (z - .5) ** 2) * 30),
                                     lambda r, z: np.cos(3 * z) * (1 - r)])


class Pair:
    """The same zero-flux operator in the library and in the oracle."""

    def __init__(self, medium, nr, nz, dev):
        kr, kz, q = sample_operator_inputs(medium, nr, nz, bc_z=1)
        g = O.Grid(nr, nz, bc_z=1)
        okr, okz, oq, _ = O.sample_medium(medium, g, rhs_index=[])
        assert np.array_equal(kr, okr) and np.array_equal(kz, okz) and np.array_equal(q, oq)
        self.t = [torch.from_numpy(x).to(dev) for x in (kr, kz, q)]
        self.op = P.ax_setup_operator(*self.t, nr, nz, bc_z=1)
        self.ora = O.Operator(okr, okz, oq, g)
        self.nr, self.nz, self.dev, self.medium = nr, nz, dev, medium

    def rhs(self):
        return sample_rhs(self.medium, self.nr, self.nz, bc_z=1)

    def close(self):
        P.ax_destroy_operator(self.op)

    def dev_array(self, x):
        return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).to(self.dev)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _orthonormal_cosine(n):
    F, _ = O.cosine_pair(n)
    C = F.copy()
    C[0] /= math.sqrt(2.0)
    return C


SHAPES = [(1, 1), (2, 3), (5, 7), (16, 33), (40, 127), (17, 300), (9, 1024)]
# FFT lengths nz: powers of two, 3/5 factors, the FP32 unrolled primes (43),
# Rader primes (61: 60 = 2^2 3 5; 97: 96 = 2^5 3) and a generic prime (211)
COS_N = [1, 2, 3, 4, 5, 7, 8, 12, 16, 43, 61, 64, 97, 100, 211, 255, 256, 1000, 1024, 2048]


@pytest.mark.parametrize("nz", COS_N)
@pytest.mark.parametrize("prec,tol", [(P.AX_PREC_FP64, 1e-13), (P.AX_PREC_FP32, 2e-6)])
def test_cosine_pair(cuda, nz, prec, tol):
    pr = Pair(_rand_medium(3), 2, nz, cuda)
    rows = 7
    x = np.random.default_rng(nz).normal(size=(rows, nz))
    C = _orthonormal_cosine(nz)
    out = torch.zeros((rows, nz), dtype=torch.float64, device=cuda)
    P.ax_apply_dst(pr.op, pr.dev_array(x), out, rows, prec)
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy(), x @ C.T) <= tol
    out.zero_()
    P.ax_apply_dst_inverse(pr.op, pr.dev_array(x), out, rows, prec)
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy(), x @ C) <= tol
    pr.close()


@pytest.mark.parametrize("nz", [1, 3, 64, 127])
def test_sine_inverse_is_the_sine_transform(cuda, nz):
    kr, kz, q = sample_operator_inputs(_rand_medium(1), 2, nz)
    op = P.ax_setup_operator(*[torch.from_numpy(v).to(cuda) for v in (kr, kz, q)], 2, nz)
    x = np.random.default_rng(nz).normal(size=(3, nz))
    out = torch.zeros((3, nz), dtype=torch.float64, device=cuda)
    P.ax_apply_dst_inverse(op, torch.from_numpy(x).to(cuda), out, 3, P.AX_PREC_FP64)
    torch.cuda.synchronize()
    assert _rel(out.cpu().numpy(), x @ O.dst1_matrix(nz)) <= 1e-13
    P.ax_destroy_operator(op)


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


@pytest.mark.parametrize("nr,nz", [(1, 1), (2, 5), (33, 64), (513, 20), (1024, 9)])
@pytest.mark.parametrize("prec,bwd", [(P.AX_PREC_FP64, 1e-14), (P.AX_PREC_FP32, 2e-6)])
@pytest.mark.parametrize("q_zero", [False, True])
def test_mode_solves(cuda, nr, nz, prec, bwd, q_zero):
    """Backward error of every mode system T_l y = b with the zero-flux
    eigenvalues (lambda_1 = 0: with q = 0 only the Dirichlet row at r = 1
    keeps T_1 definite)."""
    pr = Pair(_rand_medium(nr, q_zero), nr, nz, cuda)
    m = 2
    b = np.random.default_rng(5).normal(size=(m, nr, nz))
    out = torch.zeros((m, nr, nz), dtype=torch.float64, device=cuda)
    P.ax_apply_mode_solve(pr.op, pr.dev_array(b), out, m, prec)
    torch.cuda.synchronize()
    g = pr.ora.grid
    lam = O.mode_eigenvalues(nz, g.hz, bc_z=1)
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
    pr.close()


@pytest.mark.parametrize("nr,nz", [(1, 1), (3, 4), (20, 31), (64, 64), (65, 100), (128, 255)])
@pytest.mark.parametrize("prec,tol", [(P.AX_PREC_FP64, 1e-12), (P.AX_PREC_FP32, 1e-5)])
def test_preconditioner(cuda, nr, nz, prec, tol):
    pr = Pair(_rand_medium(nz), nr, nz, cuda)
    m = 3
    v = np.random.default_rng(9).normal(size=(m, nr, nz))
    ref = [pr.ora.apply_Binv(v[j]) for j in range(m)]
    for fn in (P.ax_apply_preconditioner, P.ax_apply_preconditioner_noalloc):
        out = torch.zeros((m, nr, nz), dtype=torch.float64, device=cuda)
        fn(pr.op, pr.dev_array(v), out, m, prec)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for j in range(m):
            assert _rel(got[j], ref[j]) <= tol
    pr.close()


def _solve(pr, f, method, tol, max_iter=5000):
    m = f.shape[0]
    u = torch.zeros(f.shape, dtype=torch.float64, device=pr.dev)
    st, info = P.ax_solve(pr.op, pr.dev_array(f), u, m, tol, max_iter, method)
    torch.cuda.synchronize()
    return st, info, u.cpu().numpy()


def _oracle_rel_res(pr, f, u):
    phi = pr.ora.phi(f)
    return np.linalg.norm(phi - pr.ora.apply_A(u)) / np.linalg.norm(phi)


def test_pcg_fp64_iterations_and_solution(cuda):
    pr = Pair(_rand_medium(11), 48, 40, cuda)
    f = pr.rhs()
    st, info, u = _solve(pr, f, P.AX_PCG_FP64, 1e-10)
    assert st == P.AX_OK
    for j in range(f.shape[0]):
        _, oi = pr.ora.solve(f[j], tol=1e-10)
        assert abs(info[j]["iters"] - oi.iters) <= 1, (info[j], oi.iters)
        assert _oracle_rel_res(pr, f[j], u[j]) <= 1e-10
    st, info, u = _solve(pr, f, P.AX_PCG_FP64, 1e-12)
    for j in range(f.shape[0]):
        ref = spl.spsolve(pr.ora.A.tocsc(), pr.ora.phi(f[j]).ravel()).reshape(pr.nr, pr.nz)
        assert _rel(u[j], ref) <= 1e-9
    pr.close()


@pytest.mark.parametrize("method", [P.AX_PCG_MIXED, P.AX_CHEB_FP64, P.AX_CHEB_MIXED])
@pytest.mark.parametrize("q_zero", [False, True])
def test_other_methods(cuda, method, q_zero):
    pr = Pair(_rand_medium(5, q_zero), 64, 50, cuda)
    f = pr.rhs()
    st, info, u = _solve(pr, f, method, 1e-8, max_iter=20000)
    assert st == P.AX_OK
    for j in range(f.shape[0]):
        assert _oracle_rel_res(pr, f[j], u[j]) <= 1e-8
    pr.close()


@pytest.mark.parametrize("method", [P.AX_PCG_FP64, P.AX_PCG_MIXED])
def test_layered_multi_rhs_512(cuda, method):
    """A 512 x 512 layered medium with 8 right-hand sides (FFT length 512)."""
    med = layered_inclusion_medium(8, 512)
    pr = Pair(med, 512, 512, cuda)
    f = pr.rhs()
    st, info, u = _solve(pr, f, method, 1e-8)
    assert st == P.AX_OK
    for j in (0, 5):
        assert _oracle_rel_res(pr, f[j], u[j]) <= 1e-8
    pr.close()


@pytest.mark.parametrize("method", [P.AX_PCG_FP64, P.AX_PCG_MIXED])
def test_batched_mixes_both_boundaries(cuda, method):
    """Instances of equal shape but different z boundary land in different
    groups; each gives the same answer as its single solve."""
    insts = batched_instances(6, sizes=(31, 64))
    pairs, fs, us, singles = [], [], [], []
    for i, (nr, nz, med) in enumerate(insts):
        bc = i % 2
        kr, kz, q = sample_operator_inputs(med, nr, nz, bc_z=bc)
        t = [torch.from_numpy(x).to(cuda) for x in (kr, kz, q)]
        op = P.ax_setup_operator(*t, nr, nz, bc_z=bc)
        P.ax_set_option(op, "small_path", 0)  # the batch's kernels for the single solves too
        g = O.Grid(nr, nz, bc_z=bc)
        ora = O.Operator(kr, kz, q, g)
        f = sample_rhs(med, nr, nz, bc_z=bc)[0]
        pairs.append((op, ora, t))
        fs.append(torch.from_numpy(f).to(cuda))
        us.append(torch.zeros((nr, nz), dtype=torch.float64, device=cuda))
    batch = P.ax_batch_create([p[0] for p in pairs])
    st, info = P.ax_batch_solve(batch, fs, us, 1e-8, 5000, method)
    torch.cuda.synchronize()
    assert st == P.AX_OK
    for j, (op, ora, _) in enumerate(pairs):
        f = fs[j].cpu().numpy()
        u1 = torch.zeros((1,) + f.shape, dtype=torch.float64, device=cuda)
        st1, info1 = P.ax_solve(op, fs[j][None], u1, 1, 1e-8, 5000, method)
        assert st1 == P.AX_OK and info1[0]["iters"] == info[j]["iters"]
        assert np.array_equal(u1[0].cpu().numpy(), us[j].cpu().numpy())
        phi = ora.phi(f)
        assert np.linalg.norm(phi - ora.apply_A(us[j].cpu().numpy())) <= 1e-8 * np.linalg.norm(phi)
    P.ax_batch_destroy(batch)
    for op, _, _ in pairs:
        P.ax_destroy_operator(op)


def _folded_reference(x, n, three):
    """The tensor-core cosine forward on the same rounded values: x in FP32,
    u = x_k + x_{n-1-k} and w = x_k - x_{n-1-k} in FP32 (the middle entry of
    odd n: u = x, w = 0), each split into BF16 hi + lo, multiplied by
    C_hi = bf16(C) (and hi by C_lo = bf16(C - C_hi) for three products):
    out[2l] from u and the even modes, out[2l+1] from w and the odd ones."""
    ne = (n + 1) // 2
    x32 = x.astype(np.float32)
    k = np.arange(ne)
    xm = x32[:, n - 1 - k]
    xk = x32[:, k]
    u = (xk + xm).astype(np.float32)
    w = (xk - xm).astype(np.float32)
    if n % 2:
        u[:, ne - 1] = xk[:, ne - 1]
        w[:, ne - 1] = 0.0
    C = _orthonormal_cosine(n)
    Ch = G.round_bf16(C)
    Cl = G.round_bf16(C - Ch)
    out = np.zeros((x.shape[0], n))
    for v, rows in ((u, np.arange(0, n, 2)), (w, np.arange(1, n, 2))):
        hi = G.round_bf16(v)
        lo = G.round_bf16((v.astype(np.float32) - hi.astype(np.float32)).astype(np.float32))
        M = Ch[rows][:, :ne]
        out[:, rows] = (hi + lo) @ M.T
        if three:
            out[:, rows] += hi @ Cl[rows][:, :ne].T
    return out


@pytest.mark.parametrize("rows,nz", [(7, 1), (5, 2), (9, 3), (130, 64), (33, 127), (260, 1024), (40, 1001)])
@pytest.mark.parametrize("prec", [P.AX_PREC_FP32_TC, P.AX_PREC_FP32_TC3])
def test_tensor_cosine_forward_matches_folded_products(cuda, rows, nz, prec):
    pr = Pair(_rand_medium(4), max(rows, 2), nz, cuda)
    x = np.random.default_rng(rows + nz).normal(size=(rows, nz))
    y = torch.zeros((rows, nz), dtype=torch.float64, device=cuda)
    P.ax_apply_dst(pr.op, pr.dev_array(x), y, rows, prec)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    three = prec == P.AX_PREC_FP32_TC3
    ref = _folded_reference(x, nz, three)
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 1e-5, err.max()
    exact = x @ _orthonormal_cosine(nz).T
    assert np.linalg.norm(got - exact) <= (1e-4 if three else 1e-2) * np.linalg.norm(exact)
    pr.close()


@pytest.mark.parametrize("prec,tol", [(P.AX_PREC_FP32_TC, 2e-2), (P.AX_PREC_FP32_TC3, 1e-4)])
def test_tensor_cosine_preconditioner_symmetric_and_close(cuda, prec, tol):
    """B^-1 through the tensor-core cosine pair is C_hi^T T^-1 C_hi: symmetric
    up to the splitting of its input, and close to the exact B^-1."""
    nr, nz = 160, 300
    pr = Pair(_rand_medium(6), nr, nz, cuda)
    rng = np.random.default_rng(8)
    u, v = rng.normal(size=(1, nr, nz)), rng.normal(size=(1, nr, nz))

    def apply(x):
        out = torch.zeros((1, nr, nz), dtype=torch.float64, device=cuda)
        P.ax_apply_preconditioner(pr.op, pr.dev_array(x), out, 1, prec)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    bu, bv = apply(u), apply(v)
    a, b = np.sum(u * bv), np.sum(bu * v)
    assert abs(a - b) <= 1e-5 * np.sqrt(np.sum(u * bu) * np.sum(v * bv))
    ex = pr.ora.apply_Binv(v[0])
    assert _rel(bv[0], ex) <= tol
    pr.close()


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("nr,nz", [(96, 80), (1500, 64)])
def test_mixed_pcg_tensor_cosine(cuda, form, nr, nz):
    pr = Pair(_rand_medium(12), nr, nz, cuda)
    f = pr.rhs()
    _, i64, _ = _solve(pr, f, P.AX_PCG_FP64, 1e-8)
    P.ax_set_option(pr.op, "dst_tensor", form)
    st, imx, u = _solve(pr, f, P.AX_PCG_MIXED, 1e-8)
    assert st == P.AX_OK
    for j in range(f.shape[0]):
        assert _oracle_rel_res(pr, f[j], u[j]) <= 1e-8
        assert imx[j]["iters"] <= 1.2 * i64[j]["iters"] + 4, (imx[j], i64[j])
    pr.close()


@pytest.mark.parametrize("fused", [0, 1])
def test_mixed_pcg_tensor_cosine_fused_and_unfused(cuda, fused):
    """The direction update p = z + beta p and x += alpha p run either in the
    inverse transform's epilogue or in the stencil and update pass: both
    reach the tolerance with the iterations of the FP64 method."""
    pr = Pair(_rand_medium(15), 200, 136, cuda)
    f = pr.rhs()
    _, i64, _ = _solve(pr, f, P.AX_PCG_FP64, 1e-8)
    P.ax_set_option(pr.op, "dst_tensor", 1)
    P.ax_set_option(pr.op, "tc_fused", fused)
    st, imx, u = _solve(pr, f, P.AX_PCG_MIXED, 1e-8)
    assert st == P.AX_OK
    for j in range(f.shape[0]):
        assert _oracle_rel_res(pr, f[j], u[j]) <= 1e-8
        assert imx[j]["iters"] <= 1.2 * i64[j]["iters"] + 4, (imx[j], i64[j])
    pr.close()


def test_tensor_cosine_rejects_long_columns(cuda):
    pr = Pair(_rand_medium(2), 4, 4100, cuda)
    with pytest.raises(P.AxError) as e:
        P.ax_set_option(pr.op, "dst_tensor", 1)
    assert e.value.status == P.AX_ERR_UNSUPPORTED
    pr.close()
