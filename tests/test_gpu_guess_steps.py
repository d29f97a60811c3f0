"""The solver-side steps of the learned initial guess against the oracle,
through the C ABI: lattice features (ax_guessnet_features, with f, and
ax_guessnet_features_pre, with g = B^-1 (r f)), the bilinear lift
(ax_guessnet_lift), one and two Adam steps of ax_guessnet_train_step, and
solves started from lifted guesses.

Tolerances (relative to the largest magnitude of the compared array):
  features, channels log kappa and q   1e-6 (FP64 sums stored in FP32)
  features, channel g / s and s        1e-6 for the raw f; 2e-4 for g from
                                       the FP32 preconditioner (1e-5 with the
                                       FFT transform, ~1e-4 with the BF16-split
                                       tensor-core transform)
  lift                                 1e-5 (FP32 lattice positions: a position
                                       up to hw carries ~hw 2^-24 in its weight)
  Adam                                 |p - p_ref| <= 1e-5 lr + 4 ulp(p) (FP32
                                       moments and update)
  guess-started solves                 oracle FP64 true residual <= 1e-8
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle import guessnet as G  # noqa: E402
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


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _maxrel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("nr,nz,hw", [(64, 64, 32), (64, 64, 64), (64, 96, 32), (60, 70, 32), (64, 70, 16),
                                      (33, 17, 8)])
def test_features_match_oracle(cuda, nr, nz, hw):
    """Cell averages where hw divides the axis, single samples where it does
    not (both, either, neither)."""
    rng = np.random.default_rng(nr * nz + hw)
    kap = np.exp(rng.normal(size=(nr, nz)))
    q = rng.uniform(size=(nr, nz))
    m = 2
    f = rng.normal(size=(m, nr, nz))
    f[1] *= 1e-7  # scale-free up to s
    x = torch.zeros((m, 3, hw, hw), dtype=torch.float32, device=cuda)
    s = torch.zeros(m, dtype=torch.float64, device=cuda)
    P.ax_guessnet_features(_t(kap, cuda), _t(q, cuda), _t(f, cuda), m, nr, nz, hw, x, s)
    torch.cuda.synchronize()
    xg, sg = x.cpu().numpy().astype(np.float64), s.cpu().numpy()
    for j in range(m):
        xr, sr = G.features(kap, q, f[j], hw)
        assert sg[j] == sr
        for ch in range(3):
            assert _maxrel(xg[j, ch], xr[ch]) <= 1e-6, (j, ch)


@pytest.mark.parametrize("nr,nz,hw", [(64, 64, 32), (64, 63, 16), (128, 127, 64)])
def test_features_pre_match_oracle(cuda, nr, nz, hw):
    med = layered_inclusion_medium(n_rhs=2, nominal_n=max(nr, nz), instance=1)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    f = sample_rhs(med, nr, nz)
    op = P.ax_setup_operator(_t(kr, cuda), _t(kz, cuda), _t(q, cuda), nr, nz)
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz))
    x = torch.zeros((2, 3, hw, hw), dtype=torch.float32, device=cuda)
    s = torch.zeros(2, dtype=torch.float64, device=cuda)
    P.ax_guessnet_features_pre(op, _t(kr, cuda), _t(q, cuda), _t(f, cuda), 2, hw, x, s)
    torch.cuda.synchronize()
    xg, sg = x.cpu().numpy().astype(np.float64), s.cpu().numpy()
    for j in range(2):
        xr, sr = G.features_pre(ora, kr, q, f[j], hw)
        assert abs(sg[j] - sr) <= 2e-4 * sr
        assert _maxrel(xg[j, 0], xr[0]) <= 1e-6 and _maxrel(xg[j, 1], xr[1]) <= 1e-6
        assert _maxrel(xg[j, 2], xr[2]) <= 2e-4, j
    P.ax_destroy_operator(op)


@pytest.mark.parametrize("hw,nr,nz", [(32, 64, 64), (32, 100, 37), (16, 16, 16), (8, 257, 129), (64, 512, 512)])
def test_lift_matches_oracle(cuda, hw, nr, nz):
    rng = np.random.default_rng(hw + nr)
    m = 2
    y = rng.normal(size=(m, hw, hw)).astype(np.float32)
    s = np.array([0.5, 3e-4])
    u = torch.zeros((m, nr, nz), dtype=torch.float64, device=cuda)
    P.ax_guessnet_lift(_t(y, cuda), m, hw, _t(s, cuda), nr, nz, u)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    for j in range(m):
        ref = G.bilinear_lift(y[j].astype(np.float64), s[j], nr, nz)
        assert _maxrel(got[j], ref) <= 1e-5, j


def test_lift_full_size_sampled_rows(cuda):
    """The 512^2 lattice lifted onto 4096^2 (the large workload's guess):
    sampled rows against the oracle's formula on those rows."""
    hw, nr, nz = 512, 4096, 4096
    rng = np.random.default_rng(5)
    y = rng.normal(size=(1, hw, hw)).astype(np.float32)
    s = np.array([2.0])
    u = torch.zeros((1, nr, nz), dtype=torch.float64, device=cuda)
    P.ax_guessnet_lift(_t(y, cuda), 1, hw, _t(s, cuda), nr, nz, u)
    torch.cuda.synchronize()
    got = u.cpu().numpy()[0]
    # rows i of the lift depend on lattice rows y0, y0 + 1 only: lift a 2-row
    # lattice band with the same fractional position and compare
    for i in rng.choice(nr, 16, replace=False):
        gy = (i + 0.5) * hw / nr - 0.5
        y0 = min(max(int(np.floor(gy)), 0), hw - 1)
        y1 = min(y0 + 1, hw - 1)
        wy = min(max(gy - y0, 0.0), 1.0)
        band = (1 - wy) * y[0, y0].astype(np.float64) + wy * y[0, y1].astype(np.float64)
        ref = G.bilinear_lift(np.tile(band, (hw, 1)), s[0], 1, nz)[0]
        assert _maxrel(got[i], ref) <= 1e-4, i  # positions up to 512: ~512 2^-24 in the weights


CH = (8, 16, 16, 32)
HW = 32


@pytest.mark.parametrize("lr", [1e-3, 3e-2])
def test_adam_steps_match_oracle(cuda, lr):
    net = P.ax_guessnet_create(HW, CH, batch_capacity=2, seed=4)
    rng = np.random.default_rng(9)
    x = torch.from_numpy(rng.normal(size=(2, 3, HW, HW)).astype(np.float32)).to(cuda)
    t = torch.from_numpy(rng.normal(size=(2, HW, HW)).astype(np.float32)).to(cuda)
    p = P.ax_guessnet_get_params(net).astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    prev = None
    for step in (1, 2):
        _, g = P.ax_guessnet_gradients(net, x, t, 2)
        g = g.astype(np.float64)
        if prev is not None:  # the step refreshed the BF16 copy the gradients use
            assert not np.array_equal(g, prev)
        prev = g
        P.ax_guessnet_train_step(net, x, t, 2, lr)
        torch.cuda.synchronize()
        got = P.ax_guessnet_get_params(net).astype(np.float64)
        ref, m, v = G.adam_step(p, g, m, v, step, lr)
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        assert (np.abs(got - ref) <= 1e-5 * lr + 4 * ulp).all(), (step, np.abs(got - ref).max())
        p = got
    P.ax_guessnet_destroy(net)


@pytest.mark.parametrize("method", [P.AX_PCG_MIXED, P.AX_PCG_FP64])
def test_guess_started_solves_meet_tolerance(cuda, method):
    """A lifted lattice guess (the oracle solution's cell averages: a good
    guess, which the gate keeps) and the untrained network's guess (a poor
    one): each solve meets 1e-8 in the oracle's FP64 true residual, the good
    guess is accepted and saves iterations."""
    nr = nz = 64
    hw = 32
    med = bumps_medium(2)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    f = sample_rhs(med, nr, nz)
    op = P.ax_setup_operator(_t(kr, cuda), _t(kz, cuda), _t(q, cuda), nr, nz)
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz))
    u_ora, _ = ora.solve(f[0], 1e-12)
    phi = ora.phi(f[0])
    fd = _t(f, cuda)
    s = torch.tensor([np.abs(u_ora).max()], dtype=torch.float64, device=cuda)
    y = (u_ora / s.item()).reshape(hw, 2, hw, 2).mean(axis=(1, 3)).astype(np.float32)[None]
    u0 = torch.zeros((1, nr, nz), dtype=torch.float64, device=cuda)
    P.ax_guessnet_lift(_t(y, cuda), 1, hw, s, nr, nz, u0)
    uz = torch.zeros_like(u0)
    st, iz = P.ax_solve(op, fd, uz, 1, 1e-8, 5000, method)
    assert st == P.AX_OK
    flags = P.AX_FLAG_USE_GUESS | P.AX_FLAG_CHECK_GUESS
    st, ig = P.ax_solve(op, fd, u0, 1, 1e-8, 5000, method, flags)
    torch.cuda.synchronize()
    assert st == P.AX_OK and ig[0]["guess_accepted"] == 1
    assert ig[0]["iters"] < iz[0]["iters"], (ig, iz)
    res = np.linalg.norm(phi - ora.apply_A(u0.cpu().numpy()[0])) / np.linalg.norm(phi)
    assert res <= 1e-8
    # the untrained network's guess through features, forward and lift
    net = P.ax_guessnet_create(hw, CH, batch_capacity=1, seed=2)
    x = torch.zeros((1, 3, hw, hw), dtype=torch.float32, device=cuda)
    sc = torch.zeros(1, dtype=torch.float64, device=cuda)
    P.ax_guessnet_features_pre(op, _t(kr, cuda), _t(q, cuda), fd, 1, hw, x, sc)
    yn = torch.zeros((1, hw, hw), dtype=torch.float32, device=cuda)
    P.ax_guessnet_forward(net, x, yn, 1)
    un = torch.zeros((1, nr, nz), dtype=torch.float64, device=cuda)
    P.ax_guessnet_lift(yn, 1, hw, sc, nr, nz, un)
    st, inn = P.ax_solve(op, fd, un, 1, 1e-8, 5000, method, flags)
    torch.cuda.synchronize()
    assert st == P.AX_OK
    res = np.linalg.norm(phi - ora.apply_A(un.cpu().numpy()[0])) / np.linalg.norm(phi)
    assert res <= 1e-8
    P.ax_guessnet_destroy(net)
    P.ax_destroy_operator(op)


@pytest.mark.parametrize("pre,target_scale", [(True, 1.0), (False, 40.0)])
def test_solve_learned_equals_its_composition(cuda, pre, target_scale):
    """ax_solve_learned (features, forward in batches of the network's
    capacity, lift with s / target_scale, gated solve) gives the same guesses,
    gate decisions, iterations and solutions, bit for bit, as the same steps
    called one by one, and meets the tolerance in the oracle's FP64 residual.
    Three right-hand sides on a network of capacity 2: two forward batches."""
    nr = nz = 64
    hw = 32
    med = layered_inclusion_medium(n_rhs=3, nominal_n=64, instance=12)
    kr, kz, q = sample_operator_inputs(med, nr, nz)
    f = sample_rhs(med, nr, nz)[:3]
    m = f.shape[0]
    op = P.ax_setup_operator(_t(kr, cuda), _t(kz, cuda), _t(q, cuda), nr, nz)
    ora = O.Operator(kr, kz, q, O.Grid(nr, nz))
    net = P.ax_guessnet_create(hw, batch_capacity=2, seed=7)
    kd, qd, fd = _t(kr, cuda), _t(q, cuda), _t(f, cuda)
    # the steps one by one
    x = torch.zeros((m, 3, hw, hw), dtype=torch.float32, device=cuda)
    s = torch.zeros(m, dtype=torch.float64, device=cuda)
    if pre:
        P.ax_guessnet_features_pre(op, kd, qd, fd, m, hw, x, s)
    else:
        P.ax_guessnet_features(kd, qd, fd, m, nr, nz, hw, x, s)
    y = torch.zeros((m, hw, hw), dtype=torch.float32, device=cuda)
    for c in range(0, m, 2):
        b = min(2, m - c)
        P.ax_guessnet_forward(net, x[c:c + b], y[c:c + b], b)
    u1 = torch.zeros_like(fd)
    P.ax_guessnet_lift(y, m, hw, s / target_scale, nr, nz, u1)
    st1, i1 = P.ax_solve(op, fd, u1, m, 1e-8, 5000, P.AX_PCG_MIXED, P.AX_FLAG_USE_GUESS | P.AX_FLAG_CHECK_GUESS)
    # in one call
    u2 = torch.full_like(fd, float("nan"))  # overwritten by the lift
    st2, i2 = P.ax_solve_learned(op, net, kd, qd, fd, u2, m, 1e-8, 5000, P.AX_PCG_MIXED, pre=pre,
                                 target_scale=target_scale)
    torch.cuda.synchronize()
    assert st1 == st2 == P.AX_OK
    assert [(a["iters"], a["guess_accepted"]) for a in i1] == [(b["iters"], b["guess_accepted"]) for b in i2]
    assert torch.equal(u1, u2)
    un = u2.cpu().numpy()
    for j in range(m):
        phi = ora.phi(f[j])
        assert np.linalg.norm(phi - ora.apply_A(un[j])) <= 1e-8 * np.linalg.norm(phi)
    assert P.ax_solve_learned(op, net, kd, qd, fd, u2, m, 1e-8, 5000, P.AX_PCG_MIXED, target_scale=0.0,
                              raise_on_error=False)[0] == P.AX_ERR_INVALID_ARG
    P.ax_guessnet_destroy(net)
    P.ax_destroy_operator(op)
