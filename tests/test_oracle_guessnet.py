"""Pins for the FP64 reference of the initial-guess network: convolution
against scipy.signal.correlate, adjoint identities, and every gradient
against central finite differences."""
import numpy as np
import pytest
import scipy.signal

from oracle import guessnet as G


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 9, 7))
    w = rng.normal(size=(3, 3, 3, 4))
    b = rng.normal(size=4)
    out = G.conv3x3(x, w, b)
    for co in range(4):
        ref = b[co] + sum(scipy.signal.correlate(x[ci], w[:, :, ci, co], mode="same") for ci in range(3))
        np.testing.assert_allclose(out[co], ref, rtol=1e-12, atol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 8, 6))
    y = rng.normal(size=(2, 4, 3))
    assert np.isclose(np.sum(G.pool2(x) * y), np.sum(x * G.pool2_backward(y)))
    assert np.isclose(np.sum(G.up2(y) * x), np.sum(y * G.up2_backward(x)))


def test_gradients_match_finite_differences():
    arch = G.architecture(ch=(2, 3, 4, 5), cin=3)
    params = G.init_params(arch, seed=3)
    rng = np.random.default_rng(4)
    # non-zero biases so that ReLU kinks are away from the probe points
    params = {k: (w, rng.normal(0, 0.1, size=b.shape)) for k, (w, b) in params.items()}
    x = rng.normal(size=(3, 16, 16))
    t = rng.normal(size=(1, 16, 16))

    def loss(p, xx):
        out, _ = G.forward(p, arch, xx)
        return G.mse_loss(out, t)[0]

    out, cache = G.forward(params, arch, x)
    _, gout = G.mse_loss(out, t)
    grads, gx = G.backward(params, arch, cache, gout)
    eps = 1e-6
    for name in ("e1a", "e2b", "b1", "d3a", "d1a", "d1b", "head"):
        w, b = params[name]
        gw, gb = grads[name]
        for idx in [tuple(rng.integers(0, s) for s in w.shape) for _ in range(4)]:
            wp, wm = w.copy(), w.copy()
            wp[idx] += eps
            wm[idx] -= eps
            fd = (loss({**params, name: (wp, b)}, x) - loss({**params, name: (wm, b)}, x)) / (2 * eps)
            assert abs(fd - gw[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, gw[idx])
        j = int(rng.integers(0, b.shape[0]))
        bp, bm = b.copy(), b.copy()
        bp[j] += eps
        bm[j] -= eps
        fd = (loss({**params, name: (w, bp)}, x) - loss({**params, name: (w, bm)}, x)) / (2 * eps)
        assert abs(fd - gb[j]) <= 1e-6 * max(1.0, abs(fd)), (name, j)
    for idx in [(0, 3, 4), (2, 15, 0), (1, 8, 8)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        fd = (loss(params, xp) - loss(params, xm)) / (2 * eps)
        assert abs(fd - gx[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_default_network_has_about_a_million_parameters():
    arch = G.architecture()
    n = sum(w.size + b.size for w, b in G.init_params(arch).values())
    assert 0.9e6 < n < 1.1e6


def test_round_bf16_ties_to_even_and_matches_torch():
    u = 2.0 ** -7  # BF16 spacing on [1, 2)
    cases = {1.0: 1.0, 1 + u / 2: 1.0, 1 + 1.5 * u: 1 + 2 * u, 1 + u / 2 + 2.0 ** -20: 1 + u,
             -(1 + 1.5 * u): -(1 + 2 * u), 3.0: 3.0, 0.0: 0.0}
    for a, want in cases.items():
        assert G.round_bf16(np.array([a]))[0] == want, a
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = (rng.normal(size=4096) * np.exp(rng.normal(size=4096) * 5)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(G.round_bf16(x), ref)


def test_store_rounding_applies_to_every_kept_activation():
    arch = G.architecture(ch=(4, 4, 4, 4))
    params = G.init_params(arch, seed=1)
    calls = []

    def store(v):
        calls.append(v.shape)
        return G.round_bf16(v)

    x = np.random.default_rng(2).normal(size=(3, 16, 16))
    out, _ = G.forward(params, arch, x, store=store)
    n_conv = sum(k in "cs" for _, _, _, k in arch)
    n_pool = sum(k == "p" for _, _, _, k in arch)
    assert len(calls) == 1 + n_conv + n_pool
    ref, _ = G.forward(params, arch, x)
    # rounding kept activations to 8 significant bits moves the output by
    # about the BF16 unit roundoff times the depth, not more
    assert 0 < np.linalg.norm(out - ref) <= 5e-2 * np.linalg.norm(ref)


def test_h1_loss_closed_forms_and_finite_differences():
    rng = np.random.default_rng(6)
    H, W = 5, 7
    t = rng.normal(size=(1, H, W))
    # lam = 0 is the mean squared error
    out = rng.normal(size=(1, H, W))
    l0, g0 = G.h1_loss(out, t, 0.0)
    lm, gm = G.mse_loss(out, t)
    assert np.isclose(l0, lm) and np.allclose(g0, gm)
    # a constant error has no edge term
    l, g = G.h1_loss(t + 0.3, t, 5.0)
    assert np.isclose(l, 0.09) and np.allclose(g, 2 * 0.3 / (H * W))
    # a ramp a*x along the last axis: H (W - 1) edges of squared difference a^2
    a = 0.2
    ramp = a * np.arange(W)[None, None, :] * np.ones((1, H, 1))
    l, _ = G.h1_loss(t + ramp, t, 3.0)
    assert np.isclose(l, (np.sum(ramp ** 2) + 3.0 * H * (W - 1) * a * a) / (H * W))
    # gradient against central differences
    lam, eps = 2.5, 1e-6
    _, g = G.h1_loss(out, t, lam)
    for idx in [(0, 0, 0), (0, 2, 3), (0, H - 1, W - 1), (0, 4, 0)]:
        op, om = out.copy(), out.copy()
        op[idx] += eps
        om[idx] -= eps
        fd = (G.h1_loss(op, t, lam)[0] - G.h1_loss(om, t, lam)[0]) / (2 * eps)
        assert abs(fd - g[idx]) <= 1e-7 * max(1.0, abs(fd))


# ---------------------------------------------------------------------------
# Solver-side steps: lattice features, lift, Adam
# ---------------------------------------------------------------------------
import os  # noqa: E402

import oracle as O  # noqa: E402


def _golden_features():
    cases = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "guess_features.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            c = cases.setdefault(parts[0], {"x": np.zeros((3, 2, 2)), "s": None})
            if parts[1] == "SCALE":
                c["s"] = float(parts[2])
            else:
                ch, py, px = map(int, parts[1:4])
                c["x"][ch, py, px] = float(parts[4])
    return cases


def test_features_hand_worked_cases():
    g = _golden_features()
    i, k = np.meshgrid(np.arange(5), np.arange(3), indexing="ij")
    x, s = G.features(np.exp(i - k), i * k, (i - 2.0) * (k + 1), 2)
    np.testing.assert_allclose(x, g["A"]["x"], rtol=0, atol=1e-15)
    assert s == g["A"]["s"]
    i, k = np.meshgrid(np.arange(4), np.arange(2), indexing="ij")
    x, s = G.features(np.exp(i + k), i * 1.0, i * (k + 1.0) - 1.0, 2)
    np.testing.assert_allclose(x, g["B"]["x"], rtol=0, atol=1e-15)
    assert s == g["B"]["s"]


def test_features_identity_lattice_and_separable_log_mean():
    rng = np.random.default_rng(2)
    kap = np.exp(rng.normal(size=(8, 8)))
    q = rng.uniform(size=(8, 8))
    f = rng.normal(size=(8, 8))
    x, s = G.features(kap, q, f, 8)            # lattice = grid: the samples themselves
    assert s == np.abs(f).max()
    np.testing.assert_allclose(x[0], np.log(kap), rtol=1e-15)
    np.testing.assert_allclose(x[2] * s, f, rtol=1e-15)
    # kappa = a(r) b(z): the cell mean of log kappa is mean log a + mean log b
    a, b = np.exp(rng.normal(size=12)), np.exp(rng.normal(size=9))
    x, _ = G.features(np.outer(a, b), np.ones((12, 9)), np.ones((12, 9)), 3)
    ref = np.log(a).reshape(3, 4).mean(1)[:, None] + np.log(b).reshape(3, 3).mean(1)[None, :]
    np.testing.assert_allclose(x[0], ref, rtol=1e-13)
    assert np.allclose(x[1], 1.0) and np.allclose(x[2], 1.0)
    # a zero right-hand side keeps s = 1
    _, s0 = G.features(kap, q, np.zeros((8, 8)), 4)
    assert s0 == 1.0


def test_features_pre_is_the_preconditioned_rhs():
    """Channel 2 holds g / s, g = B^-1 (r f): B g = phi with the dense
    assembly of B (tiny grid, lattice = grid)."""
    nr, nz = 6, 5
    grid = O.Grid(nr, nz)
    rng = np.random.default_rng(7)
    kr = 1 + rng.uniform(size=(nr, nz))
    kz = 1 + rng.uniform(size=(nr, nz + 1))
    q = rng.uniform(size=(nr, nz))
    f = rng.normal(size=(nr, nz))
    op = O.Operator(kr, kz, q, grid)
    x, s = G.features_pre(op, kr, q, f, 1)     # 1 x 1 lattice: the means over the grid
    B = O.assemble_preconditioner(op.kappa_t, op.q_t, grid).toarray()
    g = np.linalg.solve(B, op.phi(f).ravel()).reshape(nr, nz)
    assert np.isclose(s, np.abs(g).max(), rtol=1e-12)
    assert np.isclose(x[2, 0, 0], g.mean() / s, rtol=1e-10)
    assert np.isclose(x[0, 0, 0], np.log(kr).mean(), rtol=1e-14)


def test_lift_reproduces_affine_and_matches_scipy():
    from scipy.interpolate import RegularGridInterpolator
    hw, nr, nz, s = 8, 37, 50, 2.5
    c = (np.arange(hw) + 0.5) / hw
    y = 0.3 + 1.7 * c[:, None] - 0.9 * c[None, :]
    u = G.bilinear_lift(y, s, nr, nz)
    ny, nx = (np.arange(nr) + 0.5) / nr, (np.arange(nz) + 0.5) / nz
    inner_r = (ny >= c[0]) & (ny <= c[-1])
    inner_z = (nx >= c[0]) & (nx <= c[-1])
    exact = s * (0.3 + 1.7 * ny[:, None] - 0.9 * nx[None, :])
    np.testing.assert_allclose(u[np.ix_(inner_r, inner_z)], exact[np.ix_(inner_r, inner_z)], rtol=1e-12, atol=1e-14)
    # any lattice values, against scipy with the coordinates clamped to the lattice
    yr = np.random.default_rng(3).normal(size=(hw, hw))
    u = G.bilinear_lift(yr, s, nr, nz)
    rgi = RegularGridInterpolator((c, c), yr, method="linear")
    pts = np.stack(np.meshgrid(np.clip(ny, c[0], c[-1]), np.clip(nx, c[0], c[-1]), indexing="ij"), -1)
    np.testing.assert_allclose(u, s * rgi(pts), rtol=1e-12, atol=1e-14)
    # lattice = grid: the values themselves
    np.testing.assert_allclose(G.bilinear_lift(yr, s, hw, hw), s * yr, rtol=1e-15)


def test_adam_matches_torch_and_first_step_closed_form():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    p0 = rng.normal(size=20)
    grads = [rng.normal(size=20) for _ in range(3)]
    lr = 3e-3
    # first step: mhat = g, vhat = g^2, so the update is lr g / (|g| + eps)
    p1, _, _ = G.adam_step(p0, grads[0], np.zeros(20), np.zeros(20), 1, lr)
    np.testing.assert_allclose(p1, p0 - lr * grads[0] / (np.abs(grads[0]) + 1e-8), rtol=1e-14)
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(20), np.zeros(20)
    for step, g in enumerate(grads, start=1):
        opt.zero_grad()
        t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = G.adam_step(p, g, m, v, step, lr)
        np.testing.assert_allclose(p, t.detach().numpy(), rtol=1e-13, atol=1e-15)
