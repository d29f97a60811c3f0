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
