"""The initial-guess network's CUDA kernels against its FP64 reference.

The kernels keep conv weights and activations in BF16 and accumulate in
FP32, so they are compared with the FP64 reference run on the same BF16
values: conv weights rounded to BF16 and every kept activation rounded by
round_bf16 (the reference's `store`).  What remains is FP32 against FP64
accumulation, a BF16 rounding that falls the other way when the two
accumulations straddle a rounding boundary, and the first layer's weight
gradient, which reads the FP32 input rather than its BF16 copy.
Tolerances (relative, 2-norm): forward output 5e-3, every layer's weight and
bias gradient 2e-2, for the plain squared error and for the loss with the
lattice-edge (H1) term.  Against the unrounded FP64 network the gradients of the
4x4 bottleneck layers differ by up to ~25% (ReLU decisions that BF16 storage
flips), which is why the rounding is matched instead of the tolerance
widened.  The reference backward is itself pinned to finite differences in
test_oracle_guessnet.py."""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1002_3094_gb300 as P  # noqa: E402
from oracle import guessnet as G  # noqa: E402

pytestmark = pytest.mark.gpu

CH = (8, 16, 16, 32)
HW = 32


@pytest.fixture(scope="module")
def cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.load_library()
    return torch.device("cuda:0")


def _to_oracle(flat, arch):
    params, off = {}, 0
    for name, cin, cout, kind in arch:
        if kind in "cs":
            n = 9 * cin * cout
            w = flat[off:off + n].reshape(3, 3, cin, cout).astype(np.float64)
            off += n
            b = flat[off:off + cout].astype(np.float64)
            off += cout
            params[name] = (w, b)
        elif kind == "h":
            w = flat[off:off + cin].reshape(1, 1, cin, 1).astype(np.float64)
            off += cin
            b = flat[off:off + 1].astype(np.float64)
            off += 1
            params[name] = (w, b)
    assert off == flat.size
    return params


def _bf16_weights(params, arch):
    """Conv weights as the kernels hold them (BF16); the 1x1 head reads FP32."""
    out = dict(params)
    for name, cin, cout, kind in arch:
        if kind in "cs":
            w, b = params[name]
            out[name] = (G.round_bf16(w), b)
    return out


def _flat_grads(grads, arch):
    out = []
    for name, cin, cout, kind in arch:
        if kind in "csh":
            gw, gb = grads[name]
            out += [gw.ravel(), gb.ravel()]
    return np.concatenate(out)


def _inputs(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, 3, HW, HW)).astype(np.float32)
    t = rng.normal(size=(B, 1, HW, HW)).astype(np.float32)
    return x, t


def test_forward_matches_reference(cuda):
    arch = G.architecture(ch=CH)
    net = P.ax_guessnet_create(HW, CH, batch_capacity=4, seed=7)
    flat = P.ax_guessnet_get_params(net)
    params = _bf16_weights(_to_oracle(flat, arch), arch)
    x, _ = _inputs(3, 1)
    y = torch.zeros((3, HW, HW), dtype=torch.float32, device=cuda)
    P.ax_guessnet_forward(net, torch.from_numpy(x).to(cuda), y, 3)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    for b in range(3):
        ref, _ = G.forward(params, arch, x[b].astype(np.float64), store=G.round_bf16)
        assert np.linalg.norm(got[b] - ref[0]) <= 5e-3 * np.linalg.norm(ref[0])
    P.ax_guessnet_destroy(net)


def _check_gradients(cuda, h1):
    arch = G.architecture(ch=CH)
    net = P.ax_guessnet_create(HW, CH, batch_capacity=4, seed=9)
    if h1:
        P.ax_guessnet_set_loss(net, h1)
    rng = np.random.default_rng(3)
    flat = P.ax_guessnet_get_params(net)
    flat = flat + rng.normal(0, 0.05, size=flat.size).astype(np.float32) * (np.abs(flat) == 0)  # non-zero biases
    P.ax_guessnet_set_params(net, flat)
    params = _bf16_weights(_to_oracle(flat, arch), arch)
    B = 2
    x, t = _inputs(B, 5)
    loss, g = P.ax_guessnet_gradients(net, torch.from_numpy(x).to(cuda), torch.from_numpy(t).to(cuda), B)
    # reference: the loss is the mean over the batch of the per-sample loss
    gsum, lsum = None, 0.0
    for b in range(B):
        out, cache = G.forward(params, arch, x[b].astype(np.float64), store=G.round_bf16)
        lb, gout = G.h1_loss(out, t[b], h1)
        lsum += lb / B
        grads, _ = G.backward(params, arch, cache, gout / B)
        fg = _flat_grads(grads, arch)
        gsum = fg if gsum is None else gsum + fg
    assert abs(loss - lsum) <= 5e-3 * lsum
    off = 0
    for name, cin, cout, kind in arch:
        if kind not in "csh":
            continue
        nw = (9 if kind != "h" else 1) * cin * cout
        for part, n in (("w", nw), ("b", cout)):
            a, r = g[off:off + n], gsum[off:off + n]
            off += n
            assert np.linalg.norm(a - r) <= 2e-2 * np.linalg.norm(r) + 1e-7, (name, part)
    P.ax_guessnet_destroy(net)


def test_gradients_match_reference(cuda):
    _check_gradients(cuda, 0.0)


def test_h1_loss_gradients_match_reference(cuda):
    _check_gradients(cuda, 3.0)


def test_training_lowers_loss_and_checkpoint_round_trip(cuda):
    net = P.ax_guessnet_create(HW, CH, batch_capacity=4, seed=11)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(4, 3, HW, HW)).astype(np.float32)
    # a learnable target: a smoothed mix of the inputs
    t = (0.5 * x[:, 0:1] - 0.25 * x[:, 2:3]).astype(np.float32)
    xd, td = torch.from_numpy(x).to(cuda), torch.from_numpy(t).to(cuda)
    losses = [P.ax_guessnet_train_step(net, xd, td, 4, 3e-3) for _ in range(60)]
    assert losses[-1] < 0.3 * losses[0], losses[::10]
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "w.axgn")
        P.ax_guessnet_save(net, path)
        net2 = P.ax_guessnet_create(HW, CH, batch_capacity=4, seed=0)
        P.ax_guessnet_load(net2, path)
        assert np.array_equal(P.ax_guessnet_get_params(net), P.ax_guessnet_get_params(net2))
        with open(path, "r+b") as fh:  # corrupt one parameter byte: the checksum must catch it
            fh.seek(40)
            bt = fh.read(1)
            fh.seek(40)
            fh.write(bytes([bt[0] ^ 0xFF]))
        with pytest.raises(P.AxError):
            P.ax_guessnet_load(net2, path)
        P.ax_guessnet_destroy(net2)
    P.ax_guessnet_destroy(net)
