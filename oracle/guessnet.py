"""FP64 reference of the initial-guess network (forward and backward).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The network proposes the starting iterate u0 of the CG solve from (kappa, q,
f).  The paper has no such network; this module is the plain reference that
the CUDA training and inference kernels are compared against.  Everything is
written out with NumPy in FP64: 3x3 "same" convolutions as sums of shifted
arrays, ReLU, 2x2 average pooling, nearest 2x upsampling, additive skips, a
1x1 head and a mean-squared-error loss, each with its hand-derived gradient.

The CUDA network stores weights and activations in BF16 and accumulates in
FP32.  forward() takes an optional `store` rounding (round_bf16 here) applied
wherever that network writes an activation to memory: the input, each conv
output after ReLU (after the skip add for "s" layers) and each pooled map.
With store=None it is the plain FP64 network.

Tensor layout: activations (C, H, W); conv weights (3, 3, Cin, Cout) indexed
[dy + 1, dx + 1, ci, co] with out[co, y, x] = b[co] +
sum_{dy, dx, ci} w[dy+1, dx+1, ci, co] * in[ci, y+dy, x+dx] (zero padding).
"""
from __future__ import annotations

import numpy as np

# (name, cin, cout, kind): kind "c" = conv3x3 + ReLU, "s" = conv3x3 + ReLU then
# add the saved skip of the same level, "h" = 1x1 head without activation.
def architecture(ch=(24, 48, 96, 192), cin=3):
    c1, c2, c3, c4 = ch
    return [
        ("e1a", cin, c1, "c"), ("e1b", c1, c1, "c"), ("pool", 0, 0, "p"),
        ("e2a", c1, c2, "c"), ("e2b", c2, c2, "c"), ("pool", 0, 0, "p"),
        ("e3a", c2, c3, "c"), ("e3b", c3, c3, "c"), ("pool", 0, 0, "p"),
        ("b1", c3, c4, "c"), ("b2", c4, c4, "c"), ("up", 0, 0, "u"),
        ("d3a", c4, c3, "s"), ("d3b", c3, c3, "c"), ("up", 0, 0, "u"),
        ("d2a", c3, c2, "s"), ("d2b", c2, c2, "c"), ("up", 0, 0, "u"),
        ("d1a", c2, c1, "s"), ("d1b", c1, c1, "c"), ("head", c1, 1, "h"),
    ]


def conv3x3(x, w, b):
    """Zero-padded 3x3 cross-correlation: out[co] = b[co] + sum w * shifted x."""
    cin, h, wd = x.shape
    xp = np.zeros((cin, h + 2, wd + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((w.shape[3], h, wd)) + b[:, None, None]
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + h, dx:dx + wd]          # in[ci, y + dy - 1, x + dx - 1]
            out += np.einsum("ihw,io->ohw", patch, w[dy, dx])
    return out


def conv3x3_backward(x, w, gout):
    """Gradients of conv3x3 with respect to x, w and b."""
    cin, h, wd = x.shape
    xp = np.zeros((cin, h + 2, wd + 2))
    xp[:, 1:-1, 1:-1] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + h, dx:dx + wd]
            gw[dy, dx] = np.einsum("ihw,ohw->io", patch, gout)
            gxp[:, dy:dy + h, dx:dx + wd] += np.einsum("io,ohw->ihw", w[dy, dx], gout)
    return gxp[:, 1:-1, 1:-1], gw, gout.sum(axis=(1, 2))


def pool2(x):
    c, h, w = x.shape
    return x.reshape(c, h // 2, 2, w // 2, 2).mean(axis=(2, 4))


def pool2_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) * 0.25


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(g):
    c, h, w = g.shape
    return g.reshape(c, h // 2, 2, w // 2, 2).sum(axis=(2, 4))


def init_params(arch, seed=0):
    """He-normal weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, cin, cout, kind in arch:
        if kind in "csh":
            k = 1 if kind == "h" else 3
            fan_in = cin * k * k
            std = np.sqrt(2.0 / fan_in) if kind != "h" else np.sqrt(1.0 / fan_in)
            w = rng.normal(0.0, std, size=(k, k, cin, cout))
            params[name] = (w, np.zeros(cout))
    return params


def round_bf16(a):
    """Rounds to the nearest BF16 value (8 significant bits, ties to even),
    by way of FP32: the upper 16 bits of the FP32 pattern after adding half
    an ulp of the kept part (plus one if the kept part is odd)."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def forward(params, arch, x, store=None):
    """Returns (output (1, H, W), cache for backward).  `store`, if given,
    rounds every activation the network keeps in memory (see the header)."""
    st = store if store is not None else (lambda v: v)
    cache = []
    skips = []
    h = st(x)
    for name, cin, cout, kind in arch:
        if kind == "p":
            skips.append(h)
            cache.append(("p", None))
            h = st(pool2(h))
        elif kind == "u":
            cache.append(("u", None))
            h = up2(h)
        elif kind in "cs":
            w, b = params[name]
            z = conv3x3(h, w, b)
            a = np.maximum(z, 0.0)
            cache.append((name, (h, z)))
            if kind == "s":
                a = a + skips.pop()
            h = st(a)
        else:  # head: 1x1
            w, b = params[name]
            cache.append((name, (h, None)))
            h = np.einsum("ihw,io->ohw", h, w[0, 0]) + b[:, None, None]
    return h, cache


def backward(params, arch, cache, gout):
    """Gradients of every parameter given d(loss)/d(output)."""
    grads = {}
    g = gout
    skip_grads = []
    for (name, cin, cout, kind), (cname, saved) in zip(reversed(arch), reversed(cache)):
        if kind == "h":
            hin, _ = saved
            w, _ = params[name]
            grads[name] = (np.einsum("ihw,ohw->io", hin, g)[None, None], g.sum(axis=(1, 2)))
            g = np.einsum("io,ohw->ihw", w[0, 0], g)
        elif kind in "cs":
            hin, z = saved
            if kind == "s":
                skip_grads.append(g)       # the skip input receives the same gradient
            gz = g * (z > 0.0)
            gx, gw, gb = conv3x3_backward(hin, params[name][0], gz)
            grads[name] = (gw, gb)
            g = gx
        elif kind == "u":
            g = up2_backward(g)
        else:  # pool: the saved activation was also a skip source
            g = pool2_backward(g) + skip_grads.pop()
    return grads, g


def h1_loss(out, target, lam):
    """Mean squared error plus lam times the squared differences of the error
    across every edge of the lattice (the last two axes), both over the
    number of values n: (sum d^2 + lam sum_edges (d_p - d_q)^2) / n, with its
    gradient 2 (d + lam L d) / n, L the lattice graph Laplacian
    (L d)_p = sum_{q next to p} (d_p - d_q)."""
    d = np.asarray(out, dtype=np.float64) - target
    n = d.size
    dx = d[..., :, 1:] - d[..., :, :-1]
    dy = d[..., 1:, :] - d[..., :-1, :]
    loss = (np.sum(d * d) + lam * (np.sum(dx * dx) + np.sum(dy * dy))) / n
    ld = np.zeros_like(d)
    ld[..., :, 1:] += dx
    ld[..., :, :-1] -= dx
    ld[..., 1:, :] += dy
    ld[..., :-1, :] -= dy
    return float(loss), 2.0 * (d + lam * ld) / n


def mse_loss(out, target):
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size


# ---------------------------------------------------------------------------
# Solver-side steps of the learned guess: lattice features, lift, optimiser.
# The paper has no network; these are the plain definitions the library's
# features / lift kernels and its Adam step are checked against.
# ---------------------------------------------------------------------------
def lattice_index(p, n, hw):
    """Grid index range of lattice cell p along an axis of n grid points:
    cell averages when n is a multiple of hw (indices p n/hw .. p n/hw +
    n/hw - 1), else the single sample at index floor(p n / hw)."""
    if n % hw == 0:
        f = n // hw
        return list(range(p * f, p * f + f))
    return [(p * n) // hw]


def features(kappa, q, f, hw, g=None):
    """Network input of one right-hand side on an hw x hw lattice: channel 0
    the mean of log kappa, channel 1 the mean of q, channel 2 the mean of
    g / s over the grid samples of each lattice cell (lattice_index along r
    and along z), s = max |g| (1 if g = 0).  g defaults to f (raw feature);
    features_pre passes g = B^-1 (r f).  Returns (x (3, hw, hw), s)."""
    kappa = np.asarray(kappa, dtype=np.float64)
    g = np.asarray(f if g is None else g, dtype=np.float64)
    nr, nz = kappa.shape
    s = float(np.abs(g).max())
    s = s if s > 0.0 else 1.0
    x = np.zeros((3, hw, hw))
    lk = np.log(kappa)
    for py in range(hw):
        ri = lattice_index(py, nr, hw)
        for px in range(hw):
            zi = lattice_index(px, nz, hw)
            blk = np.ix_(ri, zi)
            x[0, py, px] = lk[blk].mean()
            x[1, py, px] = np.asarray(q)[blk].mean()
            x[2, py, px] = g[blk].mean() / s
    return x, s


def features_pre(op, kappa, q, f, hw):
    """features() with g = B^-1 (r f): the right-hand side after one
    application of the operator's Laplace preconditioner (Section 4.2,
    Eqs. fft_phi, eq_trid), op an oracle Operator."""
    g = op.apply_Binv(op.phi(f))
    return features(kappa, q, f, hw, g=g)


def bilinear_lift(y, s, nr, nz):
    """u[i, k] = s times the bilinear interpolation of the lattice values y
    (hw x hw) at grid node (i, k), both placed by cell centres on the unit
    square of index space: lattice value (py, px) at ((py + 1/2)/hw,
    (px + 1/2)/hw), node (i, k) at ((i + 1/2)/nr, (k + 1/2)/nz).  Beyond the
    outermost lattice centres the value is held constant (the coordinates
    are clamped to the lattice)."""
    y = np.asarray(y, dtype=np.float64)
    hw = y.shape[0]
    u = np.zeros((nr, nz))
    for i in range(nr):
        gy = (i + 0.5) * hw / nr - 0.5
        y0 = min(max(int(np.floor(gy)), 0), hw - 1)
        y1 = min(y0 + 1, hw - 1)
        wy = min(max(gy - y0, 0.0), 1.0)
        for k in range(nz):
            gx = (k + 0.5) * hw / nz - 0.5
            x0 = min(max(int(np.floor(gx)), 0), hw - 1)
            x1 = min(x0 + 1, hw - 1)
            wx = min(max(gx - x0, 0.0), 1.0)
            u[i, k] = s * ((1 - wy) * ((1 - wx) * y[y0, x0] + wx * y[y0, x1])
                           + wy * ((1 - wx) * y[y1, x0] + wx * y[y1, x1]))
    return u


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One step of Adam (Kingma and Ba, "Adam: a method for stochastic
    optimization", Algorithm 1): moments m <- b1 m + (1 - b1) g,
    v <- b2 v + (1 - b2) g^2, bias corrections 1 - b1^t and 1 - b2^t, update
    p <- p - lr mhat / (sqrt(vhat) + eps).  t counts steps from 1.  Returns
    (p, m, v) as new arrays."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
