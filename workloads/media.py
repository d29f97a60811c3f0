"""Seeded media and sources for the axisymmetric elliptic problem.

The problem (Section 2.1, Eq. main_eq) is posed on G = [0, 1] x [0, 1] in
(r, z); kappa > 0 and q >= 0 (Eq. elliptic_condition, Eq. main_problem).  The
paper's own media (the "geological fault" velocity model, Marmousi) are
available only as figures or not at all, so seeded synthetic media shaped like
them (layered, with inclusions, moderate contrast) stand in for them.

Every medium is a set of plain functions of (r, z).  Nothing here knows about
grids, stencils or solvers.  All random numbers come from
``numpy.random.default_rng(SeedSequence([SEED_ROOT, workload, instance]))``.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Sequence

import numpy as np

SEED_ROOT = 10023094

Field = Callable[[np.ndarray, np.ndarray], np.ndarray]


def _rng(workload: int, instance: int = 0) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([SEED_ROOT, workload, instance]))


def _reference_lattice(n: int = 256):
    """Cell centres of a uniform n x n lattice on [0,1]^2 (used only to rescale
    generated fields; it is not a solver grid)."""
    t = (np.arange(n) + 0.5) / n
    return np.meshgrid(t, t, indexing="ij")


@dataclasses.dataclass
class Medium:
    """kappa(r, z), q(r, z) and right-hand sides f_m(r, z), m = 0..n_rhs-1."""

    name: str
    kappa: Field
    q: Field
    sources: List[Field]
    description: str = ""

    @property
    def n_rhs(self) -> int:
        return len(self.sources)

    def f(self, r: np.ndarray, z: np.ndarray, m: int) -> np.ndarray:
        return self.sources[m](r, z)


def _gaussian(rc: float, zc: float, sigma: float, amp: float = 1.0) -> Field:
    def g(r, z):
        return amp * np.exp(-((r - rc) ** 2 + (z - zc) ** 2) / (2.0 * sigma * sigma))
    return g


def _const(c: float) -> Field:
    def g(r, z):
        return np.full(np.broadcast(r, z).shape, float(c))
    return g


def _layers(cuts: np.ndarray, values: np.ndarray) -> Field:
    """Piecewise-constant in z: layer j covers [cuts[j-1], cuts[j]) (half-open,
    so a point on an interface takes the value of the layer above it)."""
    cuts = np.asarray(cuts, dtype=np.float64)
    values = np.asarray(values, dtype=np.float64)

    def g(r, z):
        idx = np.searchsorted(cuts, np.asarray(z, dtype=np.float64), side="right")
        return np.broadcast_to(values[idx], np.broadcast(r, z).shape).copy()
    return g


def _ellipse_indicator(rc, zc, a, b, width) -> Field:
    """Smooth indicator of the ellipse ((r-rc)/a)^2 + ((z-zc)/b)^2 <= 1 with a
    logistic edge of the given width (in units of length)."""
    scale = min(a, b)

    def g(r, z):
        rho = np.sqrt(((r - rc) / a) ** 2 + ((z - zc) / b) ** 2)
        d = (rho - 1.0) * scale / width
        return 0.5 * (1.0 - np.tanh(0.5 * d))  # = 1 / (1 + exp(d)), overflow-safe
    return g


# ---------------------------------------------------------------------------
# Workload 1: three Gaussian bumps, one Gaussian source (64 x 64, FP64 PCG).
# ---------------------------------------------------------------------------
def bumps_medium(instance: int = 0) -> Medium:
    rng = _rng(1, instance)
    amps = rng.uniform(0.0, 2.0, size=3)
    centres = rng.uniform(0.0, 1.0, size=(3, 2))
    src = rng.uniform(0.1, 0.9, size=2)
    bumps = [_gaussian(c[0], c[1], 0.1, a) for a, c in zip(amps, centres)]

    def kappa(r, z):
        out = np.ones(np.broadcast(r, z).shape)
        for b in bumps:
            out = out + b(r, z)
        return out

    return Medium("bumps", kappa, _const(0.1), [_gaussian(src[0], src[1], 0.05)],
                  "kappa = 1 + 3 Gaussian bumps (amplitude U[0,2], sigma 0.1); q = 0.1; "
                  "one Gaussian source (sigma 0.05)")


# ---------------------------------------------------------------------------
# Workload 2: 8 z-layers x elliptical inclusion, q proportional to kappa,
# M point-like Gaussian sources (1024 x 1024 x 64, mixed precision).
# ---------------------------------------------------------------------------
def layered_inclusion_medium(n_rhs: int = 64, nominal_n: int = 1024, instance: int = 0,
                             eta: float = 10.0) -> Medium:
    rng = _rng(2, instance)
    cuts = np.sort(rng.uniform(0.0, 1.0, size=7))
    values = 10.0 ** rng.uniform(0.0, 1.0, size=8)
    h = 1.0 / nominal_n
    inc = _ellipse_indicator(*rng.uniform(0.2, 0.8, size=2), *rng.uniform(0.05, 0.2, size=2),
                             width=2.0 * h)
    layer = _layers(cuts, values)

    def kappa(r, z):
        return layer(r, z) * (1.0 + 4.0 * inc(r, z))

    rr, zz = _reference_lattice(512)
    kappa_geo = float(np.exp(np.mean(np.log(kappa(rr, zz)))))

    def q(r, z):
        return (0.5 * eta / kappa_geo) * kappa(r, z)

    centres = rng.uniform(0.05, 0.95, size=(n_rhs, 2))
    sources = [_gaussian(c[0], c[1], 2.0 * h) for c in centres]
    return Medium("layered_inclusion", kappa, q, sources,
                  "8 z-layers 10^U[0,1] times a x5 elliptical inclusion; "
                  "q = (eta/2) kappa / geomean(kappa), eta = 10; Gaussian sources sigma = 2/n")


# ---------------------------------------------------------------------------
# Workload 3: 256 independent instances of uneven size.
# ---------------------------------------------------------------------------
BATCH_SIZES = (127, 255, 511, 1023, 2047)


def batched_instances(count: int = 256, sizes: Sequence[int] = BATCH_SIZES):
    """Returns a list of (nr, nz, Medium); each medium has one source."""
    out = []
    for j in range(count):
        rng = _rng(3, j)
        nr = int(rng.choice(sizes))
        nz = int(rng.choice(sizes))
        n_layers = int(rng.integers(2, 9))
        contrast = rng.uniform(1.0, 20.0)
        cuts = np.sort(rng.uniform(0.0, 1.0, size=n_layers - 1))
        values = np.exp(rng.uniform(0.0, np.log(contrast), size=n_layers))
        qv = rng.uniform(0.0, 1.0)
        src = rng.uniform(0.1, 0.9, size=2)
        med = Medium(f"instance{j}", _layers(cuts, values), _const(qv),
                     [_gaussian(src[0], src[1], 0.05)],
                     "layered kappa log-uniform in [1,C], C~U[1,20]; q~U[0,1]; one Gaussian")
        out.append((nr, nz, med))
    return out


# ---------------------------------------------------------------------------
# Workload 4: log-Gaussian random field kappa (training / evaluation seeds).
# ---------------------------------------------------------------------------
def _random_fourier_field(rng: np.random.Generator, corr_len: float, n_feat: int = 256) -> Field:
    """Gaussian random field with squared-exponential covariance
    exp(-|x-y|^2 / (2 l^2)), drawn as a random Fourier feature sum."""
    omega = rng.normal(0.0, 1.0 / corr_len, size=(n_feat, 2))
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n_feat)
    amp = np.sqrt(2.0 / n_feat)

    def g(r, z):
        r = np.asarray(r, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        shape = np.broadcast(r, z).shape
        rf = np.broadcast_to(r, shape).reshape(-1)
        zf = np.broadcast_to(z, shape).reshape(-1)
        out = np.zeros(rf.shape)
        for j0 in range(0, n_feat, 32):
            arg = np.outer(rf, omega[j0:j0 + 32, 0]) + np.outer(zf, omega[j0:j0 + 32, 1]) + phase[j0:j0 + 32]
            out += np.cos(arg).sum(axis=1)
        return (amp * out).reshape(shape)
    g.omega, g.phase, g.amp = omega, phase, amp
    return g


def grf_spec(instance: int, split: str = "train") -> dict:
    """All random draws of one random-field instance: Fourier features
    (omega, phase, amp), the extremes (gmin, gmax) of the field on a fixed 64^2
    reference lattice, the contrast, q and the Gaussian sources
    (r, z, sigma, amplitude).  grf_medium builds its functions from this, and
    bulk evaluators can reproduce the same field from it."""
    rng = _rng(4 if split == "train" else 40, instance)
    g = _random_fourier_field(rng, 0.1)
    rr, zz = _reference_lattice(64)
    gv = g(rr, zz)
    spec = {"omega": g.omega, "phase": g.phase, "amp": g.amp, "gmin": float(gv.min()), "gmax": float(gv.max())}
    spec["contrast"] = float(rng.uniform(1.0, 10.0))
    spec["q"] = float(rng.uniform(0.0, 0.5))
    k = int(rng.integers(1, 5))
    spec["sources"] = [(*rng.uniform(0.1, 0.9, size=2), rng.uniform(0.02, 0.1), rng.uniform(-1.0, 1.0))
                       for _ in range(k)]
    return spec


def grf_medium(instance: int, split: str = "train") -> Medium:
    """kappa = exp(ln(C) * clip((g - gmin) / (gmax - gmin), 0, 1)) for a Gaussian
    random field g (correlation length 0.1), contrast C ~ U[1, 10]; q ~ U[0, 0.5];
    f = 1-4 Gaussians with amplitude U[-1, 1], sigma U[0.02, 0.1].  split
    'train' and 'eval' use disjoint seed streams."""
    spec = grf_spec(instance, split)
    omega, phase, amp = spec["omega"], spec["phase"], spec["amp"]
    gmin, gmax, contrast = spec["gmin"], spec["gmax"], spec["contrast"]

    def g(r, z):
        r = np.asarray(r, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        shape = np.broadcast(r, z).shape
        rf = np.broadcast_to(r, shape).reshape(-1)
        zf = np.broadcast_to(z, shape).reshape(-1)
        out = np.zeros(rf.shape)
        for j0 in range(0, omega.shape[0], 32):
            arg = np.outer(rf, omega[j0:j0 + 32, 0]) + np.outer(zf, omega[j0:j0 + 32, 1]) + phase[j0:j0 + 32]
            out += np.cos(arg).sum(axis=1)
        return (amp * out).reshape(shape)

    def kappa(r, z):
        t = (g(r, z) - gmin) / (gmax - gmin)
        return np.exp(np.log(contrast) * np.clip(t, 0.0, 1.0))

    srcs = [_gaussian(rc, zc, sg, am) for rc, zc, sg, am in spec["sources"]]

    def f(r, z):
        out = np.zeros(np.broadcast(r, z).shape)
        for s in srcs:
            out = out + s(r, z)
        return out

    return Medium(f"grf_{split}{instance}", kappa, _const(spec["q"]), [f],
                  "kappa = exp(GRF, corr 0.1) scaled to contrast U[1,10]; q~U[0,0.5]; 1-4 Gaussians")


# ---------------------------------------------------------------------------
# Workload 5: large layered medium with 4 inclusions, contrast 100.
# ---------------------------------------------------------------------------
def large_spec(instance: int = 0, n_rhs: int = 16, nominal_n: int = 4096, contrast: float = 100.0,
               split: str = "bench") -> dict:
    """All random draws of one large layered medium: the 7 layer cuts in z and
    8 layer values, 4 elliptical inclusions (centre, semi-axes, logistic edge
    width 2/n, log-factor), the extremes (lmin, lmax) of log kappa before
    rescaling on a fixed 512^2 reference lattice, and the Gaussian source
    centres (sigma 2/n).  split 'bench' is the benchmark's seed stream;
    'train' and 'eval' are disjoint streams for the learned guess.
    large_medium builds its functions from this, and bulk evaluators can
    reproduce the same medium from it."""
    rng = _rng({"bench": 5, "train": 50, "eval": 51}[split], instance)
    cuts = np.sort(rng.uniform(0.0, 1.0, size=7))
    values = np.exp(rng.uniform(0.0, np.log(10.0), size=8))
    h = 1.0 / nominal_n
    incs = []
    for _ in range(4):
        rc, zc = rng.uniform(0.15, 0.85, size=2)
        a, b = rng.uniform(0.04, 0.15, size=2)
        incs.append((float(rc), float(zc), float(a), float(b), 2.0 * h, float(rng.uniform(-1.5, 1.5))))
    spec = {"cuts": cuts, "values": values, "incs": incs, "contrast": float(contrast), "q": 0.05, "sigma": 2.0 * h}
    rr, zz = _reference_lattice(512)
    lv = _large_log_raw(spec, rr, zz)
    spec["lmin"], spec["lmax"] = float(lv.min()), float(lv.max())
    spec["centres"] = rng.uniform(0.05, 0.95, size=(n_rhs, 2))
    return spec


def _large_log_raw(spec: dict, r, z):
    out = np.log(_layers(spec["cuts"], spec["values"])(r, z))
    for rc, zc, a, b, width, lf in spec["incs"]:
        out = out + lf * _ellipse_indicator(rc, zc, a, b, width)(r, z)
    return out


def large_medium(n_rhs: int = 16, nominal_n: int = 4096, instance: int = 0,
                 contrast: float = 100.0, split: str = "bench") -> Medium:
    spec = large_spec(instance, n_rhs, nominal_n, contrast, split)
    lmin, lmax = spec["lmin"], spec["lmax"]

    def kappa(r, z):
        t = np.clip((_large_log_raw(spec, r, z) - lmin) / (lmax - lmin), 0.0, 1.0)
        return np.exp(np.log(contrast) * t)

    return Medium("large_layered", kappa, _const(spec["q"]),
                  [_gaussian(c[0], c[1], spec["sigma"]) for c in spec["centres"]],
                  "8 layers + 4 inclusions, contrast 100; q = 0.05; Gaussian sources sigma = 2/n")


# ---------------------------------------------------------------------------
# Manufactured solution (for convergence-order pins).
# ---------------------------------------------------------------------------
def manufactured_medium(q0: float = 1.0, variable_kappa: bool = True):
    """u*(r, z) = cos(pi r / 2) sin(pi z): u*_r = 0 at r = 0, u* = 0 at r = 1 and
    at z = 0, 1.  With kappa = 2 + r^2 cos(pi z) (or 1), f is chosen so that
    (1/r)(r kappa u_r)_r + (kappa u_z)_z - q u = -f holds exactly:
        f = -[kappa (u_rr + u_r / r + u_zz) + kappa_r u_r + kappa_z u_z] + q u.
    Returns (Medium, u_exact)."""
    pi = np.pi

    def u(r, z):
        return np.cos(0.5 * pi * r) * np.sin(pi * z)

    def kappa(r, z):
        if variable_kappa:
            return 2.0 + r * r * np.cos(pi * z)
        return np.ones(np.broadcast(r, z).shape)

    def f(r, z):
        r = np.asarray(r, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        s_r, c_r = np.sin(0.5 * pi * r), np.cos(0.5 * pi * r)
        s_z, c_z = np.sin(pi * z), np.cos(pi * z)
        u_r = -0.5 * pi * s_r * s_z
        u_rr = -0.25 * pi * pi * c_r * s_z
        u_zz = -pi * pi * c_r * s_z
        u_z = pi * c_r * c_z
        # sin(pi r/2)/r is smooth at r = 0 (limit pi/2); r > 0 on every grid used.
        u_r_over_r = -0.5 * pi * (s_r / r) * s_z
        if variable_kappa:
            k = 2.0 + r * r * c_z
            k_r = 2.0 * r * c_z
            k_z = -pi * r * r * s_z
        else:
            k, k_r, k_z = 1.0, 0.0, 0.0
        return -(k * (u_rr + u_r_over_r + u_zz) + k_r * u_r + k_z * u_z) + q0 * c_r * s_z

    med = Medium("manufactured", kappa, _const(q0), [f],
                 "u* = cos(pi r/2) sin(pi z), kappa = 2 + r^2 cos(pi z)")
    return med, u


def manufactured_medium_neumann(q0: float = 1.0, variable_kappa: bool = True):
    """u*(r, z) = cos(pi r / 2) cos(pi z): u*_r = 0 at r = 0, u* = 0 at r = 1 and
    u*_z = 0 at z = 0, 1 (the zero-flux z boundary of Eq. main_eq).  kappa and
    f as in manufactured_medium.  Returns (Medium, u_exact)."""
    pi = np.pi

    def u(r, z):
        return np.cos(0.5 * pi * r) * np.cos(pi * z)

    def kappa(r, z):
        if variable_kappa:
            return 2.0 + r * r * np.cos(pi * z)
        return np.ones(np.broadcast(r, z).shape)

    def f(r, z):
        r = np.asarray(r, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        s_r, c_r = np.sin(0.5 * pi * r), np.cos(0.5 * pi * r)
        s_z, c_z = np.sin(pi * z), np.cos(pi * z)
        u_r = -0.5 * pi * s_r * c_z
        u_rr = -0.25 * pi * pi * c_r * c_z
        u_zz = -pi * pi * c_r * c_z
        u_z = -pi * c_r * s_z
        u_r_over_r = -0.5 * pi * (s_r / r) * c_z
        if variable_kappa:
            k = 2.0 + r * r * c_z
            k_r = 2.0 * r * c_z
            k_z = -pi * r * r * s_z
        else:
            k, k_r, k_z = 1.0, 0.0, 0.0
        return -(k * (u_rr + u_r_over_r + u_zz) + k_r * u_r + k_z * u_z) + q0 * c_r * c_z

    med = Medium("manufactured_neumann", kappa, _const(q0), [f],
                 "u* = cos(pi r/2) cos(pi z), kappa = 2 + r^2 cos(pi z)")
    return med, u


WORKLOADS = {
    "bumps_64": dict(nr=64, nz=64, build=lambda: bumps_medium(), tol=1e-10),
    "layered_1024_m64": dict(nr=1024, nz=1024, build=lambda: layered_inclusion_medium(64, 1024), tol=1e-8),
    "large_4096_m16": dict(nr=4096, nz=4096, build=lambda: large_medium(16, 4096), tol=1e-8),
}
