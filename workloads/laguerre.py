"""Seeded inputs of the Laguerre-harmonic chain (Section 4.1): a layered
velocity model cut by an inclined fault (a stand-in for the paper's
"geological fault" model, which it gives only as a figure), constant density
rho = 1, a point source at the origin approximated by a normalised Gaussian,
and the Laguerre coefficients f_m of the source wavelet of Eq. functiont with
the paper's parameters (f_0 = 30 Hz, t_0 = 0.2 s, gamma = 4; alpha = 5,
h = 300).  Inputs only: nothing here is the solver's arithmetic.

Reading: Eq. laguerre_h's coefficient V (named the wave speed in the text) is
taken as the squared speed v^2, which makes it the coefficient of the
acoustic equation u_tt = div(v^2 grad u) + f for rho = 1; q = h^2 / (4 rho^2).
"""
from __future__ import annotations

import math

import numpy as np

from .media import Medium, _rng

ALPHA = 5
H_LAG = 300.0
F0, T0, GAMMA = 30.0, 0.2, 4.0


def fault_medium(lr: float = 2048.0, lz: float = 2048.0, instance: int = 0, h: float = H_LAG,
                 sigma: float = 4.0) -> Medium:
    """kappa = v(r, z)^2 for four layers (1500 .. 3500 m/s) whose interfaces
    drop by a throw of 8-15% of lz beyond an inclined fault plane; q = h^2/4;
    one source: a Gaussian of width `sigma` metres at the origin, normalised
    to unit integral over the half space z >= 0 with the axisymmetric volume
    element 2 pi r dr dz."""
    rng = _rng(41, instance)
    depths = np.sort(rng.uniform(0.15, 0.85, size=3)) * lz
    speeds = np.sort(rng.uniform(1500.0, 3500.0, size=4))
    r_fault, dip = rng.uniform(0.35, 0.65) * lr, math.radians(rng.uniform(55.0, 75.0))
    throw = rng.uniform(0.08, 0.15) * lz

    def kappa(r, z):
        r, z = np.broadcast_arrays(np.asarray(r, dtype=np.float64), np.asarray(z, dtype=np.float64))
        beyond = r > r_fault + z / math.tan(dip)  # hanging wall: interfaces shifted down
        zz = np.where(beyond, z - throw, z)
        layer = np.searchsorted(depths, zz, side="right")
        return speeds[layer] ** 2

    def q(r, z):
        return np.full(np.broadcast(r, z).shape, h * h / 4.0)

    norm = 1.0 / (2.0 * math.pi * sigma ** 3 * math.sqrt(math.pi / 2.0))

    def src(r, z):
        return norm * np.exp(-(np.asarray(r) ** 2 + np.asarray(z) ** 2) / (2.0 * sigma * sigma))

    return Medium("laguerre_fault", kappa, q, [src],
                  "four layers 1500-3500 m/s with an inclined fault; point source at the origin")


def source_wavelet(t):
    """Eq. functiont: exp(-(2 pi f0 (t - t0))^2 / gamma^2) sin(2 pi f0 (t - t0))."""
    s = 2.0 * math.pi * F0 * (np.asarray(t) - T0)
    return np.exp(-(s * s) / (GAMMA * GAMMA)) * np.sin(s)


def wavelet_coefficients(n: int, alpha: int = ALPHA, h: float = H_LAG, t_max: float = 0.5,
                         nt: int = 50001) -> np.ndarray:
    """f_m = int_0^inf f(t) (h t)^(-alpha/2) l_m^alpha(h t) dt, m < n (Eq.
    series_lag applied to the wavelet), by the trapezoid rule on [0, t_max]
    (the wavelet is below 1e-30 outside [0, 0.4] s), with the normalised
    functions sqrt(m! / (m + alpha)!) exp(-y/2) L_m^alpha(y) advanced by the
    three-term recurrence of the Laguerre polynomials."""
    t = np.linspace(0.0, t_max, nt)
    y = h * t
    w = source_wavelet(t) * math.sqrt(h) * (t[1] - t[0])
    w[0] *= 0.5
    w[-1] *= 0.5
    prev = np.zeros_like(y)
    cur = np.exp(-0.5 * y - 0.5 * math.lgamma(alpha + 1))
    out = np.empty(n)
    for k in range(n):
        out[k] = float(np.dot(w, cur))
        nxt = ((2 * k + 1 + alpha - y) * cur * math.sqrt((k + 1) / (k + 1 + alpha))
               - (k + alpha) * prev * math.sqrt((k + 1) * k / ((k + 1 + alpha) * (k + alpha)))) / (k + 1)
        prev, cur = cur, nxt
    return out
