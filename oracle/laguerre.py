"""FP64 oracle of the Laguerre-harmonic chain (Section 4.1).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline, never by the library.

The time-domain wave equation is expanded in the orthonormal Laguerre
functions of Eq. series_lag,

    Q_m(x) = int_0^inf u(x, t) (h t)^(-alpha/2) l_m^alpha(h t) dt,
    l_m^alpha(y) = sqrt(h m! / (m + alpha)!) y^(alpha/2) exp(-y/2) L_m^alpha(y),

and the second time derivative becomes (for a field at rest at t = 0)

    [u_tt]_m = (h^2 / 4) Q_m + h^2 a_m sum_{k<m} (m - k) w_k Q_k,
    a_m = sqrt(m! / (m + alpha)!),   w_k = sqrt((k + alpha)! / k!),

which gives Eq. laguerre_h: harmonic m solves the operator of the solver with
kappa = V, q = h^2 / (4 rho^2) and the physical right-hand side
f_m src - (h^2 / rho^2) a_m sum_{k<m} (m - k) w_k Q_k.  This module writes
the sum out directly (O(m) fields per harmonic): the library carries it in two
running fields instead.
"""
from __future__ import annotations

import math
from typing import Callable, List, Sequence

import numpy as np


def weights(m: int, alpha: int):
    """(a_m, w_m) = (sqrt(m! / (m + alpha)!), sqrt((m + alpha)! / m!)) via log-gamma."""
    lg = math.lgamma(m + alpha + 1) - math.lgamma(m + 1)
    return math.exp(-0.5 * lg), math.exp(0.5 * lg)


def laguerre_function(m: int, alpha: int, y):
    """l_m^alpha(y) / sqrt(h): sqrt(m! / (m + alpha)!) y^(alpha/2) exp(-y/2) L_m^alpha(y)
    by the three-term recurrence of the generalised Laguerre polynomials
    (L_{k+1} = ((2k + 1 + alpha - y) L_k - (k + alpha) L_{k-1}) / (k + 1)),
    normalised at every step so that nothing overflows."""
    y = np.asarray(y, dtype=np.float64)
    # psi_k = sqrt(k! / (k + alpha)!) exp(-y/2) L_k(y)
    prev = np.zeros_like(y)
    cur = np.exp(-0.5 * y - 0.5 * math.lgamma(alpha + 1))
    for k in range(m):
        nxt = ((2 * k + 1 + alpha - y) * cur * math.sqrt((k + 1) / (k + 1 + alpha))
               - (k + alpha) * prev * math.sqrt((k + 1) * k / ((k + 1 + alpha) * (k + alpha)))) / (k + 1)
        prev, cur = cur, nxt
    return cur * y ** (alpha / 2)


def second_derivative_coefficients(Q: Sequence, h: float, alpha: int) -> List:
    """[u_tt]_m for m < len(Q) from the coefficients Q_k of u (Eq. laguerre_h's
    left-hand time term), the sum written out."""
    out = []
    for m in range(len(Q)):
        a_m, _ = weights(m, alpha)
        acc = 0.0 * Q[0]
        for k in range(m):
            acc = acc + (m - k) * weights(k, alpha)[1] * Q[k]
        out.append(h * h / 4.0 * Q[m] + h * h * a_m * acc)
    return out


def harmonic_rhs(m: int, Q: Sequence[np.ndarray], c2, src, f_m: float, alpha: int) -> np.ndarray:
    """Physical right-hand side of harmonic m (Eq. laguerre_h, the solver's sign
    convention div(kappa grad u) - q u = -f):
    f_m src - c2 a_m sum_{k<m} (m - k) w_k Q_k."""
    a_m, _ = weights(m, alpha)
    acc = np.zeros_like(src, dtype=np.float64)
    for k in range(m):
        acc = acc + (m - k) * weights(k, alpha)[1] * Q[k]
    return f_m * src - c2 * a_m * acc


def chain(solve: Callable, c2, src, fm: Sequence[float], alpha: int) -> List[np.ndarray]:
    """Q_0 .. Q_{n-1}: harmonic m solved by solve(rhs, previous Q or None) with
    the right-hand side built from all earlier harmonics."""
    Q: List[np.ndarray] = []
    for m in range(len(fm)):
        rhs = harmonic_rhs(m, Q, c2, src, fm[m], alpha)
        Q.append(solve(rhs, Q[-1] if Q else None))
    return Q
