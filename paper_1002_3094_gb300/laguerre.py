"""Driver of the Laguerre-harmonic chain (Section 4.1, Eq. laguerre_h): n
sequential solves on one operator, each harmonic's right-hand side formed on
the GPU by ax_laguerre_step from two running fields, each solve started from
the previous harmonic (kept only where it lowers the initial residual).  The
weights are host scalars; every field operation runs in libaxpcg."""
from __future__ import annotations

import math
from typing import Callable, Optional, Sequence

from . import (AX_FLAG_CHECK_GUESS, AX_FLAG_USE_GUESS, AX_OK, AX_PCG_MIXED, AxError, ax_laguerre_step,
               ax_solve)


def laguerre_weights(m: int, alpha: int):
    """(a_m, w_m) = (sqrt(m! / (m + alpha)!), sqrt((m + alpha)! / m!))."""
    lg = math.lgamma(m + alpha + 1) - math.lgamma(m + 1)
    return math.exp(-0.5 * lg), math.exp(0.5 * lg)


def solve_chain(op, c2, src, fm: Sequence[float], alpha: int, tol: float, q_out, work,
                method: int = AX_PCG_MIXED, max_iter: int = 20000, warm: bool = True,
                on_harmonic: Optional[Callable] = None, stream=None):
    """Harmonics 0 .. len(fm) - 1.  c2 = h^2 / rho^2 and src are dense FP64
    device tensors [nr][nz]; q_out [1][nr][nz] receives each harmonic in turn
    (and holds the last one at the end); work is a device tensor [3][nr][nz]
    for the running fields T, S and the right-hand side (zeroed here).
    on_harmonic(m, q_out, info) is called after every solve.  Returns the
    per-harmonic solve infos."""
    work.zero_()
    T, S, f = work[0], work[1], work[2]
    q_out.zero_()
    infos = []
    # harmonic 0: T = S = 0 and no solved field yet, so the step writes f = f_0 src
    ax_laguerre_step(op, None, T, S, c2, src, 0.0, laguerre_weights(0, alpha)[0], float(fm[0]), f, stream)
    for m in range(len(fm)):
        flags = (AX_FLAG_USE_GUESS | AX_FLAG_CHECK_GUESS) if (warm and m > 0) else 0
        st, info = ax_solve(op, f.unsqueeze(0), q_out, 1, tol, max_iter, method, flags, stream=stream,
                            raise_on_error=False)
        if st != AX_OK:
            raise AxError(st, f"ax_solve (harmonic {m})")
        infos.append(info[0])
        if on_harmonic is not None:
            on_harmonic(m, q_out, info[0])
        if m + 1 < len(fm):
            ax_laguerre_step(op, q_out[0], T, S, c2, src, laguerre_weights(m, alpha)[1],
                             laguerre_weights(m + 1, alpha)[0], float(fm[m + 1]), f, stream)
    return infos
