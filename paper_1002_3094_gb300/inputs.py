"""Host-side preparation of the library's inputs from a medium description.

The library takes kappa point-sampled at cell faces and q at nodes
(Section 2.1, Eq. diff_approx1).  This module computes those sample points
for the grid of ``include/axpcg.h`` (r_i = (i - 1/2) h_r, h_r = lr/(nr + 1/2),
faces rbar_i = i h_r; z-boundary bc_z = 0: z_k = k h_z, h_z = lz/(nz + 1),
faces zbar_k = (k + 1/2) h_z; bc_z = 1: z_k = (k - 1/2) h_z, h_z = lz/nz,
faces zbar_k = k h_z) and evaluates the medium there.  No solver arithmetic
happens here.
"""
from __future__ import annotations

import numpy as np


def sample_points(nr: int, nz: int, lr: float = 1.0, lz: float = 1.0, bc_z: int = 0):
    hr = lr / (nr + 0.5)
    r_nodes = (np.arange(nr) + 0.5) * hr          # r_1 .. r_nr
    r_faces = (np.arange(nr) + 1.0) * hr          # rbar_1 .. rbar_nr
    if bc_z == 1:
        hz = lz / nz
        z_nodes = (np.arange(nz) + 0.5) * hz      # z_1 .. z_nz, cell centres
        z_faces = np.arange(nz + 1) * hz          # zbar_0 = 0 .. zbar_nz = lz
    else:
        hz = lz / (nz + 1.0)
        z_nodes = (np.arange(nz) + 1.0) * hz      # z_1 .. z_nz
        z_faces = (np.arange(nz + 1) + 0.5) * hz  # zbar_0 .. zbar_nz
    return r_nodes, r_faces, z_nodes, z_faces


def sample_operator_inputs(medium, nr: int, nz: int, lr: float = 1.0, lz: float = 1.0, bc_z: int = 0):
    """(kappa_r [nr][nz], kappa_z [nr][nz+1], q [nr][nz]) as FP64 numpy arrays."""
    rn, rf, zn, zf = sample_points(nr, nz, lr, lz, bc_z)
    kappa_r = medium.kappa(rf[:, None], zn[None, :])
    kappa_z = medium.kappa(rn[:, None], zf[None, :])
    q = medium.q(rn[:, None], zn[None, :])
    return (np.ascontiguousarray(kappa_r, dtype=np.float64), np.ascontiguousarray(kappa_z, dtype=np.float64),
            np.ascontiguousarray(q, dtype=np.float64))


def sample_rhs(medium, nr: int, nz: int, lr: float = 1.0, lz: float = 1.0, which=None, bc_z: int = 0):
    """f_m(r_i, z_k) as an FP64 array [M][nr][nz]."""
    rn, _, zn, _ = sample_points(nr, nz, lr, lz, bc_z)
    idx = range(medium.n_rhs) if which is None else which
    return np.ascontiguousarray(np.stack([medium.f(rn[:, None], zn[None, :], m) for m in idx]),
                                dtype=np.float64)
