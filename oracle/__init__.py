"""Plain FP64 CPU oracle for the Laplace-preconditioned CG / Chebyshev solver.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library and
its Python binding never import it and share no code with it.

Every function follows one passage of the paper (Terekhov, "High performance
parallel algorithm for solving elliptic equations with non-separable
variables", arXiv 1002.3094); the docstrings name the section and equation.
All functions are pinned by ``tests/test_oracle.py`` (and the Laguerre chain of
``laguerre.py`` by ``tests/test_oracle_laguerre.py``) against closed forms,
library routines, brute force on tiny grids and a manufactured solution.
"""
from . import laguerre  # noqa: F401
from .axisym import (  # noqa: F401
    Grid,
    sample_medium,
    scheme_coefficients,
    rhs_phi,
    assemble,
    preconditioner_constants,
    dst1_matrix,
    cosine_pair,
    z_transforms,
    mode_eigenvalues,
    mode_tridiagonal,
    thomas,
    precond_solve,
    assemble_preconditioner,
    pcg,
    chebyshev_bounds,
    lanczos_bounds,
    chebyshev,
    Operator,
)
