"""Exact solution of A x = b by sparse LU (oracle side).

TEST INFRASTRUCTURE ONLY: imported by tests/ and by oracle/record_aniso_reference.py,
never by the product library.

GMRES (Algorithm 1) and GMRES-IR (Algorithm 2) approximate x = A^{-1} b; the plain
definition of that target is the linear solve itself.  Here it is computed with a library
primitive: SuperLU (scipy.sparse.linalg.splu) with partial pivoting and a minimum-degree
ordering of A + A^T, in FP64.  The result carries only the direct solve's rounding error
(backward stable), so a GMRES solution's error against it is the error against the true
solution to within kappa(A) * u.

Pins (tests/test_oracle_direct.py): dense numpy.linalg.solve on small nonsymmetric systems,
a manufactured solution on a convection-diffusion stencil, and a permuted-identity case.
"""
from __future__ import annotations

import numpy as np


def direct_solve(A, b: np.ndarray) -> np.ndarray:
    """x = A^{-1} b for a CSR matrix A (attributes n, row_ptr, col_idx, vals)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    M = sp.csr_matrix((A.vals, A.col_idx, A.row_ptr), shape=(A.n, A.n)).tocsc()
    lu = sla.splu(M, permc_spec="MMD_AT_PLUS_A")
    return lu.solve(np.asarray(b, dtype=np.float64))
