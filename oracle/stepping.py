"""O1: the exact solution of A u = b by sequential time stepping.

A = B1 (x) I + B2 (x) K with lower-triangular banded Toeplitz B1, B2 (eq. 1.1,
eq. 2.5b, eq. 3.2b) is block lower triangular, so block forward substitution
in time is the classical time-stepping method that ParaDiag parallelises:

  (c1[0] I + c2[0] K) U_n = b_n - sum_{m>=1} (c1[m] U_{n-m} + c2[m] K U_{n-m}).

For the theta-method this is eq. 2.4 with uniform steps; for leap-frog it is
the two-step recurrence of eq. 3.2b.  The step matrix is factored once with a
sparse LU with partial pivoting (SuperLU), the library primitive used as the
spatial solve.  The adjoint A^T lambda = g is block upper triangular and is
solved by backward substitution in time.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from workloads import Problem

from .operators import first_columns, stencil


def solve_sequential(problem: Problem, b: np.ndarray, K=None) -> np.ndarray:
    """u = A^{-1} b by forward substitution in time; b, u of shape (Nt, S)."""
    K = stencil(problem.space) if K is None else K
    c1, c2 = first_columns(problem)
    nt, S = b.shape
    band = [m for m in range(1, nt) if c1[m] != 0.0 or c2[m] != 0.0]
    step = (c1[0] * sps.identity(S) + c2[0] * K).tocsc()
    lu = spla.splu(step)
    U = np.zeros((nt, S))
    for n in range(nt):
        rhs = np.array(b[n], dtype=np.float64)
        for m in band:
            if n - m >= 0:
                rhs -= c1[m] * U[n - m] + c2[m] * (K @ U[n - m])
        U[n] = lu.solve(rhs)
    return U


def solve_adjoint_sequential(problem: Problem, g: np.ndarray, K=None) -> np.ndarray:
    """lambda = A^{-T} g by backward substitution in time:

    (c1[0] I + c2[0] K^T) L_n = g_n - sum_{m>=1} (c1[m] L_{n+m} + c2[m] K^T L_{n+m}).
    """
    K = stencil(problem.space) if K is None else K
    KT = K.T.tocsr()
    c1, c2 = first_columns(problem)
    nt, S = g.shape
    band = [m for m in range(1, nt) if c1[m] != 0.0 or c2[m] != 0.0]
    step = (c1[0] * sps.identity(S) + c2[0] * KT).tocsc()
    lu = spla.splu(step)
    L = np.zeros((nt, S))
    for n in range(nt - 1, -1, -1):
        rhs = np.array(g[n], dtype=np.float64)
        for m in band:
            if n + m < nt:
                rhs -= c1[m] * L[n + m] + c2[m] * (KT @ L[n + m])
        L[n] = lu.solve(rhs)
    return L
