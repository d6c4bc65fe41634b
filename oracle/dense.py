"""O3: dense Kronecker forms of A and P_alpha for tiny problems (Nx*Nt small).

A = B1 (x) I + B2 (x) K (eq. 1.1) and P_alpha = C1 (x) I + C2 (x) K (eq. 1.2)
are formed explicitly with numpy.kron and solved with LAPACK's dense LU with
partial pivoting.  Nothing here uses the diagonalisation of Lemma 1.
"""
from __future__ import annotations

import numpy as np

from workloads import Problem

from .operators import circulant_matrices, stencil, time_matrices


def dense_A(problem: Problem) -> np.ndarray:
    K = stencil(problem.space).toarray()
    B1, B2 = time_matrices(problem)
    return np.kron(B1, np.eye(K.shape[0])) + np.kron(B2, K)


def dense_P(problem: Problem) -> np.ndarray:
    K = stencil(problem.space).toarray()
    C1, C2 = circulant_matrices(problem)
    return np.kron(C1, np.eye(K.shape[0])) + np.kron(C2, K)


def solve_dense(M: np.ndarray, r: np.ndarray) -> np.ndarray:
    """M^{-1} r for a time-major r of shape (Nt, S)."""
    return np.linalg.solve(M, r.reshape(-1)).reshape(r.shape)


def iteration_matrix_spectrum(problem: Problem) -> np.ndarray:
    """Eigenvalues of I - P_alpha^{-1} A (the error propagator of eq. 5.1)."""
    A = dense_A(problem)
    P = dense_P(problem)
    return np.linalg.eigvals(np.eye(A.shape[0]) - np.linalg.solve(P, A))


def preconditioned_spectrum(problem: Problem) -> np.ndarray:
    """Eigenvalues of P_alpha^{-1} A (Theorem 3.1 for leap-frog)."""
    A = dense_A(problem)
    P = dense_P(problem)
    return np.linalg.eigvals(np.linalg.solve(P, A))
