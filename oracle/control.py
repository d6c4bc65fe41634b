"""O5: heat-source inversion functional and its adjoint gradient.

For the backward-Euler all-at-once system A u = b(f) with zero initial value
and a time-independent source f, every row of b is f (eq. 2.4 with theta = 1
and f(t_n) = f), so b = (1_Nt (x) I) f.  The functional

    J(f) = 1/2 ||U_Nt - u_target||^2 + reg/2 ||f||^2        (plain Euclidean sums)

has the gradient dJ/df = sum_n lambda_n + reg f, where A^T lambda = e_Nt (x)
(U_Nt - u_target) (the transposed all-at-once solve: backward in time).
"""
from __future__ import annotations

import numpy as np

from workloads import Problem

from .operators import build_rhs, stencil
from .stepping import solve_adjoint_sequential, solve_sequential


def source_rhs(problem: Problem, f_space: np.ndarray, u0=None, K=None) -> np.ndarray:
    nt, S = problem.nt, problem.space.size
    u0 = np.zeros(S) if u0 is None else u0
    F = np.broadcast_to(np.asarray(f_space, dtype=np.float64), (nt + 1, S))
    return build_rhs(problem, u0, None, F, K)


def objective(problem: Problem, f_space, u_target, reg, K=None) -> float:
    K = stencil(problem.space) if K is None else K
    U = solve_sequential(problem, source_rhs(problem, f_space, K=K), K)
    e = U[-1] - u_target
    return 0.5 * float(e @ e) + 0.5 * reg * float(np.dot(f_space, f_space))


def gradient(problem: Problem, f_space, u_target, reg, K=None):
    """(J, dJ/df, U, lambda) with lambda from sequential backward stepping."""
    K = stencil(problem.space) if K is None else K
    U = solve_sequential(problem, source_rhs(problem, f_space, K=K), K)
    e = U[-1] - u_target
    g = np.zeros_like(U)
    g[-1] = e
    L = solve_adjoint_sequential(problem, g, K)
    J = 0.5 * float(e @ e) + 0.5 * reg * float(np.dot(f_space, f_space))
    return J, L.sum(axis=0) + reg * np.asarray(f_space), U, L
