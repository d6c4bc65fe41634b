"""O10: nonlinear problems by simplified Newton with an averaged Jacobian
(Section 1, eq. 1.4 and eq. 1.5).

Problems U' + K U + phi(U) = f with U(0) = U_0 and the pointwise reaction
term phi(u) = a1 u + a2 u^2 + a3 u^3 (coefficients a = (a1, a2, a3)).  With the
theta-method the all-at-once system (eq. 1.4 with M = I and f(U) = K U + phi(U))
is

    (B1 (x) I) u + (B2 (x) I) F(u) = b,   F(u)_n = K U_n + phi(U_n),

B1, B2 the Toeplitz matrices of the linear case, and b the linear right-hand
side with the first row also carrying -(1-theta) phi(U_0) (reading R25).

The simplified Newton iteration of eq. 1.5 replaces the Jacobian
B1 (x) I + (B2 (x) I) blkdiag(K + diag phi'(U_n)) by the alpha-circulant
P_alpha(u) = C1 (x) I + C2 (x) (K + sigma I), where the averaged Jacobian is
K + sigma I with sigma the mean of phi'(U_n(x)) over all time levels and grid
points (reading R25: the section leaves the averaging open and names time
averages; averaging over space as well keeps K + sigma I diagonalisable by the
spatial transforms, so step (b) of eq. 1.3 is unchanged up to a shift).  Each
step: r = b - (B1 (x) I) u - (B2 (x) I) F(u), du = P_alpha(u)^{-1} r, u += du.

The exact discrete solution (the fixed point) is sequential theta-stepping
with a full Newton solve of every step.
Test infrastructure only; shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from workloads import LEAPFROG, Problem

from .operators import build_rhs, first_columns, stencil
from .paradiag import Preconditioner


def reaction(u, a):
    """phi(u) = a1 u + a2 u^2 + a3 u^3."""
    a1, a2, a3 = a
    return u * (a1 + u * (a2 + u * a3))


def reaction_prime(u, a):
    """phi'(u) = a1 + 2 a2 u + 3 a3 u^2."""
    a1, a2, a3 = a
    return a1 + u * (2.0 * a2 + 3.0 * a3 * u)


def _check(problem: Problem):
    if problem.scheme == LEAPFROG:
        raise ValueError("the nonlinear form is stated for first-order (theta-method) problems")


def build_rhs_nl(problem: Problem, u0, a, f=None, K=None) -> np.ndarray:
    """b of eq. 1.4: the linear right-hand side (f at t_0..t_Nt) with
    -(1-theta) phi(U_0) added to the first row."""
    _check(problem)
    b = build_rhs(problem, u0, f=f, K=K)
    th = problem.theta_eff
    b[0] -= (1.0 - th) * reaction(np.asarray(u0, dtype=np.float64), a)
    return b


def residual_nl(problem: Problem, U: np.ndarray, b: np.ndarray, a, K=None) -> np.ndarray:
    """r = b - (B1 (x) I) u - (B2 (x) I) F(u) with F(u)_n = K U_n + phi(U_n):
    row n = b_n - sum_m c1[m] U_{n-m} - sum_m c2[m] F_{n-m} over n - m >= 0."""
    _check(problem)
    K = stencil(problem.space) if K is None else K
    U = np.asarray(U, dtype=np.float64)
    c1, c2 = first_columns(problem)
    F = (K @ U.T).T + reaction(U, a)
    r = np.array(b, dtype=np.float64, copy=True)
    for n in range(problem.nt):
        for m in range(min(2, n + 1)):
            r[n] -= c1[m] * U[n - m] + c2[m] * F[n - m]
    return r


def average_jacobian_shift(U: np.ndarray, a) -> float:
    """sigma = mean of phi'(U_n(x)) over all time levels and grid points."""
    return float(np.mean(reaction_prime(np.asarray(U, dtype=np.float64), a)))


def solve_sequential_nl(problem: Problem, b: np.ndarray, a, K=None, newton_tol=1e-14,
                        newton_maxit=50) -> np.ndarray:
    """The exact solution of eq. 1.4: step n solves
    U_n / dt + theta (K U_n + phi(U_n)) = b_n + U_{n-1} / dt - (1-theta) F(U_{n-1})
    by Newton's method with the sparse Jacobian I / dt + theta (K + diag phi'(U_n))
    (U_{-1} terms are in b_0)."""
    _check(problem)
    K = stencil(problem.space) if K is None else K
    nt, S, dt = problem.nt, problem.space.size, problem.dt
    th = problem.theta_eff
    I = sps.identity(S, format="csr")
    U = np.zeros((nt, S))
    prev = np.zeros(S)
    for n in range(nt):
        rhs = np.array(b[n], dtype=np.float64, copy=True)
        if n > 0:
            rhs += prev / dt - (1.0 - th) * (K @ prev + reaction(prev, a))
        x = prev.copy()
        for _ in range(newton_maxit):
            g = x / dt + th * (K @ x + reaction(x, a)) - rhs
            J = (I / dt + th * (K + sps.diags(reaction_prime(x, a)))).tocsc()
            dx = spla.spsolve(J, g)
            x -= dx
            if np.linalg.norm(dx) <= newton_tol * max(1.0, np.linalg.norm(x)):
                break
        U[n] = x
        prev = x
    return U


def simplified_newton(problem: Problem, b: np.ndarray, a, u_init=None, tol=1e-12, maxit=60,
                      K=None):
    """Eq. 1.5 with P_alpha(u^{k-1}) = C1 (x) I + C2 (x) (K + sigma(u^{k-1}) I),
    each correction by the three steps of eq. 1.3 (O2 with the shifted K).
    Returns (u, iterations, relative residual norms, one per residual formed)."""
    _check(problem)
    K = stencil(problem.space) if K is None else K
    U = np.zeros((problem.nt, problem.space.size)) if u_init is None else \
        np.array(u_init, dtype=np.float64, copy=True)
    nb = np.linalg.norm(b)
    hist = []
    it = 0
    while True:
        r = residual_nl(problem, U, b, a, K)
        rel = np.linalg.norm(r) / nb if nb > 0 else np.linalg.norm(r)
        hist.append(rel)
        if rel <= tol or it >= maxit:
            break
        sigma = average_jacobian_shift(U, a)
        Ks = (K + sigma * sps.identity(K.shape[0])).tocsr()
        U = U + Preconditioner(problem, Ks).apply(r)
        it += 1
    return U, it, hist
