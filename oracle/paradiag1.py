"""O6: ParaDiag-I with geometrically increasing time steps (Section 2.1.1).

The direct (non-iterative) member of the family: with the step sizes of
eq. 2.8, dt_n = dt_Nt tau^(n - Nt), the theta-method all-at-once system
(eq. 2.5a/2.5b)

    (B1 (x) I + B2 (x) K) u = b,   B1 = lower bidiagonal with 1/dt_n on the
    diagonal and -1/dt_n below it, B2 = lower bidiagonal with theta and 1-theta,

is multiplied by B2^{-1} (x) I to give (B (x) I + I (x) K) u = b~ (eq. 2.6),
B = B2^{-1} B1.  The theorem of Section 2.1.1 diagonalises B = V D V^{-1} with
D = diag(1/(theta dt_n)) and V, V^{-1} unit lower-triangular Toeplitz matrices
whose sub-diagonals are p_n and q_n in closed form.  The solve is then the
three steps of eq. 2.7:

    (a) S1 = (V^{-1} (x) I) b~,
    (b) S2_n = (1/(theta dt_n) I + K)^{-1} S1_n,  n = 1..Nt,
    (c) u = (V (x) I) S2.

Any column scaling V D~ is an eigenvector matrix as well; the section names
D~ = diag((1 + sum_{j <= Nt-n} |p_j|^2)^{-1/2}) (unit-norm columns of V).

Readings (the printed theorem is garbled for theta = 1/2):
  * q_n for theta = 1/2 is printed with a factor "q^{-n}"; it is read as
    tau^{-n}: q_n = tau^{-n} prod_{j<=n} (1 + tau^{2-j}) / (1 - tau^{-j}).  The
    reading is the one that makes V V^{-1} = I, which the tests check in exact
    rational arithmetic.
  * The source term enters as b_n = theta f(t_n) + (1-theta) f(t_{n-1}), with
    (I/dt_1 - (1-theta) K) U_0 added to row 1 (the right-hand side printed
    after eq. 2.5b for f = 0).

Layout as in ``operators``: U[n][s] of shape (Nt, S), row n standing for t_{n+1}.
Test infrastructure only; shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from workloads import BE, CN, GeometricProblem

from .operators import stencil


def theta_of(scheme: int) -> float:
    """theta of eq. 2.4: 1 for backward Euler, 1/2 for the trapezoidal rule."""
    if scheme == BE:
        return 1.0
    if scheme == CN:
        return 0.5
    raise ValueError("ParaDiag-I is stated for theta = 1 and theta = 1/2")


def geometric_steps(nt: int, dt_last: float, tau: float) -> np.ndarray:
    """dt_n = dt_Nt tau^(n - Nt), n = 1..Nt (eq. 2.8); entry n-1 holds dt_n."""
    n = np.arange(1, nt + 1, dtype=np.float64)
    return dt_last * tau ** (n - nt)


def time_matrices(dts: np.ndarray, theta: float):
    """B1, B2 of eq. 2.5b for the steps dts (dense Nt x Nt)."""
    nt = len(dts)
    B1 = np.zeros((nt, nt))
    B2 = np.zeros((nt, nt))
    for n in range(nt):
        B1[n, n] = 1.0 / dts[n]
        B2[n, n] = theta
        if n > 0:
            B1[n, n - 1] = -1.0 / dts[n]
            B2[n, n - 1] = 1.0 - theta
    return B1, B2


def eigvec_coeffs(nt: int, tau, theta):
    """p_0..p_{Nt-1} and q_0..q_{Nt-1} (p_0 = q_0 = 1) of the theorem of
    Section 2.1.1, for theta = 1 and theta = 1/2 (q for theta = 1/2 as read in
    the module header).  Plain loops, so that ``tau`` and ``theta`` may also be
    exact rationals (fractions.Fraction); floats give float64 arrays."""
    one = tau ** 0
    p = [one] * nt
    q = [one] * nt
    for n in range(1, nt):
        if theta == 1:
            den = one
            for j in range(1, n + 1):
                den = den * (1 - tau**j)
            p[n] = one / den
            q[n] = (-1) ** n * tau ** (n * (n - 1) // 2) * p[n]
        elif theta * 2 == 1:
            pn, qn = one, tau ** (-n)
            for j in range(1, n + 1):
                pn = pn * (1 + tau**j) / (1 - tau**j)
                qn = qn * (1 + tau ** (2 - j)) / (1 - tau ** (-j))
            p[n], q[n] = pn, qn
        else:
            raise ValueError("closed forms are stated for theta = 1 and theta = 1/2")
    if isinstance(tau, float):
        return np.array(p, dtype=np.float64), np.array(q, dtype=np.float64)
    return p, q


def toeplitz_lower(c: np.ndarray) -> np.ndarray:
    nt = len(c)
    T = np.zeros((nt, nt))
    for i in range(nt):
        T[i, : i + 1] = c[i::-1]
    return T


def column_scaling(p: np.ndarray) -> np.ndarray:
    """Diagonal of D~: (1 + sum_{j=1}^{Nt-n} |p_j|^2)^{-1/2}, n = 1..Nt."""
    nt = len(p)
    return np.array([(1.0 + np.sum(np.abs(p[1 : nt - n + 1]) ** 2)) ** -0.5
                     for n in range(1, nt + 1)])


def eigvec_matrices(nt: int, tau: float, theta: float, scaled: bool):
    """(V, V^{-1}); V -> V D~ and V^{-1} -> D~^{-1} V^{-1} when scaled."""
    p, q = eigvec_coeffs(nt, tau, theta)
    V = toeplitz_lower(p)
    Vi = toeplitz_lower(q)
    if scaled:
        dsc = column_scaling(p)
        V = V * dsc[None, :]
        Vi = Vi / dsc[:, None]
    return V, Vi


def eigenvalues(dts: np.ndarray, theta: float) -> np.ndarray:
    """Diagonal of D: 1/(theta dt_n)."""
    return 1.0 / (theta * dts)


def build_rhs(problem: GeometricProblem, u0, f=None, K=None) -> np.ndarray:
    """b of eq. 2.5a, shape (Nt, S); f of shape (Nt+1, S) at t_0..t_Nt or None."""
    sp = problem.space
    K = stencil(sp) if K is None else K
    th = theta_of(problem.scheme)
    dts = geometric_steps(problem.nt, problem.dt_last, problem.tau)
    nt, S = problem.nt, sp.size
    F = np.zeros((nt + 1, S)) if f is None else np.asarray(f, dtype=np.float64)
    b = np.zeros((nt, S))
    for n in range(nt):
        b[n] = th * F[n + 1] + (1.0 - th) * F[n]
    u0 = np.asarray(u0, dtype=np.float64)
    b[0] += u0 / dts[0] - (1.0 - th) * (K @ u0)
    return b


def apply_A(problem: GeometricProblem, U: np.ndarray, K=None) -> np.ndarray:
    """(B1 (x) I + B2 (x) K) u for u laid out as U[n][s]."""
    K = stencil(problem.space) if K is None else K
    th = theta_of(problem.scheme)
    B1, B2 = time_matrices(geometric_steps(problem.nt, problem.dt_last, problem.tau), th)
    KU = (K @ np.asarray(U).T).T
    return B1 @ U + B2 @ KU


def solve_sequential(problem: GeometricProblem, b: np.ndarray, K=None) -> np.ndarray:
    """Exact solution of eq. 2.5a by block forward substitution in time (the
    variable-step theta-method eq. 2.4 run step by step)."""
    K = stencil(problem.space) if K is None else K
    th = theta_of(problem.scheme)
    dts = geometric_steps(problem.nt, problem.dt_last, problem.tau)
    B1, B2 = time_matrices(dts, th)
    nt, S = b.shape
    I = sps.identity(S, format="csr")
    U = np.zeros((nt, S))
    for n in range(nt):
        rhs = np.array(b[n], dtype=np.float64)
        if n > 0:
            rhs -= B1[n, n - 1] * U[n - 1] + B2[n, n - 1] * (K @ U[n - 1])
        U[n] = spla.spsolve((B1[n, n] * I + B2[n, n] * K).tocsc(), rhs)
    return U


def solve_direct(problem: GeometricProblem, b: np.ndarray, K=None, scaled=None,
                 intermediates: bool = False):
    """ParaDiag-I: u = A^{-1} b by eq. 2.6 and the three steps of eq. 2.7.

    ``scaled`` overrides the problem's column-scaling choice.  With
    ``intermediates`` also returns (b~, S1, S2, V, V^{-1}).
    """
    sp = problem.space
    K = stencil(sp) if K is None else K
    th = theta_of(problem.scheme)
    nt = problem.nt
    dts = geometric_steps(nt, problem.dt_last, problem.tau)
    _, B2 = time_matrices(dts, th)
    use_scaling = problem.scaled if scaled is None else scaled
    V, Vi = eigvec_matrices(nt, problem.tau, th, use_scaling)
    # eq. 2.6: b~ = (B2^{-1} (x) I) b
    bt = sla.solve_triangular(B2, np.asarray(b, dtype=np.float64), lower=True)
    # step (a)
    S1 = Vi @ bt
    # step (b)
    d = eigenvalues(dts, th)
    I = sps.identity(sp.size, format="csr")
    S2 = np.zeros_like(S1)
    for n in range(nt):
        S2[n] = spla.spsolve((d[n] * I + K).tocsc(), S1[n])
    # step (c)
    U = V @ S2
    if intermediates:
        return U, (bt, S1, S2, V, Vi)
    return U
