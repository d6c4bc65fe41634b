"""Operators of the all-at-once system A u = b, A = B1 (x) M + B2 (x) K (eq. 1.1).

Layout: u is time-major, u = (U_1; ...; U_Nt) (eq. 2.5a), stored as an array
U[n][s] of shape (Nt, S), n = 0..Nt-1 standing for t_1..t_Nt, and s the
spatial index (x fastest in 2D: s = y*nx + x).  M = I (finite differences).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps

from workloads import BE, CN, LEAPFROG, PERIODIC, Problem, Space


def stencil_1d(n: int, h: float, nu: float, a: float, bc: int) -> sps.csr_matrix:
    """K = -nu d_xx + a d_x with centred differences (eq. 2.2b).

    Row j: (-nu/h^2 - a/(2h)) u_{j-1} + (2 nu/h^2) u_j + (-nu/h^2 + a/(2h)) u_{j+1}.
    Dirichlet drops the neighbours outside 0..n-1; periodic wraps them
    (the corner entries of eq. 2.2b).
    """
    lower = -nu / h**2 - a / (2.0 * h)
    main = 2.0 * nu / h**2
    upper = -nu / h**2 + a / (2.0 * h)
    K = sps.lil_matrix((n, n))
    for j in range(n):
        K[j, j] += main
        if j - 1 >= 0:
            K[j, j - 1] += lower
        elif bc == PERIODIC:
            K[j, n - 1] += lower
        if j + 1 < n:
            K[j, j + 1] += upper
        elif bc == PERIODIC:
            K[j, 0] += upper
    return K.tocsr()


def stencil(space: Space) -> sps.csr_matrix:
    """Spatial matrix K of M U' + K U = f.  2D: K = I_y (x) K_x + K_y (x) I_x
    (x fastest), i.e. the 5-point stencil with centred advection."""
    Kx = stencil_1d(space.nx, space.hx, space.nu, space.ax, space.bc_x)
    if space.dim == 1:
        return Kx
    Ky = stencil_1d(space.ny, space.hy, space.nu, space.ay, space.bc_y)
    return (sps.kron(sps.identity(space.ny), Kx) + sps.kron(Ky, sps.identity(space.nx))).tocsr()


def first_columns(problem: Problem):
    """First columns c1, c2 of the Toeplitz B1, B2 (length Nt).

    theta-method (eq. 2.5b with uniform dt): c1 = (1, -1, 0, ...)/dt,
    c2 = (theta, 1-theta, 0, ...).
    implicit leap-frog (eq. 3.2b): c1 = (1, -2, 1, 0, ...)/dt^2,
    c2 = (1/2, 0, 1/2, 0, ...).
    """
    nt, dt = problem.nt, problem.dt
    c1 = np.zeros(nt)
    c2 = np.zeros(nt)
    if problem.scheme == LEAPFROG:
        for m, v in enumerate((1.0, -2.0, 1.0)):
            if m < nt:
                c1[m] = v / dt**2
        for m, v in enumerate((0.5, 0.0, 0.5)):
            if m < nt:
                c2[m] = v
    else:
        th = problem.theta_eff
        c1[0] = 1.0 / dt
        c2[0] = th
        if nt > 1:
            c1[1] = -1.0 / dt
            c2[1] = 1.0 - th
    return c1, c2


def toeplitz_lower(c: np.ndarray) -> np.ndarray:
    """Lower-triangular Toeplitz matrix with first column c."""
    n = len(c)
    T = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1):
            T[i, j] = c[i - j]
    return T


def time_matrices(problem: Problem):
    """Dense B1, B2 (eq. 2.5b for the theta-method, eq. 3.2b for leap-frog)."""
    c1, c2 = first_columns(problem)
    return toeplitz_lower(c1), toeplitz_lower(c2)


def alpha_circulant(c: np.ndarray, alpha: float) -> np.ndarray:
    """Strang-type alpha-circulant built from the first column c of a lower
    Toeplitz matrix: below and on the diagonal C[i][j] = c[i-j]; above it the
    wrapped entry is scaled by alpha, C[i][j] = alpha*c[Nt+i-j] (eq. 1.2,
    eq. 2.11b, eq. 3.4)."""
    n = len(c)
    C = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            C[i, j] = c[i - j] if i >= j else alpha * c[n + i - j]
    return C


def circulant_matrices(problem: Problem):
    """Dense C1^(alpha), C2^(alpha) of the preconditioner P_alpha (eq. 1.2)."""
    c1, c2 = first_columns(problem)
    return alpha_circulant(c1, problem.alpha), alpha_circulant(c2, problem.alpha)


def apply_kron(T1: np.ndarray, T2: np.ndarray, K: sps.spmatrix, U: np.ndarray) -> np.ndarray:
    """(T1 (x) I + T2 (x) K) u for time-major U of shape (Nt, S):
    block row n = sum_m T1[n,m] U_m + K sum_m T2[n,m] U_m."""
    KU = (K @ U.T).T
    return T1 @ U + T2 @ KU


def apply_A(problem: Problem, U: np.ndarray, K=None) -> np.ndarray:
    """A u with A = B1 (x) I + B2 (x) K (eq. 1.1)."""
    K = stencil(problem.space) if K is None else K
    B1, B2 = time_matrices(problem)
    return apply_kron(B1, B2, K, U)


def apply_P(problem: Problem, U: np.ndarray, K=None) -> np.ndarray:
    """P_alpha u with P_alpha = C1 (x) I + C2 (x) K (eq. 1.2)."""
    K = stencil(problem.space) if K is None else K
    C1, C2 = circulant_matrices(problem)
    return apply_kron(C1, C2, K, U)


def apply_AT(problem: Problem, L: np.ndarray, K=None) -> np.ndarray:
    """A^T lambda = (B1^T (x) I + B2^T (x) K^T) lambda."""
    K = stencil(problem.space) if K is None else K
    B1, B2 = time_matrices(problem)
    return apply_kron(B1.T, B2.T, K.T.tocsr(), L)


def build_rhs(problem: Problem, u0, u1=None, f=None, K=None) -> np.ndarray:
    """Right-hand side b of eq. 1.1, shape (Nt, S).

    theta-method (eq. 2.4 written for row n = 1..Nt with uniform dt):
      b_n = theta f(t_n) + (1-theta) f(t_{n-1}),
      plus (I/dt - (1-theta) K) U_0 in row 1 (eq. 2.5a).
    leap-frog (eq. 3.2b), with the ghost value U_{-1} = U_1 - 2 dt u_1 in the
    first step and the first row halved to match B2[0][0] = 1/2:
      b_1 = U_0/dt^2 + u_1/dt + (dt/2) K u_1 + f(t_0)/2,
      b_2 = f(t_1) - U_0/dt^2 - K U_0/2,
      b_n = f(t_{n-1}) for n >= 3.
    ``f`` has shape (Nt+1, S) (values at t_0..t_Nt) or is None (zero source).
    """
    K = stencil(problem.space) if K is None else K
    nt, dt, S = problem.nt, problem.dt, problem.space.size
    u0 = np.asarray(u0, dtype=np.float64)
    F = np.zeros((nt + 1, S)) if f is None else np.asarray(f, dtype=np.float64)
    b = np.zeros((nt, S))
    if problem.scheme == LEAPFROG:
        v1 = np.zeros(S) if u1 is None else np.asarray(u1, dtype=np.float64)
        for n in range(nt):
            b[n] = F[n] if n >= 2 else 0.0
        b[0] = u0 / dt**2 + v1 / dt + (dt / 2.0) * (K @ v1) + F[0] / 2.0
        if nt > 1:
            b[1] = F[1] - u0 / dt**2 - 0.5 * (K @ u0)
    else:
        th = problem.theta_eff
        for n in range(nt):
            b[n] = th * F[n + 1] + (1.0 - th) * F[n]
        b[0] += u0 / dt - (1.0 - th) * (K @ u0)
    return b


def schemes_supported():
    return (BE, CN, LEAPFROG)
