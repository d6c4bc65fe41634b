"""O7: ParaDiag-I with the hybrid time discretisation (Section 2.1.2).

Uniform steps dt; the explicit midpoint rule for the first Nt-1 steps and one
backward-Euler step at the end (eq. neq2.9a).  The all-at-once system is
(eq. neq2.9b, neq2.9c)

    (B (x) I + I (x) K) u = b,   B = (1/dt) tridiag(-1/2, 0, 1/2) with the last
    row (..., -1, 1),  b = (U_0 / (2 dt), 0, ..., 0).

The theorem of Section 2.1.2 diagonalises B = V D V^{-1}: the eigenvalues are
lambda_n = i x_n / dt with x_n the Nt roots of P2_{Nt-1}(x) - i P1_{Nt}(x)
(Chebyshev polynomials of the second and first kind), found by Newton's
method; the eigenvectors are v_{n,l} = i^l P2_l(x_n) (eq. Vformula).  The
solve is the three steps of eq. 2.7 with these V, D:

    (a) S1 = (V^{-1} (x) I) b,  (b) S2_n = (lambda_n I + K)^{-1} S1_n,
    (c) u = (V (x) I) S2.

Readings:
  * The theorem prints the eigenvalues as i dt x_n; with the 1/dt factor of
    eq. neq2.9c they are i x_n / dt.  (The tests check B V = V D.)
  * The paper gives no starting values for Newton; here they are the
    eigenvalues of B dt from the library eigenvalue routine, polished by
    Newton steps on eq. e-value.
  * A source f (values at t_0..t_Nt) enters every row as f(t_n): rows
    1..Nt-1 are midpoint equations centred at t_n, the last row is backward
    Euler at t_Nt.
  * V^{-1} is not given in closed form; it is formed by a dense LU solve.

Second-order problems U'' + K U = f (Section 2.1.2, eq. neq2.14a/b): the hybrid
scheme applied to the first-order system W' + [[0, -I], [K, 0]] W = (0, f) with
W = (U, V) has the state rows (B U)_n - V_n = U_0/(2 dt) delta_{n1} and the
velocity rows (B V)_n + K U_n = f(t_n) + V_0/(2 dt) delta_{n1}.  Eliminating V
gives (B^2 (x) I + I (x) K) u = F_v + B F_u (B_2nd = B^2, eq. neq2.15), with
F_u = (U_0/(2 dt), 0, ...) and F_v the velocity rows' right-hand side, and the
same eigenvectors V with eigenvalues lambda_n^2.  (The elimination is the
section's; the right-hand side is written out here, reading R24.)

The exact solution of the all-at-once system (not a time-stepping recursion:
the midpoint rule needs U_{n+1} before U_1 is known, so the scheme is a
boundary value method) is a sparse LU solve of the whole system.
Test infrastructure only; shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from workloads import HybridProblem

from .operators import stencil


def time_matrix(nt: int, dt: float) -> np.ndarray:
    """B of eq. neq2.9c (dense Nt x Nt)."""
    B = np.zeros((nt, nt))
    for l in range(nt - 1):
        if l > 0:
            B[l, l - 1] = -0.5
        B[l, l + 1] = 0.5
    B[nt - 1, nt - 1] = 1.0
    if nt > 1:
        B[nt - 1, nt - 2] = -1.0
    return B / dt


def build_rhs(problem: HybridProblem, u0, f=None) -> np.ndarray:
    """b of eq. neq2.9c, shape (Nt, S); f of shape (Nt+1, S) at t_0..t_Nt or None."""
    nt, S = problem.nt, problem.space.size
    b = np.zeros((nt, S))
    if f is not None:
        F = np.asarray(f, dtype=np.float64)
        b += F[1:]
    b[0] += np.asarray(u0, dtype=np.float64) / (2.0 * problem.dt)
    return b


def apply_A(problem: HybridProblem, U: np.ndarray, K=None) -> np.ndarray:
    K = stencil(problem.space) if K is None else K
    B = time_matrix(problem.nt, problem.dt)
    return B @ U + (K @ np.asarray(U).T).T


def all_at_once_matrix(problem: HybridProblem, K=None) -> sps.csr_matrix:
    K = stencil(problem.space) if K is None else K
    B = sps.csr_matrix(time_matrix(problem.nt, problem.dt))
    S = problem.space.size
    return (sps.kron(B, sps.identity(S)) + sps.kron(sps.identity(problem.nt), K)).tocsr()


def solve_exact(problem: HybridProblem, b: np.ndarray, K=None) -> np.ndarray:
    """The exact solution of eq. neq2.9b by a sparse LU of the whole system."""
    A = all_at_once_matrix(problem, K).tocsc()
    u = spla.spsolve(A, np.asarray(b, dtype=np.float64).reshape(-1))
    return u.reshape(problem.nt, problem.space.size)


def chebyshev(n: int, x):
    """T_0..T_n and U_0..U_n at x (arrays of shape (n+1,) + x.shape) by the
    three-term recurrences T_{k+1} = 2x T_k - T_{k-1}, U likewise with U_1 = 2x."""
    x = np.asarray(x, dtype=np.complex128)
    T = np.zeros((n + 1,) + x.shape, dtype=np.complex128)
    U = np.zeros_like(T)
    T[0] = 1.0
    U[0] = 1.0
    if n >= 1:
        T[1] = x
        U[1] = 2.0 * x
    for k in range(2, n + 1):
        T[k] = 2.0 * x * T[k - 1] - T[k - 2]
        U[k] = 2.0 * x * U[k - 1] - U[k - 2]
    return T, U


def characteristic(nt: int, x):
    """g(x) = P2_{Nt-1}(x) - i P1_{Nt}(x) (eq. e-value) and g'(x), using
    T_n' = n U_{n-1} and U_n' = ((n+1) T_{n+1} - x U_n)/(x^2 - 1)."""
    T, U = chebyshev(nt, x)
    g = U[nt - 1] - 1j * T[nt]
    dU = (nt * T[nt] - x * U[nt - 1]) / (x * x - 1.0)
    dT = nt * U[nt - 1]
    return g, dU - 1j * dT


def eigen_roots(nt: int, newton_steps: int = 8) -> np.ndarray:
    """The Nt roots x_n of eq. e-value: Newton's method started from the
    eigenvalues of dt B (x = -i lambda dt)."""
    x = -1j * np.linalg.eigvals(time_matrix(nt, 1.0))
    if nt == 1:
        return x
    for _ in range(newton_steps):
        g, dg = characteristic(nt, x)
        step = g / dg
        x = x - step
        if np.max(np.abs(step)) <= 4e-16 * max(1.0, np.max(np.abs(x))):
            break
    return x


def eigenvalues(problem: HybridProblem) -> np.ndarray:
    """lambda_n = i x_n / dt (reading of the theorem of Section 2.1.2)."""
    return 1j * eigen_roots(problem.nt) / problem.dt


def eigvec_matrix(x: np.ndarray) -> np.ndarray:
    """V of eq. Vformula: V[l][n] = i^l P2_l(x_n), l = 0..Nt-1."""
    nt = len(x)
    _, U = chebyshev(nt - 1, x)
    return (1j ** np.arange(nt))[:, None] * U


def solve_direct(problem: HybridProblem, b: np.ndarray, K=None, intermediates=False):
    """ParaDiag-I with the hybrid discretisation: the three steps of eq. 2.7
    with the eigendecomposition of the theorem of Section 2.1.2."""
    sp = problem.space
    K = stencil(sp) if K is None else K
    x = eigen_roots(problem.nt)
    lam = 1j * x / problem.dt
    V = eigvec_matrix(x)
    # step (a): S1 = V^{-1} b (dense LU solve)
    S1 = np.linalg.solve(V, np.asarray(b, dtype=np.complex128))
    # step (b)
    I = sps.identity(sp.size, format="csc", dtype=np.complex128)
    Kc = K.astype(np.complex128).tocsc()
    S2 = np.zeros_like(S1)
    for n in range(problem.nt):
        S2[n] = spla.spsolve((lam[n] * I + Kc).tocsc(), S1[n])
    # step (c)
    U = V @ S2
    if intermediates:
        return U, (x, V, S1, S2)
    return U.real


# ---------------------------------------------------------------------------
# Second-order problems (B_2nd = B^2)
# ---------------------------------------------------------------------------
def time_matrix_2nd(nt: int, dt: float) -> np.ndarray:
    """B_2nd = B^2 (eq. neq2.15)."""
    B = time_matrix(nt, dt)
    return B @ B


def build_rhs_2nd(problem: HybridProblem, u0, v0, f=None) -> np.ndarray:
    """b = F_v + B F_u of the eliminated system; f of shape (Nt+1, S) at t_0..t_Nt
    or None; u0, v0 the initial value and velocity."""
    nt, S, dt = problem.nt, problem.space.size, problem.dt
    Fv = np.zeros((nt, S))
    if f is not None:
        Fv += np.asarray(f, dtype=np.float64)[1:]
    Fv[0] += np.asarray(v0, dtype=np.float64) / (2.0 * dt)
    Fu = np.zeros((nt, S))
    Fu[0] = np.asarray(u0, dtype=np.float64) / (2.0 * dt)
    return Fv + time_matrix(nt, dt) @ Fu


def apply_A_2nd(problem: HybridProblem, U: np.ndarray, K=None) -> np.ndarray:
    K = stencil(problem.space) if K is None else K
    return time_matrix_2nd(problem.nt, problem.dt) @ U + (K @ np.asarray(U).T).T


def solve_exact_2nd(problem: HybridProblem, b: np.ndarray, K=None) -> np.ndarray:
    """Sparse LU of B^2 (x) I + I (x) K (small sizes)."""
    K = stencil(problem.space) if K is None else K
    B2 = sps.csr_matrix(time_matrix_2nd(problem.nt, problem.dt))
    S = problem.space.size
    A = (sps.kron(B2, sps.identity(S)) + sps.kron(sps.identity(problem.nt), K)).tocsc()
    return spla.spsolve(A, np.asarray(b, dtype=np.float64).reshape(-1)).reshape(problem.nt, S)


def solve_direct_2nd(problem: HybridProblem, b: np.ndarray, K=None) -> np.ndarray:
    """The three steps of eq. 2.7 with B_2nd = V D^2 V^{-1}: shifts lambda_n^2."""
    sp = problem.space
    K = stencil(sp) if K is None else K
    x = eigen_roots(problem.nt)
    lam = 1j * x / problem.dt
    V = eigvec_matrix(x)
    S1 = np.linalg.solve(V, np.asarray(b, dtype=np.complex128))
    I = sps.identity(sp.size, format="csc", dtype=np.complex128)
    Kc = K.astype(np.complex128).tocsc()
    S2 = np.zeros_like(S1)
    for n in range(problem.nt):
        S2[n] = spla.spsolve((lam[n] ** 2 * I + Kc).tocsc(), S1[n])
    return (V @ S2).real
