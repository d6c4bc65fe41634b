"""O9: ParaDiag-II preconditioner for the optimal control of the wave equation
(Section 4): the saddle-point all-at-once system of the implicit leap-frog
scheme, its gamma-balanced form, the block circulant preconditioner P and
its factorisation P = P~ (blockdiag(C2, C2^T) (x) I) with the closed-form
spectral decomposition of P~ (Theorem 4); flexible GMRES on the balanced
system with P^{-1}.

Notation (the whole system multiplied by dt^2, as in the section):
  T1 = lower Toeplitz, first column (1, -2, 1, 0, ...)   (dt^2 B1 of eq. 3.2b)
  T2 = lower Toeplitz, first column (1, 0, 1, 0, ...) dt^2/2   (dt^2 B2)
  Ih = diag(1/2, 1, ..., 1),  Ic = diag(1, ..., 1, 1/2)
  A^ = [[T1, -dt^2 Ih / gamma], [dt^2 Ic, T1^T]] (x) I + blockdiag(T2, T2^T) (x) K
  balanced (similarity with diag(gamma^{1/2} I, I)):
  A  = [[T1, -beta Ih], [beta Ic, T1^T]] (x) I + blockdiag(T2, T2^T) (x) K,
  beta = dt^2 / sqrt(gamma), unknowns (gamma^{1/2} u, p);
  P  = [[C1, -beta I], [beta I, C1^T]] (x) I + blockdiag(C2, C2^T) (x) K
  with C1, C2 the Strang circulants of T1, T2 (eq. 3.3).
With the Fourier diagonalisation C = F^* diag(d) F (d_k = sum_m c_m w^{mk},
w = exp(-2 pi i/Nt)) and C^T = F^* diag(conj d) F, P~ is, per frequency k, the
2 x 2 block [[lam_k, -beta/conj(d2_k)], [beta/d2_k, lam_k]] + I (x) K with
lam_k = d1_k/d2_k (real), whose eigenvalues are lam_k +- i beta/|d2_k|
(Sigma_1, Sigma_2 of eq. 4.4b) and whose eigenvectors
Q_k = [[1, 1], [-i phibar, i phibar]], phibar = conj(d2_k)/|d2_k|, are
orthogonal (Cond_2 = 1).  P^{-1} r is then: FFT of both halves, Q_k^{-1},
2 Nt complex-shifted spatial solves, Q_k, scaling by 1/d2 and 1/conj(d2)
(the factor blockdiag(C2, C2^T)^{-1}), inverse FFT.

Readings:
  * The section's B1, B2 carry the dt^2 scaling of the saddle system; the
    printed (dt^2/2) B2 is read as dt^2 times B2 of eq. 3.2b (first column
    (1/2, 0, 1/2)).
  * Right-hand side: the section states the data (f, g, u0, u1) but not how
    they enter the discrete rows; the tests use the grid values of the exact
    solution (u = e^t sin(pi x) sin(pi y), p = (t - T)^2 sin(pi x) sin(pi y))
    at t_1..t_Nt and the right-hand side A^ applied to them, so the discrete
    solution is known exactly.
  * Mesh "(N_x, N_x, N_t)" of Table T2A: N_x intervals per direction (N_x - 1
    interior points, h = 1/N_x) and N_t time steps of dt = T/N_t (T = 2).
Test infrastructure only; shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from .operators import stencil


def time_blocks(nt: int, dt: float):
    """T1, T2 (dense Nt x Nt) and the first columns c1, c2 of their circulants."""
    c1 = np.zeros(nt)
    c2 = np.zeros(nt)
    for m, v in enumerate((1.0, -2.0, 1.0)):
        if m < nt:
            c1[m] += v
    for m, v in enumerate((1.0, 0.0, 1.0)):
        if m < nt:
            c2[m] += v * dt * dt / 2.0
    T1 = np.zeros((nt, nt))
    T2 = np.zeros((nt, nt))
    for i in range(nt):
        for m in range(min(3, i + 1)):
            T1[i, i - m] = c1[m]
            T2[i, i - m] = c2[m]
    return T1, T2, c1, c2


def circulant(c: np.ndarray) -> np.ndarray:
    n = len(c)
    return np.array([[c[(i - j) % n] for j in range(n)] for i in range(n)])


def saddle_matrix(nt: int, dt: float, gamma: float, K, balanced=True) -> sps.csr_matrix:
    """A (balanced) or A^ (eq. of Section 4) as a sparse matrix of order 2 Nt S."""
    T1, T2, _, _ = time_blocks(nt, dt)
    S = K.shape[0]
    Ih = np.eye(nt); Ih[0, 0] = 0.5
    Ic = np.eye(nt); Ic[-1, -1] = 0.5
    if balanced:
        b12, b21 = -dt * dt / np.sqrt(gamma), dt * dt / np.sqrt(gamma)
    else:
        b12, b21 = -dt * dt / gamma, dt * dt
    I = sps.identity(S)
    top = sps.hstack([sps.kron(T1, I) + sps.kron(T2, K), sps.kron(b12 * Ih, I)])
    bot = sps.hstack([sps.kron(b21 * Ic, I), sps.kron(T1.T, I) + sps.kron(T2.T, K)])
    return sps.vstack([top, bot]).tocsr()


def precond_matrix(nt: int, dt: float, gamma: float, K) -> sps.csr_matrix:
    """P = [[C1, -beta I], [beta I, C1^T]] (x) I + blockdiag(C2, C2^T) (x) K."""
    _, _, c1, c2 = time_blocks(nt, dt)
    C1, C2 = circulant(c1), circulant(c2)
    beta = dt * dt / np.sqrt(gamma)
    S = K.shape[0]
    I = sps.identity(S)
    top = sps.hstack([sps.kron(C1, I) + sps.kron(C2, K), sps.kron(-beta * np.eye(nt), I)])
    bot = sps.hstack([sps.kron(beta * np.eye(nt), I), sps.kron(C1.T, I) + sps.kron(C2.T, K)])
    return sps.vstack([top, bot]).tocsr()


def spectra(nt: int, dt: float):
    """d1_k, d2_k: eigenvalues of C1, C2 for the transform X_k = sum_n x_n w^{nk}."""
    _, _, c1, c2 = time_blocks(nt, dt)
    w = np.exp(-2j * np.pi * np.arange(nt) / nt)
    m = np.arange(nt)
    d1 = np.array([np.sum(c1 * w[k] ** m) for k in range(nt)])
    d2 = np.array([np.sum(c2 * w[k] ** m) for k in range(nt)])
    return d1, d2


def block_eigen(nt: int, dt: float, gamma: float):
    """Per frequency: lam_k = d1/d2 (real), Sigma_1,2 = lam +- i beta/|d2|, and the
    eigenvector blocks Q_k = [[1, 1], [-i phibar, i phibar]] (Theorem 4)."""
    d1, d2 = spectra(nt, dt)
    beta = dt * dt / np.sqrt(gamma)
    lam = d1 / d2
    s1 = lam + 1j * beta / np.abs(d2)
    s2 = lam - 1j * beta / np.abs(d2)
    phib = np.conj(d2) / np.abs(d2)
    Q = np.zeros((nt, 2, 2), dtype=np.complex128)
    Q[:, 0, 0] = 1.0
    Q[:, 0, 1] = 1.0
    Q[:, 1, 0] = -1j * phib
    Q[:, 1, 1] = 1j * phib
    return lam, s1, s2, Q, d2


class Preconditioner:
    """P^{-1} by the steps of Theorem 4 (the 2 Nt shifted systems factored once)."""

    def __init__(self, nt, dt, gamma, K):
        self.nt, self.K = nt, K.tocsc()
        self.lam, self.s1, self.s2, self.Q, self.d2 = block_eigen(nt, dt, gamma)
        S = K.shape[0]
        I = sps.identity(S, format="csc", dtype=np.complex128)
        Kc = K.astype(np.complex128).tocsc()
        self.lu1 = [spla.splu((self.s1[k] * I + Kc).tocsc()) for k in range(nt)]
        self.lu2 = [spla.splu((self.s2[k] * I + Kc).tocsc()) for k in range(nt)]

    def apply(self, r1: np.ndarray, r2: np.ndarray):
        nt = self.nt
        R1 = np.fft.fft(r1, axis=0)          # X_k = sum_n x_n exp(-2 pi i n k / Nt)
        R2 = np.fft.fft(r2, axis=0)
        Y1 = np.zeros_like(R1)
        Y2 = np.zeros_like(R2)
        for k in range(nt):
            Qk = self.Q[k]
            z = np.linalg.solve(Qk, np.vstack([R1[k], R2[k]]))
            yp = self.lu1[k].solve(z[0])
            ym = self.lu2[k].solve(z[1])
            y = Qk @ np.vstack([yp, ym])
            Y1[k] = y[0] / self.d2[k]
            Y2[k] = y[1] / np.conj(self.d2[k])
        return np.fft.ifft(Y1, axis=0).real, np.fft.ifft(Y2, axis=0).real


def exact_solution(space, nt: int, T: float):
    """Grid values at t_1..t_Nt of u = e^t s(x, y), p = (t - T)^2 s(x, y),
    s = sin(pi x) sin(pi y) (the section's exact optimal pair)."""
    X, Y = space.mesh()
    s = (np.sin(np.pi * X) * np.sin(np.pi * Y)).reshape(-1)
    t = (T / nt) * np.arange(1, nt + 1)
    return np.outer(np.exp(t), s), np.outer((t - T) ** 2, s)


def fgmres_op(A, Pinv, b: np.ndarray, tol=1e-7, restart=50, maxit=200):
    """Right-preconditioned flexible GMRES(restart) for the operator A with the
    preconditioner Pinv (vectors as flat arrays); modified Gram-Schmidt,
    Givens rotations; stops on the true relative residual."""
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    total = 0
    rel = 1.0
    while rel > tol and total < maxit:
        r = b - A(x)
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        jd = 0
        for j in range(m):
            Z[j] = Pinv(V[j])
            w = A(Z[j])
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            jd = j + 1
            total += 1
            if abs(g[j + 1]) / nb <= tol or total >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:jd, :jd]), g[:jd])
        x = x + Z[:jd].T @ y
        rel = np.linalg.norm(b - A(x)) / nb
    return x, total, rel


def solve(space, nt: int, T: float, gamma: float, rhs1, rhs2, tol=1e-7, K=None, side="right",
          restart=50):
    """GMRES on the balanced system with P^{-1}: returns (u, p, iterations,
    relres) for the right-hand side (rhs1, rhs2) of the unbalanced system.
    side="right": flexible GMRES on A P^{-1}, stopping on ||b - A x|| / ||b||;
    side="left": GMRES on P^{-1} A x = P^{-1} b, stopping on the preconditioned
    residual ||P^{-1}(b - A x)|| / ||P^{-1} b|| (relres is that ratio)."""
    K = stencil(space) if K is None else K
    dt = T / nt
    A = saddle_matrix(nt, dt, gamma, K, balanced=True)
    P = Preconditioner(nt, dt, gamma, K)
    S = K.shape[0]
    n = nt * S
    sg = np.sqrt(gamma)
    b = np.concatenate([sg * np.asarray(rhs1).reshape(-1), np.asarray(rhs2).reshape(-1)])
    Aop = lambda v: A @ v
    Pop = lambda v: np.concatenate([q.reshape(-1) for q in
                                    P.apply(v[:n].reshape(nt, S), v[n:].reshape(nt, S))])
    if side == "left":
        x, it, rel = fgmres_op(lambda v: Pop(Aop(v)), lambda v: v, Pop(b), tol=tol,
                               restart=restart)
    else:
        x, it, rel = fgmres_op(Aop, Pop, b, tol=tol, restart=restart)
    return x[:n].reshape(nt, S) / sg, x[n:].reshape(nt, S), it, rel
