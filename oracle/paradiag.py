"""O2: ParaDiag-II written out naively in FP64.

P_alpha^{-1} r follows Lemma 1 and the three steps of eq. 1.3 literally:
  F     = N^{-1/2} [omega^{(l1-1)(l2-1)}], omega = exp(+2 pi i / Nt)  (unitary),
  Gamma = diag(alpha^{(n-1)/Nt}), n = 1..Nt,
  V     = Gamma^{-1} F^*,  V^{-1} = F Gamma,
  D_j   = diag(sqrt(Nt) F Gamma c_j), c_j = first column of C_j^(alpha)
          (the shifted systems are factored with the closed forms of these
          diagonals, evaluated without cancellation, closed_forms.py),
  step (a) S_1 = (V^{-1} (x) I) r,
  step (b) S_{2,n} = (lambda_{1,n} I + lambda_{2,n} K)^{-1} S_{1,n}, all n = 1..Nt,
  step (c) u = (V (x) I) S_2.
The Fourier matrix is formed densely (O(Nt^2)); every one of the Nt shifted
spatial systems is solved with a complex sparse LU (no half-spectrum
shortcut, no spatial diagonalisation).

The outer solvers are the stationary iteration eq. 5.1 and flexible GMRES
(Saad's right-preconditioned FGMRES(m) with modified Gram-Schmidt) on
A u = b with P_alpha^{-1} as the preconditioner (the Krylov variant of
Section 3).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from workloads import LEAPFROG, Problem

from . import closed_forms as CF
from .operators import apply_A, first_columns, stencil


def fourier_matrix(nt: int) -> np.ndarray:
    """Unitary F of Lemma 1 with omega = exp(2 pi i / Nt).

    omega^Nt = 1, so the exponent (l1-1)(l2-1) is reduced modulo Nt in exact
    integer arithmetic before the phase is formed: the phase then stays below
    2 pi and carries one rounding of a number below 2 pi, where the unreduced
    product (up to (Nt-1)^2) would put an absolute error of about
    eps 2 pi Nt into the entries."""
    idx = np.arange(nt, dtype=np.int64)
    return np.exp(2j * np.pi * (np.outer(idx, idx) % nt) / nt) / np.sqrt(nt)


def gamma(problem: Problem) -> np.ndarray:
    """Diagonal of Gamma_alpha: alpha^{(n-1)/Nt}, n = 1..Nt (Lemma 1)."""
    return problem.alpha ** (np.arange(problem.nt) / problem.nt)


def eigenvalues(problem: Problem):
    """lambda_{j,n} = (sqrt(Nt) F Gamma c_j)_n, the diagonals D_1, D_2 of Lemma 1."""
    c1, c2 = first_columns(problem)
    F = fourier_matrix(problem.nt)
    g = gamma(problem)
    s = np.sqrt(problem.nt)
    return s * (F @ (g * c1)), s * (F @ (g * c2))


def shift_eigenvalues(problem: Problem):
    """The diagonals of Lemma 1 that step (b)'s systems are factored with:
    the closed forms (closed_forms.lemma1_eigenvalues, no cancelling digits)
    where every band entry of the first columns lies inside the matrix, else
    the definition.  The definition's sum c_j[0] + c_j[1] w + ... loses about
    log10(Nt/|ln alpha|) digits on the slow modes, where w is close to 1."""
    band = 2 if problem.scheme == LEAPFROG else 1
    if problem.nt > band:
        return CF.lemma1_eigenvalues(problem)
    return eigenvalues(problem)


class Preconditioner:
    """P_alpha^{-1} with the Nt complex shifted systems factored once."""

    def __init__(self, problem: Problem, K=None):
        self.problem = problem
        self.K = stencil(problem.space) if K is None else K
        self.F = fourier_matrix(problem.nt)
        self.g = gamma(problem)
        self.lam1, self.lam2 = shift_eigenvalues(problem)
        S = problem.space.size
        I = sps.identity(S, dtype=np.complex128)
        Kc = self.K.astype(np.complex128)
        self.lus = [spla.splu((self.lam1[n] * I + self.lam2[n] * Kc).tocsc())
                    for n in range(problem.nt)]

    def apply(self, R: np.ndarray) -> np.ndarray:
        """z = P_alpha^{-1} r for time-major r of shape (Nt, S)."""
        S1 = self.F @ (self.g[:, None] * R)                      # step (a)
        S2 = np.stack([self.lus[n].solve(S1[n]) for n in range(self.problem.nt)])  # step (b)
        Z = (self.F.conj().T @ S2) / self.g[:, None]             # step (c)
        return Z.real


def precond_apply(problem: Problem, R: np.ndarray, K=None) -> np.ndarray:
    return Preconditioner(problem, K).apply(R)


def stationary(problem: Problem, b: np.ndarray, u_init=None, tol=1e-12, maxit=50, K=None,
               history=False):
    """Stationary iteration eq. 5.1: r^k = b - A u^k, P_alpha du^k = r^k,
    u^{k+1} = u^k + du^k; stop when ||r^k||_2 / ||b||_2 <= tol.

    Returns (u, iterations, relres) and, with history=True, the list of iterates.
    """
    K = stencil(problem.space) if K is None else K
    P = Preconditioner(problem, K)
    U = np.zeros_like(b) if u_init is None else np.array(u_init, dtype=np.float64)
    nb = np.linalg.norm(b)
    hist = [U.copy()]
    it = 0
    rel = np.linalg.norm(b - apply_A(problem, U, K)) / nb
    while rel > tol and it < maxit:
        R = b - apply_A(problem, U, K)
        U = U + P.apply(R)
        it += 1
        hist.append(U.copy())
        rel = np.linalg.norm(b - apply_A(problem, U, K)) / nb
    return (U, it, rel, hist) if history else (U, it, rel)


def fgmres(problem: Problem, b: np.ndarray, tol=1e-10, restart=30, maxit=200, K=None,
           u_init=None):
    """Right-preconditioned flexible GMRES(restart) for A u = b, z_j = P^{-1} v_j.

    Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
    matrix, stop when the true relative residual ||b - A u|| / ||b|| <= tol.
    Returns (u, total inner iterations, relres).
    """
    K = stencil(problem.space) if K is None else K
    P = Preconditioner(problem, K)
    shape = b.shape
    bv = b.reshape(-1)
    nb = np.linalg.norm(bv)
    x = np.zeros_like(bv) if u_init is None else np.array(u_init, dtype=np.float64).reshape(-1)
    A = lambda v: apply_A(problem, v.reshape(shape), K).reshape(-1)
    Pinv = lambda v: P.apply(v.reshape(shape)).reshape(-1)
    total = 0
    rel = np.linalg.norm(bv - A(x)) / nb
    while rel > tol and total < maxit:
        r = bv - A(x)
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, bv.size))
        Z = np.zeros((m, bv.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        V[0] = r / beta
        j_done = 0
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
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            j_done = j + 1
            total += 1
            if abs(gvec[j + 1]) / nb <= tol or total >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), gvec[:j_done])
        x = x + Z[:j_done].T @ y
        rel = np.linalg.norm(bv - A(x)) / nb
    return x.reshape(shape), total, rel
