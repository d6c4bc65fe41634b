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
import scipy.linalg as sla
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from workloads import PERIODIC, Problem

from .operators import first_columns, stencil, stencil_1d


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


def _xmode_chunk(args):
    """Sequential time stepping of a share of the x-Fourier modes (one worker's
    part of solve_sequential_xmodes).  args = (c1, c2, band, Ky, mus, bh) with
    Ky the tridiagonal K_y (sparse), mus the eigenvalues mu_j of the share's
    modes and bh their transformed right-hand sides, shape (Nt, ny, len(mus));
    returns the transformed solution of the same shape.  The tridiagonal step
    matrix of each mode is factored once by LAPACK's LU with partial pivoting
    (zgttrf) and solved at every step (zgttrs)."""
    c1, c2, band, Ky, mus, bh = args
    nt, ny, _ = bh.shape
    Uh = np.zeros(bh.shape, dtype=np.complex128)
    Kd = Ky.diagonal(0).astype(np.complex128)
    Kl = Ky.diagonal(-1).astype(np.complex128)
    Ku = Ky.diagonal(1).astype(np.complex128)
    for q, muj in enumerate(mus):
        # step matrix c1[0] I + c2[0] (mu_j I + K_y) as its three diagonals
        dl, d, du = c2[0] * Kl, c1[0] + c2[0] * (muj + Kd), c2[0] * Ku
        dl, d, du, du2, ipiv, info = sla.lapack.zgttrf(dl, d, du)
        if info != 0:
            raise np.linalg.LinAlgError(f"singular step matrix for x-mode {q}")
        for n in range(nt):
            rhs = bh[n, :, q].copy()
            for m in band:
                if n - m >= 0:
                    v = Uh[n - m, :, q]
                    rhs -= c1[m] * v + c2[m] * (muj * v + Ky @ v)
            Uh[n, :, q], info = sla.lapack.zgttrs(dl, d, du, du2, ipiv, rhs)
    return Uh


def solve_sequential_xmodes(problem: Problem, b: np.ndarray, pool=None, chunks=1) -> np.ndarray:
    """O1 for 2D problems with x periodic, mode by mode: u = A^{-1} b.

    K = I_y (x) K_x + K_y (x) I_x with a circulant K_x, so the naive DFT along x
    (a dense matrix of exp(-2 pi i j x / nx) entries) turns A u = b into nx
    independent all-at-once systems, one per x-mode j, with K replaced by
    mu_j I + K_y, mu_j the eigenvalue of K_x for the mode exp(2 pi i j x / nx)
    (read off K_x's first row).  Each is solved by forward substitution in time
    with a tridiagonal LU with partial pivoting of its step matrix (LAPACK's
    zgttrf / zgttrs, the library primitive used as the spatial solve); the inverse DFT
    along x sums the modes back.  The modes are independent, so their time
    stepping can be spread over the processes of ``pool`` (any object with a
    ``map``) in ``chunks`` shares; time stays sequential within each mode.
    b, u of shape (Nt, S).
    """
    sp = problem.space
    if sp.dim != 2 or sp.bc_x != PERIODIC:
        raise ValueError("solve_sequential_xmodes needs a 2D problem with x periodic")
    nx, ny = sp.nx, sp.ny
    Kx = stencil_1d(nx, sp.hx, sp.nu, sp.ax, sp.bc_x).toarray()
    Ky = stencil_1d(ny, sp.hy, sp.nu, sp.ay, sp.bc_y)
    x = np.arange(nx)
    F = np.exp(-2j * np.pi * np.outer(x, x) / nx)                         # [x][j]
    mu = np.array([Kx[0] @ np.exp(2j * np.pi * j * x / nx) for j in range(nx)])
    c1, c2 = first_columns(problem)
    nt = b.shape[0]
    band = [m for m in range(1, nt) if c1[m] != 0.0 or c2[m] != 0.0]
    bh = np.asarray(b, dtype=np.float64).reshape(nt, ny, nx) @ F            # (nt, ny, nx modes)
    shares = [np.arange(i, nx, chunks) for i in range(chunks) if i < nx]
    args = [(c1, c2, band, Ky, mu[js], np.ascontiguousarray(bh[:, :, js])) for js in shares]
    parts = list(pool.map(_xmode_chunk, args)) if pool is not None else [_xmode_chunk(a) for a in args]
    Uh = np.empty_like(bh)
    for js, part in zip(shares, parts):
        Uh[:, :, js] = part
    return (np.real(Uh @ F.conj().T) / nx).reshape(nt, ny * nx)
