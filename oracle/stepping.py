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
    part of solve_sequential_xmodes).  args = (c1, c2, band, Ky, share, b) with
    share a list of (j, mu_j); returns this share's terms of the inverse DFT
    along x, a real array of shape (Nt, ny, nx)."""
    c1, c2, band, Ky, share, b = args
    nt, ny, nx = b.shape
    idx = np.arange(nx)
    out = np.zeros((nt, ny, nx))
    I = np.eye(ny)
    for j, muj in share:
        # the naive DFT of every b_n along x at frequency j
        bh = b @ np.exp(-2j * np.pi * j * idx / nx)                     # (nt, ny)
        Kj = muj * I + Ky                                                 # K on mode j
        lu = sla.lu_factor(c1[0] * I + c2[0] * Kj)
        Uh = np.zeros((nt, ny), dtype=np.complex128)
        for n in range(nt):
            rhs = bh[n].copy()
            for m in band:
                if n - m >= 0:
                    rhs -= c1[m] * Uh[n - m] + c2[m] * (Kj @ Uh[n - m])
            Uh[n] = sla.lu_solve(lu, rhs)
        # this mode's term of the inverse DFT along x
        out += np.real(Uh[:, :, None] * np.exp(2j * np.pi * j * idx / nx)[None, None, :]) / nx
    return out


def solve_sequential_xmodes(problem: Problem, b: np.ndarray, pool=None, chunks=1) -> np.ndarray:
    """O1 for 2D problems with x periodic, mode by mode: u = A^{-1} b.

    K = I_y (x) K_x + K_y (x) I_x with a circulant K_x, so the naive DFT along x
    (exp(-2 pi i j x / nx)) turns A u = b into nx independent all-at-once
    systems, one per x-mode j, with K replaced by mu_j I + K_y, mu_j the
    eigenvalue of K_x for the mode exp(2 pi i j x / nx) (read off K_x's first
    row).  Each is solved by forward substitution in time with a dense LU with
    partial pivoting of its step matrix, then the modes are summed back by the
    inverse DFT.  The modes are independent, so they can be spread over the
    processes of ``pool`` (any object with a ``map``) in ``chunks`` shares; time
    stays sequential within each mode.  b, u of shape (Nt, S).
    """
    sp = problem.space
    if sp.dim != 2 or sp.bc_x != PERIODIC:
        raise ValueError("solve_sequential_xmodes needs a 2D problem with x periodic")
    nx, ny = sp.nx, sp.ny
    Kx = stencil_1d(nx, sp.hx, sp.nu, sp.ax, sp.bc_x).toarray()
    Ky = stencil_1d(ny, sp.hy, sp.nu, sp.ay, sp.bc_y).toarray()
    x = np.arange(nx)
    mu = [(j, complex(Kx[0] @ np.exp(2j * np.pi * j * x / nx))) for j in range(nx)]
    c1, c2 = first_columns(problem)
    nt = b.shape[0]
    band = [m for m in range(1, nt) if c1[m] != 0.0 or c2[m] != 0.0]
    b3 = np.asarray(b, dtype=np.float64).reshape(nt, ny, nx)
    shares = [mu[i::chunks] for i in range(chunks)]
    args = [(c1, c2, band, Ky, share, b3) for share in shares if share]
    parts = list(pool.map(_xmode_chunk, args)) if pool is not None else [_xmode_chunk(a) for a in args]
    return np.sum(parts, axis=0).reshape(nt, ny * nx)
