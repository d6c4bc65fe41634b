"""O8: windowing (Sections 2.1.1 and 2.2; for nonlinear problems Section 1):
a long horizon as consecutive time windows, each solved exactly, window w
starting from the last time level of window w-1.

With exact window solves the windowed solution is the time-stepping solution
over the whole horizon; the GPU library solves each window by ParaDiag.
Test infrastructure only; shares no code with the CUDA library.
"""
from __future__ import annotations

import numpy as np

from workloads import GeometricProblem, Problem

from . import nonlinear as NL
from . import operators as O
from . import paradiag1 as P1
from . import stepping as ST


def windows_theta(problem: Problem, u0, nwin: int, f=None, K=None) -> np.ndarray:
    """Uniform-step theta-method windows; f of shape (nwin Nt + 1, S) or None.
    Returns U of shape (nwin, Nt, S)."""
    K = O.stencil(problem.space) if K is None else K
    nt, S = problem.nt, problem.space.size
    out = np.zeros((nwin, nt, S))
    start = np.asarray(u0, dtype=np.float64)
    for w in range(nwin):
        fw = None if f is None else np.asarray(f)[w * nt : w * nt + nt + 1]
        b = O.build_rhs(problem, start, None, fw, K)
        out[w] = ST.solve_sequential(problem, b, K)
        start = out[w, -1]
    return out


def windows_geometric(problem: GeometricProblem, u0, nwin: int, f=None, K=None) -> np.ndarray:
    """ParaDiag-I windows with the geometric steps of eq. 2.8 repeated in every
    window; f of shape (nwin Nt + 1, S) at the time points of all windows."""
    K = O.stencil(problem.space) if K is None else K
    nt, S = problem.nt, problem.space.size
    out = np.zeros((nwin, nt, S))
    start = np.asarray(u0, dtype=np.float64)
    for w in range(nwin):
        fw = None if f is None else np.asarray(f)[w * nt : w * nt + nt + 1]
        b = P1.build_rhs(problem, start, fw, K)
        out[w] = P1.solve_sequential(problem, b, K)
        start = out[w, -1]
    return out


def windows_nl(problem: Problem, u0, nwin: int, a, f=None, K=None) -> np.ndarray:
    """Nonlinear theta-method windows (eq. 1.4 in each window, O10's exact
    stepping with Newton per step); f of shape (nwin Nt + 1, S) or None.
    Returns U of shape (nwin, Nt, S)."""
    K = O.stencil(problem.space) if K is None else K
    nt, S = problem.nt, problem.space.size
    out = np.zeros((nwin, nt, S))
    start = np.asarray(u0, dtype=np.float64)
    for w in range(nwin):
        fw = None if f is None else np.asarray(f)[w * nt : w * nt + nt + 1]
        b = NL.build_rhs_nl(problem, start, a, f=fw, K=K)
        out[w] = NL.solve_sequential_nl(problem, b, a, K=K)
        start = out[w, -1]
    return out

