"""Pins of O8, windowing (CPU only): windows of uniform theta-method steps equal
one long-horizon stepping solve; windows of geometric steps reproduce the
per-mode amplification product over all windows."""
import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as CF
from oracle import operators as O
from oracle import paradiag1 as P1
from oracle import stepping as ST
from oracle import windows as WIN


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_theta_windows_equal_one_long_solve(scheme):
    sp = W.Space(dim=1, nx=24, nu=0.05, ax=0.7, bc_x=W.PERIODIC)
    nt, nwin, dt = 8, 4, 0.02
    pb = W.Problem(space=sp, nt=nt, dt=dt, scheme=scheme, alpha=0.1)
    pl = W.Problem(space=sp, nt=nt * nwin, dt=dt, scheme=scheme, alpha=0.1)
    u0 = W.uniform(W.SEED_BASE + 98, 24, -1, 1)
    f = W.uniform(W.SEED_BASE + 99, (nt * nwin + 1) * 24, -1, 1).reshape(-1, 24)
    U = WIN.windows_theta(pb, u0, nwin, f)
    ref = ST.solve_sequential(pl, O.build_rhs(pl, u0, None, f))
    assert np.abs(U.reshape(nt * nwin, 24) - ref).max() < 1e-13


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_geometric_windows_mode_amplification(scheme):
    n, j = 16, 3
    sp = W.Space(dim=1, nx=n, nu=0.05, ax=1.3, bc_x=W.PERIODIC)
    pb = W.GeometricProblem(space=sp, nt=6, dt_last=0.05, tau=1.3, scheme=scheme)
    v = np.exp(2j * np.pi * j * np.arange(n) / n)
    mu = CF.mu_periodic(n, sp.hx, 0.05, 1.3)[j]
    U = WIN.windows_geometric(pb, v.real, 3)
    R = CF.stability_function(P1.geometric_steps(6, 0.05, 1.3) * mu, P1.theta_of(scheme))
    amp = np.cumprod(np.tile(R, 3))
    ref = np.real(np.outer(amp, v))
    assert np.abs(U.reshape(18, n) - ref).max() < 1e-13


def test_nonlinear_windows_equal_long_horizon_stepping():
    # nonlinear windows solved exactly chain into the one-window stepping
    # solution over the whole horizon (the windows only cut the all-at-once
    # system; each step's equation is unchanged)
    from oracle import nonlinear as NL
    a = (-1.0, 0.5, 1.0)
    nwin, nt = 3, 8
    sp = W.Space(dim=1, nx=31, nu=1e-2, ax=0.5, bc_x=W.PERIODIC)
    pw = W.Problem(space=sp, nt=nt, dt=1.0 / 32, scheme=W.CN, alpha=1e-2)
    pl = W.Problem(space=sp, nt=nwin * nt, dt=1.0 / 32, scheme=W.CN, alpha=1e-2)
    u0 = np.sin(2 * np.pi * sp.xs())
    f = W.uniform(W.SEED_BASE + 430, (nwin * nt + 1) * 31, -1, 1).reshape(-1, 31)
    Uw = WIN.windows_nl(pw, u0, nwin, a, f)
    Ul = NL.solve_sequential_nl(pl, NL.build_rhs_nl(pl, u0, a, f=f), a)
    assert np.abs(Uw.reshape(nwin * nt, -1) - Ul).max() <= 1e-12 * np.abs(Ul).max()
