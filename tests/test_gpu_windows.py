"""GPU windowing (pd_solve_windows, pd1_solve_windows) against the oracle's
windowed stepping (O8).  Each window is a ParaDiag solve to a relative
residual of 1e-12 (ParaDiag-II) or a refined ParaDiag-I solve; the windows are
chained on the device.  Tolerance 1e-10 relative to max|u| over all windows."""
import numpy as np
import pytest

import workloads as W
from helpers import dev, host, lib_ready, make_plan, space_dict
from oracle import windows as WIN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_paradiag2_windows(pd, prec, scheme):
    sp = W.Space(dim=1, nx=63, nu=1e-2, ax=1.0, bc_x=W.PERIODIC)
    pb = W.Problem(space=sp, nt=32, dt=1.0 / 64, scheme=scheme, alpha=1e-2)
    nwin = 4
    u0 = np.sin(2 * np.pi * sp.xs())
    f = W.uniform(W.SEED_BASE + 400, (32 * nwin + 1) * 63, -1, 1).reshape(-1, 63)
    ref = WIN.windows_theta(pb, u0, nwin, f)
    plan = make_plan(pb, prec)
    u, it, rel = plan.solve_windows(dev(u0), nwin, dev(f), tol=1e-12, maxit=30)
    assert rel <= 1e-12 and it >= nwin
    assert np.abs(host(u) - ref).max() <= 1e-10 * np.abs(ref).max()
    plan.close()


def test_paradiag2_windows_2d(pd):
    sp = W.Space(dim=2, nx=33, ny=20, nu=1e-2, ax=1.0, ay=0.5, bc_x=W.PERIODIC)
    pb = W.Problem(space=sp, nt=16, dt=1.0 / 32, scheme=W.CN, alpha=1e-3)
    u0 = W.uniform(W.SEED_BASE + 401, sp.size, -1, 1)
    ref = WIN.windows_theta(pb, u0, 3)
    plan = make_plan(pb, 1)
    u, it, rel = plan.solve_windows(dev(u0), 3, tol=1e-12, maxit=30)
    assert np.abs(host(u) - ref).max() <= 1e-10 * np.abs(ref).max()
    plan.close()


def test_leapfrog_windows_unsupported(pd):
    sp = W.Space(dim=1, nx=31, nu=1.0)
    pb = W.Problem(space=sp, nt=16, dt=0.05, scheme=W.LEAPFROG, alpha=0.1)
    plan = make_plan(pb, 1)
    with pytest.raises(pd.PDError):
        plan.solve_windows(dev(np.zeros(31)), 2)
    plan.close()


@pytest.mark.parametrize("prec,scheme", [(0, W.CN), (0, W.BE), (1, W.BE)])
def test_paradiag1_windows_paper_figure(pd, prec, scheme):
    # the windowing figure: 5 windows of Nt = 32, tau = 1.16, dt_Nt = 0.05,
    # nu = 1e-3, periodic (-1, 1), u0 = exp(-30 x^2), trapezoidal rule as in the
    # figure (and backward Euler); every window refined to relres 1e-13 (the
    # direct FP64 solve alone carries ~1e-3 with the trapezoidal rule).  The
    # mixed path runs backward Euler only: with the trapezoidal rule
    # Cond(V D~) ~ 4e12 and the FP32 sweeps do not reach 1e-13.
    wl = W.pd1_ade1d(scheme=scheme)
    pb = wl.problem
    ref = WIN.windows_geometric(pb, wl.u0, 5)
    plan = pd.Plan1(space_dict(pb.space), pb.nt, pb.dt_last, pb.tau,
                    0 if scheme == W.BE else 1, True, prec)
    u, it, rel = plan.solve_windows(dev(wl.u0), 5, tol=1e-13, max_refine=20)
    assert rel <= 1e-13
    assert np.abs(host(u) - ref).max() <= 1e-10 * np.abs(ref).max()
    plan.close()
