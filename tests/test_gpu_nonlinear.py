"""GPU nonlinear solves (pd_nl_build_rhs, pd_nl_residual, pd_nl_solve: the
simplified Newton iteration of eq. 1.5 with the averaged Jacobian) against the
nonlinear oracle (O10).

  * right-hand side and residual: FP64 parity with the oracle to 1e-13
    (relative to the largest entry), the double-float residual of mixed plans
    to 1e-12; the averaged shift sigma and ||r||^2, summed in FP32, to 1e-5;
  * solves (FP64 and mixed plans) to a relative residual of 1e-11 equal the
    exact solution (sequential stepping with Newton per step) to 1e-9 of
    max|u|; on FP64 plans the number of corrections matches the oracle's
    simplified Newton within one;
  * the manufactured solution exp(-t) sin(pi x) is reproduced with the
    oracle's discretisation error;
  * the plan's linear solve is unchanged after a nonlinear solve (its
    eigenvalue table is restored); bad arguments are rejected;
  * the full 255 x 255 x 256 bench workload: the GPU iterate's residual,
    recomputed by the oracle, meets the tolerance.
"""
import numpy as np
import pytest

import workloads as W
from helpers import dev, host, lib_ready, make_plan
from oracle import nonlinear as NL

pytestmark = pytest.mark.gpu

PD_FP64, PD_MIXED = 0, 1

CASES = {
    "2d_cn_bistable": (W.nl_ade2d(nx=15, ny=13, nt=16, nu=1e-2, alpha=1e-2,
                                  reaction=(-1.0, 0.0, 1.0)), None),
    "2d_be_cubic": (W.nl_ade2d(nx=33, ny=20, nt=32, nu=1e-2, scheme=W.BE, alpha=1e-2,
                               reaction=(0.0, 0.0, 1.0)), None),
    "1d_cn_manufactured": (W.nl_manufactured1d(nx=63, nt=32), "f"),
    "1d_cn_nt12": (W.nl_manufactured1d(nx=40, nt=12, reaction=(0.3, -0.5, 1.0)), "f"),
    "1d_theta07": (W.nl_manufactured1d(nx=50, nt=20, scheme=W.THETA, theta=0.7), "f"),
}


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


def data(name):
    wl, use_f = CASES[name]
    return wl, wl.problem, wl.extra["reaction"], (wl.f if use_f else None)


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_residual_sigma_match_oracle(pd, name):
    wl, pb, a, f = data(name)
    plan = make_plan(pb, PD_FP64)
    bref = NL.build_rhs_nl(pb, wl.u0, a, f=f)
    b = plan.nl_build_rhs(a, dev(wl.u0), None if f is None else dev(f))
    assert np.abs(host(b) - bref).max() <= 1e-13 * np.abs(bref).max()
    U = W.uniform(W.SEED_BASE + 410, pb.unknowns, -1, 1).reshape(pb.nt, -1)
    rref = NL.residual_nl(pb, U, bref, a)
    r, sig, rn2 = plan.nl_residual(a, dev(bref), dev(U))
    assert np.abs(host(r) - rref).max() <= 1e-13 * np.abs(rref).max()
    # sigma and ||r||^2 are summed in FP32 (a shift and a stopping test need a
    # few digits; r itself is FP64)
    assert sig == pytest.approx(NL.average_jacobian_shift(U, a), rel=1e-5, abs=1e-6)
    assert rn2 == pytest.approx(float(np.sum(rref * rref)), rel=1e-5)
    plan.close()
    # mixed plans form the same residual in double-float arithmetic (unit
    # roundoff ~2^-48 against the largest term, here within 1e-12 of max |r|)
    pm = make_plan(pb, PD_MIXED)
    rm, sigm, _ = pm.nl_residual(a, dev(bref), dev(U))
    assert np.abs(host(rm) - rref).max() <= 1e-12 * np.abs(rref).max()
    assert sigm == pytest.approx(NL.average_jacobian_shift(U, a), rel=1e-5, abs=1e-6)
    pm.close()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", [PD_FP64, PD_MIXED])
def test_solve_matches_exact(pd, name, prec):
    wl, pb, a, f = data(name)
    b = NL.build_rhs_nl(pb, wl.u0, a, f=f)
    exact = NL.solve_sequential_nl(pb, b, a)
    plan = make_plan(pb, prec)
    u, it, rel = plan.nl_solve(a, dev(b), tol=1e-11, maxit=80)
    assert rel <= 1e-11
    assert np.abs(host(u) - exact).max() <= 1e-9 * np.abs(exact).max()
    if prec == PD_FP64:
        _, it_ref, _ = NL.simplified_newton(pb, b, a, tol=1e-11)
        assert abs(it - it_ref) <= 1, (it, it_ref)
    plan.close()


def test_manufactured_error(pd):
    wl, pb, a, f = data("1d_cn_manufactured")
    b = NL.build_rhs_nl(pb, wl.u0, a, f=f)
    err_ref = np.abs(NL.solve_sequential_nl(pb, b, a) - wl.extra["exact"]).max()
    plan = make_plan(pb, PD_MIXED)
    bg = plan.nl_build_rhs(a, dev(wl.u0), dev(f))
    u, it, rel = plan.nl_solve(a, bg, tol=1e-12, maxit=80)
    err = np.abs(host(u) - wl.extra["exact"]).max()
    assert abs(err - err_ref) <= 1e-3 * err_ref
    plan.close()


def test_linear_solve_unchanged_after_nonlinear(pd):
    wl, pb, a, f = data("2d_cn_bistable")
    plan = make_plan(pb, PD_MIXED)
    rng_b = W.uniform(W.SEED_BASE + 411, pb.unknowns, -1, 1).reshape(pb.nt, -1)
    u1, it1, rel1 = plan.solve(dev(rng_b), tol=1e-12)
    plan.nl_solve(a, dev(NL.build_rhs_nl(pb, wl.u0, a)), tol=1e-10, maxit=80)
    u2, it2, rel2 = plan.solve(dev(rng_b), tol=1e-12)
    assert it1 == it2
    assert np.array_equal(host(u1), host(u2))
    plan.close()


def test_arguments_rejected(pd):
    wl, pb, a, f = data("2d_cn_bistable")
    plan = make_plan(pb, PD_FP64)
    b = dev(NL.build_rhs_nl(pb, wl.u0, a))
    with pytest.raises(pd.PDError):
        plan.nl_solve((0.0, float("nan"), 1.0), b)
    with pytest.raises(pd.PDError):
        plan.nl_solve(a, b, tol=-1.0)
    plan.close()
    sp = W.Space(dim=1, nx=31, nu=1.0)
    lf = make_plan(W.Problem(space=sp, nt=16, dt=0.05, scheme=W.LEAPFROG, alpha=0.1), PD_FP64)
    with pytest.raises(pd.PDError):
        lf.nl_solve(a, dev(np.zeros((16, 31))))
    lf.close()


def test_not_converged_status(pd):
    wl, pb, a, f = data("2d_cn_bistable")
    plan = make_plan(pb, PD_FP64)
    b = dev(NL.build_rhs_nl(pb, wl.u0, a))
    u, it, rel = plan.nl_solve(a, b, tol=1e-14, maxit=2, allow_not_converged=True)
    assert it == 2 and rel > 1e-14
    with pytest.raises(pd.PDError):
        plan.nl_solve(a, b, tol=1e-14, maxit=2)
    plan.close()


def test_full_size_bench_workload(pd):
    import torch
    wl = W.nl_ade2d()
    pb, a = wl.problem, wl.extra["reaction"]
    plan = make_plan(pb, PD_MIXED)
    b = plan.nl_build_rhs(a, dev(wl.u0))
    u, it, rel = plan.nl_solve(a, b, tol=1e-10, maxit=80)
    assert rel <= 1e-10
    bh = host(b)
    r = NL.residual_nl(pb, host(u), bh, a)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bh)
    # the right-hand side against the oracle's
    bref = NL.build_rhs_nl(pb, wl.u0, a)
    assert np.abs(bh - bref).max() <= 1e-13 * np.abs(bref).max()
    plan.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", [PD_FP64, PD_MIXED])
def test_windows_bistable_match_oracle(pd, prec):
    # the bistable reaction phi = u^3 - u over T = 1 diverges as one window
    # (the averaged Jacobian's contraction grows with the window length) and
    # converges in four windows of T = 0.25; the windows equal the oracle's
    # exact windows (stepping with Newton per step)
    from oracle import windows as WIN
    a = (-1.0, 0.0, 1.0)
    nwin = 4
    wl = W.nl_ade2d(nx=15, ny=13, nt=16, T=0.25, nu=1e-3, alpha=1e-2, reaction=a)
    pb = wl.problem
    ref = WIN.windows_nl(pb, wl.u0, nwin, a)
    plan = make_plan(pb, prec)
    u, it, rel = plan.nl_solve_windows(a, dev(wl.u0), nwin, tol=1e-11, maxit=80)
    assert rel <= 1e-11 and it >= nwin
    assert np.abs(host(u) - ref).max() <= 1e-9 * np.abs(ref).max()
    plan.close()


def test_windows_with_source_match_oracle(pd):
    from oracle import windows as WIN
    a = (0.3, -0.5, 1.0)
    nwin, nt = 3, 12
    sp = W.Space(dim=1, nx=40, nu=1e-2, ax=0.5, bc_x=W.PERIODIC)
    pb = W.Problem(space=sp, nt=nt, dt=1.0 / 36, scheme=W.CN, alpha=1e-2)
    u0 = np.sin(2 * np.pi * sp.xs())
    f = W.uniform(W.SEED_BASE + 431, (nwin * nt + 1) * 40, -1, 1).reshape(-1, 40)
    ref = WIN.windows_nl(pb, u0, nwin, a, f)
    plan = make_plan(pb, PD_MIXED)
    u, it, rel = plan.nl_solve_windows(a, dev(u0), nwin, dev(f), tol=1e-12, maxit=80)
    assert rel <= 1e-12
    assert np.abs(host(u) - ref).max() <= 1e-10 * np.abs(ref).max()
    plan.close()
