"""GPU parity of ParaDiag-I with geometric time steps (Section 2.1.1) against
the oracle (O6), through the C ABI.

Tolerances.  The direct solve's roundoff grows like Cond_2(V) (Section
2.1.1); the oracle pin bounds the FP64 error against the exact solution
(sequential stepping) by Nt eps Cond(V~) max|u|, V~ = V D~.  The GPU FP64
solve is the same method in another summation order, so it stays within the
same bound of the exact solution, and within twice it of the oracle's direct
solve; a further 1e-12 max|u| covers the FP64 spatial solves of step (b).
The FP32 solve of the mixed path is bounded the same way with the FP32 unit
roundoff (8 Nt eps32 Cond(V~), the 8 for the FP16-split x-transform of 2D
problems).  Refined solves (residual in FP64 / double-float) must reach a
relative residual of 1e-13 and match the exact solution to 1e-10 relative.
The sweeps converge even where 8 Nt eps32 Cond(V~) exceeds one: the error
propagator of a sweep is dominated by a block lower-triangular (in time)
part, so after a transient the sweeps contract.
"""
import numpy as np
import pytest

import workloads as W
from helpers import EPS32, dev, host, lib_ready, space_dict
from oracle import paradiag1 as P1

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53
PD_BE, PD_CN, PD_FP64, PD_MIXED = 0, 1, 0, 1


def GP(dim=1, nx=15, ny=1, nu=0.05, ax=0.0, ay=0.0, bcx=W.DIRICHLET, nt=8, dt_last=0.05,
       tau=1.5, scheme=W.BE, scaled=True, lx=1.0):
    sp = W.Space(dim=dim, nx=nx, ny=ny, nu=nu, ax=ax, ay=ay, bc_x=bcx, lx=lx)
    return W.GeometricProblem(space=sp, nt=nt, dt_last=dt_last, tau=tau, scheme=scheme,
                              scaled=scaled)


CASES = {
    "1d_dirichlet_be_127x8": GP(nx=127, nu=0.02, ax=1.0, nt=8, tau=1.5),
    "1d_dirichlet_cn_200x20": GP(nx=200, nu=0.02, ax=1.0, nt=20, tau=1.3, scheme=W.CN),
    "1d_dirichlet_be_300x32_unscaled": GP(nx=300, nu=0.01, ax=0.5, nt=32, tau=1.16, scaled=False),
    "1d_periodic_be_128x12": GP(nx=128, nu=1e-2, ax=1.0, bcx=W.PERIODIC, lx=2.0, nt=12, tau=1.3),
    "1d_single_step": GP(nx=50, nu=0.1, nt=1, dt_last=0.02, tau=1.2),
    "2d_xper_be_33x20x16": GP(dim=2, nx=33, ny=20, nu=1e-2, ax=1.0, ay=0.5, bcx=W.PERIODIC,
                              nt=16, tau=1.3),
    "2d_xdir_cn_17x15x7": GP(dim=2, nx=17, ny=15, nu=0.05, ay=0.3, nt=7, tau=1.5, scheme=W.CN),
}


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


def make_plan1(pb, precision):
    import paradiag_gb300 as pd
    return pd.Plan1(space_dict(pb.space), pb.nt, pb.dt_last, pb.tau,
                    PD_BE if pb.scheme == W.BE else PD_CN, pb.scaled, precision)


def data(pb, seed):
    S = pb.space.size
    u0 = W.uniform(seed, S, -1, 1)
    f = W.uniform(seed + 1, (pb.nt + 1) * S, -1, 1).reshape(pb.nt + 1, S)
    return u0, f


def cond_v(pb):
    V, _ = P1.eigvec_matrices(pb.nt, pb.tau, P1.theta_of(pb.scheme), pb.scaled)
    return np.linalg.cond(V)


@pytest.mark.parametrize("name", sorted(CASES))
def test_pd1_direct_fp64_matches_oracle(pd, name):
    pb = CASES[name]
    u0, f = data(pb, W.SEED_BASE + 200)
    b = P1.build_rhs(pb, u0, f)
    ref = P1.solve_direct(pb, b)
    exact = P1.solve_sequential(pb, b)
    plan = make_plan1(pb, PD_FP64)
    u, it, _ = plan.solve(dev(b))
    assert it == 0
    ug = host(u)
    scale = np.abs(exact).max()
    bound = pb.nt * EPS64 * cond_v(pb) * scale + 1e-12 * scale
    assert np.abs(ug - exact).max() <= bound
    assert np.abs(ug - ref).max() <= 2 * bound
    plan.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_pd1_mixed_direct_within_fp32_bound(pd, name):
    pb = CASES[name]
    u0, f = data(pb, W.SEED_BASE + 201)
    b = P1.build_rhs(pb, u0, f)
    exact = P1.solve_sequential(pb, b)
    plan = make_plan1(pb, PD_MIXED)
    u, _, _ = plan.solve(dev(b))
    scale = np.abs(exact).max()
    assert np.abs(host(u) - exact).max() <= 8 * pb.nt * EPS32 * cond_v(pb) * scale
    plan.close()


REFINE = ["1d_dirichlet_be_127x8", "1d_dirichlet_cn_200x20", "1d_dirichlet_be_300x32_unscaled",
          "1d_periodic_be_128x12", "1d_single_step", "2d_xper_be_33x20x16",
          "2d_xdir_cn_17x15x7"]


@pytest.mark.parametrize("name", REFINE)
@pytest.mark.parametrize("prec", [PD_FP64, PD_MIXED])
def test_pd1_refined_matches_exact(pd, name, prec):
    pb = CASES[name]
    u0, f = data(pb, W.SEED_BASE + 202)
    b = P1.build_rhs(pb, u0, f)
    exact = P1.solve_sequential(pb, b)
    plan = make_plan1(pb, prec)
    u, it, rel = plan.solve(dev(b), tol=1e-13, max_refine=20)
    assert rel <= 1e-13
    ug = host(u)
    assert np.abs(ug - exact).max() <= 1e-10 * np.abs(exact).max()
    # the relative residual reported agrees with the oracle's operator
    r = b - P1.apply_A(pb, ug)
    rr = np.linalg.norm(r) / np.linalg.norm(b)
    assert rr <= 4 * max(rel, 1e-15) + 1e-14
    plan.close()


def test_pd1_refinement_removes_the_roundoff_of_the_paper_window(pd):
    # the windowing figure's window: Nt = 32, tau = 1.16, dt_Nt = 0.05, CN,
    # Cond(V~) ~ 1e12: the direct FP64 solve carries ~1e-4 of roundoff, which
    # FP64 residual sweeps remove
    wl = W.pd1_ade1d()
    pb = wl.problem
    b = P1.build_rhs(pb, wl.u0)
    exact = P1.solve_sequential(pb, b)
    scale = np.abs(exact).max()
    plan = make_plan1(pb, PD_FP64)
    u, _, rel0 = plan.solve(dev(b), tol=0.0, max_refine=0)
    e0 = np.abs(host(u) - exact).max() / scale
    assert e0 <= pb.nt * EPS64 * cond_v(pb)
    u, it, rel = plan.solve(dev(b), tol=1e-14, max_refine=10)
    e1 = np.abs(host(u) - exact).max() / scale
    assert rel <= 1e-14 and e1 <= 1e-11 and e1 < 1e-3 * e0, (e0, e1, it)
    plan.close()


@pytest.mark.parametrize("name", ["1d_dirichlet_cn_200x20", "1d_periodic_be_128x12",
                                  "2d_xper_be_33x20x16", "2d_xdir_cn_17x15x7"])
def test_pd1_apply_A_and_rhs_match_oracle(pd, name):
    pb = CASES[name]
    u0, f = data(pb, W.SEED_BASE + 203)
    plan = make_plan1(pb, PD_FP64)
    bg = host(plan.build_rhs(dev(u0), dev(f)))
    br = P1.build_rhs(pb, u0, f)
    assert np.abs(bg - br).max() <= 1e-13 * np.abs(br).max()
    assert np.abs(host(plan.build_rhs(dev(u0))) - P1.build_rhs(pb, u0)).max() <= \
        1e-13 * np.abs(br).max()
    U = W.uniform(W.SEED_BASE + 204, pb.nt * pb.space.size, -1, 1).reshape(pb.nt, -1)
    yg = host(plan.apply_A(dev(U)))
    yr = P1.apply_A(pb, U)
    assert np.abs(yg - yr).max() <= 1e-13 * np.abs(yr).max()
    plan.close()


def test_pd1_step_sizes_and_condition(pd):
    pb = CASES["1d_dirichlet_cn_200x20"]
    plan = make_plan1(pb, PD_FP64)
    d = np.array(plan.step_sizes())
    ref = P1.geometric_steps(pb.nt, pb.dt_last, pb.tau)
    assert np.abs(d - ref).max() <= 1e-15 * ref.max()
    assert plan.condition() >= 0.999 * cond_v(pb)
    plan.close()


def test_pd1_full_size_window(pd):
    # the 2D window measured by the benchmark: 255 x 255 grid, Nt = 32,
    # tau = 1.16, dt_Nt = 0.05, backward Euler, mixed precision with
    # refinement; checked by its FP64 residual (GPU apply_A, a separate kernel)
    # and against the exact solution at a sample of spatial points
    import torch
    wl = W.pd1_ade2d()
    pb = wl.problem
    plan = make_plan1(pb, PD_MIXED)
    bd = plan.build_rhs(dev(wl.u0))
    u, it, rel = plan.solve(bd, tol=1e-12, max_refine=20)
    assert rel <= 1e-12
    r = bd - plan.apply_A(u)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(bd)) <= 2e-12
    exact = P1.solve_sequential(pb, P1.build_rhs(pb, wl.u0))
    ug = host(u)
    idx = W.splitmix64(W.SEED_BASE + 205, 512) % np.uint64(pb.space.size)
    idx = idx.astype(np.int64)
    assert np.abs(ug[:, idx] - exact[:, idx]).max() <= 1e-10 * np.abs(exact).max()
    plan.close()
