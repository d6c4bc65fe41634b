"""GPU parity of ParaDiag-I with the hybrid midpoint + backward-Euler
discretisation (Section 2.1.2) against the oracle (O7), through the C ABI.

The plan finds the eigenvalues by a fixed point on the angle form of the
characteristic equation plus Newton steps, and V^{-1} from closed-form left
eigenvectors; the oracle uses Newton from library eigenvalues and a dense LU
for V^{-1}, so the two share no step.  Tolerances as for the geometric-step
variant: the direct FP64 solve within 10 Nt eps Cond(V) max|u| (+1e-12 max|u|
for step (b)) of the exact solution (sparse LU of the whole system) and within
twice that of the oracle's direct solve; the FP32 direct solve within
8 Nt eps32 Cond(V) max|u|; refined solves to a relative residual of 1e-13 and
1e-10 of the exact solution.
"""
import numpy as np
import pytest

import workloads as W
from helpers import EPS32, dev, host, lib_ready, space_dict
from oracle import hybrid as H

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53
PD_FP64, PD_MIXED = 0, 1


def HP(dim=1, nx=31, ny=1, nu=0.02, ax=0.0, ay=0.0, bcx=W.DIRICHLET, nt=16, T=0.5, lx=1.0):
    sp = W.Space(dim=dim, nx=nx, ny=ny, nu=nu, ax=ax, ay=ay, bc_x=bcx, lx=lx)
    return W.HybridProblem(space=sp, nt=nt, dt=T / nt)


CASES = {
    "1d_dirichlet_adv_31x16": HP(nx=31, nu=0.02, ax=1.0, nt=16),
    "1d_periodic_paper_256x64": W.hybrid_ade1d().problem,
    "1d_odd_nt_45x33": HP(nx=45, nu=0.05, ax=0.5, nt=33),
    "1d_nt1": HP(nx=20, nu=0.1, nt=1, T=0.01),
    "1d_nt2": HP(nx=20, nu=0.1, nt=2, T=0.02),
    "1d_nt3": HP(nx=130, nu=0.1, ax=1.0, nt=3, T=0.03),
    "1d_nt300_127": HP(nx=127, nu=1e-2, ax=1.0, nt=300, T=1.0),
    "2d_xper_33x20x40": HP(dim=2, nx=33, ny=20, nu=1e-2, ax=1.0, ay=0.5, bcx=W.PERIODIC, nt=40),
    "2d_xdir_17x15x9": HP(dim=2, nx=17, ny=15, nu=0.05, ay=0.3, nt=9),
}


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


def make(pb, precision):
    import paradiag_gb300 as pd
    return pd.PlanHybrid(space_dict(pb.space), pb.nt, pb.dt, precision)


def data(pb, seed):
    S = pb.space.size
    u0 = W.uniform(seed, S, -1, 1)
    f = W.uniform(seed + 1, (pb.nt + 1) * S, -1, 1).reshape(pb.nt + 1, S)
    return u0, f


def cond_v(pb):
    return np.linalg.cond(H.eigvec_matrix(H.eigen_roots(pb.nt)))


@pytest.mark.parametrize("name", sorted(CASES))
def test_hybrid_eigenvalues_match_oracle(pd, name):
    pb = CASES[name]
    plan = make(pb, PD_FP64)
    lam = np.array(plan.eigenvalues())
    ref = H.eigenvalues(pb)
    # match every GPU eigenvalue to its nearest oracle eigenvalue (a bijection)
    d = np.abs(lam[:, None] - ref[None, :])
    j = d.argmin(axis=1)
    assert len(set(j.tolist())) == pb.nt
    assert np.max(d[np.arange(pb.nt), j]) <= 1e-9 * np.abs(ref).max()
    assert plan.condition() >= 0.99 * cond_v(pb)
    plan.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_hybrid_direct_fp64_matches_oracle(pd, name):
    pb = CASES[name]
    u0, f = data(pb, W.SEED_BASE + 300)
    b = H.build_rhs(pb, u0, f)
    exact = H.solve_exact(pb, b)
    ref = H.solve_direct(pb, b)
    plan = make(pb, PD_FP64)
    u, it, _ = plan.solve(dev(b))
    assert it == 0
    ug = host(u)
    scale = np.abs(exact).max()
    bound = 10 * pb.nt * EPS64 * cond_v(pb) * scale + 1e-12 * scale
    assert np.abs(ug - exact).max() <= bound
    assert np.abs(ug - ref).max() <= 2 * bound
    plan.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_hybrid_mixed_direct_within_fp32_bound(pd, name):
    pb = CASES[name]
    u0, f = data(pb, W.SEED_BASE + 301)
    b = H.build_rhs(pb, u0, f)
    exact = H.solve_exact(pb, b)
    plan = make(pb, PD_MIXED)
    u, _, _ = plan.solve(dev(b))
    scale = np.abs(exact).max()
    assert np.abs(host(u) - exact).max() <= 8 * pb.nt * EPS32 * cond_v(pb) * scale
    plan.close()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", [PD_FP64, PD_MIXED])
def test_hybrid_refined_matches_exact(pd, name, prec):
    pb = CASES[name]
    u0, f = data(pb, W.SEED_BASE + 302)
    b = H.build_rhs(pb, u0, f)
    exact = H.solve_exact(pb, b)
    plan = make(pb, prec)
    u, it, rel = plan.solve(dev(b), tol=1e-13, max_refine=20)
    assert rel <= 1e-13
    ug = host(u)
    assert np.abs(ug - exact).max() <= 1e-10 * np.abs(exact).max()
    r = b - H.apply_A(pb, ug)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 4 * max(rel, 1e-15) + 1e-14
    plan.close()


@pytest.mark.parametrize("name", ["1d_dirichlet_adv_31x16", "1d_periodic_paper_256x64",
                                  "2d_xper_33x20x40", "1d_nt1"])
def test_hybrid_apply_A_and_rhs_match_oracle(pd, name):
    pb = CASES[name]
    u0, f = data(pb, W.SEED_BASE + 303)
    plan = make(pb, PD_FP64)
    bg = host(plan.build_rhs(dev(u0), dev(f)))
    br = H.build_rhs(pb, u0, f)
    assert np.abs(bg - br).max() <= 1e-13 * np.abs(br).max()
    assert np.abs(host(plan.build_rhs(dev(u0))) - H.build_rhs(pb, u0)).max() <= \
        1e-13 * np.abs(br).max()
    U = W.uniform(W.SEED_BASE + 304, pb.nt * pb.space.size, -1, 1).reshape(pb.nt, -1)
    yg = host(plan.apply_A(dev(U)))
    yr = H.apply_A(pb, U)
    assert np.abs(yg - yr).max() <= 1e-13 * np.abs(yr).max()
    plan.close()


def test_hybrid_full_size_window(pd):
    # the benchmark's hybrid workload: 255 x 255 grid, Nt = 256, T = 1,
    # mixed precision with refinement, checked by an independent FP64 residual
    import torch
    wl = W.hybrid_ade2d()
    pb = wl.problem
    plan = make(pb, PD_MIXED)
    bd = plan.build_rhs(dev(wl.u0))
    u, it, rel = plan.solve(bd, tol=1e-12, max_refine=20)
    assert rel <= 1e-12
    r = bd - plan.apply_A(u)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(bd)) <= 2e-12
    plan.close()
