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
from oracle.operators import stencil

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
    # tensor-core time contractions: K = Nt of 304 (ragged K chunk, two N
    # blocks), 131 points (ragged row block); 2D Dirichlet x with Nt = 64
    "1d_nt304_131": HP(nx=131, nu=1e-2, ax=1.0, nt=304, T=1.0),
    "2d_xdir_17x9x64": HP(dim=2, nx=17, ny=9, nu=0.05, ay=0.3, nt=64),
}

# cases whose mixed plan runs steps (a) and (c) on the tensor cores (mixed,
# Nt a multiple of 16 and at least 32, at least 128 spatial points)
TC_CASES = sorted(n for n, pb in CASES.items()
                  if pb.nt % 16 == 0 and pb.nt >= 32 and pb.space.size >= 128)


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


def make(pb, precision, tc=None):
    import paradiag_gb300 as pd
    plan = pd.PlanHybrid(space_dict(pb.space), pb.nt, pb.dt, precision)
    if tc is not None:
        plan.set_tensor_cores(tc)
    return plan


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


def test_hybrid_tensor_core_engine_selection(pd):
    import paradiag_gb300 as lib
    assert TC_CASES == ["1d_nt304_131", "1d_periodic_paper_256x64", "2d_xdir_17x9x64"]
    for name, pb in CASES.items():
        plan = make(pb, PD_MIXED)
        assert plan.tensor_cores == (name in TC_CASES)
        if name not in TC_CASES:
            with pytest.raises(lib.PDError) as e:
                plan.set_tensor_cores(True)
            assert e.value.status == lib.PD_ERR_UNSUPPORTED
        plan.set_tensor_cores(False)
        assert not plan.tensor_cores
        plan.close()
        p64 = make(pb, PD_FP64)
        assert not p64.tensor_cores
        p64.close()


@pytest.mark.parametrize("name", TC_CASES)
def test_hybrid_tensor_core_and_cuda_core_engines_agree(pd, name):
    """Direct mixed solves with either engine of the time contractions: both
    within the FP32 bound of the exact solution, and within twice that bound
    of each other; refined with either engine to the same residual."""
    pb = CASES[name]
    u0, f = data(pb, W.SEED_BASE + 305)
    b = H.build_rhs(pb, u0, f)
    exact = H.solve_exact(pb, b)
    scale = np.abs(exact).max()
    bound = 8 * pb.nt * EPS32 * cond_v(pb) * scale
    out = {}
    for tc in (True, False):
        plan = make(pb, PD_MIXED, tc)
        u, _, _ = plan.solve(dev(b))
        out[tc] = host(u)
        assert np.abs(out[tc] - exact).max() <= bound, tc
        u, it, rel = plan.solve(dev(b), tol=1e-13, max_refine=20)
        assert rel <= 1e-13
        assert np.abs(host(u) - exact).max() <= 1e-10 * scale
        plan.close()
    assert np.abs(out[True] - out[False]).max() <= 2 * bound


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
    assert plan.tensor_cores
    u, it, rel = plan.solve(bd, tol=1e-12, max_refine=20)
    assert rel <= 1e-12
    r = bd - plan.apply_A(u)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(bd)) <= 2e-12
    plan.close()


# ---- second-order problems (B_2nd = B^2) ----

WAVE = {
    "2d_dirichlet_15x15x16": W.HybridProblem(space=W.Space(dim=2, nx=15, ny=15, nu=1.0),
                                             nt=16, dt=2.0 / 16),
    "1d_dirichlet_63x33": W.HybridProblem(space=W.Space(dim=1, nx=63, nu=1.0), nt=33, dt=1.0 / 33),
    "2d_xper_33x20x8": W.HybridProblem(space=W.Space(dim=2, nx=33, ny=20, nu=0.5,
                                                     bc_x=W.PERIODIC), nt=8, dt=0.05),
    "1d_nt2": W.HybridProblem(space=W.Space(dim=1, nx=20, nu=1.0), nt=2, dt=0.1),
}


def make2(pb, precision):
    import paradiag_gb300 as pd
    return pd.PlanHybrid(space_dict(pb.space), pb.nt, pb.dt, precision, order=2)


def refine_tol(pb, b, exact, precision):
    """Residual tolerance the refinement can reach: the residual is formed in
    double-float (unit roundoff 2^-48) for the mixed path, so its floor is a few
    units times || |A| |u| || / || b ||, which B^2's (1/dt^2) entries make
    ~1e2..1e3 for these problems."""
    if precision == PD_FP64:
        return 1e-13
    K = stencil(pb.space)
    Au = np.abs(H.time_matrix_2nd(pb.nt, pb.dt)) @ np.abs(exact) + (abs(K) @ np.abs(exact).T).T
    return max(1e-13, 8 * 2.0 ** -48 * np.linalg.norm(Au) / np.linalg.norm(b))


@pytest.mark.parametrize("name", sorted(WAVE))
def test_wave_apply_and_rhs_match_oracle(pd, name):
    pb = WAVE[name]
    S = pb.space.size
    u0 = W.uniform(W.SEED_BASE + 310, S, -1, 1)
    v0 = W.uniform(W.SEED_BASE + 311, S, -1, 1)
    f = W.uniform(W.SEED_BASE + 312, (pb.nt + 1) * S, -1, 1).reshape(pb.nt + 1, S)
    plan = make2(pb, PD_FP64)
    br = H.build_rhs_2nd(pb, u0, v0, f)
    bg = host(plan.build_rhs_wave(dev(u0), dev(v0), dev(f)))
    assert np.abs(bg - br).max() <= 1e-13 * np.abs(br).max()
    U = W.uniform(W.SEED_BASE + 313, pb.nt * S, -1, 1).reshape(pb.nt, S)
    yr = H.apply_A_2nd(pb, U)
    assert np.abs(host(plan.apply_A(dev(U))) - yr).max() <= 1e-13 * np.abs(yr).max()
    plan.close()


@pytest.mark.parametrize("name", sorted(WAVE))
@pytest.mark.parametrize("prec", [PD_FP64, PD_MIXED])
def test_wave_solve_matches_exact(pd, name, prec):
    pb = WAVE[name]
    S = pb.space.size
    b = H.build_rhs_2nd(pb, W.uniform(W.SEED_BASE + 314, S, -1, 1),
                        W.uniform(W.SEED_BASE + 315, S, -1, 1),
                        W.uniform(W.SEED_BASE + 316, (pb.nt + 1) * S, -1, 1).reshape(pb.nt + 1, S))
    exact = H.solve_exact_2nd(pb, b)
    plan = make2(pb, prec)
    u, it, _ = plan.solve(dev(b))
    cond = cond_v(pb)
    scale = np.abs(exact).max()
    eps = EPS64 if prec == PD_FP64 else EPS32
    assert np.abs(host(u) - exact).max() <= 16 * pb.nt * eps * cond * scale + 1e-12 * scale
    tol = refine_tol(pb, b, exact, prec)
    u, it, rel = plan.solve(dev(b), tol=tol, max_refine=20)
    assert rel <= tol
    assert np.abs(host(u) - exact).max() <= 1e-10 * scale
    plan.close()


@pytest.mark.parametrize("nt", [16, 64])
def test_wave_table_ex2tab1_errors(pd, nt):
    # the errors of Table Ex2Tab1 (2D wave equation, T = 2), GPU mixed solve
    # refined to a 1e-10 residual on a 31 x 31 grid (the spatial discretisation is exact
    # for the solution's spatial factor)
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "ex2tab1_wave_hybrid.json")))
    err_ref = dict(zip(gold["nt"], gold["error"]))[nt]
    wl = W.hybrid_wave2d(n=32, nt=nt)
    pb = wl.problem
    plan = make2(pb, PD_MIXED)
    b = plan.build_rhs_wave(dev(wl.u0), dev(wl.u1), dev(wl.f))
    u, it, rel = plan.solve(b, tol=1e-10, max_refine=20)
    t = pb.dt * np.arange(1, nt + 1)
    err = np.abs(host(u) - np.outer(np.sin(2 * np.pi * t), wl.extra["phi"])).max()
    assert abs(err - err_ref) <= 0.01 * err_ref, (nt, err, err_ref)
    plan.close()
