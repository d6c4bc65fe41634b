"""The allocation-free preconditioner entry point (pd_apply_precond_noalloc).

Some callers cannot call cudaMalloc: code that runs while an application's
memory pool is frozen, plug-ins whose host application owns every device
allocation, or code inside a region where allocation is not allowed.  They
cannot create a plan, which allocates its tables and workspace.  This entry
point applies z = P_alpha^{-1} r for 1D Dirichlet problems using only a fixed
device array inside the library.

Checked here, through the C ABI:
  * on two calls in a row (the second reusing the array the first left
    behind), it agrees with the plan-based pd_apply_precond within the
    preconditioner tolerance of the parity tests (64 eps32 kappa / alpha), for
    every time scheme: backward Euler, Crank-Nicolson, the theta-method with
    theta = 0.7 and leap-frog (band 2);
  * at the largest Nt it accepts (4096) it agrees with the oracle's naive
    ParaDiag (O2) directly;
  * Nt = 8192 and nx = 5000 are rejected as unsupported, a problem too large
    for the array is rejected with the size it needs, and a NaN in r is
    reported as PD_ERR_NONFINITE.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from helpers import EPS32, SCHEME_TO_PD, dev, host, lib_ready, make_plan, relerr
from oracle import closed_forms as CF
from oracle import operators as O
from oracle import paradiag as PD

pytestmark = pytest.mark.gpu


def _kappa(pb):
    K = O.stencil(pb.space).toarray()
    l1, l2 = CF.lemma1_eigenvalues(pb)
    I = np.eye(K.shape[0])
    return max(np.linalg.cond(l1[k] * I + l2[k] * K) for k in range(pb.nt // 2 + 1))


def _noalloc(pd, pb, r_dev, z_dev):
    import torch
    sp = pb.space
    space = pd.pd_space(1, sp.nx, 1, sp.nu, sp.ax, 0.0, pd.PD_DIRICHLET, pd.PD_DIRICHLET,
                        sp.lx, 1.0)
    st, need = pd.pd_apply_precond_noalloc(space, pb.nt, pb.dt, pb.alpha,
                                           SCHEME_TO_PD[pb.scheme], pb.theta_eff,
                                           ctypes.c_void_p(r_dev.data_ptr()),
                                           ctypes.c_void_p(z_dev.data_ptr()),
                                           torch.cuda.current_stream().cuda_stream)
    return st, need


def _problem(nx, nt, scheme, alpha, nu=1e-2, ax=1.0, T=1.0, theta=1.0):
    sp = W.Space(dim=1, nx=nx, nu=nu, ax=ax, bc_x=W.DIRICHLET)
    return W.Problem(space=sp, nt=nt, dt=T / nt, scheme=scheme, alpha=alpha, theta=theta)


SCHEMES = {
    "be": lambda nx, nt: _problem(nx, nt, W.BE, 1e-2),
    "cn": lambda nx, nt: _problem(nx, nt, W.CN, 1e-2),
    "theta07": lambda nx, nt: _problem(nx, nt, W.THETA, 1e-2, theta=0.7),
    "leapfrog": lambda nx, nt: _problem(nx, nt, W.LEAPFROG, 0.1, nu=1.0, ax=0.0, T=2.0),
}


@pytest.mark.parametrize("scheme", sorted(SCHEMES))
def test_noalloc_matches_plan_on_two_calls(scheme):
    import torch
    pd = lib_ready()
    problems = [SCHEMES[scheme](300, 128), SCHEMES[scheme](127, 64)]   # larger first
    for i, pb in enumerate(problems):
        r = W.uniform(W.SEED_BASE + 100 + i, pb.unknowns, -1.0, 1.0).reshape(pb.nt, -1)
        rd = dev(r)
        zn = torch.full_like(rd, float("nan"))
        st, need = _noalloc(pd, pb, rd, zn)
        assert st == pd.PD_OK, (st, need)
        assert 0 < need <= (8 << 20)
        plan = make_plan(pb, pd.PD_MIXED)
        zp = host(plan.apply_precond(rd))
        plan.close()
        tol = 64 * EPS32 * _kappa(pb) / pb.alpha
        err = relerr(host(zn), zp)
        print(f"NOALLOC {scheme} call={i} vs plan err={err:.3e} tol={tol:.3e}")
        assert err <= tol


def test_noalloc_largest_nt_matches_oracle():
    import torch
    pd = lib_ready()
    pb = _problem(15, 4096, W.BE, 1e-2, nu=0.1)
    r = W.uniform(W.SEED_BASE + 110, pb.unknowns, -1.0, 1.0).reshape(pb.nt, -1)
    zref = PD.precond_apply(pb, r)
    rd = dev(r)
    z = torch.full_like(rd, float("nan"))
    st, need = _noalloc(pd, pb, rd, z)
    assert st == pd.PD_OK, (st, need)
    tol = 64 * EPS32 * _kappa(pb) / pb.alpha
    err = relerr(host(z), zref)
    print(f"NOALLOC nt=4096 vs O2 err={err:.3e} tol={tol:.3e}")
    assert err <= tol


def test_noalloc_rejections():
    import torch
    pd = lib_ready()
    rd = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    st, _ = _noalloc(pd, _problem(15, 8192, W.BE, 1e-2), rd, rd)
    assert st == pd.PD_ERR_UNSUPPORTED
    st, _ = _noalloc(pd, _problem(5000, 64, W.BE, 1e-2), rd, rd)
    assert st == pd.PD_ERR_UNSUPPORTED
    st, need = _noalloc(pd, _problem(4096, 1024, W.BE, 1e-2), rd, rd)  # ~16.8 MB > 8 MiB
    assert st == pd.PD_ERR_ARG
    assert need > (8 << 20)


def test_noalloc_reports_nonfinite_input():
    import torch
    pd = lib_ready()
    pb = _problem(63, 32, W.BE, 1e-2)
    r = W.uniform(W.SEED_BASE + 120, pb.unknowns, -1.0, 1.0).reshape(pb.nt, -1)
    r[5, 7] = np.nan
    rd = dev(r)
    z = torch.empty_like(rd)
    st, _ = _noalloc(pd, pb, rd, z)
    assert st == pd.PD_ERR_NONFINITE
    # the next call on clean data succeeds: the status word is cleared per call
    r[5, 7] = 0.0
    st, _ = _noalloc(pd, pb, dev(r), z)
    assert st == pd.PD_OK
