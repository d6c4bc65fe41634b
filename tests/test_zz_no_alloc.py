"""The allocation-free preconditioner entry point (pd_apply_precond_noalloc).

Callers that cannot call cudaMalloc (a frozen memory pool, a host application
that owns all device memory, a region where allocation is not allowed) cannot
create a plan.  This entry point applies z = P_alpha^{-1} r for 1D Dirichlet
problems using only a fixed device array inside the library.  It must agree
with the plan-based pd_apply_precond within the preconditioner tolerance used
by the other tests (64 eps32 kappa / alpha), on two calls in a row that reuse
the same array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from helpers import EPS32, SCHEME_TO_PD, dev, host, lib_ready, make_plan, relerr
from oracle import closed_forms as CF
from oracle import operators as O

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


def test_noalloc_matches_plan_on_two_calls():
    import torch
    pd = lib_ready()
    problems = [W.ade1d(nx=300, nt=128, scheme=W.CN, alpha=1e-2).problem,   # larger first
                W.ade1d(nx=127, nt=64, scheme=W.BE, alpha=1e-2).problem]
    for i, pb in enumerate(problems):
        r = W.uniform(100 + i, pb.unknowns, -1.0, 1.0).reshape(pb.nt, -1)
        rd = dev(r)
        zn = torch.full_like(rd, float("nan"))
        st, need = _noalloc(pd, pb, rd, zn)
        assert st == pd.PD_OK, (st, need)
        assert 0 < need <= (8 << 20)
        plan = make_plan(pb, pd.PD_MIXED)
        zp = host(plan.apply_precond(rd))
        plan.close()
        tol = 64 * EPS32 * _kappa(pb) / pb.alpha
        assert relerr(host(zn), zp) <= tol


def test_noalloc_rejects_oversized_problem():
    import torch
    pd = lib_ready()
    pb = W.ade1d(nx=4096, nt=1024).problem          # ~16.8 MB of spectrum > 8 MiB
    rd = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    st, need = _noalloc(pd, pb, rd, rd)
    assert st == pd.PD_ERR_ARG
    assert need > (8 << 20)
