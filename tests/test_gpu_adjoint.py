"""Parity of the transposed all-at-once solve A^T lambda = g (backward in time)
and of the autograd gradient with the oracle (sequential backward stepping)."""
import numpy as np
import pytest

import workloads as W
from helpers import dev, host, lib_ready, make_plan, rel2
from oracle import control as C
from oracle import stepping as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["ade1d", "ade2d", "wave1d"])
def test_adjoint_solve_matches_backward_stepping(pd, prec, name):
    w = {"ade1d": W.ade1d(nx=63, nt=32), "ade2d": W.ade2d(nx=15, ny=13, nt=16),
         "wave1d": W.wave1d(nx=63, nt=64)}[name]
    pb = w.problem
    g = np.random.default_rng(8).standard_normal((pb.nt, pb.space.size))
    lref = S.solve_adjoint_sequential(pb, g)
    plan = make_plan(pb, pd.PD_FP64 if prec == "fp64" else pd.PD_MIXED)
    mode = pd.PD_GMRES if name == "wave1d" else pd.PD_STATIONARY
    lam, it, rel = plan.adjoint_solve(dev(g), mode=mode, tol=1e-12, maxit=60)
    assert rel2(host(lam), lref) <= 1e-10, rel2(host(lam), lref)
    plan.close()


def test_autograd_gradient_heat_source(pd):
    import torch
    w = W.heat2d_control(nx=15, nt=16)
    pb = w.problem
    tgt = w.extra["u_target"]
    f = w.extra["f_probe"]
    J_ref, g_ref, _, _ = C.gradient(pb, f, tgt, 1e-4)
    plan = make_plan(pb, pd.PD_MIXED)
    fd = dev(f).requires_grad_(True)
    b = fd.unsqueeze(0).expand(pb.nt, -1).contiguous()      # b_n = f (BE, u0 = 0)
    u = pd.PDSolve.apply(plan, b, pd.PD_STATIONARY, 1e-13, 60)
    e = u[-1] - dev(tgt)
    J = 0.5 * (e * e).sum() + 0.5e-4 * (fd * fd).sum()
    J.backward()
    assert abs(float(J) - J_ref) <= 1e-10 * abs(J_ref)
    assert rel2(host(fd.grad), g_ref) <= 1e-9, rel2(host(fd.grad), g_ref)
    plan.close()
