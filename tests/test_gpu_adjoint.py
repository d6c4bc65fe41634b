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
    assert abs(float(J.detach()) - J_ref) <= 1e-10 * abs(J_ref)
    assert rel2(host(fd.grad), g_ref) <= 1e-9, rel2(host(fd.grad), g_ref)
    plan.close()


def test_autograd_gradient_heat_source_full_size(pd):
    """The heat-source inversion at its full size: 127 x 127 grid (Dirichlet,
    nu = 1), backward Euler, Nt = 128 (2,064,512 unknowns).  Mixed plan: the
    x-transform runs on the tensor cores (nx >= 16 and 65 x 127 >= 128 spectrum
    rows), in the forward solve and in the transposed solve of the backward
    pass.  J and dJ/df against O5 (sequential forward and backward stepping),
    and four central differences of J against <dJ/df, d> (J is quadratic in f,
    so central differences are exact up to the solves' error at any h).
    The solves stop at a relative residual of 1e-11: at this grid Dt ||K|| is
    about 1e3, so the double-float residual (48-bit significand) of the
    transposed solve, whose right-hand side is rough (U_Nt - u_target at the last
    level only), has a floor near 2^-48 (1 + Dt ||K||) ~ 4e-12."""
    import torch
    w = W.heat2d_control()
    pb = w.problem
    assert (pb.space.nx, pb.space.ny, pb.nt) == (127, 127, 128)
    tgt = w.extra["u_target"]
    f = w.extra["f_probe"]
    reg = w.extra["reg"]
    J_ref, g_ref, _, _ = C.gradient(pb, f, tgt, reg)
    plan = make_plan(pb, pd.PD_MIXED)
    tg = dev(tgt)

    def J_of(fd):
        b = fd.unsqueeze(0).expand(pb.nt, -1).contiguous()      # b_n = f (BE, u0 = 0)
        u = pd.PDSolve.apply(plan, b, pd.PD_STATIONARY, 1e-11, 60)
        e = u[-1] - tg
        return 0.5 * (e * e).sum() + 0.5 * reg * (fd * fd).sum()

    fd = dev(f).requires_grad_(True)
    J = J_of(fd)
    J.backward()
    grad = host(fd.grad)
    Jv = float(J.detach())
    print(f"CFG4 J={Jv:.12e} J_ref={J_ref:.12e} grad_rel2={rel2(grad, g_ref):.3e}")
    assert abs(Jv - J_ref) <= 1e-10 * abs(J_ref)
    assert rel2(grad, g_ref) <= 1e-9, rel2(grad, g_ref)
    h = 1e-3
    with torch.no_grad():
        for i in range(4):
            d = dev(W.uniform(W.SEED_BASE + 40 + i, pb.space.size, -1.0, 1.0))
            fdiff = (float(J_of(fd + h * d)) - float(J_of(fd - h * d))) / (2 * h)
            dot = float((fd.grad * d).sum())
            assert abs(fdiff - dot) <= 1e-7 * max(abs(dot), 1e-30), (i, fdiff, dot)
    plan.close()


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_adjoint_advective_periodic_2d_tensor_core(pd, scheme):
    """A^T lambda = g for 2D advection-diffusion with x periodic and advection in
    both directions, where K^T != K (the transposed solve runs with reversed
    advection and its own x-eigentransform tables).  48 x 20 grid, Nt = 32: the
    mixed plan takes the tensor-core x-transform (nx >= 16, 17 x 20 spectrum
    rows >= 128).  Against sequential backward stepping (O5)."""
    sp = W.Space(dim=2, nx=48, ny=20, nu=1e-2, ax=1.0, ay=0.5, bc_x=W.PERIODIC,
                 bc_y=W.DIRICHLET)
    pb = W.Problem(space=sp, nt=32, dt=1.0 / 32, scheme=scheme, alpha=1e-3)
    g = W.uniform(W.SEED_BASE + 50 + scheme, pb.unknowns, -1.0, 1.0).reshape(pb.nt, -1)
    lref = S.solve_adjoint_sequential(pb, g)
    for prec in (pd.PD_MIXED, pd.PD_FP64):
        plan = make_plan(pb, prec)
        lam, it, rel = plan.adjoint_solve(dev(g), tol=1e-12, maxit=60)
        e = rel2(host(lam), lref)
        print(f"ADJ2D scheme={scheme} prec={prec} iterations={it} rel2={e:.3e}")
        assert e <= 1e-10, e
        plan.close()
