"""Parity at the full size of the 2D advection-diffusion workload: 255 x 255 grid
(x periodic, y Dirichlet), nu = 1e-3, velocity (1, 0.5), Crank-Nicolson, Nt = 256,
T = 1, alpha = 1e-3, seeded Gaussian bump, zero source -- 16,646,400 space-time
unknowns.

Both plans (mixed: FP32 preconditioner with the tensor-core x-transform and a
double-float residual; FP64) solve A u = b (eq. 1.1) by the stationary iteration
eq. 5.1 from a zero guess, in the launch configuration the benchmark times
(pd_solve_async: the CUDA-graph solve), and are compared element by element with
O1, the exact solution of the all-at-once system by sequential time stepping.
The bar: ||u - u_O1||_2 / ||u_O1||_2 <= 1e-10 and max |u - u_O1| / max |u_O1|
<= 1e-10.  The right-hand side is built on each side from the same u0 (pd_build_rhs
on the GPU, eq. 2.4 in the oracle).
"""
import numpy as np
import pytest

import workloads as W
from helpers import dev, host, lib_ready, make_plan, rel2, relerr
from oracle import operators as O
from oracle import stepping as S

pytestmark = pytest.mark.gpu

TOL_RES = 1e-11     # relative residual of the solve (the benchmark's setting)
TOL_ERR = 1e-10     # relative error against the oracle


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


@pytest.fixture(scope="module")
def headline():
    w = W.ade2d()
    pb = w.problem
    assert (pb.space.nx, pb.space.ny, pb.nt) == (255, 255, 256)
    uref = S.solve_sequential(pb, O.build_rhs(pb, w.u0, None, None))
    return w, uref


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_headline_solve_matches_sequential_stepping(pd, headline, prec):
    import torch
    w, uref = headline
    pb = w.problem
    plan = make_plan(pb, pd.PD_MIXED if prec == "mixed" else pd.PD_FP64)
    b = plan.build_rhs(dev(w.u0))
    u = torch.zeros_like(b)
    plan.solve_async(b, u, tol=TOL_RES, maxit=40)
    it, rel = plan.result()
    un = host(u).reshape(pb.nt, -1)
    e2, emax = rel2(un, uref), relerr(un, uref)
    print(f"HEADLINE {prec} iterations={it} relres={rel:.3e} rel2={e2:.3e} maxrel={emax:.3e}")
    assert rel <= TOL_RES
    assert e2 <= TOL_ERR, e2
    assert emax <= TOL_ERR, emax
    # a second solve on the same plan (the graph is reused) gives the same iterate
    u2 = torch.zeros_like(b)
    plan.solve_async(b, u2, tol=TOL_RES, maxit=40)
    plan.result()
    assert rel2(host(u2).reshape(pb.nt, -1), uref) <= TOL_ERR
    plan.close()
