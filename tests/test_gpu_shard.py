"""The slab-distributed stationary solve (paradiag_gb300.shard) with every
rank in this process on one GPU (the in-process exchange: the collectives are
local copies, and no kernel of one rank waits on another's).  Each rank runs
its residual, time transforms and x-transforms on a plan of its grid lines
plus halos and its share of step (b) on a plan of the whole grid, through
pd_precond_forward / pd_precond_solve_rows / pd_precond_backward; the
assembled solution must match the oracle's sequential time stepping (O1) to
1e-10 relative, for 1, 2 and 3 ranks, on a 2D periodic-x problem (mixed and
FP64 plans, the mixed x-transform on the tensor cores) and a 1D Dirichlet one."""
import numpy as np
import pytest

import workloads as W
from helpers import SCHEME_TO_PD, dev, host, lib_ready, rel2, space_dict
from oracle import operators as O
from oracle import stepping as S

pytestmark = pytest.mark.gpu


def _solve_sharded(pd, w, world, precision, tol):
    import torch
    from paradiag_gb300 import shard
    pb = w.problem
    sp = pb.space
    space = space_dict(sp)
    lines, pts = (sp.ny, sp.nx) if sp.dim == 2 else (sp.nx, 1)
    layout = shard.SlabLayout(lines, pts, pb.nt // 2 + 1, world)
    ranks = [shard.RankState(pd, torch, space, pb.nt, pb.dt, pb.alpha, SCHEME_TO_PD[pb.scheme],
                             pb.theta_eff, precision, layout, r, "cuda") for r in range(world)]
    solver = shard.ShardedSolver(pd, torch, ranks, shard.LocalExchange(torch))
    b = O.build_rhs(pb, w.u0, w.u1, w.f).reshape(pb.nt, lines, pts)
    solver.set_rhs([dev(b[:, rk.l0:rk.l1, :].reshape(pb.nt, -1)) for rk in ranks])
    it, rel = solver.solve(tol=tol, maxit=40)
    u = np.concatenate([host(solver.owned(rk, rk.u)).reshape(pb.nt, rk.ys, pts) for rk in ranks],
                       axis=1).reshape(pb.nt, -1)
    for rk in ranks:
        rk.close()
    return u, it, rel


@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_sharded_2d_matches_sequential(world, prec):
    pd = lib_ready()
    w = W.ade2d(nx=33, ny=24, nt=32, nu=1e-2, alpha=1e-3)
    pb = w.problem
    uref = S.solve_sequential(pb, O.build_rhs(pb, w.u0, None, None))
    u, it, rel = _solve_sharded(pd, w, world, pd.PD_MIXED if prec == "mixed" else pd.PD_FP64,
                                1e-12)
    e = rel2(u, uref)
    print(f"SHARD2D world={world} prec={prec} iterations={it} relres={rel:.2e} rel2={e:.2e}")
    assert e <= 1e-10, e


@pytest.mark.parametrize("world", [1, 2, 3])
def test_sharded_1d_matches_sequential(world):
    pd = lib_ready()
    w = W.ade1d(nx=63, nt=32)
    pb = w.problem
    uref = S.solve_sequential(pb, O.build_rhs(pb, w.u0, None, w.f))
    u, it, rel = _solve_sharded(pd, w, world, pd.PD_MIXED, 1e-12)
    e = rel2(u, uref)
    print(f"SHARD1D world={world} iterations={it} relres={rel:.2e} rel2={e:.2e}")
    assert e <= 1e-10, e
