"""Shared helpers for the GPU parity tests: plans from workloads.Problem and
numpy <-> torch transfers.  The oracle and the GPU library are only compared
here, never mixed."""
import numpy as np

import workloads as W

SCHEME_TO_PD = {W.BE: 0, W.CN: 1, W.THETA: 2, W.LEAPFROG: 3}
EPS32 = 2.0 ** -24


def lib_ready():
    import paradiag_gb300 as pd
    pd.build()
    return pd


def space_dict(sp: W.Space):
    return dict(dim=sp.dim, nx=sp.nx, ny=sp.ny, nu=sp.nu, ax=sp.ax, ay=sp.ay, bc_x=sp.bc_x,
                bc_y=sp.bc_y, lx=sp.lx, ly=sp.ly)


def make_plan(problem: W.Problem, precision):
    import paradiag_gb300 as pd
    return pd.Plan(space_dict(problem.space), problem.nt, problem.dt, problem.alpha,
                   SCHEME_TO_PD[problem.scheme], problem.theta_eff, precision)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def relerr(x, ref):
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300))


def rel2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))
