"""Parity of the batched solve (many 1D problems of uneven nx, Nt and nu in one
set of launches) with the oracle's sequential time stepping, problem by
problem.  Tolerance 1e-10 relative per problem (the solver stops at a relative
residual of 1e-11 mixed / 1e-12 FP64)."""
import numpy as np
import pytest

import workloads as W
from helpers import dev, host, lib_ready, rel2
from oracle import operators as O
from oracle import stepping as S

pytestmark = pytest.mark.gpu


def _problems(count, seed, pow2=True):
    return W.batched(count=count, seed=seed, pow2=pow2)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_matches_sequential(prec):
    pd = lib_ready()
    import torch
    wls = _problems(10, 4242)
    # systems from 63 to 1023 rows, so several tridiagonal lane classes are present
    wls.append(W.ade1d(nx=1023, nt=64, nu=1e-3, scheme=W.BE, alpha=1e-2, seed=9, name="big"))
    wls.append(W.ade1d(nx=400, nt=32, nu=1e-2, scheme=W.BE, alpha=1e-2, seed=10, name="mid"))
    wls.append(W.ade1d(nx=63, nt=1024, nu=1e-1, scheme=W.BE, alpha=1e-2, seed=11, name="long"))
    probs = [dict(space=dict(nx=w.problem.space.nx, nu=w.problem.space.nu, ax=w.problem.space.ax),
                  nt=w.problem.nt, dt=w.problem.dt, alpha=w.problem.alpha, scheme=0, theta=1.0)
             for w in wls]
    batch = pd.Batch(probs, pd.PD_MIXED if prec == "mixed" else pd.PD_FP64)
    u0 = np.concatenate([w.u0 for w in wls])
    f = np.concatenate([w.f.reshape(-1) for w in wls])
    b = batch.build_rhs(dev(u0), dev(f))
    l0 = batch.launches()
    # The mixed path forms the residual in double-float (48-bit significand), so
    # member i bottoms out near 2^-48 (1 + dt_i ||K_i||_inf) relative; it runs to
    # that floor (tol 0, 12 sweeps) and every member must be within 16x of it.
    # The FP64 path stops at 1e-12.
    if prec == "mixed":
        u, it, rel = batch.solve(b, tol=0.0, maxit=12, allow_not_converged=True)
        for i, w in enumerate(wls):
            K = O.stencil(w.problem.space)
            floor = 2.0 ** -48 * (1.0 + w.problem.dt * abs(K).sum(axis=1).max())
            assert batch.relres()[i] <= 16 * floor, (i, batch.relres()[i], floor)
    else:
        u, it, rel = batch.solve(b, tol=1e-12, maxit=30)
        assert rel <= 1e-12
    # one launch per kernel type per sweep: time forward, the device-side
    # convergence check of the graph (mixed path), one per tridiagonal lane
    # class, time inverse.  A system of n rows is split over the smallest
    # power-of-two number of lanes that holds it in chunks of at most 32 rows
    # (mixed) or 16 rows (FP64).
    rows = 32 if prec == "mixed" else 16
    classes = {int(np.ceil(np.log2(max(1, -(-w.problem.space.nx // rows))))) for w in wls}
    # the time kernels run one persistent launch per tile-footprint class
    # (4, 8 or 16 complex elements per thread; tiles of N x TX reals with
    # TX = min(32, budget / N), budget 8192 mixed / 2048 FP64)
    budget = 8192 if prec == "mixed" else 2048
    tcls = set()
    for w in wls:
        n = w.problem.nt
        tx = max(2, min(32, budget // n))
        e = -(-(n * (tx // 2)) // 256)
        tcls.add(0 if e <= 4 else 1 if e <= 8 else 2)
    per_sweep = len(tcls) + 1 + len(classes) + len(tcls)
    assert batch.launches() - l0 <= per_sweep * it + len(classes) + 6
    assert batch.uses_graph() == (prec == "mixed")
    uh = host(u)
    bh = host(b)
    off = batch.offsets
    for i, w in enumerate(wls):
        pb = w.problem
        bref = O.build_rhs(pb, w.u0, None, w.f)
        assert rel2(bh[off[i]:off[i + 1]].reshape(pb.nt, -1), bref) <= 1e-14
        uref = S.solve_sequential(pb, bref)
        err = rel2(uh[off[i]:off[i + 1]].reshape(pb.nt, -1), uref)
        assert err <= 1e-10, (i, pb.space.nx, pb.nt, err)
    batch.close()


def test_batch_rejects_mixed_bands_and_2d():
    pd = lib_ready()
    base = dict(space=dict(nx=31, nu=0.1), nt=16, dt=1 / 16, alpha=0.1, theta=1.0)
    with pytest.raises(pd.PDError) as ei:
        pd.Batch([dict(base, scheme=0), dict(base, scheme=3)])
    assert ei.value.status == pd.PD_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_integer_nt_reading(prec):
    # Nt drawn uniformly from the integers (non-powers of two use Bluestein)
    pd = lib_ready()
    wls = W.batched(count=8, seed=777, pow2=False)
    assert any((w.problem.nt & (w.problem.nt - 1)) != 0 for w in wls)
    probs = [dict(space=dict(nx=w.problem.space.nx, nu=w.problem.space.nu, ax=w.problem.space.ax),
                  nt=w.problem.nt, dt=w.problem.dt, alpha=w.problem.alpha, scheme=0, theta=1.0)
             for w in wls]
    batch = pd.Batch(probs, pd.PD_MIXED if prec == "mixed" else pd.PD_FP64)
    u0 = np.concatenate([w.u0 for w in wls])
    f = np.concatenate([w.f.reshape(-1) for w in wls])
    b = batch.build_rhs(dev(u0), dev(f))
    if prec == "mixed":
        u, it, rel = batch.solve(b, tol=0.0, maxit=12, allow_not_converged=True)
    else:
        u, it, rel = batch.solve(b, tol=1e-12, maxit=30)
    uh = host(u)
    off = batch.offsets
    for i, w in enumerate(wls):
        pb = w.problem
        uref = S.solve_sequential(pb, O.build_rhs(pb, w.u0, None, w.f))
        err = rel2(uh[off[i]:off[i + 1]].reshape(pb.nt, -1), uref)
        assert err <= 1e-10, (i, pb.space.nx, pb.nt, err)
    batch.close()


def test_batch_autotuned_matches_sequential():
    """A mixed batch of more than 2^18 unknowns chooses its tile widths and
    tridiagonal lane counts by timing at creation (per group of members with
    one transform length / one lane class); the solve with those shapes must
    still give every member the oracle's solution, and the per-kernel sweep
    profile reports three positive times."""
    pd = lib_ready()
    wls = W.batched(count=12, seed=31337, pow2=False)
    assert sum(w.problem.unknowns for w in wls) >= 1 << 18
    probs = [dict(space=dict(nx=w.problem.space.nx, nu=w.problem.space.nu, ax=w.problem.space.ax),
                  nt=w.problem.nt, dt=w.problem.dt, alpha=w.problem.alpha, scheme=0, theta=1.0)
             for w in wls]
    batch = pd.Batch(probs, pd.PD_MIXED)
    assert batch.tuned()
    u0 = np.concatenate([w.u0 for w in wls])
    f = np.concatenate([w.f.reshape(-1) for w in wls])
    b = batch.build_rhs(dev(u0), dev(f))
    import torch
    ms = batch.profile_sweep(b, torch.zeros_like(b), reps=2)
    assert len(ms) == 3 and all(t > 0 for t in ms), ms
    # as in the first test: run to the double-float residual floor of every
    # member, then compare with the oracle
    u, it, rel = batch.solve(b, tol=0.0, maxit=12, allow_not_converged=True)
    uh = host(u)
    off = batch.offsets
    for i, w in enumerate(wls):
        pb = w.problem
        K = O.stencil(pb.space)
        floor = 2.0 ** -48 * (1.0 + pb.dt * abs(K).sum(axis=1).max())
        assert batch.relres()[i] <= 16 * floor, (i, batch.relres()[i], floor)
        uref = S.solve_sequential(pb, O.build_rhs(pb, w.u0, None, w.f))
        err = rel2(uh[off[i]:off[i + 1]].reshape(pb.nt, -1), uref)
        assert err <= 1e-10, (i, pb.space.nx, pb.nt, err)
    batch.close()
