"""Time tiles split over a thread-block cluster (pd_plan_time_cluster).

A power-of-two Nt may have its FFT along t split over CR blocks: block c forms
the time rows [c N/CR, (c+1) N/CR), one radix-CR step of the transform goes
through distributed shared memory, and each block finishes a length-N/CR FFT
(decimation in frequency; the inverse in reverse).  The operator is still
z = P_alpha^{-1} r of eq. 1.3, so every cluster size is compared with the
oracle's Lemma-1 application (dense Fourier matrix), within the bound the
preconditioner parity tests use (2 eps kappa (1 + log2 Nt) / alpha, see
test_gpu_precond), and the solves with Nt beyond one block's tile with the
oracle's sequential time stepping.
"""
import zlib

import numpy as np
import pytest

import workloads as W
from helpers import EPS32, dev, host, lib_ready, make_plan, rel2, relerr
from oracle import closed_forms as CF
from oracle import operators as O
from oracle import paradiag as PD
from oracle import stepping as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


def problem(nx, nt, scheme=W.BE, alpha=1e-2, nu=0.05, ax=1.0, T=1.0):
    sp = W.Space(dim=1, nx=nx, nu=nu, ax=ax)
    return W.Problem(space=sp, nt=nt, dt=T / nt, scheme=scheme, alpha=alpha)


def kappa(pb):
    K = O.stencil(pb.space).toarray()
    l1, l2 = CF.lemma1_eigenvalues(pb)
    I = np.eye(K.shape[0])
    return max(np.linalg.cond(l1[k] * I + l2[k] * K) for k in range(pb.nt // 2 + 1))


def test_default_time_cluster_rule(pd):
    # one block per tile while its tile keeps 8 columns; then the smallest
    # cluster giving 8 columns (8 blocks at most); Bluestein lengths never split
    cases = [(pd.PD_MIXED, 1024, 1), (pd.PD_MIXED, 2048, 2), (pd.PD_MIXED, 4096, 4),
             (pd.PD_MIXED, 8192, 8), (pd.PD_MIXED, 32768, 8), (pd.PD_MIXED, 1000, 1),
             (pd.PD_FP64, 256, 1), (pd.PD_FP64, 512, 2), (pd.PD_FP64, 2048, 8),
             (pd.PD_FP64, 8192, 8), (pd.PD_FP64, 1000, 1)]
    for prec, nt, cr in cases:
        plan = make_plan(problem(7, nt), prec)
        assert plan.time_cluster == cr, (prec, nt, plan.time_cluster)
        tx = plan.tuning()[0]
        budget = 8192 if prec == pd.PD_MIXED else 2048
        if cr > 1:
            assert tx == budget * cr // nt
        plan.close()
    # beyond 8 blocks of two columns: unsupported
    for prec, nt in [(pd.PD_MIXED, 65536), (pd.PD_FP64, 16384)]:
        with pytest.raises(pd.PDError) as e:
            make_plan(problem(7, nt), prec)
        assert e.value.status == pd.PD_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_time_cluster_matches_oracle(pd, prec):
    # Nt = 1024, 33 columns (ragged: the last tile is partly padding)
    pb = problem(33, 1024, scheme=W.CN, alpha=1e-2)
    r = W.uniform(W.SEED_BASE + zlib.crc32(b"time_cluster") % 1000, pb.unknowns,
                  -1.0, 1.0).reshape(pb.nt, -1)
    zref = PD.precond_apply(pb, r)
    eps = 2.0 ** -53 if prec == "fp64" else EPS32
    tol = 2.0 * eps * kappa(pb) * (1.0 + np.log2(pb.nt)) / pb.alpha
    plan = make_plan(pb, pd.PD_FP64 if prec == "fp64" else pd.PD_MIXED)
    budget = 2048 if prec == "fp64" else 8192
    valid = {1} | {cr for cr in (2, 4, 8) if 2 <= budget * cr // pb.nt <= 32}
    assert valid == ({1, 2, 4, 8} if prec == "fp64" else {1, 2, 4})
    outs = {}
    for cr in (1, 2, 4, 8):
        if cr not in valid:
            with pytest.raises(pd.PDError) as e:
                plan.set_time_cluster(cr)
            assert e.value.status == pd.PD_ERR_UNSUPPORTED
            continue
        plan.set_time_cluster(cr)
        assert plan.time_cluster == cr
        z = host(plan.apply_precond(dev(r)))
        err = relerr(z, zref)
        print(f"TIME_CLUSTER {prec} cr={cr} tx={plan.tuning()[0]} err={err:.3e} tol={tol:.3e}")
        assert err <= tol, (prec, cr, err, tol)
        outs[cr] = z
    with pytest.raises(pd.PDError) as e:
        plan.set_time_cluster(3)
    assert e.value.status == pd.PD_ERR_ARG
    if prec == "mixed":
        # a cluster plan keeps its tile width
        plan.set_time_cluster(2)
        tx, lanes, rows = plan.get_tuning()
        with pytest.raises(pd.PDError) as e:
            plan.set_tuning(tx // 2, lanes, rows)
        assert e.value.status == pd.PD_ERR_ARG
        plan.set_tuning(tx, lanes, rows)
    plan.close()


@pytest.mark.parametrize("prec,nt,scheme", [("mixed", 8192, W.BE), ("mixed", 32768, W.CN),
                                            ("fp64", 8192, W.BE)])
def test_long_time_axis_solve_matches_sequential(pd, prec, nt, scheme):
    # Nt beyond one block's tile (4096 mixed, 2048 FP64), solved to 1e-12
    w = W.ade1d(nx=7, nt=nt, nu=1e-2, a=1.0, scheme=scheme, alpha=1e-2, T=1.0)
    pb = w.problem
    b = O.build_rhs(pb, w.u0, w.u1, w.f)
    uref = S.solve_sequential(pb, b)
    plan = make_plan(pb, pd.PD_FP64 if prec == "fp64" else pd.PD_MIXED)
    assert plan.time_cluster == 8
    u, it, rel = plan.solve(dev(b), tol=1e-12, maxit=40)
    err = rel2(host(u), uref)
    print(f"LONG_NT {prec} nt={nt} iters={it} relres={rel:.2e} err={err:.2e}")
    assert rel <= 1e-12
    assert err <= 1e-10, (err, it)
    plan.close()
