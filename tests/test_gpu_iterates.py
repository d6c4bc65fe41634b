"""Per-iteration parity of the stationary iteration eq. 5.1: the GPU iterate u^k
after k sweeps (maxit = k) against the oracle's k-th iterate, from the random
initial guess in [-20, 20] of the paper's waveform-relaxation experiment.

Tolerance.  u^k = u^{k-1} + P^{-1} r^{k-1}, so every sweep adds the evaluation
error of the preconditioner, at most tol_P ||u^j - u^{j-1}|| with
tol_P = 64 eps kappa / alpha as in the preconditioner test (eps of the
preconditioner's arithmetic: FP32 on the mixed path, FP64 otherwise; kappa the
largest condition number of the shifted systems).  Later sweeps carry an
earlier error along with the contraction of I - P^{-1} A (Theorem 5.1: rate
<= alpha / (1 - alpha) < 1 per mode), so the test bound is
||u^k_gpu - u^k_oracle|| <= 4 tol_P sum_{j <= k} ||u^j - u^{j-1}||.
"""
import numpy as np
import pytest

import workloads as W
from helpers import EPS32, dev, host, lib_ready, make_plan
from oracle import closed_forms as CF
from oracle import operators as O
from oracle import paradiag as PD

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53


def P(dim=1, nx=15, ny=1, nu=0.1, ax=0.0, ay=0.0, bcx=W.DIRICHLET, nt=16, T=1.0,
      scheme=W.BE, alpha=1e-2):
    sp = W.Space(dim=dim, nx=nx, ny=ny, nu=nu, ax=ax, ay=ay, bc_x=bcx)
    return W.Problem(space=sp, nt=nt, dt=T / nt, scheme=scheme, alpha=alpha)


CASES = {
    "1d_be_127x64": P(nx=127, nu=1e-2, ax=1.0, nt=64, alpha=1e-2),
    "1d_leapfrog_63x32": P(nx=63, nu=1.0, nt=32, T=2.0, scheme=W.LEAPFROG, alpha=0.1),
    "2d_cn_periodic_x_15x13x16": P(dim=2, nx=15, ny=13, nu=1e-2, ax=1.0, ay=0.5,
                                    bcx=W.PERIODIC, nt=16, scheme=W.CN, alpha=1e-3),
    "2d_tc_cn_periodic_33x20x32": P(dim=2, nx=33, ny=20, nu=1e-2, ax=1.0, ay=0.5,
                                    bcx=W.PERIODIC, nt=32, scheme=W.CN, alpha=1e-3),
}


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


def kappa(pb):
    """max_k cond_2(lambda_1k I + lambda_2k K) over the Lemma 1 eigenvalues."""
    K = O.stencil(pb.space).toarray()
    l1, l2 = CF.lemma1_eigenvalues(pb)
    I = np.eye(K.shape[0])
    return max(np.linalg.cond(l1[k] * I + l2[k] * K) for k in range(pb.nt // 2 + 1))


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_stationary_iterates_match_oracle(pd, name, prec):
    pb = CASES[name]
    K = O.stencil(pb.space)
    shape = (pb.nt, pb.space.size)
    n = pb.nt * pb.space.size
    b = W.uniform(W.SEED_BASE + 77, n, -1.0, 1.0).reshape(shape)
    u0 = W.uniform(W.SEED_BASE + 78, n, -20.0, 20.0).reshape(shape)
    _, _, _, hist = PD.stationary(pb, b, u_init=u0, tol=0.0, maxit=3, K=K, history=True)
    eps = EPS32 if prec == "mixed" else EPS64
    tol_p = 64.0 * eps * kappa(pb) / pb.alpha
    plan = make_plan(pb, pd.PD_MIXED if prec == "mixed" else pd.PD_FP64)
    steps = 0.0
    for k in (1, 2, 3):
        u, it, _ = plan.solve(dev(b), dev(u0), tol=0.0, maxit=k, allow_not_converged=True)
        assert it == k
        steps += np.linalg.norm(hist[k] - hist[k - 1])
        err = np.linalg.norm(host(u) - hist[k])
        assert err <= 4.0 * tol_p * steps, (k, err, tol_p * steps)
    plan.close()
