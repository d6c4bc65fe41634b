"""Parity of z = P_alpha^{-1} r (eq. 1.3) between the CUDA path and the oracle's
naive Lemma-1 application (dense Fourier matrix, sparse LU per frequency).

Tolerances.  The transform has Cond_2(V) <= 1/alpha (eq. 2.13) and each
shifted system lambda_1 I + lambda_2 K has a 2-norm condition number kappa_k,
so a backward-stable evaluation in precision eps gives a relative error of
order eps * kappa / alpha with kappa = max_k kappa_k (computed here from the
dense shifted matrices); the FFTs add a factor growing like log2 M, M the
transform length (Nt, or Bluestein's M = 2^ceil(log2(2 Nt - 1))).  The bound
checked is 2 eps kappa (1 + log2 M) / alpha with eps = 2^-53 (FP64 path) or
2^-24 (mixed path: FP32 transforms and solves).  The measured max-norm
errors sit between about 1/1300 and 1/5 of it; every case prints its error and
the ratio err / (eps kappa / alpha).
The invariant P z = r is checked relative to |P| |z| (entrywise absolute
values), the natural scale of the rounding error of the product, against
64 eps kappa / alpha (at least 1e-12).
"""
import zlib

import numpy as np
import pytest

import workloads as W
from helpers import EPS32, dev, host, lib_ready, make_plan, relerr
from oracle import closed_forms as CF
from oracle import operators as O
from oracle import paradiag as PD

pytestmark = pytest.mark.gpu


def P(dim=1, nx=15, ny=1, nu=0.1, ax=0.0, ay=0.0, bcx=W.DIRICHLET, nt=16, T=1.0,
      scheme=W.BE, alpha=1e-2):
    sp = W.Space(dim=dim, nx=nx, ny=ny, nu=nu, ax=ax, ay=ay, bc_x=bcx)
    return W.Problem(space=sp, nt=nt, dt=T / nt, scheme=scheme, alpha=alpha)


CASES = {
    "1d_be_ade_127x64": P(nx=127, nu=1e-2, ax=1.0, nt=64, alpha=1e-2),
    "1d_cn_ragged_37x16": P(nx=37, nu=3e-2, ax=0.7, nt=16, scheme=W.CN, alpha=1e-3),
    "1d_leapfrog_63x32": P(nx=63, nu=1.0, nt=32, T=2.0, scheme=W.LEAPFROG, alpha=0.1),
    "1d_leapfrog_alpha1": P(nx=31, nu=1.0, nt=16, T=2.0, scheme=W.LEAPFROG, alpha=1.0),
    "1d_periodic_be_24x8": P(nx=24, nu=1e-2, ax=1.0, bcx=W.PERIODIC, nt=8, alpha=1e-2),
    "1d_nt1": P(nx=20, nt=1, alpha=0.5),
    "1d_nt2": P(nx=20, nt=2, scheme=W.CN, alpha=0.05),
    "1d_nx1": P(nx=1, nt=8),
    "1d_nx600_multiwarp": P(nx=600, nu=1e-3, ax=1.0, nt=8, alpha=1e-2),
    "1d_nx400_two_warps": P(nx=400, nu=1e-2, ax=1.0, nt=32, alpha=1e-2),
    "1d_nx511_two_warps": P(nx=511, nu=1e-2, ax=1.0, nt=16, alpha=1e-2),
    "1d_nx1023_multiwarp": P(nx=1023, nu=1.0, nt=16, T=2.0, scheme=W.LEAPFROG, alpha=0.1),
    "1d_nt512": P(nx=33, nu=0.05, ax=1.0, nt=512, alpha=1e-2),
    # non-power-of-two Nt (Bluestein): even, odd, prime, and the largest class
    "1d_bluestein_nt12": P(nx=31, nu=0.05, ax=1.0, nt=12, alpha=1e-2),
    "1d_bluestein_nt3": P(nx=17, nu=0.05, ax=1.0, nt=3, scheme=W.CN, alpha=1e-2),
    "1d_bluestein_nt63_cn": P(nx=40, nu=0.02, ax=1.0, nt=63, scheme=W.CN, alpha=1e-3),
    "1d_bluestein_nt97_leapfrog": P(nx=63, nu=1.0, nt=97, T=2.0, scheme=W.LEAPFROG, alpha=0.1),
    "1d_bluestein_nt1000": P(nx=47, nu=0.05, ax=1.0, nt=1000, alpha=1e-2),
    "2d_bluestein_cn_periodic_20x9x20": P(dim=2, nx=20, ny=9, nu=1e-2, ax=1.0, ay=0.5,
                                          bcx=W.PERIODIC, nt=20, scheme=W.CN, alpha=1e-3),
    "2d_cn_periodic_x_15x13x16": P(dim=2, nx=15, ny=13, nu=1e-2, ax=1.0, ay=0.5,
                                    bcx=W.PERIODIC, nt=16, scheme=W.CN, alpha=1e-3),
    "2d_be_dirichlet_sym_11x9x8": P(dim=2, nx=11, ny=9, nu=1.0, nt=8, alpha=1e-2),
    "2d_lf_dirichlet_sym_9x7x8": P(dim=2, nx=9, ny=7, nu=1.0, nt=8, T=2.0,
                                   scheme=W.LEAPFROG, alpha=0.1),
    # x-transform on the tensor cores in the mixed path (nx >= 16, >= 128 spectrum rows)
    "2d_tc_cn_periodic_33x20x32": P(dim=2, nx=33, ny=20, nu=1e-2, ax=1.0, ay=0.5,
                                    bcx=W.PERIODIC, nt=32, scheme=W.CN, alpha=1e-3),
    "2d_tc_be_dirichlet_sym_40x17x16": P(dim=2, nx=40, ny=17, nu=1.0, nt=16, alpha=1e-2),
    "2d_tc_cn_periodic_255x4x64": P(dim=2, nx=255, ny=4, nu=1e-3, ax=1.0, ay=0.5,
                                    bcx=W.PERIODIC, nt=64, scheme=W.CN, alpha=1e-3),
    "1d_tc_periodic_200x256": P(nx=200, nu=1e-2, ax=1.0, bcx=W.PERIODIC, nt=256, alpha=1e-2),
    # time tiles split over a thread-block cluster (the plans' default shapes:
    # mixed Nt = 2048 / 4096 take 2 / 4 blocks per tile; FP64 Nt = 1024 / 2048
    # / 4096 take 4 / 8 / 8, Nt = 512 two)
    "1d_cluster_cn_nt2048": P(nx=9, nu=0.05, ax=1.0, nt=2048, scheme=W.CN, alpha=1e-2),
    "1d_cluster_be_nt4096": P(nx=13, nu=0.02, ax=1.0, nt=4096, alpha=1e-2),
    "1d_cluster_leapfrog_nt1024": P(nx=21, nu=1.0, nt=1024, T=2.0, scheme=W.LEAPFROG, alpha=0.1),
    "2d_cluster_cn_periodic_9x3x2048": P(dim=2, nx=9, ny=3, nu=1e-2, ax=1.0, ay=0.5,
                                         bcx=W.PERIODIC, nt=2048, scheme=W.CN, alpha=1e-3),
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


def abs_product_scale(pb, z):
    """max of |C1| (x) I + |C2| (x) |K| applied to |z|: the scale of P z."""
    K = abs(O.stencil(pb.space))
    C1, C2 = O.circulant_matrices(pb)
    return np.abs(O.apply_kron(np.abs(C1), np.abs(C2), K, np.abs(z))).max()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_precond_matches_oracle(pd, name, prec):
    pb = CASES[name]
    # a fixed seed per case (crc32 of its name), the same in every process
    r = W.uniform(W.SEED_BASE + zlib.crc32(name.encode()) % 1000, pb.unknowns,
                  -1.0, 1.0).reshape(pb.nt, -1)
    zref = PD.precond_apply(pb, r)
    plan = make_plan(pb, pd.PD_FP64 if prec == "fp64" else pd.PD_MIXED)
    z = host(plan.apply_precond(dev(r)))
    kap = kappa(pb)
    eps = 2.0 ** -53 if prec == "fp64" else EPS32
    M = pb.nt if pb.nt & (pb.nt - 1) == 0 else 1 << int(np.ceil(np.log2(2 * pb.nt - 1)))
    tol = 2.0 * eps * kap * (1.0 + np.log2(M)) / pb.alpha
    err = relerr(z, zref)
    print(f"PRECOND_ERR {name} {prec} err={err:.3e} eps_kappa_over_alpha={eps * kap / pb.alpha:.3e}"
          f" ratio={err / (eps * kap / pb.alpha):.3e} of_bound={err / tol:.3e}")
    assert err <= tol, (name, prec, err, tol, kap)
    # invariant P z = r, evaluated by the oracle in FP64, relative to |P||z|
    pz = O.apply_P(pb, z)
    res = np.abs(pz - r).max() / abs_product_scale(pb, z)
    tol_inv = max(64 * eps * kap / pb.alpha, 1e-12)
    assert res <= tol_inv, (res, tol_inv)
    plan.close()


# every case with an x-eigentransform (2D, or periodic 1D) under each engine
# its mixed plan offers: the tensor-core GEMM where available and the FP32 FFT
XFORM_CASES = sorted(n for n, pb in CASES.items()
                     if pb.space.dim == 2 or pb.space.bc_x == W.PERIODIC)


@pytest.mark.parametrize("name", XFORM_CASES)
def test_precond_each_xform_engine_matches_oracle(pd, name):
    pb = CASES[name]
    r = W.uniform(W.SEED_BASE + zlib.crc32(name.encode()) % 1000, pb.unknowns,
                  -1.0, 1.0).reshape(pb.nt, -1)
    zref = PD.precond_apply(pb, r)
    kap = kappa(pb)
    M = pb.nt if pb.nt & (pb.nt - 1) == 0 else 1 << int(np.ceil(np.log2(2 * pb.nt - 1)))
    tol = 2.0 * EPS32 * kap * (1.0 + np.log2(M)) / pb.alpha
    plan = make_plan(pb, pd.PD_MIXED)
    nx, rows = pb.space.nx, (pb.nt // 2 + 1) * (pb.space.ny if pb.space.dim == 2 else 1)
    has_tc = nx >= 16 and rows >= 128
    engines = [pd.PD_XFORM_FFT] + ([pd.PD_XFORM_TENSOR] if has_tc else [])
    assert plan.xform_engine == (pd.PD_XFORM_TENSOR if has_tc else pd.PD_XFORM_FFT)
    zs = {}
    for eng in engines:
        plan.set_xform_engine(eng)
        assert plan.xform_engine == eng
        zs[eng] = host(plan.apply_precond(dev(r)))
        err = relerr(zs[eng], zref)
        print(f"XFORM_ENGINE {name} engine={eng} err={err:.3e} of_bound={err / tol:.3e}")
        assert err <= tol, (name, eng, err, tol)
    if not has_tc:
        with pytest.raises(pd.PDError) as e:
            plan.set_xform_engine(pd.PD_XFORM_TENSOR)
        assert e.value.status == pd.PD_ERR_UNSUPPORTED
    plan.close()


def test_xform_engine_rules(pd):
    # FP64 2D plans take the FFT; plans without an x-transform report -1 and
    # refuse either engine; invalid engine values are argument errors
    sp = W.Space(dim=2, nx=33, ny=20, nu=1e-2, ax=1.0, ay=0.5, bc_x=W.PERIODIC)
    pb = W.Problem(space=sp, nt=32, dt=1.0 / 32, scheme=W.CN, alpha=1e-3)
    p64 = make_plan(pb, pd.PD_FP64)
    assert p64.xform_engine == pd.PD_XFORM_FFT
    with pytest.raises(pd.PDError) as e:
        p64.set_xform_engine(pd.PD_XFORM_TENSOR)
    assert e.value.status == pd.PD_ERR_UNSUPPORTED
    with pytest.raises(pd.PDError) as e:
        p64.set_xform_engine(7)
    assert e.value.status == pd.PD_ERR_ARG
    p64.close()
    p1 = make_plan(CASES["1d_be_ade_127x64"], pd.PD_MIXED)
    assert p1.xform_engine == -1
    for eng in (pd.PD_XFORM_TENSOR, pd.PD_XFORM_FFT):
        with pytest.raises(pd.PDError) as e:
            p1.set_xform_engine(eng)
        assert e.value.status == pd.PD_ERR_UNSUPPORTED
    p1.close()
