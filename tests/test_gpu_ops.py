"""Parity of the FP64 all-at-once operator kernels (apply A, A^T, residual,
right-hand side) with the oracle.  Both sides are FP64 with the same operation
count per entry up to ordering, so the tolerance is 1e-13 of the scale."""
import numpy as np
import pytest

import workloads as W
from helpers import dev, host, lib_ready, make_plan, relerr
from oracle import operators as O

pytestmark = pytest.mark.gpu


def probs():
    return {
        "1d_be_adv": W.ade1d(nx=31, nt=8, scheme=W.BE),
        "1d_cn_adv": W.ade1d(nx=29, nt=9 - 1, scheme=W.CN),
        "1d_theta": None,
        "2d_cn_perx": W.ade2d(nx=13, ny=11, nt=8),
        "1d_wave": W.wave1d(nx=33, nt=16),
        "2d_heat": W.heat2d_control(nx=9, nt=8),
    }


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


@pytest.mark.parametrize("name", ["1d_be_adv", "1d_cn_adv", "2d_cn_perx", "1d_wave", "2d_heat"])
def test_apply_A_AT_residual_rhs(pd, name):
    w = probs()[name]
    pb = w.problem
    plan = make_plan(pb, pd.PD_FP64)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((pb.nt, pb.space.size))
    b = rng.standard_normal((pb.nt, pb.space.size))
    assert relerr(host(plan.apply_A(dev(U))), O.apply_A(pb, U)) <= 1e-13
    assert relerr(host(plan.apply_A(dev(U), transpose=True)), O.apply_AT(pb, U)) <= 1e-13
    assert relerr(host(plan.residual(dev(b), dev(U))), b - O.apply_A(pb, U)) <= 1e-13
    f = w.f if w.f is not None else rng.standard_normal((pb.nt + 1, pb.space.size))
    bref = O.build_rhs(pb, w.u0, w.u1, f)
    bg = host(plan.build_rhs(dev(w.u0), None if w.u1 is None else dev(w.u1), dev(f)))
    assert relerr(bg, bref) <= 1e-13
    plan.close()
