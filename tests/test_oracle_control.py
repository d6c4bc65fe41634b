"""Pins of O5 (heat-source inversion gradient by the adjoint) (CPU only)."""
import numpy as np

import workloads as W
from oracle import control as C


def test_gradient_matches_central_differences():
    w = W.heat2d_control(nx=15, nt=16)
    pb = w.problem
    tgt = w.extra["u_target"]
    f = w.extra["f_probe"]
    J, g, _, _ = C.gradient(pb, f, tgt, 1e-4)
    assert abs(J - C.objective(pb, f, tgt, 1e-4)) <= 1e-14 * abs(J)
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal(f.size)
        fd = (C.objective(pb, f + h * d, tgt, 1e-4) - C.objective(pb, f - h * d, tgt, 1e-4)) / (2 * h)
        # J is quadratic in f: central differences are exact up to roundoff ~ eps |J| / h
        assert abs(fd - g @ d) <= 1e-8 * (abs(g @ d) + abs(J))


def test_gradient_quadratic_identity():
    # J(f + d) - J(f) - g.d = 1/2 d^T H d >= 0 exactly for this convex quadratic
    w = W.heat2d_control(nx=9, nt=8)
    pb = w.problem
    tgt = w.extra["u_target"]
    f = w.extra["f_probe"]
    J, g, _, _ = C.gradient(pb, f, tgt, 1e-4)
    d = np.random.default_rng(6).standard_normal(f.size)
    q1 = C.objective(pb, f + d, tgt, 1e-4) - J - g @ d
    q2 = C.objective(pb, f + 2 * d, tgt, 1e-4) - J - 2 * (g @ d)
    assert q1 > 0 and abs(q2 / q1 - 4.0) < 1e-8
