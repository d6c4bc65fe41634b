"""Pins of O6, ParaDiag-I with geometric time steps (Section 2.1.1), CPU only.

The closed forms of the theorem are checked in exact rational arithmetic
(V V^{-1} = I and the eigen-relation B1 V = B2 V D, column by column), the
variable-step stepping against the per-mode amplification factors and against
the uniform-step oracle, and the three-step solve against a dense Kronecker
solve and against stepping within the roundoff bound Nt eps Cond(V).
"""
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as CF
from oracle import operators as O
from oracle import paradiag1 as P1
from oracle import stepping as ST

EPS = 2.0 ** -53


def GP(dim=1, nx=15, ny=1, nu=0.05, ax=0.0, ay=0.0, bcx=W.DIRICHLET, nt=8, dt_last=0.05,
       tau=1.5, scheme=W.BE, scaled=True, lx=1.0):
    sp = W.Space(dim=dim, nx=nx, ny=ny, nu=nu, ax=ax, ay=ay, bc_x=bcx, lx=lx)
    return W.GeometricProblem(space=sp, nt=nt, dt_last=dt_last, tau=tau, scheme=scheme,
                              scaled=scaled)


def test_geometric_steps():
    nt, dl, tau = 12, 0.05, 1.16
    d = P1.geometric_steps(nt, dl, tau)
    assert d[-1] == dl
    assert np.allclose(d[1:] / d[:-1], tau, rtol=1e-15, atol=0)
    # total length: the geometric sum dt_Nt (1 - tau^-Nt) / (1 - 1/tau)
    assert abs(d.sum() - dl * (1 - tau ** -nt) / (1 - 1 / tau)) < 1e-15


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_time_matrices_structure(theta):
    d = P1.geometric_steps(7, 0.1, 1.3)
    B1, B2 = P1.time_matrices(d, theta)
    one = np.ones(7)
    # difference quotients annihilate constants except in the first row
    e1 = np.zeros(7); e1[0] = 1.0 / d[0]
    assert np.allclose(B1 @ one, e1, rtol=0, atol=1e-13)
    # theta-weights sum to one except in the first row
    w = np.ones(7); w[0] = theta
    assert np.allclose(B2 @ one, w, rtol=0, atol=0)
    # row n of B1 applied to t_n (linear in time) gives 1 (exact derivative)
    t = np.cumsum(d)
    assert np.allclose((B1 @ t)[1:], 1.0, rtol=1e-12)


@pytest.mark.parametrize("tau", [Fraction(3, 2), Fraction(6, 5), Fraction(7, 4)])
@pytest.mark.parametrize("theta", [Fraction(1), Fraction(1, 2)])
def test_closed_forms_exact(tau, theta):
    nt = 10
    p, q = P1.eigvec_coeffs(nt, tau, theta)
    # V V^{-1} = I for lower-triangular Toeplitz matrices: the convolution of
    # the first columns is the unit vector (exact, so the reading of q_n for
    # theta = 1/2 is checked without roundoff)
    for n in range(nt):
        conv = sum(p[m] * q[n - m] for m in range(n + 1))
        assert conv == (1 if n == 0 else 0), (n, conv)
    # eigen-relation B1 v_k = (1/(theta dt_k)) B2 v_k for the column v_k of V
    # (entries p_{n-k} below the diagonal), rows n > k of eq. 2.5b, with
    # dt_n = tau^n (B = V D V^{-1} is invariant under a common scale of the steps)
    dt = [tau ** n for n in range(nt)]
    for k in range(nt):
        v = [Fraction(0)] * k + [p[n - k] for n in range(k, nt)]
        lam = 1 / (theta * dt[k])
        for n in range(k + 1, nt):
            lhs = (v[n] - v[n - 1]) / dt[n]
            rhs = lam * (theta * v[n] + (1 - theta) * v[n - 1])
            assert lhs == rhs, (k, n)


def test_closed_forms_first_terms():
    # theta = 1: p_1 = 1/(1 - tau), q_1 = -p_1; theta = 1/2: p_1 = (1 + tau)/(1 - tau)
    tau = 1.25
    p, q = P1.eigvec_coeffs(4, tau, 1.0)
    assert p[1] == pytest.approx(1 / (1 - tau), rel=1e-15)
    assert q[1] == pytest.approx(-p[1], rel=1e-15)
    assert p[2] == pytest.approx(1 / ((1 - tau) * (1 - tau**2)), rel=1e-15)
    p, q = P1.eigvec_coeffs(4, tau, 0.5)
    assert p[1] == pytest.approx((1 + tau) / (1 - tau), rel=1e-15)
    assert q[1] == pytest.approx(-p[1], rel=1e-15)


@pytest.mark.parametrize("theta", [1.0, 0.5])
@pytest.mark.parametrize("scaled", [False, True])
def test_eigendecomposition_float(theta, scaled):
    nt, tau = 12, 1.4
    d = P1.geometric_steps(nt, 0.05, tau)
    B1, B2 = P1.time_matrices(d, theta)
    B = np.linalg.solve(B2, B1)
    V, Vi = P1.eigvec_matrices(nt, tau, theta, scaled)
    D = np.diag(P1.eigenvalues(d, theta))
    cond = np.linalg.cond(V)
    assert np.abs(V @ Vi - np.eye(nt)).max() < 10 * nt * EPS * cond
    rel = np.linalg.norm(B @ V - V @ D) / (np.linalg.norm(B) * np.linalg.norm(V))
    assert rel < 10 * nt * EPS * cond
    if scaled:
        assert np.allclose(np.linalg.norm(V, axis=0), 1.0, rtol=1e-14)


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_stepping_mode_solution(scheme):
    # periodic Fourier mode v, f = 0: U_n = prod_{m<=n} R(dt_m mu) v
    n, j = 16, 3
    pb = GP(nx=n, nu=0.05, ax=1.3, bcx=W.PERIODIC, nt=10, dt_last=0.08, tau=1.3, scheme=scheme)
    v = np.exp(2j * np.pi * j * np.arange(n) / n)
    mu = CF.mu_periodic(n, pb.space.hx, 0.05, 1.3)[j]
    th = P1.theta_of(scheme)
    U = P1.solve_sequential(pb, P1.build_rhs(pb, v.real))
    amp = np.cumprod(CF.stability_function(P1.geometric_steps(10, 0.08, 1.3) * mu, th))
    ref = np.real(np.outer(amp, v))
    assert np.abs(U - ref).max() < 1e-13


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_stepping_steady_state(scheme):
    # U_0 = phi/mu and f = phi for an eigenmode phi: every U_n = phi/mu
    pb = GP(nx=15, nu=0.2, nt=9, dt_last=0.1, tau=1.7, scheme=scheme)
    x = pb.space.xs()
    phi = np.sin(2 * np.pi * x)
    mu = np.sort(CF.mu_dirichlet(15, pb.space.hx, 0.2, 0.0).real)[1]
    F = np.broadcast_to(phi, (10, 15))
    U = P1.solve_sequential(pb, P1.build_rhs(pb, phi / mu, F))
    assert np.abs(U - phi / mu).max() < 1e-13


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_uniform_limit_matches_uniform_oracle(scheme):
    # tau = 1 gives uniform steps: rhs and stepping agree with the uniform oracle
    sp = W.Space(dim=1, nx=20, nu=0.03, ax=0.7)
    pb = W.GeometricProblem(space=sp, nt=11, dt_last=0.04, tau=1.0, scheme=scheme)
    pu = W.Problem(space=sp, nt=11, dt=0.04, scheme=scheme, alpha=0.1)
    u0 = W.uniform(W.SEED_BASE + 90, 20, -1, 1)
    f = W.uniform(W.SEED_BASE + 91, 12 * 20, -1, 1).reshape(12, 20)
    b = P1.build_rhs(pb, u0, f)
    assert np.allclose(b, O.build_rhs(pu, u0, None, f), rtol=0, atol=1e-13)
    assert np.allclose(P1.solve_sequential(pb, b), ST.solve_sequential(pu, b), rtol=0, atol=1e-12)
    U = P1.solve_sequential(pb, b)
    assert np.allclose(P1.apply_A(pb, U), O.apply_A(pu, U), rtol=0, atol=1e-10)


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
@pytest.mark.parametrize("scaled", [False, True])
def test_direct_matches_dense_kron(scheme, scaled):
    pb = GP(nx=6, nu=0.3, ax=0.8, nt=5, dt_last=0.1, tau=1.6, scheme=scheme, scaled=scaled)
    K = O.stencil(pb.space).toarray()
    th = P1.theta_of(scheme)
    d = P1.geometric_steps(5, 0.1, 1.6)
    B1, B2 = P1.time_matrices(d, th)
    A = np.kron(B1, np.eye(6)) + np.kron(B2, K)
    b = W.uniform(W.SEED_BASE + 92, 30, -1, 1)
    ref = np.linalg.solve(A, b).reshape(5, 6)
    U = P1.solve_direct(pb, b.reshape(5, 6))
    assert np.abs(U - ref).max() < 1e-12 * np.abs(ref).max()
    # the factorisation behind eq. 2.7
    V, Vi = P1.eigvec_matrices(5, 1.6, th, scaled)
    lhs = np.kron(V, np.eye(6)) @ (np.kron(np.diag(P1.eigenvalues(d, th)), np.eye(6))
                                    + np.kron(np.eye(5), K)) @ np.kron(Vi, np.eye(6))
    rhs = np.kron(np.linalg.solve(B2, B1), np.eye(6)) + np.kron(np.eye(5), K)
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(rhs).max()


CASES = {
    "1d_dirichlet_adv": GP(nx=31, nu=0.02, ax=1.0, nt=8, dt_last=0.05, tau=1.5),
    "1d_periodic_paper": GP(nx=64, nu=1e-2, ax=1.0, bcx=W.PERIODIC, lx=2.0, nt=12,
                            dt_last=0.05, tau=1.3),
    "2d_small": GP(dim=2, nx=9, ny=7, nu=0.05, ax=0.5, nt=10, dt_last=0.05, tau=1.4),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_direct_matches_stepping_within_roundoff(name, scheme):
    base = CASES[name]
    pb = W.GeometricProblem(space=base.space, nt=base.nt, dt_last=base.dt_last, tau=base.tau,
                            scheme=scheme)
    S = pb.space.size
    u0 = W.uniform(W.SEED_BASE + 93, S, -1, 1)
    f = W.uniform(W.SEED_BASE + 94, (pb.nt + 1) * S, -1, 1).reshape(pb.nt + 1, S)
    b = P1.build_rhs(pb, u0, f)
    ref = P1.solve_sequential(pb, b)
    U = P1.solve_direct(pb, b)
    V, _ = P1.eigvec_matrices(pb.nt, pb.tau, P1.theta_of(scheme), True)
    bound = pb.nt * EPS * np.linalg.cond(V) * np.abs(ref).max()
    assert np.abs(U - ref).max() <= max(bound, 1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("scheme,cond_lo", [(W.BE, 1e5), (W.CN, 1e12)])
def test_paper_window_roundoff(scheme, cond_lo):
    # the window of the windowing figure (Nt = 32, tau = 1.16, dt_Nt = 0.05,
    # nu = 1e-3, periodic (-1, 1), u0 = exp(-30 x^2)): Cond(V) is large and
    # the error of the direct solve tracks it (roundoff ~ Cond_2(V))
    wl = W.pd1_ade1d(scheme=scheme)
    pb = wl.problem
    b = P1.build_rhs(pb, wl.u0)
    ref = P1.solve_sequential(pb, b)
    U = P1.solve_direct(pb, b)
    V, _ = P1.eigvec_matrices(pb.nt, pb.tau, P1.theta_of(scheme), True)
    cond = np.linalg.cond(V)
    assert cond > cond_lo
    err = np.abs(U - ref).max() / np.abs(ref).max()
    assert err <= pb.nt * EPS * cond
    # far larger than for a well-conditioned window of the same problem
    pb2 = W.GeometricProblem(space=pb.space, nt=8, dt_last=0.05, tau=1.5, scheme=scheme)
    b2 = P1.build_rhs(pb2, wl.u0)
    r2 = P1.solve_sequential(pb2, b2)
    e2 = np.abs(P1.solve_direct(pb2, b2) - r2).max() / np.abs(r2).max()
    assert e2 < 1e-11 and err > 100 * e2


def test_column_scaling_same_solution():
    pb = GP(nx=31, nu=0.02, ax=1.0, nt=10, dt_last=0.05, tau=1.4, scheme=W.CN)
    b = P1.build_rhs(pb, np.sin(np.pi * pb.space.xs()))
    u1 = P1.solve_direct(pb, b, scaled=True)
    u0 = P1.solve_direct(pb, b, scaled=False)
    V, _ = P1.eigvec_matrices(10, 1.4, 0.5, False)
    assert np.abs(u1 - u0).max() <= 10 * 10 * EPS * np.linalg.cond(V) * np.abs(u0).max()
