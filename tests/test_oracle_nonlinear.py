"""Pins of the nonlinear oracle (O10: eq. 1.4 and the simplified Newton
iteration eq. 1.5 with an averaged Jacobian).

The pins that tie it to something other than itself:
  * a linear reaction phi(u) = a1 u is the linear problem with K + a1 I, solved
    by the pinned linear oracles (sequential stepping O1, stationary iteration
    O2): same right-hand side, same solution, and -- because the averaged
    Jacobian is then exactly K + a1 I -- the same iterates;
  * the manufactured solution u = exp(-t) sin(pi x): errors fall as dt^2 + h^2
    for Crank-Nicolson and as dt for backward Euler and theta = 0.7;
  * sequential stepping with Newton per step equals a full Newton solve of the
    whole all-at-once system (an independent algorithm for eq. 1.4);
  * the averaged shift of a constant field is phi' at that value.
"""
import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

import workloads as W
from oracle import nonlinear as NL
from oracle import operators as O
from oracle import paradiag as PD
from oracle import stepping as ST


def small2d(nt=16, scheme=W.CN, reaction=(-1.0, 0.0, 1.0), theta=None):
    wl = W.nl_ade2d(nx=15, ny=13, nt=nt, nu=1e-2, scheme=scheme, alpha=1e-2, reaction=reaction)
    if theta is not None:   # a general theta-method on the same data
        pb = W.Problem(space=wl.problem.space, nt=nt, dt=wl.problem.dt, scheme=W.THETA,
                       alpha=1e-2, theta=theta)
        wl = W.Workload(wl.name, pb, wl.u0, None, None, wl.seed, extra=wl.extra)
    return wl


def test_reaction_and_derivative():
    a = (0.3, -1.2, 2.5)
    u = np.linspace(-2, 2, 41)
    assert np.allclose(NL.reaction(u, a), 0.3 * u - 1.2 * u**2 + 2.5 * u**3, rtol=0, atol=1e-14)
    h = 1e-6
    fd = (NL.reaction(u + h, a) - NL.reaction(u - h, a)) / (2 * h)
    assert np.allclose(NL.reaction_prime(u, a), fd, rtol=0, atol=1e-8)


def test_average_shift_of_constant_field():
    a = (0.5, 1.0, 2.0)
    for c in (-1.5, 0.0, 0.7):
        U = np.full((8, 20), c)
        assert NL.average_jacobian_shift(U, a) == pytest.approx(0.5 + 2.0 * c + 6.0 * c * c, abs=1e-14)
    assert NL.average_jacobian_shift(np.random.default_rng(0).normal(size=(4, 9)), (0.8, 0.0, 0.0)) \
        == pytest.approx(0.8, abs=1e-15)


@pytest.mark.parametrize("scheme", [W.BE, W.CN, W.THETA])
def test_linear_reaction_is_the_shifted_linear_problem(scheme):
    a1 = 0.7
    wl = small2d(scheme=scheme, reaction=(a1, 0.0, 0.0),
                 theta=0.7 if scheme == W.THETA else None)
    pb = wl.problem
    K = O.stencil(pb.space)
    Ks = (K + a1 * sps.identity(K.shape[0])).tocsr()
    f = W.uniform(W.SEED_BASE + 400, (pb.nt + 1) * pb.space.size, -1, 1).reshape(pb.nt + 1, -1)
    b = NL.build_rhs_nl(pb, wl.u0, (a1, 0, 0), f=f)
    assert np.allclose(b, O.build_rhs(pb, wl.u0, f=f, K=Ks), rtol=0, atol=1e-12)
    U = W.uniform(W.SEED_BASE + 401, pb.unknowns, -1, 1).reshape(pb.nt, -1)
    r = NL.residual_nl(pb, U, b, (a1, 0, 0))
    assert np.allclose(r, b - O.apply_A(pb, U, K=Ks), rtol=0, atol=1e-11)
    u_nl = NL.solve_sequential_nl(pb, b, (a1, 0, 0))
    u_lin = ST.solve_sequential(pb, b, K=Ks)
    assert np.abs(u_nl - u_lin).max() <= 1e-12 * np.abs(u_lin).max()
    # sigma = a1 exactly: the iterates are those of the linear stationary iteration
    u_sn, it, hist = NL.simplified_newton(pb, b, (a1, 0, 0), tol=1e-12)
    u_st, it_st, _ = PD.stationary(pb, b, tol=1e-12, K=Ks)
    assert it == it_st
    assert np.abs(u_sn - u_st).max() <= 1e-12 * np.abs(u_st).max()


@pytest.mark.parametrize("scheme,sizes,ratio,first", [
    (W.CN, [(15, 8), (31, 16), (63, 32)], (3.6, 4.5), 2.5e-3),
    (W.BE, [(255, 8), (255, 16), (255, 32)], (1.8, 2.2), 4e-3),
    (W.THETA, [(255, 8), (255, 16), (255, 32)], (1.8, 2.2), 1.5e-3),   # theta = 0.7
])
def test_manufactured_solution_convergence(scheme, sizes, ratio, first):
    errs = []
    for nx, nt in sizes:
        wl = W.nl_manufactured1d(nx=nx, nt=nt, scheme=scheme,
                                 theta=0.7 if scheme == W.THETA else 1.0)
        pb = wl.problem
        a = wl.extra["reaction"]
        b = NL.build_rhs_nl(pb, wl.u0, a, f=wl.f)
        U = NL.solve_sequential_nl(pb, b, a)
        errs.append(np.abs(U - wl.extra["exact"]).max())
    assert errs[0] < first, errs
    for e0, e1 in zip(errs, errs[1:]):
        assert ratio[0] < e0 / e1 < ratio[1], errs


def test_sequential_equals_full_newton_on_the_all_at_once_system():
    wl = small2d(nt=8, reaction=(-1.0, 0.5, 1.0))
    pb = wl.problem
    a = wl.extra["reaction"]
    b = NL.build_rhs_nl(pb, wl.u0, a)
    U = NL.solve_sequential_nl(pb, b, a)
    assert np.linalg.norm(NL.residual_nl(pb, U, b, a)) <= 1e-12 * np.linalg.norm(b)
    # full Newton: Jacobian B1 (x) I + (B2 (x) I) blkdiag(K + diag phi'(U_n))
    K = O.stencil(pb.space)
    B1, B2 = O.time_matrices(pb)
    S = pb.space.size
    X = np.zeros_like(U)
    for _ in range(30):
        r = NL.residual_nl(pb, X, b, a)
        D = sps.block_diag([K + sps.diags(NL.reaction_prime(X[n], a)) for n in range(pb.nt)])
        J = (sps.kron(sps.csr_matrix(B1), sps.identity(S)) +
             sps.kron(sps.csr_matrix(B2), sps.identity(S)) @ D).tocsc()
        dx = spla.spsolve(J, r.reshape(-1)).reshape(pb.nt, S)
        X += dx
        if np.abs(dx).max() <= 1e-15 * np.abs(X).max():
            break
    assert np.abs(X - U).max() <= 1e-12 * np.abs(U).max()


@pytest.mark.parametrize("scheme", [W.BE, W.CN, W.THETA])
def test_simplified_newton_reaches_the_exact_solution(scheme):
    wl = small2d(scheme=scheme, theta=0.7 if scheme == W.THETA else None)
    pb = wl.problem
    a = wl.extra["reaction"]
    b = NL.build_rhs_nl(pb, wl.u0, a)
    U, it, hist = NL.simplified_newton(pb, b, a, tol=1e-12)
    assert hist[-1] <= 1e-12 and it <= 20
    # linear convergence: every step reduces the residual
    assert all(h1 < h0 for h0, h1 in zip(hist, hist[1:]))
    Ue = NL.solve_sequential_nl(pb, b, a)
    assert np.abs(U - Ue).max() <= 1e-10 * np.abs(Ue).max()


def test_leapfrog_rejected():
    sp = W.Space(dim=1, nx=7)
    pb = W.Problem(space=sp, nt=4, dt=0.1, scheme=W.LEAPFROG, alpha=0.1)
    with pytest.raises(ValueError):
        NL.residual_nl(pb, np.zeros((4, 7)), np.zeros((4, 7)), (0, 0, 1))
