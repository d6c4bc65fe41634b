"""Pins of O2 (naive ParaDiag-II), O3 (dense Kronecker) and the convergence
theory (CPU only)."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as CF
from oracle import dense as D
from oracle import operators as O
from oracle import paradiag as PD
from oracle import stepping as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prob(scheme, nx=6, ny=1, nt=8, alpha=0.05, dim=1, bcx=W.DIRICHLET):
    lf = scheme == W.LEAPFROG
    sp = W.Space(dim=dim, nx=nx, ny=ny, nu=0.1, ax=0.0 if lf else 1.0, ay=0.0 if lf else 0.5,
                 bc_x=bcx)
    return W.Problem(space=sp, nt=nt, dt=1.0 / nt, scheme=scheme, alpha=alpha)


@pytest.mark.parametrize("scheme", [W.BE, W.CN, W.LEAPFROG])
@pytest.mark.parametrize("alpha", [1.0, 0.1, 1e-3])
@pytest.mark.parametrize("dim", [1, 2])
def test_precond_naive_equals_dense(scheme, alpha, dim):
    pb = _prob(scheme, nx=5, ny=(4 if dim == 2 else 1), nt=8, alpha=alpha, dim=dim,
               bcx=(W.PERIODIC if dim == 2 else W.DIRICHLET))
    r = np.random.default_rng(4).standard_normal((pb.nt, pb.space.size))
    z = PD.precond_apply(pb, r)
    zd = D.solve_dense(D.dense_P(pb), r)
    assert np.abs(z - zd).max() <= 1e-10 * np.abs(zd).max()
    # the invariant P z = r
    assert np.abs(O.apply_P(pb, z) - r).max() <= 1e-9 * np.abs(r).max()


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
@pytest.mark.parametrize("alpha", [1e-2, 0.1, 0.4])
def test_stationary_rate_closed_form(scheme, alpha):
    # rho(I - P^{-1} A) = max_mu |alpha R^Nt/(1 - alpha R^Nt)| (rank-one per mode, eq. 5.1)
    pb = _prob(scheme, nx=15, nt=16, alpha=alpha)
    sp = pb.space
    mus = CF.mu_dirichlet(sp.nx, sp.hx, sp.nu, sp.ax)
    rho = CF.stationary_rate(mus, pb.dt, pb.nt, alpha, pb.theta_eff)
    ev = D.iteration_matrix_spectrum(pb)
    assert abs(np.abs(ev).max() - rho) <= 1e-9 * max(rho, 1e-12) + 1e-14
    # Theorem 5.1 (|R| <= 1): rho <= alpha/(1-alpha), the trapezoidal bound of Theorem 1.2
    assert rho <= alpha / (1 - alpha) * (1 + 1e-12)
    if scheme == W.BE:
        # Theorem 1.2 (BE) with the discrete damping (1 + dt r)^{-Nt} in place of its
        # dt -> 0 limit e^{-T r}, r = min Re mu
        q = (1 + pb.dt * mus.real.min()) ** (-pb.nt)
        assert rho <= alpha * q / (1 - alpha * q) * (1 + 1e-12)


def test_theorem31_spectrum_and_annulus():
    pb = _prob(W.LEAPFROG, nx=7, nt=12, alpha=0.2)
    sp = pb.space
    mus = CF.mu_dirichlet(sp.nx, sp.hx, sp.nu, 0.0).real
    ev = D.preconditioned_spectrum(pb)
    unit = np.abs(ev - 1.0) < 1e-9
    assert unit.sum() == (pb.nt - 2) * sp.nx
    th = CF.theorem31_spectrum(mus, pb.dt, pb.nt, pb.alpha)
    rest = ev[~unit]
    assert np.abs(rest[:, None] - th[None, :]).min(axis=1).max() < 1e-10
    lo, hi = CF.theorem31_annulus(pb.alpha)
    assert np.all(np.abs(rest - 1) >= lo - 1e-12) and np.all(np.abs(rest - 1) <= hi + 1e-12)


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
@pytest.mark.parametrize("a", [1.0, 0.0])
def test_stationary_converges_to_sequential(scheme, a):
    w = W.ade1d(nx=31, nt=16, scheme=scheme, alpha=0.1, nu=0.05, a=a)
    pb = w.problem
    b = O.build_rhs(pb, w.u0, None, w.f)
    u_ex = S.solve_sequential(pb, b)
    u, it, rel, hist = PD.stationary(pb, b, tol=1e-13, maxit=30, history=True)
    assert rel <= 1e-13 and it <= 12
    assert np.abs(u - u_ex).max() <= 1e-12 * np.abs(u_ex).max()
    if a != 0.0:
        return   # K non-normal: the max-norm contraction is not the spectral radius
    # symmetric K: after the first step the error lies in the range of the per-mode
    # rank-one propagator and then contracts by the closed-form rate
    sp = pb.space
    rho = CF.stationary_rate(CF.mu_dirichlet(sp.nx, sp.hx, sp.nu, sp.ax), pb.dt, pb.nt,
                             pb.alpha, pb.theta_eff)
    e1 = np.abs(hist[1] - u_ex).max()
    e2 = np.abs(hist[2] - u_ex).max()
    assert e2 <= 10 * rho * e1 + 1e-14 * np.abs(u_ex).max()
    assert e2 >= 0.01 * rho * e1


def test_random_initial_guess_like_fig_13a():
    # the WR experiment starts from a random guess uniform in [-20, 20] (Section 2.2)
    w = W.ade1d(nx=31, nt=32, scheme=W.CN, alpha=1e-2)
    pb = w.problem
    b = O.build_rhs(pb, w.u0, None, w.f)
    g = W.uniform(7, pb.unknowns, -20.0, 20.0).reshape(pb.nt, -1)
    u, it, rel = PD.stationary(pb, b, u_init=g, tol=1e-12, maxit=20)
    assert rel <= 1e-12 and it <= 8


def test_fgmres_table_t4a_iterations():
    gold = json.load(open(os.path.join(GOLDEN, "t4a_wave2d_gmres.json")))
    n = 31
    sp = W.Space(dim=2, nx=n, ny=n, nu=1.0)
    pb = W.Problem(space=sp, nt=n + 1, dt=2.0 / (n + 1), scheme=W.LEAPFROG, alpha=gold["alpha"])
    X, Y = sp.mesh()
    ph = (np.sin(np.pi * X) * np.sin(np.pi * Y)).reshape(-1)
    t = np.arange(pb.nt + 1) * pb.dt
    F = np.outer(np.exp(t), (1 + 2 * np.pi**2) * ph)
    K = O.stencil(sp)
    b = O.build_rhs(pb, ph, ph, F, K)
    u, it, rel = PD.fgmres(pb, b, tol=1e-10, restart=30, maxit=60, K=K)
    assert it == gold["iterations_alpha_0.1"][0]
    assert rel <= 1e-10
    u_ex = S.solve_sequential(pb, b, K)
    assert np.abs(u - u_ex).max() <= 1e-9 * np.abs(u_ex).max()
    # alpha = 1 (Strang circulant) needs more iterations (Table T4A)
    pb1 = W.Problem(space=sp, nt=n + 1, dt=2.0 / (n + 1), scheme=W.LEAPFROG, alpha=1.0)
    _, it1, _ = PD.fgmres(pb1, b, tol=1e-10, restart=30, maxit=60, K=K)
    assert it1 > it
