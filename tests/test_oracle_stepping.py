"""Pins of O1 (sequential stepping), the right-hand side and the adjoint (CPU only)."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as CF
from oracle import dense as D
from oracle import operators as O
from oracle import stepping as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_theta_mode_solution_dirichlet(scheme):
    # K sin(pi x) = mu_1 sin(pi x) (a = 0) => U_n = R(dt mu_1)^n sin(pi x), f = 0
    sp = W.Space(dim=1, nx=31, nu=0.7)
    pb = W.Problem(space=sp, nt=20, dt=0.01, scheme=scheme, alpha=0.1)
    x = sp.xs()
    phi = np.sin(np.pi * x)
    mu1 = CF.mu_dirichlet(31, sp.hx, 0.7, 0.0).real.min()
    U = S.solve_sequential(pb, O.build_rhs(pb, phi))
    R = CF.stability_function(pb.dt * mu1, pb.theta_eff)
    ref = np.outer(R ** np.arange(1, 21), phi)
    assert np.abs(U - ref).max() < 1e-13


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_theta_mode_solution_periodic_advection(scheme):
    n, j = 16, 2
    sp = W.Space(dim=1, nx=n, nu=0.05, ax=1.3, bc_x=W.PERIODIC)
    pb = W.Problem(space=sp, nt=12, dt=0.02, scheme=scheme, alpha=0.1)
    v = np.exp(2j * np.pi * j * np.arange(n) / n)
    mu = CF.mu_periodic(n, sp.hx, 0.05, 1.3)[j]
    U = S.solve_sequential(pb, O.build_rhs(pb, v.real))
    R = CF.stability_function(pb.dt * mu, pb.theta_eff)
    ref = np.real(np.outer(R ** np.arange(1, 13), v))
    assert np.abs(U - ref).max() < 1e-13


@pytest.mark.parametrize("scheme", [W.BE, W.CN])
def test_theta_constant_source(scheme):
    # U_0 = 0, f = phi constant: U_n = (1 - R^n) phi / mu
    sp = W.Space(dim=1, nx=15, nu=0.2)
    pb = W.Problem(space=sp, nt=9, dt=0.05, scheme=scheme, alpha=0.1)
    phi = np.sin(2 * np.pi * sp.xs())
    mu = CF.mu_dirichlet(15, sp.hx, 0.2, 0.0).real
    mu2 = np.sort(mu)[1]
    F = np.broadcast_to(phi, (10, 15))
    U = S.solve_sequential(pb, O.build_rhs(pb, np.zeros(15), None, F))
    R = CF.stability_function(pb.dt * mu2, pb.theta_eff)
    ref = np.outer((1 - R ** np.arange(1, 10)) / mu2, phi)
    assert np.abs(U - ref).max() < 1e-13


@pytest.mark.parametrize("scheme,order", [(W.BE, 1.0), (W.CN, 2.0)])
def test_theta_convergence_order_manufactured(scheme, order):
    # u = sin(pi x) cos(t) + x(1-x) e^{-t}; f = u_t - nu u_xx + a u_x (time dependent source)
    nu, a, T = 0.1, 0.5, 0.5
    u = lambda x, t: np.sin(np.pi * x) * np.cos(t) + x * (1 - x) * np.exp(-t)
    ut = lambda x, t: -np.sin(np.pi * x) * np.sin(t) - x * (1 - x) * np.exp(-t)
    ux = lambda x, t: np.pi * np.cos(np.pi * x) * np.cos(t) + (1 - 2 * x) * np.exp(-t)
    uxx = lambda x, t: -np.pi**2 * np.sin(np.pi * x) * np.cos(t) - 2 * np.exp(-t)
    errs = []
    for k in range(3):
        nt = 16 * 2**k
        nx = (255 if scheme == W.BE else 8 * 2**k * 4 - 1)
        sp = W.Space(dim=1, nx=nx, nu=nu, ax=a)
        pb = W.Problem(space=sp, nt=nt, dt=T / nt, scheme=scheme, alpha=0.1)
        x = sp.xs()
        t = np.arange(nt + 1) * pb.dt
        F = np.array([ut(x, s) - nu * uxx(x, s) + a * ux(x, s) for s in t])
        U = S.solve_sequential(pb, O.build_rhs(pb, u(x, 0.0), None, F))
        errs.append(np.abs(U - np.array([u(x, s) for s in t[1:]])).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - order) < 0.2), orders


def test_leapfrog_mode_solution_with_velocity():
    # per eigenmode: U_n = cos(n th) U_0 + (dt / sin th) sin(n th) u_1, cos th = 1/(1 + dt^2 mu/2)
    sp = W.Space(dim=1, nx=31, nu=1.0)
    pb = W.Problem(space=sp, nt=40, dt=0.05, scheme=W.LEAPFROG, alpha=0.1)
    x = sp.xs()
    p1, p3 = np.sin(np.pi * x), np.sin(3 * np.pi * x)
    mus = np.sort(CF.mu_dirichlet(31, sp.hx, 1.0, 0.0).real)
    th1 = CF.leapfrog_mode_angle(mus[0], pb.dt)
    th3 = CF.leapfrog_mode_angle(mus[2], pb.dt)
    U = S.solve_sequential(pb, O.build_rhs(pb, p1, 0.7 * p3))
    n = np.arange(1, 41)
    ref = (np.outer(np.cos(n * th1), p1)
           + np.outer(pb.dt / np.sin(th3) * np.sin(n * th3), 0.7 * p3))
    assert np.abs(U - ref).max() < 1e-12


def test_leapfrog_second_order_like_table_t4a():
    # Table T4A reports second order (1.9, 1.9, 2.0, 2.0) for the leap-frog all-at-once
    # system with the exact solution sin(pi x) sin(pi y) e^t; same problem in 2D, small meshes.
    gold = json.load(open(os.path.join(GOLDEN, "t4a_wave2d_gmres.json")))
    errs = []
    for n in (15, 31, 63):
        sp = W.Space(dim=2, nx=n, ny=n, nu=1.0)
        pb = W.Problem(space=sp, nt=n + 1, dt=2.0 / (n + 1), scheme=W.LEAPFROG, alpha=0.1)
        X, Y = sp.mesh()
        ph = (np.sin(np.pi * X) * np.sin(np.pi * Y)).reshape(-1)
        t = np.arange(pb.nt + 1) * pb.dt
        F = np.outer(np.exp(t), (1 + 2 * np.pi**2) * ph)
        U = S.solve_sequential(pb, O.build_rhs(pb, ph, ph, F))
        e = U - np.outer(np.exp(t[1:]), ph)
        errs.append(np.max(np.sqrt(sp.hx**2 * np.sum(e * e, axis=1))))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders >= min(gold["orders"]) - 0.15) and np.all(orders <= 2.15), orders
    # same magnitude as the printed error at the coarsest printed mesh (within a factor 2)
    assert 0.5 < errs[1] / gold["errors_alpha_0.1"][0] < 2.0


@pytest.mark.parametrize("scheme", [W.BE, W.CN, W.LEAPFROG])
def test_sequential_equals_dense_solve(scheme):
    sp = W.Space(dim=2, nx=4, ny=3, nu=0.2, ax=(0 if scheme == W.LEAPFROG else 1.0),
                 ay=(0 if scheme == W.LEAPFROG else -0.5), bc_x=W.PERIODIC)
    pb = W.Problem(space=sp, nt=7, dt=0.1, scheme=scheme, alpha=0.1)
    b = np.random.default_rng(2).standard_normal((7, 12))
    U = S.solve_sequential(pb, b)
    assert np.abs(U - D.solve_dense(D.dense_A(pb), b)).max() < 1e-12
    L = S.solve_adjoint_sequential(pb, b)
    assert np.abs(L - D.solve_dense(D.dense_A(pb).T, b)).max() < 1e-12


@pytest.mark.parametrize("scheme", [W.BE, W.CN, W.LEAPFROG])
def test_adjoint_dot_product(scheme):
    sp = W.Space(dim=1, nx=40, nu=0.05, ax=(0 if scheme == W.LEAPFROG else 1.0))
    pb = W.Problem(space=sp, nt=30, dt=0.02, scheme=scheme, alpha=0.1)
    rng = np.random.default_rng(3)
    b, g = rng.standard_normal((30, 40)), rng.standard_normal((30, 40))
    lhs = np.sum(S.solve_sequential(pb, b) * g)
    rhs = np.sum(b * S.solve_adjoint_sequential(pb, g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("scheme", [W.BE, W.CN, W.LEAPFROG])
def test_xmodes_stepping_matches_dense_kronecker(scheme):
    """The mode-by-mode O1 (naive DFT along a periodic x, dense LU per mode)
    equals the dense Kronecker solve of A u = b (O3) on a tiny 2D problem with
    advection in both directions, and the sparse-LU stepping."""
    sp = W.Space(dim=2, nx=6, ny=5, nu=0.05, ax=1.0, ay=0.5, bc_x=W.PERIODIC)
    pb = W.Problem(space=sp, nt=8, dt=0.05, scheme=scheme, alpha=0.1)
    b = W.uniform(W.SEED_BASE + 60, pb.unknowns, -1.0, 1.0).reshape(pb.nt, -1)
    u_dense = D.solve_dense(D.dense_A(pb), b)
    u_modes = S.solve_sequential_xmodes(pb, b, chunks=3)
    assert np.abs(u_modes - u_dense).max() <= 1e-12 * np.abs(u_dense).max()
    assert np.abs(S.solve_sequential(pb, b) - u_dense).max() <= 1e-12 * np.abs(u_dense).max()


def test_xmodes_stepping_process_pool():
    """The same solve with its modes spread over two spawned processes."""
    import multiprocessing as mp
    sp = W.Space(dim=2, nx=9, ny=7, nu=0.02, ax=1.0, ay=0.5, bc_x=W.PERIODIC)
    pb = W.Problem(space=sp, nt=6, dt=0.1, scheme=W.CN, alpha=0.1)
    b = W.uniform(W.SEED_BASE + 61, pb.unknowns, -1.0, 1.0).reshape(pb.nt, -1)
    with mp.get_context("spawn").Pool(2) as pool:
        u = S.solve_sequential_xmodes(pb, b, pool=pool, chunks=2)
    ref = S.solve_sequential(pb, b)
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()
