"""Pins of O7, ParaDiag-I with the hybrid midpoint + backward-Euler time
discretisation (Section 2.1.2), CPU only.

B is pinned by the printed B^2 of eq. neq2.15 (golden fixture) and by exact
derivatives of linear functions; the Newton roots by the characteristic
equation, their count, the conjugate pairing and the trace of B; the closed-form
V by B V = V D; Cond(V) by the O(Nt^2) bound of the theorem; the three-step
solve by a sparse LU of the whole system and a dense Kronecker solve; the
discretisation by its second-order accuracy and steady states.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as CF
from oracle import hybrid as H
from oracle import operators as O

EPS = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def HP(dim=1, nx=31, ny=1, nu=0.02, ax=0.0, ay=0.0, bcx=W.DIRICHLET, nt=16, T=0.5, lx=1.0):
    sp = W.Space(dim=dim, nx=nx, ny=ny, nu=nu, ax=ax, ay=ay, bc_x=bcx, lx=lx)
    return W.HybridProblem(space=sp, nt=nt, dt=T / nt)


@pytest.mark.parametrize("nt", [6, 8, 13])
def test_b_squared_matches_the_printed_matrix(nt):
    g = json.load(open(os.path.join(GOLDEN, "hybrid_b2nd.json")))
    dt = 0.01
    B = H.time_matrix(nt, dt)
    M = np.rint(4.0 * dt * dt * (B @ B)).astype(int)
    assert np.allclose(4.0 * dt * dt * (B @ B), M, atol=1e-12)
    P = np.zeros((nt, nt), dtype=int)
    for r, row in enumerate(g["first_rows"]):
        P[r, : len(row)] = row
    c = g["interior_row"]
    for r in range(len(g["first_rows"]), nt - len(g["last_rows_right_aligned"])):
        P[r, r - 2 : r + 3] = c
    for j, row in enumerate(g["last_rows_right_aligned"]):
        r = nt - len(g["last_rows_right_aligned"]) + j
        P[r, nt - len(row):] = row
    assert np.array_equal(M, P)


def test_time_matrix_differentiates_linear_functions():
    nt, dt = 9, 0.1
    B = H.time_matrix(nt, dt)
    t = dt * np.arange(1, nt + 1)          # t_1..t_Nt with t_0 = 0 folded into b
    assert np.allclose(B @ t, 1.0, rtol=1e-13)
    assert np.allclose(B @ np.ones(nt), np.r_[0.5 / dt, np.zeros(nt - 1)], atol=1e-12)


@pytest.mark.parametrize("nt", [1, 2, 3, 8, 17, 64, 200])
def test_roots_of_the_characteristic_equation(nt):
    x = H.eigen_roots(nt)
    assert len(x) == nt
    if nt > 1:
        g, _ = H.characteristic(nt, x)
        _, U = H.chebyshev(nt, x)
        assert np.max(np.abs(g) / np.max(np.abs(U), axis=0)) < 1e-12
        # distinct roots
        d = np.abs(x[:, None] - x[None, :]) + np.eye(nt)
        assert d.min() > 1e-8
    # B is real: the roots come in pairs x, -conj(x); trace(dt B) = 1 = sum i x
    assert np.max(np.min(np.abs(x[:, None] + np.conj(x)[None, :]), axis=1)) < 1e-10
    assert abs(np.sum(x) + 1j) < 1e-10 * nt
    # stable shifts: Re(lambda) = -Im(x)/dt > 0
    assert np.all(x.imag < 0)


@pytest.mark.parametrize("nt", [2, 5, 16, 64, 128])
def test_closed_form_eigendecomposition(nt):
    dt = 0.02
    x = H.eigen_roots(nt)
    V = H.eigvec_matrix(x)
    D = np.diag(1j * x / dt)
    B = H.time_matrix(nt, dt)
    rel = np.linalg.norm(B @ V - V @ D) / (np.linalg.norm(B) * np.linalg.norm(V))
    assert rel < 10 * nt * EPS * np.linalg.cond(V)
    assert np.allclose(V[0], 1.0)             # v_{n,0} = 1


def test_condition_number_growth():
    ns = [8, 16, 32, 64, 128, 256]
    c = [np.linalg.cond(H.eigvec_matrix(H.eigen_roots(n))) for n in ns]
    for n, cn in zip(ns, c):
        assert cn <= n * n                   # O(Nt^2), the theorem's bound (constant 1)
    slope = np.polyfit(np.log(ns[2:]), np.log(c[2:]), 1)[0]
    assert 1.5 < slope < 2.0                 # the section reports ~1.75 in practice


CASES = {
    "1d_dirichlet_adv": HP(nx=31, nu=0.02, ax=1.0, nt=16),
    "1d_periodic_paper": HP(nx=64, nu=1e-3, ax=1.0, bcx=W.PERIODIC, lx=2.0, nt=40, T=0.5),
    "2d_small": HP(dim=2, nx=9, ny=7, nu=0.05, ax=0.5, nt=12),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_direct_matches_exact_solution(name):
    pb = CASES[name]
    S = pb.space.size
    u0 = W.uniform(W.SEED_BASE + 95, S, -1, 1)
    f = W.uniform(W.SEED_BASE + 96, (pb.nt + 1) * S, -1, 1).reshape(pb.nt + 1, S)
    b = H.build_rhs(pb, u0, f)
    ref = H.solve_exact(pb, b)
    U = H.solve_direct(pb, b)
    cond = np.linalg.cond(H.eigvec_matrix(H.eigen_roots(pb.nt)))
    assert np.abs(U - ref).max() <= pb.nt * EPS * cond * np.abs(ref).max() * 10
    assert np.abs(H.apply_A(pb, ref) - b).max() <= 1e-10 * np.abs(b).max()


def test_direct_matches_dense_kron():
    pb = HP(nx=5, nu=0.3, ax=0.8, nt=6, T=0.3)
    K = O.stencil(pb.space).toarray()
    A = np.kron(H.time_matrix(6, pb.dt), np.eye(5)) + np.kron(np.eye(6), K)
    b = W.uniform(W.SEED_BASE + 97, 30, -1, 1)
    ref = np.linalg.solve(A, b).reshape(6, 5)
    assert np.abs(H.solve_direct(pb, b.reshape(6, 5)) - ref).max() < 1e-12 * np.abs(ref).max()


def test_second_order_in_time():
    # periodic Fourier mode v, f = 0: the exact semi-discrete solution is
    # exp(-mu t) v; the hybrid scheme is uniformly second order (max over t_n)
    n, j, T = 16, 2, 0.5
    sp = W.Space(dim=1, nx=n, nu=0.05, ax=0.7, bc_x=W.PERIODIC)
    mu = CF.mu_periodic(n, sp.hx, 0.05, 0.7)[j]
    v = np.exp(2j * np.pi * j * np.arange(n) / n)
    errs = []
    for nt in (20, 40, 80, 160):
        pb = W.HybridProblem(space=sp, nt=nt, dt=T / nt)
        U = H.solve_exact(pb, H.build_rhs(pb, v.real))
        t = pb.dt * np.arange(1, nt + 1)
        ex = np.real(np.outer(np.exp(-mu * t), v))
        errs.append(np.abs(U - ex).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(ratios > 3.5) and np.all(ratios < 4.5), ratios


def test_steady_state_is_preserved():
    pb = HP(nx=15, nu=0.2, nt=11)
    x = pb.space.xs()
    phi = np.sin(2 * np.pi * x)
    mu = np.sort(CF.mu_dirichlet(15, pb.space.hx, 0.2, 0.0).real)[1]
    F = np.broadcast_to(phi, (12, 15))
    U = H.solve_exact(pb, H.build_rhs(pb, phi / mu, F))
    assert np.abs(U - phi / mu).max() < 1e-12


# ---- second-order problems: B_2nd = B^2 (eq. neq2.15) ----

def test_second_order_elimination_consistency():
    # for the solution U of (B^2 + K) U = F_v + B F_u, the velocity V = B U - F_u
    # solves the first-order velocity rows B V + K U = F_v (eq. neq2.14b)
    pb = HP(dim=2, nx=7, ny=6, nu=1.0, nt=9, T=0.4)
    K = O.stencil(pb.space)
    S = pb.space.size
    u0 = W.uniform(W.SEED_BASE + 110, S, -1, 1)
    v0 = W.uniform(W.SEED_BASE + 111, S, -1, 1)
    f = W.uniform(W.SEED_BASE + 112, (pb.nt + 1) * S, -1, 1).reshape(pb.nt + 1, S)
    b = H.build_rhs_2nd(pb, u0, v0, f)
    U = H.solve_exact_2nd(pb, b, K)
    B = H.time_matrix(pb.nt, pb.dt)
    Fu = np.zeros((pb.nt, S)); Fu[0] = u0 / (2 * pb.dt)
    Fv = f[1:].copy(); Fv[0] += v0 / (2 * pb.dt)
    Vv = B @ U - Fu
    assert np.abs(B @ Vv + (K @ U.T).T - Fv).max() < 1e-10 * np.abs(Fv).max()


@pytest.mark.parametrize("nt", [5, 12])
def test_second_order_direct_matches_exact(nt):
    pb = HP(dim=2, nx=8, ny=7, nu=1.0, nt=nt, T=0.5)
    S = pb.space.size
    b = H.build_rhs_2nd(pb, W.uniform(W.SEED_BASE + 113, S, -1, 1),
                        W.uniform(W.SEED_BASE + 114, S, -1, 1))
    ref = H.solve_exact_2nd(pb, b)
    U = H.solve_direct_2nd(pb, b)
    assert np.abs(U - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("nt", [4, 8, 16, 32, 64])
def test_table_ex2tab1_errors(nt):
    # the printed errors of the second-order hybrid ParaDiag-I (max over all grid
    # points and time levels); the 5-point Laplacian is exact for the solution's
    # spatial factor, so a 31 x 31 grid reproduces the dx = 1/512 column
    gold = json.load(open(os.path.join(GOLDEN, "ex2tab1_wave_hybrid.json")))
    err_ref = dict(zip(gold["nt"], gold["error"]))[nt]
    wl = W.hybrid_wave2d(n=32, nt=nt)
    pb = wl.problem
    b = H.build_rhs_2nd(pb, wl.u0, wl.u1, wl.f)
    U = H.solve_direct_2nd(pb, b)
    t = pb.dt * np.arange(1, nt + 1)
    ex = np.outer(np.sin(2 * np.pi * t), wl.extra["phi"])
    err = np.abs(U - ex).max()
    assert abs(err - err_ref) <= 0.01 * err_ref, (nt, err, err_ref)
