"""Pins of the oracle's spatial and temporal operators (CPU only).

K is pinned by closed-form spectra and by its truncation error against the
PDE; B1/B2/C1/C2 by Lemma 1 (closed-form eigenvalues and the factorisation
C = V D V^{-1}) and by the paper's explicit WR right-hand side (eq. 2.11b).
"""
import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as CF
from oracle import operators as O
from oracle import paradiag as PD


def test_splitmix64_published_vector():
    # Reference outputs of SplitMix64 seeded with 1234567 (the public C reference).
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    assert [int(v) for v in W.splitmix64(1234567, 5)] == ref


@pytest.mark.parametrize("nu,a", [(1e-2, 1.0), (1.0, 0.0), (3e-3, -2.0)])
def test_periodic_K_spectrum(nu, a):
    n = 17
    h = 1.0 / n
    K = O.stencil_1d(n, h, nu, a, W.PERIODIC).toarray()
    ev = np.linalg.eigvals(K)
    mu = CF.mu_periodic(n, h, nu, a)
    d = np.abs(ev[:, None] - mu[None, :]).min(axis=1)
    assert d.max() < 1e-9 * np.abs(mu).max()
    # eigenvector check fixes the sign of the advection term
    j = 3
    v = np.exp(2j * np.pi * j * np.arange(n) / n)
    assert np.allclose(K @ v, mu[j] * v, rtol=0, atol=1e-9 * np.abs(mu).max())


@pytest.mark.parametrize("nu,a", [(1e-2, 1.0), (1.0, 0.0), (1e-3, 1.0)])
def test_dirichlet_K_spectrum(nu, a):
    n = 15
    h = 1.0 / (n + 1)
    K = O.stencil_1d(n, h, nu, a, W.DIRICHLET).toarray()
    ev = np.linalg.eigvals(K)
    mu = CF.mu_dirichlet(n, h, nu, a)
    d = np.abs(ev[:, None] - mu[None, :]).min(axis=1)
    assert d.max() < 1e-7 * np.abs(mu).max()


def test_K_truncation_error_second_order():
    # K u ~ -nu u'' + a u' for u = sin(2 pi x) + x (1 - x) e^x on interior points
    nu, a = 0.3, 1.7
    errs = []
    for n in (31, 63, 127):
        sp = W.Space(dim=1, nx=n, nu=nu, ax=a)
        x = sp.xs()
        u = lambda x: np.sin(2 * np.pi * x) + x * (1 - x) * np.exp(x)
        du = lambda x: 2 * np.pi * np.cos(2 * np.pi * x) + (1 - x - x * x) * np.exp(x)
        d2u = lambda x: -4 * np.pi**2 * np.sin(2 * np.pi * x) + (-3 * x - x * x) * np.exp(x)
        # boundary values are 0 (Dirichlet) for this u at x = 0 and 1
        Ku = O.stencil(sp) @ u(x)
        errs.append(np.abs(Ku - (-nu * d2u(x) + a * du(x))).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.9)


def test_2d_K_is_kronecker_sum():
    sp = W.Space(dim=2, nx=7, ny=5, nu=0.1, ax=1.0, ay=0.5, bc_x=W.PERIODIC, bc_y=W.DIRICHLET)
    K = O.stencil(sp).toarray()
    mx = CF.mu_periodic(7, sp.hx, 0.1, 1.0)
    my = CF.mu_dirichlet(5, sp.hy, 0.1, 0.5)
    mu = (mx[None, :] + my[:, None]).reshape(-1)
    ev = np.linalg.eigvals(K)
    d = np.abs(ev[:, None] - mu[None, :]).min(axis=1)
    assert d.max() < 1e-8 * np.abs(mu).max()
    # x is the fast index: row s couples to s+1 (x+1) and s+nx (y+1)
    row = K[2 * 7 + 3]
    assert row[2 * 7 + 4] == pytest.approx(-0.1 / sp.hx**2 + 1.0 / (2 * sp.hx))
    assert row[3 * 7 + 3] == pytest.approx(-0.1 / sp.hy**2 + 0.5 / (2 * sp.hy))


@pytest.mark.parametrize("scheme", [W.BE, W.CN, W.LEAPFROG])
@pytest.mark.parametrize("alpha", [1.0, 0.1, 1e-3])
def test_lemma1_eigenvalues_closed_form(scheme, alpha):
    pb = W.Problem(space=W.Space(dim=1, nx=3), nt=16, dt=0.05, scheme=scheme, alpha=alpha)
    l1, l2 = PD.eigenvalues(pb)
    c1, c2 = CF.lemma1_eigenvalues(pb)
    assert np.abs(l1 - c1).max() <= 1e-13 * np.abs(c1).max()
    assert np.abs(l2 - c2).max() <= 1e-14


@pytest.mark.parametrize("scheme", [W.BE, W.CN, W.LEAPFROG])
def test_lemma1_factorisation(scheme):
    # C_j = V D_j V^{-1}, V = Gamma^{-1} F^*, with D_j from the closed forms
    pb = W.Problem(space=W.Space(dim=1, nx=3), nt=12, dt=0.1, scheme=scheme, alpha=0.02)
    C1, C2 = O.circulant_matrices(pb)
    F = PD.fourier_matrix(pb.nt)
    g = PD.gamma(pb)
    V = np.diag(1 / g) @ F.conj().T
    Vi = F @ np.diag(g)
    d1, d2 = CF.lemma1_eigenvalues(pb)
    assert np.allclose(V @ np.diag(d1) @ Vi, C1, atol=1e-10 * np.abs(C1).max())
    assert np.allclose(V @ np.diag(d2) @ Vi, C2, atol=1e-12)
    # eq. 2.13: Cond_2(V) <= 1/alpha
    assert np.linalg.cond(V) <= 1 / pb.alpha * (1 + 1e-12)


def test_wr_rhs_matches_eq_2_11b():
    # eq. 2.11b: b^{k-1} = ((U0 - alpha U^{k-1}_Nt)(I/dt - (1-theta) A), 0, ..., 0), f = 0;
    # the stationary step P u^k = (P - A) u^{k-1} + b must have exactly this right side.
    for scheme in (W.BE, W.CN):
        sp = W.Space(dim=1, nx=9, nu=0.05, ax=1.0)
        pb = W.Problem(space=sp, nt=10, dt=0.1, scheme=scheme, alpha=0.03)
        K = O.stencil(sp)
        rng = np.random.default_rng(1)
        u0 = rng.standard_normal(9)
        U = rng.standard_normal((10, 9))
        b = O.build_rhs(pb, u0, K=K)
        lhs = O.apply_P(pb, U, K) - O.apply_A(pb, U, K) + b
        th = pb.theta_eff
        w = u0 - pb.alpha * U[-1]
        ref = np.zeros_like(U)
        ref[0] = w / pb.dt - (1 - th) * (K @ w)
        assert np.allclose(lhs, ref, atol=1e-12 * np.abs(ref).max())


def test_leapfrog_circulant_corner_eq_3_4():
    # eq. 3.4: first row (1, ..., alpha, -2 alpha)/dt^2 and (1/2)(1, ..., alpha, 0);
    # second row (-2, 1, ..., alpha)/dt^2 and (1/2)(0, 1, ..., alpha).
    pb = W.Problem(space=W.Space(dim=1, nx=2), nt=6, dt=0.5, scheme=W.LEAPFROG, alpha=0.3)
    C1, C2 = O.circulant_matrices(pb)
    s = pb.dt**2
    assert np.allclose(C1[0] * s, [1, 0, 0, 0, 0.3, -0.6])
    assert np.allclose(C1[1] * s, [-2, 1, 0, 0, 0, 0.3])
    assert np.allclose(C2[0] * 2, [1, 0, 0, 0, 0.3, 0])
    assert np.allclose(C2[1] * 2, [0, 1, 0, 0, 0, 0.3])
