"""Pins of the oracle's Lemma 1 tables against 50-digit evaluations.

Lemma 1: D_j = diag(sqrt(Nt) F Gamma c_j), i.e. lambda_{j,n} = sum_m c_j[m] w_n^m
with w_n = alpha^{1/Nt} omega^n, omega = exp(2 pi i/Nt), and F the unitary
Fourier matrix [omega^{(l1-1)(l2-1)}]/sqrt(Nt).  The oracle evaluates the
eigenvalues by their closed forms written without cancellation
(closed_forms.lemma1_eigenvalues) and forms F with the exponent reduced modulo
Nt.  Here both are compared with the same quantities computed by mpmath at 50
significant digits straight from the definitions: the slow modes (n near 0 and
near Nt, where w is close to 1) and long time axes are where a cancelling
evaluation loses digits, so they are sampled explicitly.
"""
import numpy as np
import pytest

import workloads as W
from oracle import closed_forms as CF
from oracle import paradiag as PD

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50

EPS = 2.0 ** -53


def lam_exact(pb, n):
    """sum_m c_j[m] w_n^m at 50 digits (the first columns of the theta-method
    and leap-frog matrices, eq. 2.5b / eq. 3.2b)."""
    nt = pb.nt
    w = mp.mpf(pb.alpha) ** (mp.mpf(1) / nt) * mp.expjpi(mp.mpf(2 * n) / nt)
    dt = mp.mpf(pb.dt)
    if pb.scheme == W.LEAPFROG:
        return (1 - 2 * w + w * w) / dt**2, (1 + w * w) / 2
    th = mp.mpf(pb.theta_eff)
    return (1 - w) / dt, th + (1 - th) * w


def rel(a, b):
    return float(abs(mp.mpc(complex(a)) - b) / abs(b))


@pytest.mark.parametrize("scheme,theta", [(W.BE, None), (W.CN, None), (W.THETA, 0.7),
                                          (W.LEAPFROG, None)])
@pytest.mark.parametrize("nt", [16, 1000, 4096, 32768])
@pytest.mark.parametrize("alpha", [1e-2, 1e-3, 0.5])
def test_closed_forms_to_50_digits(scheme, theta, nt, alpha):
    kw = {} if theta is None else {"theta": theta}
    pb = W.Problem(space=W.Space(dim=1, nx=3), nt=nt, dt=1.0 / nt, scheme=scheme, alpha=alpha, **kw)
    l1, l2 = CF.lemma1_eigenvalues(pb)
    for n in sorted({0, 1, 2, 3, nt // 4, nt // 2 - 1, nt // 2, nt // 2 + 1, nt - 3, nt - 2, nt - 1}):
        e1, e2 = lam_exact(pb, n)
        # a few roundings of order-one terms: well under 1e-15 relative
        assert rel(l1[n], e1) <= 16 * EPS, (n, rel(l1[n], e1))
        assert rel(l2[n], e2) <= 16 * EPS, (n, rel(l2[n], e2))


def test_conjugate_pairs_hold():
    # lambda_{Nt-n} = conj(lambda_n) for real first columns; the angle taken in
    # (-pi, pi] makes the two evaluations mirror images
    pb = W.Problem(space=W.Space(dim=1, nx=3), nt=4096, dt=1.0 / 4096, scheme=W.BE, alpha=1e-2)
    l1, l2 = CF.lemma1_eigenvalues(pb)
    n = np.arange(1, pb.nt)
    assert (np.abs(l1[pb.nt - n] - np.conj(l1[n])) / np.abs(l1[n])).max() <= 8 * EPS
    assert (np.abs(l2[pb.nt - n] - np.conj(l2[n])) / np.abs(l2[n])).max() <= 8 * EPS


@pytest.mark.parametrize("nt", [255, 4096])
def test_fourier_matrix_entries_to_50_digits(nt):
    F = PD.fourier_matrix(nt)
    rng = np.random.default_rng(7)
    idx = list(rng.integers(0, nt, size=(40, 2))) + [(nt - 1, nt - 1), (nt - 1, nt - 2), (1, 1)]
    s = mp.sqrt(nt)
    for l1, l2 in idx:
        exact = mp.expjpi(mp.mpf(2 * int(l1) * int(l2)) / nt) / s
        err = abs(mp.mpc(complex(F[l1, l2])) - exact)
        # the phase 2 pi q/Nt (q < Nt) carries about 2 eps relative, i.e. up to
        # 4 pi eps absolute, then exp and the division: 16 eps / sqrt(Nt) at most
        # (the unreduced exponent would put about 2 pi eps Nt / sqrt(Nt) there)
        assert float(err) <= 16 * EPS / np.sqrt(nt), (l1, l2, float(err))
