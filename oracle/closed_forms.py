"""O4: closed forms that pin the oracle (and, through it, the GPU path).

* Lemma 1 eigenvalues in closed form.  With w_n = alpha^{1/Nt} omega^n,
  omega = exp(2 pi i/Nt), the diagonal of D_j is sum_m c_j[m] w_n^m, so
    theta-method: lambda_1 = (1 - w)/dt,      lambda_2 = theta + (1-theta) w,
    leap-frog:    lambda_1 = (1 - w)^2/dt^2,  lambda_2 = (1 + w^2)/2
  (every band entry of the first columns inside the matrix: Nt > band).
* Eigenvalues of the centred 1D operators: periodic (circulant)
    mu_j = (2 nu/h^2)(1 - cos(2 pi j/n)) + i (a/h) sin(2 pi j/n),
  and Dirichlet (tridiagonal Toeplitz tridiag(l, d, u))
    mu_j = d + 2 sqrt(l u) cos(pi j/(n+1)), j = 1..n.
* One-step schemes (Section 5, eq. 5.3): on an eigenmode K v = mu v the
  theta-method advances by R(z) = (1 - (1-theta) z)/(1 + theta z), z = dt mu.
  The error of eq. 5.1 is a rank-one perturbation per mode, and its only
  nonzero eigenvalue is -alpha R^Nt / (1 - alpha R^Nt), so
    rho(I - P_alpha^{-1} A) = max_mu |alpha R^Nt / (1 - alpha R^Nt)|,
  which satisfies the bounds of Theorem 1.2 and Theorem 5.1 when |R| <= 1.
* Theorem 3.1 (leap-frog): sigma(P_alpha^{-1} A) is (Nt-2) Nx ones together with
  1/(1 - alpha exp(+-i Nt theta_j)), theta_j = arctan(sqrt(lambda_j^2 - 1)),
  lambda_j the eigenvalues of I + (dt^2/2) K.
* Leap-frog mode solution with u_1 = 0, f = 0: U_n = cos(n theta) U_0 with
  cos(theta) = 1/(1 + dt^2 mu/2) (the characteristic roots of the recurrence
  of eq. 3.2b have modulus one).
"""
from __future__ import annotations

import numpy as np

from workloads import LEAPFROG, Problem


def cos_sin_2pi(n, den):
    """(cos, sin)(2 pi n / den) for integers n, den, with the angle reduced exactly:
    4 n = q den + r with |r| <= den/2 (integers), so the angle is q quarter turns
    plus pi r / (2 den), |pi r / (2 den)| <= pi/4, whose cosine and sine keep their
    full relative accuracy (also where the result is small, e.g. sin near pi)."""
    n = np.asarray(n, dtype=np.int64)
    q = (4 * n + den // 2) // den
    r = 4 * n - q * den
    t = np.pi * r / (2.0 * den)
    c, s = np.cos(t), np.sin(t)
    q = q % 4
    cos = np.select([q == 0, q == 1, q == 2], [c, -s, -c], s)
    sin = np.select([q == 0, q == 1, q == 2], [s, c, -s], -c)
    return cos, sin


def lemma1_eigenvalues(problem: Problem):
    """The closed forms above, evaluated so that no digits cancel.

    w = e^{x + i y} with x = ln(alpha)/Nt, y = 2 pi n/Nt.  For the slow modes
    w is close to 1 (|1 - w_0| is about |ln alpha|/Nt), and 1 - w formed by
    subtraction would carry a relative error of about eps Nt/|ln alpha|.  The
    real parts are written as sums of terms of one sign instead:
      Re(1 - w)            = 2 sin^2(y/2) - expm1(x) cos y,
      Re(theta + (1-theta) w) = 2 theta cos^2(y/2) + (1 - 2 theta) cos y
                                + (1 - theta) expm1(x) cos y,
      Re((1 + w^2)/2)      = cos^2 y + expm1(2x) cos(2y)/2,
    and the imaginary parts are -e^x sin y, (1-theta) e^x sin y and
    e^{2x} sin(2y)/2.  The sines and cosines of y/2, y and 2y come from
    cos_sin_2pi, the angle reduced in integers."""
    nt, dt, a = problem.nt, problem.dt, problem.alpha
    x = np.log(a) / nt
    n = np.arange(nt)
    cy, sy = cos_sin_2pi(n, nt)
    ch, sh = cos_sin_2pi(n, 2 * nt)
    one_m_w = (2.0 * sh ** 2 - np.expm1(x) * cy) - 1j * np.exp(x) * sy
    if problem.scheme == LEAPFROG:
        c2, s2 = cos_sin_2pi(2 * n, nt)
        l2 = cy ** 2 + 0.5 * np.expm1(2 * x) * c2 + 0.5j * np.exp(2 * x) * s2
        return one_m_w ** 2 / dt**2, l2
    th = problem.theta_eff
    l2 = (2 * th * ch ** 2 + (1 - 2 * th) * cy + (1 - th) * np.expm1(x) * cy
          + 1j * (1 - th) * np.exp(x) * sy)
    return one_m_w / dt, l2


def mu_periodic(n: int, h: float, nu: float, a: float) -> np.ndarray:
    t = 2.0 * np.pi * np.arange(n) / n
    return (2.0 * nu / h**2) * (1.0 - np.cos(t)) + 1j * (a / h) * np.sin(t)


def mu_dirichlet(n: int, h: float, nu: float, a: float) -> np.ndarray:
    lo = -nu / h**2 - a / (2.0 * h)
    d = 2.0 * nu / h**2
    up = -nu / h**2 + a / (2.0 * h)
    j = np.arange(1, n + 1)
    return d + 2.0 * np.sqrt(complex(lo * up)) * np.cos(np.pi * j / (n + 1))


def stability_function(z, theta: float):
    """R(z) of the theta-method written as U_{n+1} = R U_n (eq. 5.3 up to sign)."""
    return (1.0 - (1.0 - theta) * z) / (1.0 + theta * z)


def stationary_rate(mus: np.ndarray, dt: float, nt: int, alpha: float, theta: float) -> float:
    """max over modes of |alpha R^Nt / (1 - alpha R^Nt)|."""
    R = stability_function(dt * np.asarray(mus), theta)
    q = alpha * R**nt
    return float(np.max(np.abs(q / (1.0 - q))))


def theorem31_spectrum(mus: np.ndarray, dt: float, nt: int, alpha: float) -> np.ndarray:
    """The 2 Nx non-unit eigenvalues of P_alpha^{-1} A for leap-frog."""
    lam = 1.0 + 0.5 * dt**2 * np.asarray(mus, dtype=np.float64)
    th = np.arctan(np.sqrt(lam**2 - 1.0))
    return np.concatenate([1.0 / (1.0 - alpha * np.exp(1j * nt * th)),
                           1.0 / (1.0 - alpha * np.exp(-1j * nt * th))])


def theorem31_annulus(alpha: float):
    """Inner and outer radii of the annulus |z - 1| of Theorem 3.1 (alpha < 1)."""
    return alpha / (1.0 + alpha), alpha / (1.0 - alpha)


def leapfrog_mode_angle(mu: float, dt: float) -> float:
    return float(np.arccos(1.0 / (1.0 + 0.5 * dt**2 * mu)))
