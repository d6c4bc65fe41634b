"""Seeded synthetic workloads for the ParaDiag-II all-at-once solver.

This module holds problem descriptions and seeded input generators only: grid
sizes, physical parameters, initial data and source terms.  It contains none
of the method's arithmetic (no operators, no time stepping, no transforms), so
both the CPU oracle and the GPU path can take their inputs from here without
sharing any of the computation that is checked.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds.  A double in [0, 1) is the top 53 bits of
the output times 2^-53.

Problem families (the paper's model problems):
  * advection-diffusion u_t = nu*Lap(u) - a.grad(u) + f  (Section 2, eq. 2.1 and
    eq. 2.14), theta-method in time (eq. 2.4), with uniform steps or with the
    geometrically increasing steps of ParaDiag-I (Section 2.1.1, eq. 2.8), or the
    hybrid midpoint + backward-Euler discretisation (Section 2.1.2, eq. neq2.9a);
  * wave equation u_tt = Lap(u) + f (Section 3, eq. 3.1), implicit leap-frog
    in time (eq. 3.2b).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

DIRICHLET = 0
PERIODIC = 1

BE, CN, THETA, LEAPFROG = 0, 1, 2, 3
SCHEME_NAMES = {BE: "backward-euler", CN: "crank-nicolson", THETA: "theta", LEAPFROG: "leapfrog"}

SEED_BASE = 20200519

_MASK = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First ``n`` outputs of SplitMix64 started from ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``n`` doubles uniform in [lo, hi) from SplitMix64(seed)."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


@dataclasses.dataclass(frozen=True)
class Space:
    """Spatial grid of the semi-discrete system M U' + K U = f with M = I.

    dim 1: nx unknowns in x.  dim 2: ny*nx unknowns, x fastest (index y*nx + x).
    Dirichlet directions hold the interior points x_j = j*h, j = 1..n, with
    h = L/(n+1); periodic directions hold x_j = j*h, j = 0..n-1, with h = L/n.
    K = -nu*Lap_h + a.grad_h with second-order centred differences.
    """
    dim: int
    nx: int
    ny: int = 1
    nu: float = 1.0
    ax: float = 0.0
    ay: float = 0.0
    bc_x: int = DIRICHLET
    bc_y: int = DIRICHLET
    lx: float = 1.0
    ly: float = 1.0

    @property
    def size(self) -> int:
        return self.nx * (self.ny if self.dim == 2 else 1)

    @property
    def hx(self) -> float:
        return self.lx / (self.nx if self.bc_x == PERIODIC else self.nx + 1)

    @property
    def hy(self) -> float:
        return self.ly / (self.ny if self.bc_y == PERIODIC else self.ny + 1)

    def xs(self) -> np.ndarray:
        j = np.arange(self.nx, dtype=np.float64)
        return j * self.hx if self.bc_x == PERIODIC else (j + 1.0) * self.hx

    def ys(self) -> np.ndarray:
        j = np.arange(self.ny, dtype=np.float64)
        return j * self.hy if self.bc_y == PERIODIC else (j + 1.0) * self.hy

    def mesh(self):
        """(X, Y) arrays of shape [ny][nx] (2D only)."""
        return np.meshgrid(self.xs(), self.ys(), indexing="xy")


@dataclasses.dataclass(frozen=True)
class Problem:
    """All-at-once problem A u = b, A = B1 (x) I + B2 (x) K (eq. 1.1)."""
    space: Space
    nt: int
    dt: float
    scheme: int
    alpha: float
    theta: float = 1.0

    @property
    def unknowns(self) -> int:
        return self.space.size * self.nt

    @property
    def theta_eff(self) -> float:
        if self.scheme == BE:
            return 1.0
        if self.scheme == CN:
            return 0.5
        return self.theta


@dataclasses.dataclass(frozen=True)
class GeometricProblem:
    """All-at-once theta-method system with geometrically increasing steps
    (Section 2.1.1), the problem ParaDiag-I solves directly: ``nt`` steps, the
    last one of length ``dt_last``, consecutive steps in the ratio ``tau > 1``
    (eq. 2.8).  ``scaled`` selects the column-scaled eigenvector matrix
    V D~ of the same section."""
    space: Space
    nt: int
    dt_last: float
    tau: float
    scheme: int
    scaled: bool = True

    @property
    def unknowns(self) -> int:
        return self.space.size * self.nt

    @property
    def theta_eff(self) -> float:
        return 1.0 if self.scheme == BE else 0.5


@dataclasses.dataclass(frozen=True)
class HybridProblem:
    """All-at-once system of the hybrid time discretisation of Section 2.1.2:
    explicit midpoint steps for n = 1..Nt-1 and one backward-Euler step at the
    end, uniform step ``dt`` (eq. neq2.9a)."""
    space: Space
    nt: int
    dt: float

    @property
    def unknowns(self) -> int:
        return self.space.size * self.nt


@dataclasses.dataclass
class Workload:
    """A problem plus its seeded data.

    u0: [S] initial value; u1: [S] initial velocity (wave only) or None;
    f: [nt+1][S] source at t_0..t_nt or None (zero source).
    """
    name: str
    problem: Problem
    u0: np.ndarray
    u1: Optional[np.ndarray]
    f: Optional[np.ndarray]
    seed: int
    extra: dict = dataclasses.field(default_factory=dict)


def sine_mode_source(seed: int, x: np.ndarray, modes: int = 8) -> np.ndarray:
    """f(x) = sum_{m=1..modes} c_m sin(m pi x), c_m uniform in [-1, 1)."""
    c = uniform(seed, modes, -1.0, 1.0)
    m = np.arange(1, modes + 1, dtype=np.float64)
    return np.sin(np.pi * np.outer(x, m)) @ c


def ade1d(nx=127, nt=64, T=1.0, nu=1e-2, a=1.0, scheme=BE, alpha=1e-2, seed=SEED_BASE + 0,
          name="ade1d") -> Workload:
    """1D advection-diffusion on (0,1), Dirichlet, u0 = sin(pi x), time-independent
    source on 8 seeded sine modes."""
    sp = Space(dim=1, nx=nx, nu=nu, ax=a, bc_x=DIRICHLET)
    pb = Problem(space=sp, nt=nt, dt=T / nt, scheme=scheme, alpha=alpha)
    x = sp.xs()
    u0 = np.sin(np.pi * x)
    fx = sine_mode_source(seed, x)
    f = np.broadcast_to(fx, (nt + 1, nx)).copy()
    return Workload(name, pb, u0, None, f, seed)


def ade2d(nx=255, ny=255, nt=256, T=1.0, nu=1e-3, ax=1.0, ay=0.5, scheme=CN, alpha=1e-3,
          seed=SEED_BASE + 1, name="ade2d") -> Workload:
    """2D advection-diffusion, x periodic (nx points, h = 1/nx), y Dirichlet
    (ny interior points, h = 1/(ny+1)), Gaussian bump u0 = exp(-20 r^2) with a
    seeded centre in [0.3, 0.7)^2, zero source."""
    sp = Space(dim=2, nx=nx, ny=ny, nu=nu, ax=ax, ay=ay, bc_x=PERIODIC, bc_y=DIRICHLET)
    pb = Problem(space=sp, nt=nt, dt=T / nt, scheme=scheme, alpha=alpha)
    x0, y0 = uniform(seed, 2, 0.3, 0.7)
    X, Y = sp.mesh()
    u0 = np.exp(-20.0 * ((X - x0) ** 2 + (Y - y0) ** 2)).reshape(-1)
    return Workload(name, pb, u0, None, None, seed, extra={"center": (x0, y0)})


def batch_instances(count=64, seed=SEED_BASE + 2, pow2=False, nx_range=(63, 1023),
                    nt_range=(32, 1024)):
    """Sizes and viscosities of the batched 1D instances.

    Integer reading: nx uniform on {63..1023}, nt uniform on {32..1024}.
    pow2 reading: nx from {63,127,...,1023}, nt from {32,...,1024}.
    nu = 10^U[-3,-1].  Returns a list of (nx, nt, nu, seed_i).
    """
    r = uniform(seed, 3 * count)
    out = []
    for i in range(count):
        if pow2:
            nxs = [2 ** p - 1 for p in range(6, 11) if nx_range[0] <= 2 ** p - 1 <= nx_range[1]]
            nts = [2 ** p for p in range(5, 11) if nt_range[0] <= 2 ** p <= nt_range[1]]
            nx = nxs[min(int(r[3 * i] * len(nxs)), len(nxs) - 1)]
            nt = nts[min(int(r[3 * i + 1] * len(nts)), len(nts) - 1)]
        else:
            nx = nx_range[0] + min(int(r[3 * i] * (nx_range[1] - nx_range[0] + 1)),
                                   nx_range[1] - nx_range[0])
            nt = nt_range[0] + min(int(r[3 * i + 1] * (nt_range[1] - nt_range[0] + 1)),
                                   nt_range[1] - nt_range[0])
        nu = 10.0 ** (-3.0 + 2.0 * r[3 * i + 2])
        out.append((nx, nt, nu, seed * 1000 + i))
    return out


def batched(count=64, seed=SEED_BASE + 2, pow2=False, **kw):
    """The batched 1D advection-diffusion workload: a list of Workloads."""
    wls = []
    for i, (nx, nt, nu, s) in enumerate(batch_instances(count, seed, pow2, **kw)):
        wls.append(ade1d(nx=nx, nt=nt, nu=nu, a=1.0, scheme=BE, alpha=1e-2, seed=s,
                         name=f"batch{i}"))
    return wls


def heat2d_control(nx=127, nt=128, T=1.0, seed=SEED_BASE + 3, name="heat2d"):
    """2D heat equation (nu = 1, Dirichlet all sides) for the source inversion
    J(f) = 1/2 ||u(T) - u_target||^2 + 1/2 * 1e-4 ||f||^2; u0 = 0.

    Returns the workload with ``f`` = a seeded control probe (uniform [-1,1),
    time independent) and ``extra['u_target']`` = a sum of 4 Gaussians with
    amplitude in [0.5, 1), centre in [0.2, 0.8)^2 and profile exp(-50 r^2).
    """
    sp = Space(dim=2, nx=nx, ny=nx, nu=1.0, bc_x=DIRICHLET, bc_y=DIRICHLET)
    pb = Problem(space=sp, nt=nt, dt=T / nt, scheme=BE, alpha=1e-2)
    X, Y = sp.mesh()
    r = uniform(seed, 12)
    tgt = np.zeros_like(X)
    for g in range(4):
        amp = 0.5 + 0.5 * r[3 * g]
        cx = 0.2 + 0.6 * r[3 * g + 1]
        cy = 0.2 + 0.6 * r[3 * g + 2]
        tgt += amp * np.exp(-50.0 * ((X - cx) ** 2 + (Y - cy) ** 2))
    fprobe = uniform(seed + 7, sp.size, -1.0, 1.0)
    f = np.broadcast_to(fprobe, (nt + 1, sp.size)).copy()
    u0 = np.zeros(sp.size)
    return Workload(name, pb, u0, None, f, seed,
                    extra={"u_target": tgt.reshape(-1), "f_probe": fprobe, "reg": 1e-4})


def wave1d(nx=1023, nt=1024, T=2.0, alpha=0.1, seed=SEED_BASE + 4, name="wave1d"):
    """1D wave u_tt = u_xx on (0,1), Dirichlet, u0 = exp(-100 (x-0.5)^2), u_t(0) = 0."""
    sp = Space(dim=1, nx=nx, nu=1.0, bc_x=DIRICHLET)
    pb = Problem(space=sp, nt=nt, dt=T / nt, scheme=LEAPFROG, alpha=alpha)
    x = sp.xs()
    u0 = np.exp(-100.0 * (x - 0.5) ** 2)
    u1 = np.zeros(nx)
    return Workload(name, pb, u0, u1, None, seed)


def pd1_ade1d(nx=128, nt=32, tau=1.16, dt_last=0.05, nu=1e-3, scheme=CN, scaled=True,
              seed=SEED_BASE + 5, name="pd1_ade1d") -> Workload:
    """The ParaDiag-I example of Section 2.1.1: u_t - nu u_xx + u_x = 0 on (-1, 1),
    periodic (eq. 2.1, the grid x_j = -1 + j h, h = 2/nx), u0 = exp(-30 x^2),
    geometric steps (eq. 2.8).  Defaults: the window of the windowing figure
    (Nt = 32, tau = 1.16, dt_Nt = 0.05, nu = 1e-3, trapezoidal rule)."""
    sp = Space(dim=1, nx=nx, nu=nu, ax=1.0, bc_x=PERIODIC, lx=2.0)
    pb = GeometricProblem(space=sp, nt=nt, dt_last=dt_last, tau=tau, scheme=scheme, scaled=scaled)
    x = sp.xs() - 1.0
    u0 = np.exp(-30.0 * x * x)
    return Workload(name, pb, u0, None, None, seed)


def pd1_ade2d(nx=255, ny=255, nt=32, tau=1.16, dt_last=0.05, nu=1e-3, ax=1.0, ay=0.5,
              scheme=BE, scaled=True, seed=SEED_BASE + 6, name="pd1_ade2d") -> Workload:
    """One ParaDiag-I window on the 2D advection-diffusion grid of ``ade2d``
    (x periodic, y Dirichlet, seeded Gaussian bump, zero source) with geometric
    steps (eq. 2.8); backward Euler by default."""
    sp = Space(dim=2, nx=nx, ny=ny, nu=nu, ax=ax, ay=ay, bc_x=PERIODIC, bc_y=DIRICHLET)
    pb = GeometricProblem(space=sp, nt=nt, dt_last=dt_last, tau=tau, scheme=scheme, scaled=scaled)
    x0, y0 = uniform(seed, 2, 0.3, 0.7)
    X, Y = sp.mesh()
    u0 = np.exp(-20.0 * ((X - x0) ** 2 + (Y - y0) ** 2)).reshape(-1)
    return Workload(name, pb, u0, None, None, seed, extra={"center": (x0, y0)})


def hybrid_ade1d(nx=256, nt=64, T=1.0, nu=1e-3, seed=SEED_BASE + 7,
                  name="hybrid_ade1d") -> Workload:
    """The hybrid ParaDiag-I example of Section 2.1.2: eq. 2.1 (periodic on (-1, 1),
    u_t - nu u_xx + u_x = 0, u0 = exp(-30 x^2)) with dx = 1/128 (nx = 256), the
    midpoint + backward-Euler discretisation with nt uniform steps over [0, T]."""
    sp = Space(dim=1, nx=nx, nu=nu, ax=1.0, bc_x=PERIODIC, lx=2.0)
    pb = HybridProblem(space=sp, nt=nt, dt=T / nt)
    x = sp.xs() - 1.0
    return Workload(name, pb, np.exp(-30.0 * x * x), None, None, seed)


def hybrid_ade2d(nx=255, ny=255, nt=256, T=1.0, nu=1e-3, ax=1.0, ay=0.5, seed=SEED_BASE + 8,
                 name="hybrid_ade2d") -> Workload:
    """The hybrid ParaDiag-I discretisation on the 2D grid of ``ade2d`` (x periodic,
    y Dirichlet, seeded Gaussian bump, zero source), nt uniform steps over [0, T]."""
    sp = Space(dim=2, nx=nx, ny=ny, nu=nu, ax=ax, ay=ay, bc_x=PERIODIC, bc_y=DIRICHLET)
    pb = HybridProblem(space=sp, nt=nt, dt=T / nt)
    x0, y0 = uniform(seed, 2, 0.3, 0.7)
    X, Y = sp.mesh()
    u0 = np.exp(-20.0 * ((X - x0) ** 2 + (Y - y0) ** 2)).reshape(-1)
    return Workload(name, pb, u0, None, None, seed, extra={"center": (x0, y0)})


def hybrid_wave2d(n=512, nt=512, T=2.0, seed=SEED_BASE + 9, name="hybrid_wave2d") -> Workload:
    """The second-order hybrid ParaDiag-I experiment of Section 2.1.2: u_tt - Lap u = f
    on (0,1)^2, Dirichlet, dx = dy = 1/n ((n-1)^2 interior points), T = 2,
    u0 = 0, u_t(0) = 2 pi x(x-1)y(y-1), f such that u = x(x-1)y(y-1) sin(2 pi t).
    ``f`` holds the source at t_0..t_nt; ``u1`` the initial velocity."""
    sp = Space(dim=2, nx=n - 1, ny=n - 1, nu=1.0, bc_x=DIRICHLET, bc_y=DIRICHLET)
    pb = HybridProblem(space=sp, nt=nt, dt=T / nt)
    X, Y = sp.mesh()
    phi = (X * (X - 1.0) * Y * (Y - 1.0)).reshape(-1)
    q = (X * (X - 1.0) + Y * (Y - 1.0)).reshape(-1)
    t = (T / nt) * np.arange(nt + 1)
    st = np.sin(2.0 * np.pi * t)
    f = np.outer(st, -4.0 * np.pi**2 * phi - 2.0 * q)
    return Workload(name, pb, np.zeros_like(phi), 2.0 * np.pi * phi, f, seed,
                    extra={"phi": phi, "T": T})


def nl_manufactured1d(nx=63, nt=32, T=1.0, nu=1.0, reaction=(0.5, 1.0, 2.0), scheme=CN,
                      alpha=1e-2, theta=1.0, seed=SEED_BASE + 10,
                      name="nl_manufactured1d") -> Workload:
    """U' + K U + phi(U) = f on (0,1), Dirichlet, K = -nu d_xx, with the cubic
    reaction phi(u) = a1 u + a2 u^2 + a3 u^3 and f chosen so that the exact
    solution is u = exp(-t) sin(pi x).  ``extra``: the reaction coefficients
    and the exact solution at t_1..t_nt."""
    sp = Space(dim=1, nx=nx, nu=nu, bc_x=DIRICHLET)
    pb = Problem(space=sp, nt=nt, dt=T / nt, scheme=scheme, alpha=alpha, theta=theta)
    x = sp.xs()
    t = (T / nt) * np.arange(nt + 1)
    u = np.outer(np.exp(-t), np.sin(np.pi * x))
    a1, a2, a3 = reaction
    f = -u + nu * np.pi**2 * u + u * (a1 + u * (a2 + u * a3))
    return Workload(name, pb, u[0].copy(), None, f, seed,
                    extra={"reaction": tuple(reaction), "exact": u[1:].copy()})


def nl_ade2d(nx=255, ny=255, nt=256, T=1.0, nu=1e-3, ax=1.0, ay=0.5, scheme=CN, alpha=1e-3,
             reaction=(0.0, 0.0, 1.0), seed=SEED_BASE + 1, name="nl_ade2d") -> Workload:
    """The ade2d grid and data (Gaussian bump, zero source) with a cubic
    reaction, by default phi(u) = u^3 (coefficients (a1, a2, a3) in ``extra``)."""
    w = ade2d(nx=nx, ny=ny, nt=nt, T=T, nu=nu, ax=ax, ay=ay, scheme=scheme, alpha=alpha,
              seed=seed, name=name)
    return Workload(name, w.problem, w.u0, None, None, seed,
                    extra={"reaction": tuple(reaction), "center": w.extra["center"]})


def named(name: str, **kw) -> Workload:
    """The five named workloads at their full sizes (keyword overrides allowed)."""
    table = {
        "ade1d_be": lambda: ade1d(**kw),
        "ade2d_cn": lambda: ade2d(**kw),
        "heat2d_control": lambda: heat2d_control(**kw),
        "wave1d_leapfrog": lambda: wave1d(**kw),
        "pd1_ade1d": lambda: pd1_ade1d(**kw),
        "pd1_ade2d": lambda: pd1_ade2d(**kw),
        "hybrid_ade1d": lambda: hybrid_ade1d(**kw),
        "hybrid_ade2d": lambda: hybrid_ade2d(**kw),
        "hybrid_wave2d": lambda: hybrid_wave2d(**kw),
        "nl_manufactured1d": lambda: nl_manufactured1d(**kw),
        "nl_ade2d": lambda: nl_ade2d(**kw),
    }
    return table[name]()


def workload_summary(w: Workload) -> dict:
    p = w.problem
    s = p.space
    if isinstance(p, HybridProblem):
        return {"name": w.name, "dim": s.dim, "nx": s.nx, "ny": s.ny if s.dim == 2 else 1,
                "nt": p.nt, "dt": p.dt, "scheme": "midpoint + backward Euler (hybrid)",
                "nu": s.nu, "ax": s.ax, "ay": s.ay, "unknowns": p.unknowns, "seed": w.seed}
    if isinstance(p, GeometricProblem):
        return {"name": w.name, "dim": s.dim, "nx": s.nx, "ny": s.ny if s.dim == 2 else 1,
                "nt": p.nt, "dt_last": p.dt_last, "tau": p.tau, "scheme": SCHEME_NAMES[p.scheme],
                "column_scaling": p.scaled, "nu": s.nu, "ax": s.ax, "ay": s.ay,
                "unknowns": p.unknowns, "seed": w.seed}
    return {"name": w.name, "dim": s.dim, "nx": s.nx, "ny": s.ny if s.dim == 2 else 1,
            "nt": p.nt, "dt": p.dt, "scheme": SCHEME_NAMES[p.scheme], "alpha": p.alpha,
            "nu": s.nu, "ax": s.ax, "ay": s.ay, "unknowns": p.unknowns, "seed": w.seed}

