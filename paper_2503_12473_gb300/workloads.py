"""Seeded synthetic workloads: initial data and problem sizes.

This module serves both the CUDA path and the CPU oracle and therefore holds
none of the method's arithmetic: no basis, quadrature, flux, damping or time
stepping.  It only defines the physical initial data (as point-value functions
of conserved variables) and the problem descriptions.

Workloads (sizes and data):
  * ``advection_1d``  -- u_t + u_x = 0, u0 = sin(x) on [0, 2pi], periodic, 128 cells,
    P^2, SSP-RK3, CFL 0.1, T = 2pi (one period).
  * ``shu_osher_1d``  -- 1D Euler, gamma = 1.4, [-5, 5] transmissive, 4000 cells,
    (rho, v, p) = (3.857143, 2.629369, 10.33333) for x < -4, else
    (1 + 0.2 sin 5x, 0, 1) (the Shu-Osher data of Section 4), T = 1.8.
  * ``burgers_1d``    -- u_t + (u^2/2)_x = 0, u0 = sin x + 0.5 on [0, 2pi] periodic,
    P^3, classical RK4, CFL 0.31, T = 0.6 (the Table 2 accuracy test).
  * ``euler_wave_1d`` -- 1D Euler density wave (1 + 0.2 sin x, 1, 1), periodic.
  * ``riemann_2d``    -- 2D Euler four-quadrant Riemann data split at (0.8, 0.8) on
    [0,1]^2 transmissive, 1024^2, Q^2, CFL 0.1, 200 steps.
  * ``batched_2d``    -- 256 periodic 2D Euler problems with seeded sizes and data.
  * ``vortex_2d``     -- isentropic vortex (strength 5) on uniform flow (1,1),
    [0,10]^2 periodic, 256^2.
  * ``two_blast_waves_1d`` -- 1D Euler, [0, 1] between reflective walls, 960
    cells, P^2, SSP-RK3, CFL 0.3 (Section 4's value for P^2 on discontinuous
    data), (rho, v, p) = (1, 0, 1e3) for x < 0.1, (1, 0, 1e-2) in between,
    (1, 0, 1e2) for x > 0.9 (the two-blast-wave data of Section 4), T = 0.038.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Callable, Optional

import numpy as np

GAMMA = 1.4

# system / basis / boundary codes shared by the two sides' problem descriptions
ADVECTION, BURGERS, EULER = 0, 1, 2
BASIS_Q, BASIS_P = 0, 1
PERIODIC, TRANSMISSIVE, REFLECTIVE = 0, 1, 2


@dataclass
class Workload:
    """A problem: mesh, discretisation parameters and initial data."""
    name: str
    dim: int
    nx: int
    ny: int
    k: int
    system: int
    bc: int
    ax: float
    bx: float
    ay: float = 0.0
    by: float = 1.0
    basis: int = BASIS_Q
    gamma: float = GAMMA
    adv: tuple = (1.0, 0.0)
    cfl: float = 0.1
    rk: int = 3
    oe: int = 1
    T: float = 0.0          # end time (0: none)
    steps: int = 0          # step count when T == 0
    u0: Optional[Callable] = field(default=None, repr=False)  # xy [n, dim] -> conserved [n, F]

    @property
    def nfields(self) -> int:
        return self.dim + 2 if self.system == EULER else 1

    @property
    def nmodes(self) -> int:
        if self.dim == 1:
            return self.k + 1
        return (self.k + 1) ** 2 if self.basis == BASIS_Q else (self.k + 1) * (self.k + 2) // 2

    @property
    def sides(self):
        """Boundary condition of each side (x-low, x-high, y-low, y-high)."""
        b = self.bc
        return tuple(b) if isinstance(b, (tuple, list)) else (b, b, b, b)

    @property
    def state_shape(self):
        """Both meshes in the padded layout: one more column (row) where the low
        x (y) side is a reflective wall (the dual cell centred on it)."""
        nxs = self.nx + (self.sides[0] == REFLECTIVE)
        nys = (self.ny + (self.sides[2] == REFLECTIVE)) if self.dim == 2 else 1
        return (2, self.nfields, self.nmodes, nys, nxs)

    @property
    def dofs(self) -> int:
        return int(np.prod(self.state_shape))

    def resized(self, nx: int, ny: Optional[int] = None, **kw) -> "Workload":
        return replace(self, nx=nx, ny=(ny if ny is not None else (nx if self.dim == 2 else 1)), **kw)


# ----------------------------------------------------------- conversions ----

def prim_to_cons_1d(rho, v, p, gamma=GAMMA):
    return np.stack([rho, rho * v, p / (gamma - 1.0) + 0.5 * rho * v * v], axis=-1)


def prim_to_cons_2d(rho, u, v, p, gamma=GAMMA):
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)], axis=-1)


def _wrap(x, a, b):
    L = b - a
    return a + np.mod(x - a, L)


# ------------------------------------------------------------- initial data --

def sine_1d(period: float = 2.0 * math.pi, a: float = 0.0):
    def f(xy):
        x = np.asarray(xy, dtype=np.float64).reshape(len(xy), -1)[:, 0]
        return np.sin(2.0 * math.pi * (x - a) / period)[:, None]
    return f


def burgers_sine(offset: float = 0.5):
    """u0 = sin x + offset (the Burgers accuracy test of Table 2)."""
    def f(xy):
        x = np.asarray(xy, dtype=np.float64).reshape(len(xy), -1)[:, 0]
        return (np.sin(x) + offset)[:, None]
    return f


def density_wave_1d(gamma=GAMMA, amp: float = 0.2):
    """Smooth 1D Euler data (rho, v, p) = (1 + amp sin x, 1, 1), 2 pi periodic."""
    def f(xy):
        x = np.asarray(xy, dtype=np.float64).reshape(len(xy), -1)[:, 0]
        return prim_to_cons_1d(1.0 + amp * np.sin(x), np.ones_like(x), np.ones_like(x), gamma)
    return f


def shu_osher(gamma=GAMMA):
    def f(xy):
        x = np.asarray(xy, dtype=np.float64).reshape(len(xy), -1)[:, 0]
        left = x < -4.0
        rho = np.where(left, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
        v = np.where(left, 2.629369, 0.0)
        p = np.where(left, 10.33333, 1.0)
        return prim_to_cons_1d(rho, v, p, gamma)
    return f


def two_blast_waves(gamma=GAMMA):
    """(rho, v, p) = (1, 0, 1e3) for x < 0.1, (1, 0, 1e-2) for 0.1 < x < 0.9,
    (1, 0, 1e2) for x > 0.9."""
    def f(xy):
        x = np.asarray(xy, dtype=np.float64).reshape(len(xy), -1)[:, 0]
        p = np.where(x < 0.1, 1e3, np.where(x > 0.9, 1e2, 1e-2))
        return prim_to_cons_1d(np.ones_like(x), np.zeros_like(x), p, gamma)
    return f


def riemann_quadrants(gamma=GAMMA, x0=0.8, y0=0.8):
    """Four constant states split at (x0, y0): NE, NW, SW, SE as (rho, u, v, p)."""
    ne = (1.5, 0.0, 0.0, 1.5)
    nw = (0.5323, 1.206, 0.0, 0.3)
    sw = (0.138, 1.206, 1.206, 0.029)
    se = (0.5323, 0.0, 1.206, 0.3)

    def f(xy):
        xy = np.asarray(xy, dtype=np.float64)
        x, y = xy[:, 0], xy[:, 1]
        east, north = x >= x0, y >= y0
        out = np.empty((len(x), 4))
        for st, m in ((ne, east & north), (nw, ~east & north), (sw, ~east & ~north), (se, east & ~north)):
            out[m] = prim_to_cons_2d(np.full(m.sum(), st[0]), np.full(m.sum(), st[1]), np.full(m.sum(), st[2]),
                                     np.full(m.sum(), st[3]), gamma)
        return out
    return f


def steady_wave_2d(gamma=GAMMA):
    """(rho, u, v, p) = (1 + 0.2 sin(pi (x - y)), 1, 1, 1): an exact steady solution."""
    def f(xy):
        xy = np.asarray(xy, dtype=np.float64)
        rho = 1.0 + 0.2 * np.sin(math.pi * (xy[:, 0] - xy[:, 1]))
        one = np.ones_like(rho)
        return prim_to_cons_2d(rho, one, one, one, gamma)
    return f


def isentropic_vortex(gamma=GAMMA, eps=5.0, centre=(5.0, 5.0), vel=(1.0, 1.0), L=10.0, t=0.0):
    """Isentropic vortex of strength eps on uniform flow `vel` with rho = p = 1 at
    infinity, translated to time t on the periodic square [0, L]^2:
      du = eps/(2 pi) exp((1 - r^2)/2) (-ybar, xbar),
      dT = -(gamma - 1) eps^2 / (8 gamma pi^2) exp(1 - r^2),
      rho = (1 + dT)^(1/(gamma-1)), p = rho^gamma."""
    def f(xy):
        xy = np.asarray(xy, dtype=np.float64)
        cx = centre[0] + vel[0] * t
        cy = centre[1] + vel[1] * t
        # nearest periodic image of the centre
        xb = xy[:, 0] - cx
        yb = xy[:, 1] - cy
        xb = xb - L * np.round(xb / L)
        yb = yb - L * np.round(yb / L)
        r2 = xb * xb + yb * yb
        du = eps / (2.0 * math.pi) * np.exp(0.5 * (1.0 - r2))
        dT = -(gamma - 1.0) * eps * eps / (8.0 * gamma * math.pi * math.pi) * np.exp(1.0 - r2)
        T = 1.0 + dT
        rho = T ** (1.0 / (gamma - 1.0))
        p = rho ** gamma
        return prim_to_cons_2d(rho, vel[0] - yb * du, vel[1] + xb * du, p, gamma)
    return f


def constant_state(values):
    vals = np.asarray(values, dtype=np.float64)

    def f(xy):
        return np.broadcast_to(vals, (len(xy), len(vals))).copy()
    return f


# ------------------------------------------------------------ batched data --

@dataclass
class BatchInstance:
    n: int
    a: np.ndarray        # amplitudes a_j, j = 1..3
    kv: np.ndarray       # integer wave vectors k_j, shape [3, 2]
    centre: np.ndarray   # circle centre
    radius: float
    vel: np.ndarray      # (u, v)


BATCH_SIZES = (64, 96, 128, 192, 256, 384, 512)


def batched_instances(seed: int = 0, count: int = 256, sizes=BATCH_SIZES):
    """Seeded parameters of the batched periodic 2D Euler problems:
    N uniform in `sizes`; a_j ~ U[-1,1]; k_j in {-3..3}^2 minus 0; circle
    centre ~ U[0,1]^2, radius ~ U[0.1,0.25] (+0.5 density inside);
    (u, v) ~ U[-0.5,0.5]^2; p = 1."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(sizes))
        a = rng.uniform(-1.0, 1.0, 3)
        kv = np.zeros((3, 2), dtype=np.int64)
        for j in range(3):
            while True:
                kk = rng.integers(-3, 4, 2)
                if kk[0] != 0 or kk[1] != 0:
                    break
            kv[j] = kk
        centre = rng.uniform(0.0, 1.0, 2)
        radius = float(rng.uniform(0.1, 0.25))
        vel = rng.uniform(-0.5, 0.5, 2)
        out.append(BatchInstance(n, a, kv, centre, radius, vel))
    return out


def batched_ic(inst: BatchInstance, gamma=GAMMA):
    def f(xy):
        xy = np.asarray(xy, dtype=np.float64)
        x = _wrap(xy[:, 0], 0.0, 1.0)
        y = _wrap(xy[:, 1], 0.0, 1.0)
        rho = np.ones_like(x)
        for j in range(3):
            rho = rho + 0.2 * inst.a[j] * np.sin(2.0 * math.pi * (inst.kv[j, 0] * x + inst.kv[j, 1] * y))
        dx = x - inst.centre[0]
        dy = y - inst.centre[1]
        dx = dx - np.round(dx)
        dy = dy - np.round(dy)
        rho = rho + 0.5 * (dx * dx + dy * dy < inst.radius ** 2)
        return prim_to_cons_2d(rho, np.full_like(x, inst.vel[0]), np.full_like(x, inst.vel[1]),
                               np.ones_like(x), gamma)
    return f


# ---------------------------------------------------------------- random ----

def random_modal(shape, seed: int, scale: float = 1.0, decay: float = 0.5, nmode_axis: int = 2):
    """Seeded N(0, scale^2) modal coefficients, higher modes scaled by decay^index."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(shape) * scale
    nm = shape[nmode_axis]
    s = np.array([decay ** m for m in range(nm)])
    sh = [1] * len(shape)
    sh[nmode_axis] = nm
    return u * s.reshape(sh)


def counter_uniform(shape, seed: int) -> np.ndarray:
    """Seeded values uniform in [-1, 1) that are the same on every machine and
    numpy version: element i is SplitMix64 (Steele, Lea and Flood, "Fast
    splittable pseudorandom number generators", OOPSLA 2014) of the counter
    seed * 2^32 + i, its top 53 bits read as a fraction in [0, 1), then
    mapped by 2 x - 1 (all steps exact in integer and binary arithmetic)."""
    n = int(np.prod(shape))
    with np.errstate(over="ignore"):
        z = np.arange(n, dtype=np.uint64) + np.uint64(seed) * np.uint64(1 << 32)
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (2.0 * u - 1.0).reshape(shape)


def perturbation(shape, seed: int, amp: float = 1e-3):
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal(shape)


# ------------------------------------------------------------- workloads ----

def advection_1d(n: int = 128) -> Workload:
    return Workload("advection_1d_p2_128", 1, n, 1, 2, ADVECTION, PERIODIC, 0.0, 2.0 * math.pi,
                    adv=(1.0, 0.0), cfl=0.1, T=2.0 * math.pi, u0=sine_1d(2.0 * math.pi))


def shu_osher_1d(n: int = 4000) -> Workload:
    return Workload("euler_1d_shu_osher_p2_4000", 1, n, 1, 2, EULER, TRANSMISSIVE, -5.0, 5.0, cfl=0.1, T=1.8,
                    u0=shu_osher())


def two_blast_waves_1d(n: int = 960) -> Workload:
    return Workload(f"euler_1d_two_blast_waves_p2_{n}", 1, n, 1, 2, EULER, (REFLECTIVE, REFLECTIVE, PERIODIC, PERIODIC),
                    0.0, 1.0, cfl=0.3, T=0.038, u0=two_blast_waves())


def burgers_1d(n: int = 128, k: int = 3) -> Workload:
    return Workload(f"burgers_1d_p{k}_{n}", 1, n, 1, k, BURGERS, PERIODIC, 0.0, 2.0 * math.pi, cfl=0.31, rk=4,
                    T=0.6, u0=burgers_sine(0.5))


def euler_wave_1d(n: int = 128, k: int = 2) -> Workload:
    return Workload(f"euler_1d_wave_p{k}_{n}", 1, n, 1, k, EULER, PERIODIC, 0.0, 2.0 * math.pi, cfl=0.1,
                    T=0.5, u0=density_wave_1d())


def steady_wave_2d_workload(n: int = 1024, k: int = 3, basis: int = BASIS_P) -> Workload:
    """The smooth 2D Euler test of Table 4 on [0, 2]^2, periodic, with the
    (k+1)-order RK method and the accuracy-test CFL number of Section 4."""
    rk = {1: 2, 2: 3, 3: 4}[k]
    cfl = {1: 0.45, 2: 0.33, 3: 0.31}[k]
    return Workload(f"euler_2d_steady_wave_{'QP'[basis]}{k}_{n}", 2, n, n, k, EULER, PERIODIC, 0.0, 2.0, 0.0, 2.0,
                    basis=basis, cfl=cfl, rk=rk, T=10.0, u0=steady_wave_2d())


def riemann_2d(n: int = 1024, steps: int = 200) -> Workload:
    return Workload(f"euler_2d_riemann_q2_{n}", 2, n, n, 2, EULER, TRANSMISSIVE, 0.0, 1.0, 0.0, 1.0, cfl=0.1,
                    steps=steps, u0=riemann_quadrants())


def vortex_2d(n: int = 256, steps: int = 400) -> Workload:
    return Workload(f"euler_2d_vortex_q2_{n}", 2, n, n, 2, EULER, PERIODIC, 0.0, 10.0, 0.0, 10.0, cfl=0.1,
                    steps=steps, u0=isentropic_vortex())


def batch_workloads(seed: int = 0, count: int = 256, steps: int = 100, sizes=BATCH_SIZES):
    out = []
    for q, inst in enumerate(batched_instances(seed, count, sizes)):
        out.append(Workload(f"batched_{q}_{inst.n}", 2, inst.n, inst.n, 2, EULER, PERIODIC, 0.0, 1.0, 0.0, 1.0,
                            cfl=0.1, steps=steps, u0=batched_ic(inst)))
    return out
