"""Pins of the oracle's reflective walls (the walls of Section 4's blast-wave and
wall-bounded tests; the paper does not say how the overlapping meshes are
closed at a wall).

The reading: a reflective wall is the restriction of the mirror-extended
problem.  Mirror the data across the wall (density, tangential momentum and
energy even, the normal momentum odd): the Euler equations keep that symmetry,
and the solution restricted to the original domain is the wall-bounded one.
Closing a box with walls on both sides of a direction makes the extended
problem periodic with twice the period, so a reflective run on [0, 1] must
equal, cell for cell, the periodic run on [0, 2] with the mirrored data.  The
dual mesh of the extended problem has a cell centred on each wall: the
reflective mesh stores it (the slot after its last cell for a low-side wall;
the last dual cell for a high-side wall), and sigma and avg are those of the
extended domain (that cell counts half, a normal momentum averages to 0).

These tests check that equality to rounding for 1D and 2D Euler, with the OE
step, for a box closed in x and y and for walls in x with y periodic; and that
the comparison discriminates (a copy closure instead of the mirror misses).
"""
import numpy as np
import pytest

from oracle import oracle as O

GAMMA = 1.4


def _cons1(rho, v, p):
    return np.stack([rho, rho * v, p / (GAMMA - 1.0) + 0.5 * rho * v * v], axis=-1)


def _cons2(rho, u, v, p):
    return np.stack([rho, rho * u, rho * v, p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v)], axis=-1)


def _ic1(xs):
    """1D: a density and pressure pulse near the left wall, flow towards the right wall."""
    x = xs[:, 0]
    rho = 1.0 + 0.5 * np.exp(-((x - 0.3) / 0.08) ** 2) + 0.2 * (x > 0.62)
    v = 0.4 * np.sin(np.pi * x) + 0.2
    p = 1.0 + 0.8 * np.exp(-((x - 0.25) / 0.1) ** 2)
    return _cons1(rho, v, p)


def _ic2(xy):
    """2D: an off-centre pressure pulse and a density step, a shear flow."""
    x, y = xy[:, 0], xy[:, 1]
    rho = 1.0 + 0.4 * np.exp(-((x - 0.3) ** 2 + (y - 0.65 * 0.75) ** 2) / 0.02) + 0.3 * (x + 0.4 * y > 0.7)
    u = 0.3 * np.sin(np.pi * y / 0.75) + 0.1
    v = -0.2 * np.cos(np.pi * x) + 0.15
    p = 1.0 + 0.6 * np.exp(-((x - 0.35) ** 2 + (y - 0.3) ** 2) / 0.03)
    return _cons2(rho, u, v, p)


def _mirror(fn, dim, walls_x, period_x, walls_y=None, period_y=None):
    """The mirror-extended initial data of fn on [0, 2 Lx] (x [0, 2 Ly]):
    fold every point back into [0, L] and negate the normal momentum."""
    def f(pts):
        pts = np.array(pts, dtype=np.float64)
        neg_x = np.zeros(len(pts), bool)
        neg_y = np.zeros(len(pts), bool)
        if walls_x:
            x = np.mod(pts[:, 0], 2 * period_x)
            neg_x = x > period_x
            pts[:, 0] = np.where(neg_x, 2 * period_x - x, x)
        if walls_y:
            y = np.mod(pts[:, 1], 2 * period_y)
            neg_y = y > period_y
            pts[:, 1] = np.where(neg_y, 2 * period_y - y, y)
        out = fn(pts)
        out[neg_x, 1] *= -1.0
        if dim == 2:
            out[neg_y, 2] *= -1.0
        return out
    return f


def _run(p, fn, nsteps):
    u0 = O.project_fn(p, fn)
    u, _, done, st = O.advance(p, u0, 0.0, 0.0, nsteps)
    assert st == O.OK and done == nsteps
    return u


def _dual_map(n, walls):
    """Extended-periodic dual index of each stored dual index of the walled
    mesh (vertex v = i + 1 for i < n; the slot n is vertex 0 = extended 2n)."""
    idx = list(range(n))
    if walls:
        idx.append(2 * n - 1)
    return np.array(idx)


def _restrict(u_ext, nx, ny, walls_x, walls_y, dim):
    """The walled layout's cells taken from the extended periodic state."""
    F, M = u_ext.shape[1], u_ext.shape[2]
    if dim == 1:
        prim = u_ext[0][..., :nx]
        dual = u_ext[1][..., _dual_map(nx, walls_x)]
        out = np.zeros((2, F, M, 1, nx + walls_x))
        out[0, ..., :nx] = prim
        out[1] = dual
        return out
    jx = _dual_map(nx, walls_x)
    jy = _dual_map(ny, walls_y) if walls_y else np.arange(ny)
    out = np.zeros((2, F, M, ny + walls_y, nx + walls_x))
    out[0, :, :, :ny, :nx] = u_ext[0][:, :, :ny, :nx]
    out[1] = u_ext[1][:, :, jy][:, :, :, jx]
    return out


def _rel(a, b):
    """max |a - b| / max |b| per field (arrays [..., F, M, ny, nx])."""
    ax = tuple(i for i in range(a.ndim) if i != a.ndim - 4)
    return (np.abs(a - b).max(axis=ax) / np.abs(b).max(axis=ax)).max()


def test_reflective_1d_is_the_mirrored_periodic_problem():
    n, steps = 24, 12
    walled = O.Problem(dim=1, nx=n, ny=1, k=2, system=O.EULER, bc=O.REFLECTIVE, oe=1, rk=3, ax=0.0, bx=1.0,
                       gamma=GAMMA, cfl=0.1)
    ext = O.Problem(dim=1, nx=2 * n, ny=1, k=2, system=O.EULER, bc=O.PERIODIC, oe=1, rk=3, ax=0.0, bx=2.0,
                    gamma=GAMMA, cfl=0.1)
    assert walled.shape == (2, 3, 3, 1, n + 1)
    a = _run(walled, _ic1, steps)
    b = _restrict(_run(ext, _mirror(_ic1, 1, True, 1.0), steps), n, 1, 1, 0, 1)
    assert _rel(a[0, ..., :n], b[0, ..., :n]) < 1e-12
    assert _rel(a[1], b[1]) < 1e-12
    assert np.all(a[0, ..., n:] == 0.0)  # the primal mesh's unused slot
    # the wall-centred dual cells keep the mirror symmetry: normal momentum
    # and the odd modes of the even fields vanish there (to rounding)
    for c in (n - 1, n):
        assert abs(a[1, 1, 0, 0, c]) < 1e-12 and abs(a[1, 0, 1, 0, c]) < 1e-12
    # the comparison discriminates: a copy closure (transmissive) misses
    trans = O.Problem(dim=1, nx=n, ny=1, k=2, system=O.EULER, bc=O.TRANSMISSIVE, oe=1, rk=3, ax=0.0, bx=1.0,
                      gamma=GAMMA, cfl=0.1)
    c = _run(trans, _ic1, steps)
    assert _rel(c[0], b[0, ..., :n]) > 1e-6


@pytest.mark.parametrize("walls_y", [True, False])
def test_reflective_2d_is_the_mirrored_periodic_problem(walls_y):
    nx, ny, Ly, steps = 8, 6, 0.75, 3
    bc = (O.REFLECTIVE, O.REFLECTIVE, O.REFLECTIVE if walls_y else O.PERIODIC,
          O.REFLECTIVE if walls_y else O.PERIODIC)
    walled = O.Problem(dim=2, nx=nx, ny=ny, k=2, basis=O.BASIS_Q, system=O.EULER, bc=bc, oe=1, rk=3,
                       ax=0.0, bx=1.0, ay=0.0, by=Ly, gamma=GAMMA, cfl=0.1)
    ext = O.Problem(dim=2, nx=2 * nx, ny=2 * ny if walls_y else ny, k=2, basis=O.BASIS_Q, system=O.EULER,
                    bc=O.PERIODIC, oe=1, rk=3, ax=0.0, bx=2.0, ay=0.0, by=2 * Ly if walls_y else Ly, gamma=GAMMA,
                    cfl=0.1)
    assert walled.shape == (2, 4, 9, ny + walls_y, nx + 1)
    a = _run(walled, _ic2, steps)
    b = _restrict(_run(ext, _mirror(_ic2, 2, True, 1.0, walls_y, Ly), steps), nx, ny, 1, int(walls_y), 2)
    assert _rel(a[0, :, :, :ny, :nx], b[0, :, :, :ny, :nx]) < 1e-12
    assert _rel(a[1], b[1]) < 1e-12


def test_reflective_needs_a_velocity_and_paired_periodic_sides():
    for kw in (dict(dim=1, system=O.ADVECTION, bc=O.REFLECTIVE), dict(dim=1, system=O.BURGERS, bc=O.REFLECTIVE),
               dict(dim=2, system=O.EULER, bc=(O.PERIODIC, O.REFLECTIVE, O.PERIODIC, O.PERIODIC))):
        with pytest.raises(ValueError):
            O.Problem(nx=4, ny=4, **kw).c()
    # one wall and one outflow side in a direction is a valid mix
    p = O.Problem(dim=2, nx=4, ny=4, system=O.EULER, bc=(O.REFLECTIVE, O.TRANSMISSIVE, O.PERIODIC, O.PERIODIC))
    p.c()
    assert p.shape == (2, 4, 9, 4, 5)
