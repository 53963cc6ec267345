"""Pins of the oracle's sigma_K (Section 2.2): the L-infinity distance of a
field from its domain average, and its reading for a field that is constant up
to rounding.

sigma_K = ||u_h - avg(u_h)||_inf, the OE coefficients divide by it, and they
vanish where it is 0.  The oracle takes the max over the Gauss points of every
cell and counts a sigma at or below 2^-40 of the field's magnitude as 0: a
field that is constant in exact arithmetic carries a few ulps of rounding noise
after the projection, and its computed sigma is then a few ulps too.

Checked here: sigma against the plain definition, evaluated independently from
the point values (orc_eval_cells) and the cell-average mean; the floor on both
sides of 2^-40; and that a rounding-noisy uniform density (Section 4's
two-blast-wave start) steps like the exactly constant one.  Also the
multi-index sum in delta^2 (each multi-index once), by a closed-form ratio
that a multinomial (rotation-invariant) weighting of the mixed derivative
fails.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

GAMMA = 1.4


def _problem(n=48, **kw):
    base = dict(dim=1, nx=n, ny=1, k=2, system=O.EULER, bc=O.PERIODIC, oe=1, rk=3, ax=0.0, bx=1.0, gamma=GAMMA,
                cfl=0.1)
    base.update(kw)
    return O.Problem(**base)


def _state(p, rho_fn, v=0.3, pr=1.0):
    def fn(xs):
        x = xs[:, 0]
        rho = rho_fn(x)
        vel = v + 0.2 * np.sin(2 * np.pi * x)
        return np.stack([rho, rho * vel, pr / (GAMMA - 1.0) + 0.5 * rho * vel * vel], axis=-1)
    return O.project_fn(p, fn)


def _sigma_by_definition(p, u):
    """max over the Gauss points of |u - avg| per mesh and field, avg = the mean
    of the cell averages (uniform cells, periodic: every stored cell counts)."""
    x, _ = O.gauss(p.k + 1)
    out = np.zeros((2, p.nfields))
    for mesh in range(2):
        n = p.nx
        vals = O.eval_cells(p, u, mesh, x)[0, :n]      # [n, nq, F]
        avg = u[mesh, :, 0, 0, :n].mean(axis=1)        # [F]
        out[mesh] = np.abs(vals - avg).max(axis=(0, 1))
    return out


def test_sigma_is_the_sup_distance_from_the_domain_average():
    p = _problem()
    u = _state(p, lambda x: 1.0 + 0.3 * np.cos(2 * np.pi * x) + 0.1 * (x > 0.4))
    _, sigma, avg, st = O.oe_coefficients(p, u)
    assert st == O.OK
    ref = _sigma_by_definition(p, u)
    # |u - avg| cancels: compare to rounding of the field's magnitude
    mag = np.abs(u[:, :, 0]).max(axis=(0, 2, 3))
    assert (np.abs(sigma - ref) <= 1e-13 * mag).all(), (sigma, ref)
    assert (sigma > 0.05).all()
    np.testing.assert_allclose(avg, u[:, :, 0, 0, :p.nx].mean(axis=2), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("amp,floored", [(1e-14, True), (2e-13, True), (1e-11, False), (1e-9, False)])
def test_sigma_floor_at_2_pow_minus_40_of_the_magnitude(amp, floored):
    """A density of relative variation amp: sigma counts as 0 when it is at
    most 2^-40 (9.1e-13) times the magnitude, and is the plain distance
    otherwise.  The momentum and energy fields vary and keep their sigma."""
    p = _problem()
    u = _state(p, lambda x: 2.0 * (1.0 + amp * np.sin(2 * np.pi * x)))
    _, sigma, _, st = O.oe_coefficients(p, u)
    assert st == O.OK
    ref = _sigma_by_definition(p, u)
    assert (ref[:, 0] <= 2.0 ** -40 * 2.0 * (1 + amp)).all() == floored
    if floored:
        assert (sigma[:, 0] == 0.0).all()
    else:
        np.testing.assert_allclose(sigma[:, 0], ref[:, 0], rtol=1e-3)
    mag = np.abs(u[:, 1:, 0]).max(axis=(0, 2, 3))
    assert (np.abs(sigma[:, 1:] - ref[:, 1:]) <= 1e-13 * mag).all()


def test_rounding_noise_in_a_uniform_density_does_not_damp():
    """Section 4's two-blast-wave start: density 1 everywhere, whose projection
    leaves an ulp above 1 in the averages and ~1e-16 in the higher modes.  One
    step from it equals one step from the exactly constant density to
    rounding; a sigma of a few ulps would instead damp every mode of every cell
    (the momentum after one step then differs by percents)."""
    from paper_2503_12473_gb300 import workloads as W
    w = W.two_blast_waves_1d(240)
    p = O.Problem(dim=1, nx=w.nx, ny=1, k=2, system=O.EULER, bc=w.bc, oe=1, rk=3, ax=w.ax, bx=w.bx, cfl=w.cfl)
    noisy = O.project_fn(p, w.u0)
    clean = noisy.copy()
    clean[0, 0, 0, 0, :w.nx] = 1.0
    clean[1, 0, 0, 0, :] = 1.0
    clean[:, 0, 1:] = 0.0
    assert np.abs(noisy - clean).max() > 0.0  # the projection did leave noise
    _, sg, _, _ = O.oe_coefficients(p, noisy)
    assert (sg[:, 0] == 0.0).all()
    a, *_ = O.advance(p, noisy, 0.0, w.T, 1)
    b, *_ = O.advance(p, clean, 0.0, w.T, 1)
    rel = np.abs(a - b).max(axis=(0, 2, 3, 4)) / np.abs(b).max(axis=(0, 2, 3, 4))
    assert rel.max() < 1e-13, rel


def _delta2_of_local_quadratic(coef):
    """delta^2 of a primal cell of a periodic 4 x 4 Q^2 advection mesh whose
    primal cells all hold the same local polynomial (modal coefficients coef
    at (a, b), Q^2 index 3 b + a) plus a large linear part 1e6 P_1(xi), and
    whose dual mesh is 0: u^C - u^D on every half-face is the cell's own
    polynomial, sigma is set by the linear part (the same for every coef to
    1e-6), and the second derivatives are constants."""
    p = O.Problem(dim=2, nx=4, ny=4, k=2, basis=O.BASIS_Q, system=O.ADVECTION, bc=O.PERIODIC, adv_x=1.0,
                  adv_y=1.0, cfl=0.1)
    u = p.zeros()
    u[0, 0, 1] = 1e6  # (a, b) = (1, 0)
    for (a, b), c in coef.items():
        u[0, 0, 3 * b + a] += c
    delta, sigma, _, st = O.oe_coefficients(p, u)
    assert st == O.OK
    return delta[0, 1, 2, 2], sigma[0, 0]


def test_delta2_is_the_plain_multi_index_sum():
    """Section 2.2's delta^m integrates (sum over |alpha| = m of
    (d^alpha (u^C - u^D))^2)^(1/2): for m = 2 the multi-indices (2,0), (1,1),
    (0,2), each once.  A face integrand that is constant makes delta^2
    proportional to that square root: xi eta (only the mixed derivative, 1)
    against (xi^2 - eta^2)/2 = (P_2(xi) - P_2(eta))/3 (the pure ones, 1 and -1)
    gives sqrt(1 / 2) -- the same rotated function, so a rotation-invariant
    (multinomial, Frobenius) sum would give 1."""
    d_mixed, s1 = _delta2_of_local_quadratic({(1, 1): 1.0})
    d_pure, s2 = _delta2_of_local_quadratic({(2, 0): 1.0 / 3.0, (0, 2): -1.0 / 3.0})
    assert abs(s1 / s2 - 1.0) < 1e-5
    assert d_mixed > 0.0 and d_pure > 0.0
    assert abs(d_mixed / d_pure - math.sqrt(0.5)) < 1e-5, d_mixed / d_pure
