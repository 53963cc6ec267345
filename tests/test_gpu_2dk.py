"""Degree-generic 2D CUDA path: Q^k and P^k for k = 1, 2, 3, advection,
Burgers and Euler, every RK method, against the CPU oracle through the C-ABI.

Tolerances (relative L1 per field over all modal coefficients of both meshes):
1e-12 for single operator applications (RHS, OE step), 1e-10 after a few full
steps of smooth data, 1e-9 for the discontinuous Riemann data.  Meshes of
37 x 13 cells span two 32-cell block columns and a ragged 4-row block tail.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_12473_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2503_12473_gb300 import oecdg
    oecdg.load()


def _ctx(w):
    from paper_2503_12473_gb300 import oecdg as G
    return G.Context(G.desc_from_workload(w))


def _oracle_problem(w):
    return O.Problem(dim=w.dim, nx=w.nx, ny=w.ny, k=w.k, basis=w.basis, system=w.system, bc=w.bc, oe=w.oe,
                     rk=w.rk, ax=w.ax, bx=w.bx, ay=w.ay, by=w.by, gamma=w.gamma, adv_x=w.adv[0], adv_y=w.adv[1],
                     cfl=w.cfl)


def rel_l1(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).sum(axis=(0, 2, 3, 4)) / np.maximum(np.abs(b).sum(axis=(0, 2, 3, 4)), 1e-300)


def _sin2(xy):
    return (np.sin(np.pi * (xy[:, 0] + xy[:, 1])) ** 2)[:, None]


def _wl(sys, k, basis, rk=3, nx=37, ny=13):
    if sys == W.ADVECTION:
        return W.Workload("adv2d", 2, nx, ny, k, W.ADVECTION, W.PERIODIC, 0.0, 1.0, 0.0, 1.0, basis=basis,
                          adv=(1.0, 1.0), cfl=0.2, rk=rk, u0=_sin2)
    if sys == W.BURGERS:
        return W.Workload("burgers2d", 2, nx, ny, k, W.BURGERS, W.PERIODIC, 0.0, 2.0, 0.0, 2.0, basis=basis,
                          cfl=0.2, rk=rk,
                          u0=lambda xy: (0.5 + 0.25 * np.sin(np.pi * (xy[:, 0] + xy[:, 1])))[:, None])
    return W.Workload("euler2d", 2, nx, ny, k, W.EULER, W.PERIODIC, 0.0, 2.0, 0.0, 2.0, basis=basis, cfl=0.2, rk=rk,
                      u0=W.steady_wave_2d())


def _both(w, seed=None, amp=1e-3):
    ctx = _ctx(w)
    p = _oracle_problem(w)
    ug = ctx.project(w.u0)
    uo = O.project_fn(p, w.u0)
    if seed is not None:
        pert = W.perturbation(uo.shape, seed, amp)
        ug = ug + torch.from_numpy(pert).cuda()
        uo = uo + pert
    return ctx, p, ug, uo


KB = [(k, b) for k in (1, 2, 3) for b in (W.BASIS_Q, W.BASIS_P) if (k, b) != (2, W.BASIS_Q)]


@pytest.mark.parametrize("k,basis", KB)
def test_quad_points_and_projection_2dk(k, basis):
    w = _wl(W.EULER, k, basis)
    ctx, p, ug, uo = _both(w)
    n = ctx.cdg_quad_points(None)
    assert n == 2 * 37 * 13 * 4 * (k + 1) ** 2
    xy = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    ctx.cdg_quad_points(xy)
    np.testing.assert_allclose(xy.cpu().numpy(), O.quad_points(p), rtol=0, atol=1e-14)
    assert ug.shape == uo.shape
    assert rel_l1(ug.cpu().numpy(), uo).max() < 1e-13


@pytest.mark.parametrize("sys", [W.ADVECTION, W.BURGERS, W.EULER])
@pytest.mark.parametrize("k,basis", KB)
def test_rhs_and_oe_parity_2dk(sys, k, basis):
    """cdg_rhs, cdg_oe_coefficients (delta^0..delta^k, sigma) and cdg_oe_damp on
    perturbed data."""
    w = _wl(sys, k, basis)
    ctx, p, ug, uo = _both(w, seed=41 + 3 * k + basis, amp=1e-2 if sys != W.EULER else 1e-3)
    tm = 1.7e-3
    Lg = torch.empty_like(ug)
    ctx.cdg_rhs(ug, tm, Lg)
    assert rel_l1(Lg.cpu().numpy(), O.rhs(p, uo, tm)).max() < 1e-12
    dg = torch.zeros((2, w.ny, w.nx, k + 1), dtype=torch.float64, device="cuda")
    sg = torch.zeros((2, w.nfields), dtype=torch.float64, device="cuda")
    ctx.cdg_oe_coefficients(ug, dg, sg)
    do, so, ao, st = O.oe_coefficients(p, uo)
    assert st == O.OK
    np.testing.assert_allclose(sg.cpu().numpy(), so, rtol=1e-11)
    d = dg.cpu().numpy()
    for m in range(k + 1):
        assert np.abs(d[..., m] - do[..., m]).max() <= 1e-11 * max(np.abs(do[..., m]).max(), 1e-300), m
    ctx.cdg_set_dt(0.6 * tm, tm)
    out = torch.empty_like(ug)
    ctx.cdg_oe_damp(ug, out)
    ref, st = O.oe(p, uo, 0.6 * tm)
    assert rel_l1(out.cpu().numpy(), ref).max() < 1e-12


STEP_CASES = [
    (W.EULER, 1, W.BASIS_Q, 2), (W.EULER, 1, W.BASIS_P, 2), (W.EULER, 2, W.BASIS_P, 3),
    (W.EULER, 3, W.BASIS_P, 4), (W.EULER, 3, W.BASIS_Q, 4), (W.EULER, 2, W.BASIS_Q, 4),
    (W.ADVECTION, 3, W.BASIS_Q, 4), (W.ADVECTION, 2, W.BASIS_P, 1), (W.BURGERS, 1, W.BASIS_P, 2),
    (W.BURGERS, 2, W.BASIS_Q, 3),
]


@pytest.mark.parametrize("sys,k,basis,rk", STEP_CASES)
def test_step_parity_2dk(sys, k, basis, rk):
    w = _wl(sys, k, basis, rk)
    ctx, p, ug, uo = _both(w)
    ctx.cdg_step(ug, 0.0, 0.0, 4)
    ref, t, n, st = O.advance(p, uo, 0.0, 0.0, 4)
    assert st == O.OK and n == 4
    err = rel_l1(ug.cpu().numpy(), ref)
    assert err.max() < 1e-10, err
    assert abs(ctx.cdg_get_time() - t) <= 1e-14 * max(t, 1.0)


@pytest.mark.parametrize("k,basis", [(1, W.BASIS_P), (3, W.BASIS_Q)])
def test_step_parity_2dk_riemann_transmissive(k, basis):
    """Discontinuous four-quadrant data, transmissive boundaries."""
    w = W.riemann_2d(n=34).resized(34, 21, k=k, basis=basis, rk=3)
    ctx, p, ug, uo = _both(w)
    ctx.cdg_step(ug, 0.0, 0.0, 3)
    ref, t, n, st = O.advance(p, uo, 0.0, 0.0, 3)
    assert st == O.OK
    assert rel_l1(ug.cpu().numpy(), ref).max() < 1e-9


def test_generic_q2_rk3_matches_tiled_q2():
    """Q^2 SSP-RK3 through the generic kernels (reached with RK4's sibling
    entry point cdg_rk_combine on an RK4 context) agrees with the tiled Q^2
    kernels to rounding: one stage each, same tau."""
    from paper_2503_12473_gb300 import oecdg as G
    w = _wl(W.EULER, 2, W.BASIS_Q, rk=3, nx=40, ny=24)
    tiled = _ctx(w)
    generic = G.Context(G.desc_from_workload(w, rk=4))
    u = tiled.project(w.u0)
    pert = torch.from_numpy(W.perturbation(tuple(u.shape), 5, 1e-3)).cuda()
    u = u + pert
    for c in (tiled, generic):
        c.cdg_set_dt(2e-3, 2.5e-3)
    a = torch.empty_like(u)
    b = torch.empty_like(u)
    ul = u * 1.001
    tiled.cdg_rk_stage(1, u, ul, a)
    generic.cdg_rk_combine(ul, [u, ul], [0.75, 0.25], 0.25, b)
    assert rel_l1(a.cpu().numpy(), b.cpu().numpy()).max() < 1e-13
    tiled.cdg_oe_damp(a, ul)
    generic.cdg_oe_damp(a, u)
    assert rel_l1(ul.cpu().numpy(), u.cpu().numpy()).max() < 1e-13


def test_adjoint_refuses_generic_configurations():
    from paper_2503_12473_gb300 import oecdg as G
    w = _wl(W.EULER, 3, W.BASIS_Q, rk=3, nx=16, ny=16)
    ctx = _ctx(w)
    u = ctx.project(w.u0)
    with pytest.raises(G.CdgError) as e:
        ctx.cdg_step_adjoint(u, u.clone(), torch.empty_like(u))
    assert e.value.status == G.CDG_EUNSUPPORTED


@pytest.mark.parametrize("case", ["tiled_q2_riemann", "generic_p3_rk4", "tiled_q2_no_oe"])
def test_step_graph_equals_step_2d(case):
    """cdg_step_graph replays one captured step; results equal cdg_step_async
    bit for bit on the tiled Q^2 kernels (with and without the OE step, whose
    absence puts a copy node in the graph) and on the generic P^3 kernels with
    RK4's extra stage buffers."""
    from paper_2503_12473_gb300 import oecdg as G
    if case == "generic_p3_rk4":
        w = _wl(W.EULER, 3, W.BASIS_P, rk=4, nx=40, ny=20)
        over = {}
    else:
        w = W.riemann_2d(n=48).resized(48, 36)
        over = {"oe": 0} if case == "tiled_q2_no_oe" else {}
    st = torch.cuda.Stream()
    ctx = G.Context(G.desc_from_workload(w, **over), stream=st)
    with torch.cuda.stream(st):
        u0 = ctx.project(w.u0)
        a = u0.clone()
        b = u0.clone()
    ctx.cdg_step_async(a, 0.0, 0.0, 5)
    ctx.cdg_step_graph(b, 0.0, 0.0, 5)
    assert ctx.cdg_check_status() == G.CDG_OK
    assert torch.equal(a, b)


def _pk_eval(coef, k, g):
    """Values of a P^k expansion (modes by total degree, then decreasing a) at
    the tensor points g x g of every cell: coef [M, ny, nx] -> [ny, nx, q, q]."""
    V = np.polynomial.legendre.legvander(g, k)  # [q, k+1]
    out = 0.0
    m = 0
    for s in range(k + 1):
        for a in range(s, -1, -1):
            b = s - a
            out = out + coef[m][:, :, None, None] * V[None, None, :, b][..., :, None] * V[None, None, :, a][..., None, :]
            m += 1
    return out


def _l1_error(u, k, n, L, exact):
    g, wq = np.polynomial.legendre.leggauss(k + 2)
    v = _pk_eval(u[0, 0], k, g)  # primal mesh, first field
    h = L / n
    xs = (np.arange(n)[None, :, None, None] + 0.5 + 0.5 * g[None, None, None, :]) * h
    ys = (np.arange(n)[:, None, None, None] + 0.5 + 0.5 * g[None, None, :, None]) * h
    e = np.abs(v - exact(xs, ys))
    return float(np.sum(e * np.outer(wq, wq)[None, None] / 4)) / (n * n)


@pytest.mark.parametrize("case", ["euler_steady_wave", "advection"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_pk_orders_2d(case, k):
    """The P^k scheme with its (k+1)-order RK method converges at order ~k+1
    (the error estimate of Section 3.3; Tables 3 and 4): l1 error of the first
    field over the primal cells at meshes 16^2 and 32^2, observed order > k + 0.5."""
    errs = []
    for n in (16, 32):
        if case == "advection":
            w = W.Workload("adv", 2, n, n, k, W.ADVECTION, W.PERIODIC, 0.0, 1.0, 0.0, 1.0, basis=W.BASIS_P,
                           adv=(1.0, 1.0), cfl={1: 0.45, 2: 0.33, 3: 0.31}[k], rk=k + 1, u0=_sin2)
            T, L = 0.25, 1.0
            exact = lambda x, y: np.sin(np.pi * (x + y - 2 * T)) ** 2
        else:
            w = W.steady_wave_2d_workload(n, k, W.BASIS_P)
            T, L = 0.5, 2.0
            exact = lambda x, y: 1 + 0.2 * np.sin(np.pi * (x - y))
        ctx = _ctx(w)
        u = ctx.project(w.u0)
        t = 0.0
        while t < T:
            ctx.cdg_step(u, t, T, 256)
            t = ctx.cdg_get_time()
        errs.append(_l1_error(u.cpu().numpy(), k, n, L, exact))
    rate = math.log2(errs[0] / errs[1])
    assert rate > k + 0.5, (errs, rate)
