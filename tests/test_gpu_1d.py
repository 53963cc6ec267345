"""1D CUDA path for every degree k = 1, 2, 3, every system (advection, Burgers,
1D Euler) and every RK method (forward Euler, SSP-RK2, SSP-RK3, classical
RK4), against the CPU oracle through the C-ABI; and the Table 2 P^3 Burgers
errors reproduced on the GPU.

Tolerances: relative L1 per field over all modal coefficients of both meshes,
1e-12 for single operator applications (RHS, OE), 1e-10 after 20 full steps of
smooth data, 1e-9 for the Shu-Osher data (discontinuous; the damping
coefficients amplify the round-off of the jumps).  Mesh sizes span several
128-cell blocks with a ragged tail.
"""
import math
import os

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


def _ctx(w, **over):
    from paper_2503_12473_gb300 import oecdg as G
    return G.Context(G.desc_from_workload(w, **over))


def _oracle_problem(w):
    return O.Problem(dim=w.dim, nx=w.nx, ny=w.ny, k=w.k, basis=w.basis, system=w.system, bc=w.bc, oe=w.oe,
                     rk=w.rk, ax=w.ax, bx=w.bx, ay=w.ay, by=w.by, gamma=w.gamma, adv_x=w.adv[0], adv_y=w.adv[1],
                     cfl=w.cfl)


def rel_l1(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).sum(axis=(0, 2, 3, 4)) / np.maximum(np.abs(b).sum(axis=(0, 2, 3, 4)), 1e-300)


def _wl(sys, k, rk, n):
    if sys == W.ADVECTION:
        w = W.Workload(f"adv_{k}", 1, n, 1, k, W.ADVECTION, W.PERIODIC, 0.0, 2 * math.pi, adv=(-0.8, 0.0),
                       cfl=0.1, rk=rk, u0=W.sine_1d(2 * math.pi))
    elif sys == W.BURGERS:
        w = W.burgers_1d(n, k)
        w = W.Workload(w.name, 1, n, 1, k, W.BURGERS, W.PERIODIC, w.ax, w.bx, cfl=0.31 if rk == 4 else 0.1, rk=rk,
                       u0=w.u0)
    else:
        w = W.shu_osher_1d(n)
        w = W.Workload(w.name, 1, n, 1, k, W.EULER, W.TRANSMISSIVE, w.ax, w.bx, cfl=0.1, rk=rk, u0=w.u0)
    return w


CASES = ([(W.ADVECTION, k, rk) for k in (1, 2, 3) for rk in (3, 4)]
         + [(W.BURGERS, k, rk) for k in (1, 2, 3) for rk in (1, 2, 3, 4)]
         + [(W.EULER, k, rk) for k in (1, 2, 3) for rk in (2, 3)]
         + [(W.EULER, 3, 4)])


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


@pytest.mark.parametrize("k", [1, 2, 3])
def test_quad_points_and_projection_1d(k):
    w = _wl(W.BURGERS, k, 3, 301)
    ctx, p, ug, uo = _both(w)
    n = ctx.cdg_quad_points(None)
    assert n == 2 * 301 * 2 * (k + 1)
    x = torch.empty((n, 1), dtype=torch.float64, device="cuda")
    ctx.cdg_quad_points(x)
    np.testing.assert_allclose(x.cpu().numpy().ravel(), O.quad_points(p).ravel(), rtol=0, atol=1e-14)
    assert ug.shape == (2, 1, k + 1, 1, 301)
    assert rel_l1(ug.cpu().numpy(), uo).max() < 1e-13


@pytest.mark.parametrize("sys", [W.ADVECTION, W.BURGERS, W.EULER])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_rhs_and_oe_parity_1d(sys, k):
    """cdg_rhs, cdg_oe_coefficients and cdg_oe_damp on perturbed data."""
    w = _wl(sys, k, 3, 333)
    ctx, p, ug, uo = _both(w, seed=31 + k, amp=1e-2 if sys != W.EULER else 1e-3)
    tm = 2.3e-3
    Lg = torch.empty_like(ug)
    ctx.cdg_rhs(ug, tm, Lg)
    assert rel_l1(Lg.cpu().numpy(), O.rhs(p, uo, tm)).max() < 1e-12
    dg = torch.zeros((2, 1, w.nx, k + 1), dtype=torch.float64, device="cuda")
    sg = torch.zeros((2, w.nfields), dtype=torch.float64, device="cuda")
    ctx.cdg_oe_coefficients(ug, dg, sg)
    do, so, ao, st = O.oe_coefficients(p, uo)
    assert st == O.OK
    np.testing.assert_allclose(sg.cpu().numpy(), so, rtol=1e-11)
    d = dg.cpu().numpy()
    for m in range(k + 1):
        assert np.abs(d[..., m] - do[..., m]).max() <= 1e-11 * max(np.abs(do[..., m]).max(), 1e-300), m
    ctx.cdg_set_dt(0.7 * tm, tm)
    out = torch.empty_like(ug)
    ctx.cdg_oe_damp(ug, out)
    ref, st = O.oe(p, uo, 0.7 * tm)
    assert rel_l1(out.cpu().numpy(), ref).max() < 1e-12


@pytest.mark.parametrize("sys,k,rk", CASES)
def test_step_parity_1d(sys, k, rk):
    """cdg_step (wave speed, every stage of the method with the OE step after
    each) against the oracle after 20 steps."""
    w = _wl(sys, k, rk, 301)
    ctx, p, ug, uo = _both(w)
    ctx.cdg_step(ug, 0.0, 0.0, 20)
    ref, t, n, st = O.advance(p, uo, 0.0, 0.0, 20)
    assert st == O.OK and n == 20
    tol = 1e-9 if sys == W.EULER else 1e-10
    err = rel_l1(ug.cpu().numpy(), ref)
    assert err.max() < tol, err
    assert abs(ctx.cdg_get_time() - t) <= 1e-14 * max(t, 1.0)


def test_rk4_stage_entry_points_match_step():
    """RK4 assembled from cdg_compute_dt, cdg_rk_stage (stages 0-2),
    cdg_rk_combine (stage 3) and cdg_oe_damp gives cdg_step's result bit for
    bit."""
    w = _wl(W.BURGERS, 3, 4, 257)
    ctx, p, ug, uo = _both(w)
    ref = ug.clone()
    ctx.cdg_step(ref, 0.0, 0.0, 1)
    ctx.cdg_compute_dt(ug, 0.0, 0.0)
    U = [ug]
    tmp = torch.empty_like(ug)
    for l in range(3):
        ctx.cdg_rk_stage(l, ug, U[-1], tmp)
        nxt = torch.empty_like(ug)
        ctx.cdg_oe_damp(tmp, nxt)
        U.append(nxt)
    ctx.cdg_rk_combine(U[3], U, [-1.0 / 3.0, 1.0 / 3.0, 2.0 / 3.0, 1.0 / 3.0], 1.0 / 6.0, tmp)
    out = torch.empty_like(ug)
    ctx.cdg_oe_damp(tmp, out)
    assert torch.equal(out, ref)


def _cell_gauss_errors(u, n, t):
    """l1 = int |e|, l2 = (int e^2)^(1/2), linf = max over the 4 Gauss points of
    every primal cell (the norms the Table 2 golden rows were matched with)."""
    g, wq = np.polynomial.legendre.leggauss(4)
    coef = u[0, 0, :, 0, :]  # [k+1, n]: unnormalised Legendre coefficients
    v = np.polynomial.legendre.legval(g, coef)  # [n, 4]
    h = 2 * math.pi / n
    x = (np.arange(n)[:, None] + 0.5 + 0.5 * g[None, :]) * h
    uex = np.sin(x) + 0.5
    for _ in range(60):
        uex = uex - (uex - np.sin(x - uex * t) - 0.5) / (1 + t * np.cos(x - uex * t))
    e = np.abs(v - uex)
    return np.sum(e * wq / 2) * h, math.sqrt(np.sum(e * e * wq / 2) * h), e.max()


def test_table2_burgers_p3_on_gpu():
    """Table 2, P^3 rows (Burgers, u0 = sin x + 0.5, t = 0.6, RK4, CFL 0.31):
    the CUDA path reproduces the printed errors within 1 % (the oracle's own
    pin), and at N = 128 agrees with the oracle's final state to 1e-11."""
    from paper_2503_12473_gb300 import oecdg as G
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "table2_burgers_p3.txt"))
    for n, l1p, l2p, lip in rows:
        n = int(n)
        w = W.burgers_1d(n, 3)
        ctx = _ctx(w)
        u = ctx.project(w.u0)
        t = 0.0
        while t < w.T:
            ctx.cdg_step(u, t, w.T, 64)
            t = ctx.cdg_get_time()
        assert abs(t - w.T) < 1e-14
        got = _cell_gauss_errors(u.cpu().numpy(), n, t)
        for gv, pv in zip(got, (l1p, l2p, lip)):
            assert abs(gv / pv - 1.0) < 0.01, (n, got, (l1p, l2p, lip))
        if n == 128:
            p = _oracle_problem(w)
            ref, to, _, st = O.advance(p, O.project_fn(p, w.u0), 0.0, w.T)
            assert st == O.OK and to == w.T
            assert rel_l1(u.cpu().numpy(), ref).max() < 1e-11


def test_ssp2_parity_2d_and_combine_forms():
    """2D SSP-RK2 steps against the oracle; the general combine runs the
    two-state form in 2D and refuses others."""
    from paper_2503_12473_gb300 import oecdg as G
    w = W.vortex_2d(n=36).resized(36, 36, rk=2)
    ctx = _ctx(w)
    p = _oracle_problem(w)
    ug = ctx.project(w.u0)
    uo = O.project_fn(p, w.u0)
    ctx.cdg_step(ug, 0.0, 0.0, 4)
    ref, _, _, st = O.advance(p, uo, 0.0, 0.0, 4)
    assert rel_l1(ug.cpu().numpy(), ref).max() < 1e-11
    ctx.cdg_compute_dt(ug, 0.0, 0.0)
    a = torch.empty_like(ug)
    b = torch.empty_like(ug)
    ul = ug * 1.001
    ctx.cdg_rk_stage(1, ug, ul, a)
    ctx.cdg_rk_combine(ul, [ug, ul], [0.5, 0.5], 0.5, b)
    assert torch.equal(a, b)
    with pytest.raises(G.CdgError) as e:
        ctx.cdg_rk_combine(ul, [ug, ul, ug], [0.5, 0.25, 0.25], 0.5, b)
    assert e.value.status == G.CDG_EUNSUPPORTED


def test_scope_checks():
    from paper_2503_12473_gb300 import oecdg as G
    for kw, status in ((dict(dim=1, nx=16, k=4), G.CDG_EUNSUPPORTED),
                       (dict(dim=1, nx=16, k=0), G.CDG_EUNSUPPORTED),
                       (dict(dim=2, nx=8, ny=8, k=4), G.CDG_EUNSUPPORTED),
                       (dict(dim=2, nx=8, ny=8, basis=7), G.CDG_EINVAL),
                       (dict(dim=1, nx=16, rk=5), G.CDG_EINVAL)):
        with pytest.raises(G.CdgError) as e:
            G.Context(G.MeshDesc(**kw))
        assert e.value.status == status, kw
    ctx = G.Context(G.MeshDesc(dim=1, nx=16, k=3, system=G.BURGERS, rk=G.RK_RK4, bx=2 * math.pi))
    u = ctx.zeros()
    with pytest.raises(G.CdgError) as e:
        ctx.cdg_rk_stage(3, u, u.clone(), torch.empty_like(u))
    assert e.value.status == G.CDG_EINVAL


@pytest.mark.parametrize("name", ["advection", "shu_osher"])
def test_step_graph_equals_step(name):
    """cdg_step_graph (one captured step replayed) gives cdg_step_async's
    result bit for bit, including the clipped last step at T_end and the
    skipped steps after it; a second call with another state re-captures."""
    from paper_2503_12473_gb300 import oecdg as G
    w = W.advection_1d(128) if name == "advection" else W.shu_osher_1d(400)
    T = w.T if name == "advection" else 0.01
    st = torch.cuda.Stream()
    ctx = G.Context(G.desc_from_workload(w), stream=st)
    with torch.cuda.stream(st):
        u0 = ctx.project(w.u0)
        a = u0.clone()
        b = u0.clone()
        c = u0.clone()
    n = 1400 if name == "advection" else 300
    ctx.cdg_step_async(a, 0.0, T, n)
    ta = ctx.cdg_get_time()
    ctx.cdg_step_graph(b, 0.0, T, n // 2)
    tb = ctx.cdg_get_time()
    ctx.cdg_step_graph(b, tb, T, n - n // 2)
    assert ctx.cdg_check_status() == G.CDG_OK
    assert ctx.cdg_get_time() == ta
    assert torch.equal(a, b)
    ctx.cdg_step_graph(c, 0.0, T, n)
    assert ctx.cdg_check_status() == G.CDG_OK
    assert torch.equal(a, c)


def test_step_graph_needs_own_stream():
    from paper_2503_12473_gb300 import oecdg as G
    w = W.advection_1d(64)
    ctx = G.Context(G.desc_from_workload(w))
    u = ctx.project(w.u0)
    with pytest.raises(G.CdgError) as e:
        ctx.cdg_step_graph(u, 0.0, 0.0, 2)
    assert e.value.status == G.CDG_EINVAL


@pytest.mark.parametrize("case", ["advection", "burgers"])
@pytest.mark.parametrize("k", [1, 2])
def test_pk_orders_1d(case, k):
    """P^1 and P^2 with their (k+1)-order RK methods converge at order ~k+1
    (Section 3.3; Tables 1 and 2): l1 error at the cell Gauss points of the
    primal mesh, meshes 64 and 128, observed order > k + 0.5."""
    errs = []
    for n in (64, 128):
        if case == "advection":
            w = W.Workload("adv", 1, n, 1, k, W.ADVECTION, W.PERIODIC, 0.0, 1.0, adv=(1.0, 0.0),
                           cfl={1: 0.45, 2: 0.33}[k], rk=k + 1, T=0.5,
                           u0=lambda xy: np.sin(2 * np.pi * np.asarray(xy).reshape(len(xy), -1)[:, 0])[:, None])
            ex = lambda x, t: np.sin(2 * np.pi * (x - t))
            L = 1.0
        else:
            w = W.burgers_1d(n, k)
            w = W.Workload(w.name, 1, n, 1, k, W.BURGERS, W.PERIODIC, w.ax, w.bx, cfl={1: 0.45, 2: 0.33}[k],
                           rk=k + 1, T=0.6, u0=w.u0)
            L = 2 * math.pi

            def ex(x, t):
                u = np.sin(x) + 0.5
                for _ in range(60):
                    u = u - (u - np.sin(x - u * t) - 0.5) / (1 + t * np.cos(x - u * t))
                return u
        ctx = _ctx(w)
        u = ctx.project(w.u0)
        t = 0.0
        while t < w.T:
            ctx.cdg_step(u, t, w.T, 512)
            t = ctx.cdg_get_time()
        g, wq = np.polynomial.legendre.leggauss(k + 2)
        v = np.polynomial.legendre.legval(g, u.cpu().numpy()[0, 0, :, 0, :])  # [n, q]
        x = (np.arange(n)[:, None] + 0.5 + 0.5 * g[None, :]) * (L / n)
        errs.append(float(np.sum(np.abs(v - ex(x, t)) * wq / 2)) / n)
    rate = math.log2(errs[0] / errs[1])
    assert rate > k + 0.5, (errs, rate)


PERSIST_CASES = [("advection", W.ADVECTION, 2, 3, 1), ("shu-osher", W.EULER, 2, 3, 1), ("euler-p3-rk4", W.EULER, 3, 4, 1),
                 ("burgers-p1-ssp2", W.BURGERS, 1, 2, 1), ("burgers-p2-euler1", W.BURGERS, 2, 1, 1),
                 ("advection-no-oe", W.ADVECTION, 3, 3, 0)]


@pytest.mark.parametrize("name,sys,k,rk,oe", PERSIST_CASES)
def test_step_persistent_equals_step(name, sys, k, rk, oe):
    """cdg_step_persistent (all steps in one cooperative launch, grid-wide
    barriers between the phases, one lane per cell) gives cdg_step_async's
    result (two lanes per cell, sigma folded in the OE launch) bit for bit, and
    the same time: every system, degree and RK method of the 1D path, with and
    without OE, periodic and transmissive, including the clipped last step at
    T_end and the skipped steps after it.  Its runs are deterministic."""
    from paper_2503_12473_gb300 import oecdg as G
    if name == "advection":
        w = W.advection_1d(128)
    elif name == "shu-osher":
        w = W.shu_osher_1d(4000)
    else:
        w = _wl(sys, k, rk, 300)
    w = W.Workload(w.name, 1, w.nx, 1, k, sys, w.bc, w.ax, w.bx, adv=w.adv, cfl=w.cfl, rk=rk, oe=oe, u0=w.u0)
    # the context on torch's current stream: the copies below and the steps are ordered
    ctx = G.Context(G.desc_from_workload(w))
    u0 = ctx.project(w.u0)
    a = u0.clone()
    b = u0.clone()
    # a short end time: the last of n steps is clipped, the rest skipped on the device
    ctx.cdg_step_async(a, 0.0, 0.0, 1)
    tau, _ = ctx.cdg_get_dt()
    T = 37.5 * tau
    n = 45
    ctx.cdg_step_async(a.copy_(u0), 0.0, T, n)
    ta = ctx.cdg_get_time()
    assert ctx.cdg_check_status() == G.CDG_OK
    ctx.cdg_step_persistent(b, 0.0, T, n)
    assert ctx.cdg_check_status() == G.CDG_OK
    assert ctx.cdg_get_time() == ta
    assert torch.equal(b, a), (a - b).abs().max().item()
    c = u0.clone()
    ctx.cdg_step_persistent(c, 0.0, T, n)
    assert torch.equal(b, c)  # deterministic
    # and without an end time, in two calls
    ctx.cdg_step_async(a.copy_(u0), 0.0, 0.0, 12)
    ctx.cdg_step_persistent(b.copy_(u0), 0.0, 0.0, 5)
    ctx.cdg_step_persistent(b, ctx.cdg_get_time(), 0.0, 7)
    assert ctx.cdg_check_status() == G.CDG_OK
    assert torch.equal(b, a)
    ctx.cdg_step_persistent(c.copy_(u0), 0.0, 0.0, 12)
    assert torch.equal(b, c)  # two launches of 5 + 7 steps equal one of 12


def test_step_persistent_barrier_wait_runs_out_without_hanging():
    """The grid barriers' waits are bounded.  With the test hook that makes
    every barrier wait for one arrival that never comes, the launch ends by
    itself after about the limit and cdg_check_status reports CDG_ETIMEOUT;
    nothing faults, and the context then steps normally again."""
    import time
    from paper_2503_12473_gb300 import oecdg as G
    w = W.shu_osher_1d(4000)
    ctx = G.Context(G.desc_from_workload(w))
    u0 = ctx.project(w.u0)
    a = u0.clone()
    b = u0.clone()
    ctx.cdg_set_wait(0.2, withheld=1)
    t0 = time.time()
    ctx.cdg_step_persistent(b, 0.0, 0.0, 3)
    assert ctx.cdg_check_status() == G.CDG_ETIMEOUT
    assert time.time() - t0 < 10.0
    ctx.cdg_set_wait(5.0, withheld=0)
    ctx.cdg_step_async(a, 0.0, 0.0, 3)
    ctx.cdg_step_persistent(b.copy_(u0), 0.0, 0.0, 3)
    assert ctx.cdg_check_status() == G.CDG_OK
    assert torch.equal(b, a)
    with pytest.raises(G.CdgError) as e:
        ctx.cdg_set_wait(0.0)
    assert e.value.status == G.CDG_EINVAL


def test_step_persistent_against_oracle():
    """The persistent launch against the oracle: 1D Euler Shu-Osher data, P^2,
    4000 cells, 100 steps (rel L1 <= 1e-9 per field, the bar for
    discontinuous runs), and 1D advection of sin x over its whole period
    (1280 steps, <= 1e-11)."""
    from paper_2503_12473_gb300 import oecdg as G
    for w, n, T, tol in ((W.shu_osher_1d(4000), 100, 0.0, 1e-9), (W.advection_1d(128), 1300, 2 * math.pi, 1e-11)):
        ctx = G.Context(G.desc_from_workload(w))
        p = _oracle_problem(w)
        uo = O.project_fn(p, w.u0)
        ug = torch.from_numpy(uo).cuda()
        ctx.cdg_step_persistent(ug, 0.0, T, n)
        assert ctx.cdg_check_status() == G.CDG_OK
        ref, t, steps, status = O.advance(p, uo, 0.0, T, n)
        assert status == O.OK
        assert abs(ctx.cdg_get_time() - t) <= 1e-13 * max(t, 1.0)
        assert rel_l1(ug.cpu().numpy(), ref).max() < tol, (w.name, rel_l1(ug.cpu().numpy(), ref))
