"""Parity at the full sizes of the measured workloads, in the launch
configuration bench.py times (a context bound to its own non-blocking stream).

* 1D advection, P^2, 128 cells, T = 2 pi (1280 steps): whole run against the
  oracle, rel L1 <= 1e-11.
* 1D Euler Shu-Osher, 4000 cells: the first 100 steps against the oracle
  (rel L1 <= 1e-9); the whole run to T = 1.8 by properties (status, end time,
  physical cell averages).
* 2D Euler four-quadrant Riemann, Q^2, 1024^2: the oracle is too slow for
  whole-mesh steps, so every operator is checked on sampled cells the oracle
  computes one by one (RHS, delta, sigma/avg over the whole meshes, the OE
  step, tau) on a seeded synthetic full-size state; the 200-step run by
  properties (status; the data's symmetry under x <-> y with u <-> v, which
  the scheme keeps in exact arithmetic).
* 256 batched meshes (seed 0 sizes): batched launch equals per-instance
  launches bit for bit on sampled instances; the smallest matches the oracle.
* Adjoint, 256^2 vortex, 400 steps, 20 checkpoints: directional derivatives
  against central differences (h = 1e-8) on seeded directions, rel <= 2e-5
  (finite differences through the OE step's kinks resolve no more; the
  per-step adjoint is checked to 1e-7 in test_gpu_adjoint.py).
"""
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


def _bench_ctx(w, **over):
    """A context as bench.py makes it: bound to its own stream."""
    from paper_2503_12473_gb300 import oecdg as G
    stream = torch.cuda.Stream()
    return G.Context(G.desc_from_workload(w, **over), stream=stream), stream


def _oracle_problem(w):
    return O.Problem(dim=w.dim, nx=w.nx, ny=w.ny, k=w.k, basis=w.basis, system=w.system, bc=w.bc, oe=w.oe,
                     rk=w.rk, ax=w.ax, bx=w.bx, ay=w.ay, by=w.by, gamma=w.gamma, adv_x=w.adv[0], adv_y=w.adv[1],
                     cfl=w.cfl)


def rel_l1(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).sum(axis=(0, 2, 3, 4)) / np.maximum(np.abs(b).sum(axis=(0, 2, 3, 4)), 1e-300)


def test_advection_1d_full_run():
    w = W.advection_1d(128)
    ctx, st = _bench_ctx(w)
    p = _oracle_problem(w)
    with torch.cuda.stream(st):
        ug = ctx.project(w.u0)
        ctx.cdg_step(ug, 0.0, w.T, 1300)
    t = ctx.cdg_get_time()
    ref, to, steps, status = O.advance(p, O.project_fn(p, w.u0), 0.0, w.T)
    assert status == O.OK and steps == 1280 and to == w.T
    assert abs(t - w.T) < 1e-13
    assert rel_l1(ug.cpu().numpy(), ref).max() < 1e-11


def test_shu_osher_1d_full_size():
    w = W.shu_osher_1d(4000)
    ctx, st = _bench_ctx(w)
    p = _oracle_problem(w)
    with torch.cuda.stream(st):
        ug = ctx.project(w.u0)
        u = ug.clone()
        ctx.cdg_step(ug, 0.0, w.T, 100)
    ref, _, steps, status = O.advance(p, O.project_fn(p, w.u0), 0.0, w.T, 100)
    assert status == O.OK and steps == 100
    assert rel_l1(ug.cpu().numpy(), ref).max() < 1e-9
    # the whole run: every call's status, the exact end time, physical averages
    with torch.cuda.stream(st):
        t = 0.0
        while t < w.T:
            ctx.cdg_step(u, t, w.T, 4096)
            t = ctx.cdg_get_time()
    assert abs(t - w.T) < 1e-13
    a = u[:, :, 0, 0].cpu().numpy()  # [mesh, field, cell] averages
    rho, m, E = a[:, 0], a[:, 1], a[:, 2]
    p_ = 0.4 * (E - 0.5 * m * m / rho)
    assert rho.min() > 0.5 and rho.max() < 5.0 and p_.min() > 0.5


# ------------------------------------------------------------ 2D 1024^2 ----

N2 = 1024


def _synthetic_full_state(w, seed):
    """Seeded synthetic 2D Euler Q^2 state on both meshes: the four quadrant
    states as cell averages (sampled at the cell centres) plus a seeded
    perturbation of every modal coefficient."""
    n = w.nx
    h = 1.0 / n
    out = np.zeros(w.state_shape)
    for mesh in range(2):
        c = (np.arange(n) + 0.5 + 0.5 * mesh) * h
        X, Y = np.meshgrid(c, c)
        vals = w.u0(np.stack([X.ravel(), Y.ravel()], axis=1)).reshape(n, n, 4)
        out[mesh, :, 0] = np.moveaxis(vals, -1, 0)
    pert = W.perturbation(out.shape, seed, 1e-3)
    pert[:, :, 0] *= 0.5
    return out + pert


def _sample_cells(n, seed, count=1500):
    """Seeded random cells, boundary rows and columns, cells beside the
    discontinuity lines x, y = 0.8 and on 32 x 4 tile edges."""
    rng = np.random.default_rng(seed)
    cells = set()
    for _ in range(count):
        cells.add((int(rng.integers(2)), int(rng.integers(n)), int(rng.integers(n))))
    for mesh in range(2):
        for q in range(0, n, 37):
            for c in ((0, q), (n - 1, q), (q, 0), (q, n - 1)):
                cells.add((mesh, c[0], c[1]))
        for q in range(0, n, 53):
            for d in (-2, -1, 0, 1):
                cells.add((mesh, int(0.8 * n) + d, q))
                cells.add((mesh, q, int(0.8 * n) + d))
            cells.update({(mesh, 31, q), (mesh, 32, q), (mesh, q, 3), (mesh, q, 4)})
    return np.array(sorted(cells), dtype=np.int32)


def _gather(u, cells):
    """u [2, F, M, ny, nx] at (mesh, i, j) rows -> [n, F, M]."""
    return u[cells[:, 0], :, :, cells[:, 2], cells[:, 1]]


@pytest.fixture(scope="module")
def full2d():
    w = W.riemann_2d(n=N2)
    ctx, st = _bench_ctx(w)
    return w, ctx, st, _oracle_problem(w), _synthetic_full_state(w, 17), _sample_cells(N2, 5)


def test_full_size_rhs_sampled(full2d):
    w, ctx, st, p, u, cells = full2d
    tm = 2.3e-5
    with torch.cuda.stream(st):
        ug = torch.from_numpy(u).cuda()
        Lg = torch.empty_like(ug)
        ctx.cdg_rhs(ug, tm, Lg)
    st.synchronize()
    got = _gather(Lg.cpu().numpy(), cells)
    ref = O.rhs_cells(p, u, tm, cells)
    err = np.abs(got - ref).sum(axis=(0, 2)) / np.abs(ref).sum(axis=(0, 2))
    assert err.max() < 1e-12, err


def test_full_size_oe_sampled(full2d):
    w, ctx, st, p, u, cells = full2d
    tau, tm = 2.0e-5, 2.3e-5
    with torch.cuda.stream(st):
        ug = torch.from_numpy(u).cuda()
        dg = torch.zeros((2, N2, N2, 3), dtype=torch.float64, device="cuda")
        sg = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
        ctx.cdg_oe_coefficients(ug, dg, sg)
        ctx.cdg_set_dt(tau, tm)
        out = torch.empty_like(ug)
        ctx.cdg_oe_damp(ug, out)
    st.synchronize()
    d, s, a, usig, status = O.oe_cells(p, u, tau, cells)
    assert status == O.OK
    # sigma and avg reduce 2^20 cell values per mesh in different orders
    np.testing.assert_allclose(sg.cpu().numpy(), s, rtol=1e-10)
    dgot = dg.cpu().numpy()[cells[:, 0], cells[:, 2], cells[:, 1]]
    for m in range(3):
        assert np.abs(dgot[:, m] - d[:, m]).max() <= 1e-10 * np.abs(d[:, m]).max(), m
    got = _gather(out.cpu().numpy(), cells)
    err = np.abs(got - usig).sum(axis=(0, 2)) / np.abs(usig).sum(axis=(0, 2))
    assert err.max() < 1e-12, err


def test_full_size_dt(full2d):
    w, ctx, st, p, u, cells = full2d
    with torch.cuda.stream(st):
        ug = torch.from_numpy(u).cuda()
        ctx.cdg_compute_dt(ug, 0.0, 0.0)
    tau, tm = ctx.cdg_get_dt()
    ref, status = O.tau_max(p, u)
    assert status == O.OK
    assert abs(tm - ref) <= 1e-14 * ref and tau == tm


def test_full_size_run_properties():
    """The measured run itself: projected four-quadrant data, 200 steps."""
    w = W.riemann_2d(n=N2)
    ctx, st = _bench_ctx(w)
    with torch.cuda.stream(st):
        u = ctx.project(w.u0)
        ctx.cdg_step(u, 0.0, 0.0, 200)
    t = ctx.cdg_get_time()
    assert 0.0 < t < 0.01
    a = u.cpu().numpy()
    # x <-> y: cell (i, j) <-> (j, i), mode (a, b) <-> (b, a), rho u <-> rho v
    tr = a.reshape(2, 4, 3, 3, N2, N2).transpose(0, 1, 3, 2, 5, 4).reshape(a.shape)[:, [0, 2, 1, 3]]
    err = rel_l1(tr, a)
    assert err.max() < 1e-9, err
    avg = a[:, :, 0]
    rho = avg[:, 0]
    p_ = 0.4 * (avg[:, 3] - 0.5 * (avg[:, 1] ** 2 + avg[:, 2] ** 2) / rho)
    assert rho.min() > 0.0 and p_.min() > 0.0


# -------------------------------------------------------------- batched ----

def test_batched_full_size():
    """The 256 meshes of the batched workload (seed 0 sizes 64^2..512^2) on
    seeded synthetic states: a constant physical state plus a 1e-3 Gaussian
    perturbation of every coefficient, drawn by a seeded device generator."""
    from paper_2503_12473_gb300 import oecdg as G
    wls = W.batch_workloads(seed=0, count=256, steps=2)
    descs = [G.desc_from_workload(w) for w in wls]
    gen = torch.Generator(device="cuda").manual_seed(0)
    base = torch.tensor([1.0, 0.2, -0.1, 2.5], dtype=torch.float64, device="cuda")
    us = []
    for w in wls:
        u = 1e-3 * torch.randn(w.state_shape, generator=gen, dtype=torch.float64, device="cuda")
        u[:, :, 0] += base[None, :, None, None]
        us.append(u)
    u0 = [u.clone() for u in us]
    b = G.Batch(descs)
    b.cdg_batch_step(us, 2, use_graph=True)
    assert b.cdg_batch_check_status() == G.CDG_OK
    same_tiles = b.cdg_batch_rows() == 4  # the single-mesh kernels use 4-row tiles
    rng = np.random.default_rng(1)
    for q in sorted(set(int(x) for x in rng.choice(len(wls), 8, replace=False))):
        v = u0[q].clone()
        G.Context(descs[q]).cdg_step(v, 0.0, 0.0, 2)
        if same_tiles:
            assert torch.equal(v, us[q]), q
        else:
            assert ((v - us[q]).abs().sum() / v.abs().sum()).item() < 1e-13, q
    small = min(range(len(wls)), key=lambda q: wls[q].nx * wls[q].ny)
    p = _oracle_problem(wls[small])
    ref, _, _, status = O.advance(p, u0[small].cpu().numpy(), 0.0, 0.0, 2)
    assert status == O.OK
    assert rel_l1(us[small].cpu().numpy(), ref).max() < 1e-9


# -------------------------------------------------------------- adjoint ----

def test_adjoint_full_size_vs_fd():
    from paper_2503_12473_gb300 import oecdg as G
    from paper_2503_12473_gb300.autograd import rollout
    w = W.vortex_2d(n=256)
    ctx = G.Context(G.desc_from_workload(w))
    base = ctx.project(w.u0)
    nsteps = 400
    target = base.clone()
    ctx.cdg_step(target, 0.0, 0.0, nsteps)
    rho_t = target[:, 0].clone()
    u = base + torch.from_numpy(W.perturbation(tuple(base.shape), 3, 1e-3)).cuda()
    u0 = u.clone().requires_grad_(True)
    uT = rollout(u0, ctx, nsteps)
    (0.5 * ((uT[:, 0] - rho_t) ** 2).sum()).backward()
    grad = u0.grad.detach()

    def L(x):
        y = x.clone()
        ctx.cdg_step(y, 0.0, 0.0, nsteps)
        return 0.5 * ((y[:, 0] - rho_t) ** 2).sum().item()

    gen = torch.Generator(device="cpu").manual_seed(64)
    for _ in range(2):
        d = torch.randn(tuple(u.shape), generator=gen, dtype=torch.float64).cuda()
        eps = 1e-8
        fd = (L(u + eps * d) - L(u - eps * d)) / (2 * eps)
        an = (grad * d).sum().item()
        assert abs(an - fd) <= 2e-5 * abs(fd), (an, fd)


def test_conservation_full_size_periodic():
    """Conservation (Section 3.3): with periodic boundaries the total of every
    conserved variable over both meshes, sum_K |K| u_K,00, is constant up to
    round-off; the 256^2 vortex workload over 100 steps, in bench.py's launch
    configuration."""
    w = W.vortex_2d(n=256)
    ctx, st = _bench_ctx(w)
    with torch.cuda.stream(st):
        u = ctx.project(w.u0)
        tot0 = u[:, :, 0].sum(dim=(0, 2, 3)).cpu().numpy()
        scale = u[:, :, 0].abs().sum(dim=(0, 2, 3)).cpu().numpy()
        ctx.cdg_step(u, 0.0, 0.0, 100)
        tot1 = u[:, :, 0].sum(dim=(0, 2, 3)).cpu().numpy()
    assert np.all(np.abs(tot1 - tot0) <= 1e-12 * scale), (tot0, tot1)
