"""The hand-written adjoint of one OECDG step (cdg_step_adjoint) and the
checkpointed multi-step gradient.

The OE step is not smooth: the damping coefficients take |u^C - u^D|, square
roots of sums of squares, a max over the fields and a global max / min (sigma),
and the time step a max over cells.  A finite difference whose step straddles
one of those kinks does not measure the derivative (its forward and backward
one-sided differences split apart).  The OE checks therefore use states with a
5% offset between the meshes' averages (fewer sign changes of u^C - u^D) and a
smaller step; without the OE step the scheme is smooth and any state is used."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_12473_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _setup(n=20, oe=1, offset=0.05):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2503_12473_gb300 import oecdg as G
    w = W.vortex_2d(n=n)
    desc = G.desc_from_workload(w, cfl=0.2, oe=oe)
    ctx = G.Context(desc)
    u = ctx.project(w.u0)
    u = u + torch.from_numpy(W.perturbation(tuple(u.shape), 5, 1e-3)).cuda()
    u[1, :, 0] *= 1.0 + offset
    return G, w, desc, ctx, u


def _step(ctx, u, n=1):
    v = u.clone()
    ctx.cdg_step(v, 0.0, 0.0, n)
    return v


@pytest.mark.parametrize("oe,offset", [(1, 0.05), (0, 0.0)])
def test_step_adjoint_dot_product_vs_gpu_fd(oe, offset):
    G, w, desc, ctx, u = _setup(oe=oe, offset=offset)
    gen = torch.Generator(device="cpu").manual_seed(11)
    lam = torch.randn(tuple(u.shape), generator=gen, dtype=torch.float64).cuda()
    v = torch.randn(tuple(u.shape), generator=gen, dtype=torch.float64).cuda()
    adj = torch.empty_like(u)
    ctx.cdg_step_adjoint(u, lam, adj)
    torch.cuda.synchronize()
    lhs = (adj * v).sum().item()
    # with OE, steps of 1e-6 and above straddle kinks of the damping
    # coefficients (the forward and backward differences split apart there);
    # at 1e-7 the central difference converges to the adjoint
    eps = 1e-7 if oe else 1e-6
    fd = (_step(ctx, u + eps * v) - _step(ctx, u - eps * v)) / (2 * eps)
    rhs = (lam * fd).sum().item()
    assert abs(lhs - rhs) <= (1e-6 if oe else 1e-7) * abs(rhs), (lhs, rhs)


def test_step_adjoint_vs_oracle_fd():
    """<lam, J_oracle v> by central differences of the oracle's step against
    <J^T lam, v> from the CUDA adjoint (each side projects the data itself)."""
    G, w, desc, ctx, u = _setup(n=12)
    p = O.Problem(dim=2, nx=12, ny=12, k=2, system=O.EULER, bc=O.PERIODIC, bx=10.0, by=10.0, cfl=0.2)
    uo = O.project_fn(p, w.u0) + W.perturbation(tuple(u.shape), 5, 1e-3)
    uo[1, :, 0] *= 1.05
    rng = np.random.default_rng(3)
    lam = rng.standard_normal(uo.shape)
    v = rng.standard_normal(uo.shape)
    adj = torch.empty_like(u)
    ctx.cdg_step_adjoint(u, torch.from_numpy(lam).cuda(), adj)
    torch.cuda.synchronize()
    lhs = float((adj.cpu().numpy() * v).sum())
    eps = 1e-6
    a, *_ = O.advance(p, uo + eps * v, 0.0, 0.0, 1)
    b, *_ = O.advance(p, uo - eps * v, 0.0, 0.0, 1)
    rhs = float((lam * (a - b) / (2 * eps)).sum())
    assert abs(lhs - rhs) <= 1e-7 * abs(rhs), (lhs, rhs)


def _oracle_of(desc):
    return O.Problem(dim=desc.dim, nx=desc.nx, ny=desc.ny, k=desc.k, basis=desc.basis, system=desc.system,
                     bc=desc.bc, oe=desc.oe, rk=desc.rk, ax=desc.ax, bx=desc.bx, ay=desc.ay, by=desc.by,
                     gamma=desc.gamma, adv_x=desc.adv_x, adv_y=desc.adv_y, cfl=desc.cfl)


@pytest.mark.parametrize("system,nx,ny", [(W.ADVECTION, 6, 5), (W.EULER, 4, 3)])
def test_step_adjoint_equals_oracle_adjoint(system, nx, ny):
    """The oracle's own adjoint of one step, J^T lam, with J formed column by
    column by complex-step runs of the oracle (no difference quotient, no
    truncation error), against cdg_step_adjoint, element by element.  Seeded
    state with every modal coefficient perturbed, OE on, tau from the state."""
    from paper_2503_12473_gb300 import oecdg as G
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    w = W.Workload("adjoint_small", 2, nx, ny, 2, system, W.PERIODIC, 0.0, 2.0, 0.0, 2.0, adv=(1.0, 0.6), cfl=0.2)
    desc = G.desc_from_workload(w)
    u = W.random_modal(w.state_shape, 4, 0.05)
    if system == W.EULER:
        u[:, 0, 0] += 1.0
        u[:, 3, 0] += 2.5
    lam = W.random_modal(w.state_shape, 9, 1.0)
    ref, st = O.step_adjoint(_oracle_of(desc), u, lam)
    assert st == O.OK
    ctx = G.Context(desc)
    got = torch.empty(w.state_shape, dtype=torch.float64, device="cuda")
    ctx.cdg_step_adjoint(torch.from_numpy(u).cuda(), torch.from_numpy(lam).cuda(), got)
    torch.cuda.synchronize()
    g = got.cpu().numpy()
    assert np.abs(g - ref).sum() <= 1e-10 * np.abs(ref).sum()
    assert np.abs(g - ref).max() <= 1e-9 * np.abs(ref).max()


def test_step_adjoint_dot_products_vs_oracle_jvp():
    """On a 20 x 20 vortex state: <lam, J v> with J v from the complex-step
    oracle against <J^T lam, v> from the CUDA adjoint, 64 seeded directions, to
    1e-11 (measured: max 1.6e-12, median 7e-15).
    Both sides get the same host-built state (oracle projection + seeded
    perturbation, 5% offset between the meshes)."""
    from paper_2503_12473_gb300 import oecdg as G
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    w = W.vortex_2d(n=20)
    desc = G.desc_from_workload(w, cfl=0.2)
    p = _oracle_of(desc)
    u = O.project_fn(p, w.u0) + W.perturbation(w.state_shape, 5, 1e-3)
    u[1, :, 0] *= 1.05
    rng = np.random.default_rng(12)
    lam = rng.standard_normal(u.shape)
    ctx = G.Context(desc)
    adj = torch.empty(w.state_shape, dtype=torch.float64, device="cuda")
    ctx.cdg_step_adjoint(torch.from_numpy(u).cuda(), torch.from_numpy(lam).cuda(), adj)
    torch.cuda.synchronize()
    a = adj.cpu().numpy()
    for _ in range(64):
        v = rng.standard_normal(u.shape)
        _, jv, st = O.step_jvp(p, u, v)
        assert st == O.OK
        lhs = float((a * v).sum())
        rhs = float((lam * jv).sum())
        assert abs(lhs - rhs) <= 1e-11 * abs(rhs), (lhs, rhs)


def test_adjoint_gtau_matches_fd_of_fixed_tau_step():
    """The returned adjoints of tau and tau_max: compare with central
    differences of one step at a fixed (tau, tau_max) through cdg_set_dt and
    the stage / OE entry points."""
    G, w, desc, ctx, u = _setup()
    gen = torch.Generator(device="cpu").manual_seed(4)
    lam = torch.randn(tuple(u.shape), generator=gen, dtype=torch.float64).cuda()
    adj = torch.empty_like(u)
    gt = torch.zeros(2, dtype=torch.float64, device="cuda")
    ctx.cdg_step_adjoint(u, lam, adj, gt)
    ctx.cdg_compute_dt(u, 0.0, 0.0)
    tau, tm = ctx.cdg_get_dt()

    def step_fixed(t, tmx):
        ctx.cdg_set_dt(t, tmx)
        un = u.clone()
        s = u.clone()
        h = torch.empty_like(u)
        for l in range(3):
            ctx.cdg_rk_stage(l, un, s, h)
            ctx.cdg_oe_damp(h, s)
        return s

    e = 1e-6 * tau
    d_tau = ((lam * (step_fixed(tau + e, tm) - step_fixed(tau - e, tm))).sum() / (2 * e)).item()
    d_tm = ((lam * (step_fixed(tau, tm + e) - step_fixed(tau, tm - e))).sum() / (2 * e)).item()
    got = gt.tolist()
    assert abs(got[0] - d_tau) <= 1e-6 * abs(d_tau), (got, d_tau)
    assert abs(got[1] - d_tm) <= 1e-6 * abs(d_tm), (got, d_tm)


def test_checkpointed_rollout_equals_stepwise_chain():
    """sqrt(n) checkpointing recomputes the same states: the rollout's gradient
    equals the chain of cdg_step_adjoint over all stored states."""
    from paper_2503_12473_gb300.autograd import rollout
    G, w, desc, ctx, u = _setup(n=16)
    nsteps = 10
    gen = torch.Generator(device="cpu").manual_seed(21)
    lam = torch.randn(tuple(u.shape), generator=gen, dtype=torch.float64).cuda()
    u0 = u.clone().requires_grad_(True)
    uT = rollout(u0, ctx, nsteps)
    (uT * lam).sum().backward()
    states = [u.clone()]
    for _ in range(nsteps - 1):
        states.append(_step(ctx, states[-1]))
    g = lam.clone()
    nxt = torch.empty_like(g)
    for s in reversed(states):
        ctx.cdg_step_adjoint(s, g, nxt)
        g, nxt = nxt, g
    assert torch.equal(u0.grad, g)
    assert torch.equal(uT.detach(), _step(ctx, u, nsteps))


def test_rollout_gradient_vs_fd_without_oe():
    """Gradient of 0.5 ||rho(T) - rho_target||^2 (rho modal coefficients of both
    meshes) through 9 steps with checkpoints, against central differences in
    seeded directions (the scheme without the OE step is smooth)."""
    from paper_2503_12473_gb300.autograd import rollout
    G, w, desc, ctx, u = _setup(n=16, oe=0, offset=0.0)
    nsteps = 9
    target = _step(ctx, u, nsteps)[:, 0] + 0.01
    u0 = u.clone().requires_grad_(True)
    uT = rollout(u0, ctx, nsteps)
    loss = 0.5 * ((uT[:, 0] - target) ** 2).sum()
    loss.backward()
    grad = u0.grad.detach()

    def L(x):
        y = _step(ctx, x, nsteps)
        return 0.5 * ((y[:, 0] - target) ** 2).sum().item()

    gen = torch.Generator(device="cpu").manual_seed(21)
    for _ in range(4):
        d = torch.randn(tuple(u.shape), generator=gen, dtype=torch.float64).cuda()
        eps = 1e-6
        fd = (L(u + eps * d) - L(u - eps * d)) / (2 * eps)
        an = (grad * d).sum().item()
        assert abs(an - fd) <= 1e-6 * abs(fd), (an, fd)


def test_rollout_gradient_vs_fd_with_oe():
    """With the OE step, over several steps the |u^C - u^D| kinks are met by
    any finite difference; at h = 1e-8 the directional derivatives still agree
    to 1e-4."""
    from paper_2503_12473_gb300.autograd import rollout
    G, w, desc, ctx, u = _setup(n=16)
    nsteps = 6
    target = _step(ctx, u, nsteps)[:, 0] + 0.01
    u0 = u.clone().requires_grad_(True)
    uT = rollout(u0, ctx, nsteps)
    (0.5 * ((uT[:, 0] - target) ** 2).sum()).backward()
    grad = u0.grad.detach()

    def L(x):
        y = _step(ctx, x, nsteps)
        return 0.5 * ((y[:, 0] - target) ** 2).sum().item()

    gen = torch.Generator(device="cpu").manual_seed(8)
    for _ in range(3):
        d = torch.randn(tuple(u.shape), generator=gen, dtype=torch.float64).cuda()
        eps = 1e-8
        fd = (L(u + eps * d) - L(u - eps * d)) / (2 * eps)
        an = (grad * d).sum().item()
        assert abs(an - fd) <= 1e-4 * abs(fd), (an, fd)
