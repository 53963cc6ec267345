"""cdg_oe_damp_noalloc, the OE step for callers that cannot allocate device
memory (for example code inside a host application whose memory manager owns
the device heap, or a latency-critical path that must not allocate while it
runs): it takes no context and keeps its scratch in a fixed array inside the
library.  Checked against the context-based cdg_oe_damp through the C-ABI, on
two calls in a row (the second call reuses the array the first one left
behind).  This file is collected last so that a run stopping at the first
failure has run every other test before it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel_l1(a, b):
    num = (a - b).abs().sum(dim=(0, 2, 3, 4))
    den = b.abs().sum(dim=(0, 2, 3, 4))
    return (num / den).max().item()


@pytest.mark.parametrize("which", ["riemann_2d", "shu_osher_1d"])
def test_noalloc_oe_matches_context_oe(which):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2503_12473_gb300 import oecdg as G
    from paper_2503_12473_gb300 import workloads as W
    w = W.riemann_2d(n=72).resized(72, 44) if which == "riemann_2d" else W.shu_osher_1d(700)
    desc = G.desc_from_workload(w)
    ctx = G.Context(desc)
    u = ctx.project(w.u0)
    states = [u, u + torch.from_numpy(W.perturbation(tuple(u.shape), 3, 1e-3)).cuda()]
    for q, uh in enumerate(states):  # two calls in a row
        tau = 1e-3 * (q + 1)
        ctx.cdg_set_dt(tau, tau)
        ref = torch.empty_like(uh)
        ctx.cdg_oe_damp(uh, ref)
        got = torch.full_like(uh, float("nan"))
        G.cdg_oe_damp_noalloc(desc, uh, tau, got)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        # the two paths sum the global average in different orders: 1e-12
        assert _rel_l1(got, ref) < 1e-12
        assert torch.equal(got[:, :, 0], uh[:, :, 0])  # averages untouched


def test_noalloc_rejects_meshes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2503_12473_gb300 import oecdg as G
    desc = G.MeshDesc(dim=2, nx=1200, ny=1200)
    u = torch.zeros(desc.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(G.CdgError) as e:
        G.cdg_oe_damp_noalloc(desc, u, 1e-3, torch.empty_like(u))
    assert e.value.status == G.CDG_EINVAL


@pytest.mark.parametrize("which", ["euler_2d_512x2729", "advection_1d_5589504"])
def test_noalloc_accepts_the_largest_mesh_its_scratch_holds(which):
    """The largest meshes within the documented limit (2D Euler: 1,397,248 cells
    per mesh; 1D advection: 5,589,504) run and match cdg_oe_damp; one block of
    256 cells more is refused (checked on the host in test_abi.py)."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2503_12473_gb300 import oecdg as G
    from paper_2503_12473_gb300 import workloads as W
    if which.startswith("euler"):
        desc = G.MeshDesc(dim=2, nx=512, ny=2729, system=G.EULER, bc=G.PERIODIC)
        # physical state: a smooth density wave plus a seeded perturbation
        u = torch.zeros(desc.shape, dtype=torch.float64, device="cuda")
        x = torch.linspace(0.0, 6.283185307179586, desc.nx, dtype=torch.float64, device="cuda")
        u[:, 0, 0] = 1.0 + 0.2 * torch.sin(x)
        u[:, 3, 0] = 2.5
        u[:, :, 1:] = torch.from_numpy(W.perturbation((2, 4, 8, desc.ny, desc.nx), 5, 1e-3)).cuda()
    else:
        desc = G.MeshDesc(dim=1, nx=5589504, ny=1, system=G.ADVECTION, bc=G.PERIODIC, adv_x=1.0)
        u = torch.from_numpy(W.random_modal(desc.shape, 6)).cuda()
    assert desc.nx * desc.ny in (1397248, 5589504)
    ctx = G.Context(desc)
    tau = 2e-3
    ctx.cdg_set_dt(tau, tau)
    ref = torch.empty_like(u)
    ctx.cdg_oe_damp(u, ref)
    got = torch.full_like(u, float("nan"))
    G.cdg_oe_damp_noalloc(desc, u, tau, got)
    torch.cuda.synchronize()
    assert torch.isfinite(got).all()
    assert _rel_l1(got, ref) < 1e-12
    assert torch.equal(got[:, :, 0], u[:, :, 0])
