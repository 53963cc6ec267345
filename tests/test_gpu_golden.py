"""Parity over the stated step counts of the discontinuous workloads, against
end states the CPU oracle wrote offline (tests/golden/make_goldens.py runs
only oracle/; whole-mesh oracle steps are far too slow to run inside a test).

* 2D Euler four-quadrant Riemann data, Q^2, transmissive, 130 x 130 cells
  (ragged in both directions of the 32 x 4 cell tiles), 200 SSP-RK3 + OE steps.
* 1D Euler Shu-Osher data, P^2, 4000 cells, to T = 1.8 (34,627 steps), as
  bench.py runs it: one CUDA graph per step.
* The 8 smallest instances of the seed-0 batch (periodic 2D Euler Q^2, 64^2,
  their own data), 100 steps through the batched path.
* A 20-step checkpointed rollout's gradient (5 checkpoints) on a 16^2 vortex:
  <v_i, J^T lam> from the CUDA adjoint against <lam, J v_i> from the
  complex-step oracle, 16 seeded directions.

Each run starts from the oracle's own projection of the same point values
(the CUDA projection is checked in test_gpu_parity.py).  Tolerance (the
GPU <-> oracle bar for discontinuous runs): relative L1 per field over all
modal coefficients of both meshes <= 1e-9; the max element error is reported
beside it.  Stored values carry at most 7.3e-12 relative rounding
(tests/golden/golden_io.py), far below the bar.
"""
import os
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_12473_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import golden_io  # noqa: E402
import make_goldens as MG  # noqa: E402

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2503_12473_gb300 import oecdg
    oecdg.load()


def _golden(name):
    path = os.path.join(HERE, "golden", name)
    assert os.path.exists(path), f"missing golden {name}: run tests/golden/make_goldens.py"
    return golden_io.load(path)


def _compare(got, ref, what):
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape
    assert np.isfinite(got).all(), what
    num = np.abs(got - ref).sum(axis=(0, 2, 3, 4))
    den = np.abs(ref).sum(axis=(0, 2, 3, 4))
    rel = num / den
    maxel = np.abs(got - ref).max(axis=(0, 2, 3, 4)) / np.abs(ref).max(axis=(0, 2, 3, 4))
    print(f"{what}: rel L1 per field {np.array2string(rel, precision=2)}, "
          f"max element error / max |u| per field {np.array2string(maxel, precision=2)}")
    assert rel.max() <= TOL, (what, rel, maxel)
    return rel, maxel


def _ctx(w):
    """A context as bench.py makes it: bound to its own stream."""
    from paper_2503_12473_gb300 import oecdg as G
    stream = torch.cuda.Stream()
    return G.Context(G.desc_from_workload(w), stream=stream), stream


def test_riemann_2d_200_steps_against_oracle():
    w = MG.riemann_workload()
    arrays, meta = _golden(f"riemann_q2_{MG.RIEMANN_N}_{MG.RIEMANN_STEPS}steps.npz")
    assert meta["steps"] == MG.RIEMANN_STEPS and (meta["nx"], meta["ny"]) == (w.nx, w.ny)
    p = MG.oracle_problem(w)
    u0 = O.project_fn(p, w.u0)
    ctx, st = _ctx(w)
    with torch.cuda.stream(st):
        u = torch.from_numpy(u0).to("cuda", non_blocking=False)
        ctx.cdg_step(u, 0.0, 0.0, MG.RIEMANN_STEPS)
    st.synchronize()
    t = ctx.cdg_get_time()
    assert abs(t - meta["t_final"]) <= 1e-12 * meta["t_final"], (t, meta["t_final"])
    _compare(u.cpu().numpy(), arrays["u"], "riemann 130^2, 200 steps")


def test_shu_osher_to_final_time_against_oracle():
    w = MG.shu_workload()
    arrays, meta = _golden("shu_osher_p2_4000_T1.8.npz")
    assert meta["t_final"] == w.T
    p = MG.oracle_problem(w)
    u0 = O.project_fn(p, w.u0)
    ctx, st = _ctx(w)
    with torch.cuda.stream(st):
        u = torch.from_numpy(u0).to("cuda")
        # the graph path bench.py times; steps past T_end are skipped on the device
        ctx.cdg_step_graph(u, 0.0, w.T, meta["steps"] + 20)
    st.synchronize()
    assert ctx.cdg_check_status() == 0
    assert ctx.cdg_get_time() == w.T
    _compare(u.cpu().numpy(), arrays["u"], f"shu-osher 4000 cells, {meta['steps']} steps to T = 1.8")


def test_batched_smallest_instances_against_oracle():
    from paper_2503_12473_gb300 import oecdg as G
    idx, ws = MG.smallest_batch_indices()
    descs, states, refs = [], [], []
    for q in idx:
        w = ws[q]
        arrays, meta = _golden(f"batched_seed0_{q}_{w.nx}_{MG.BATCH_STEPS}steps.npz")
        assert meta["steps"] == MG.BATCH_STEPS
        p = MG.oracle_problem(w)
        descs.append(G.desc_from_workload(w))
        states.append(torch.from_numpy(O.project_fn(p, w.u0)).cuda())
        refs.append(arrays["u"])
    b = G.Batch(descs)
    b.cdg_batch_step(states, MG.BATCH_STEPS, use_graph=True)
    assert b.cdg_batch_check_status() == G.CDG_OK
    for q, u, r in zip(idx, states, refs):
        _compare(u.cpu().numpy(), r, f"batched instance {q} ({u.shape[-1]}^2), {MG.BATCH_STEPS} steps")


def test_checkpointed_rollout_gradient_against_complex_step_oracle():
    from paper_2503_12473_gb300 import oecdg as G
    from paper_2503_12473_gb300.autograd import rollout
    arrays, meta = _golden(f"adjoint_vortex_{MG.ADJ_N}_{MG.ADJ_STEPS}steps.npz")
    w, _, _, lam, dirs = MG.adjoint_case()
    u0 = arrays["u0"]  # the state the oracle differentiated, bit for bit
    ctx = G.Context(G.desc_from_workload(w))
    x = torch.from_numpy(u0).cuda().requires_grad_(True)
    nseg = 5
    uT = rollout(x, ctx, MG.ADJ_STEPS, segment=MG.ADJ_STEPS // nseg)
    (uT * torch.from_numpy(lam).cuda()).sum().backward()
    g = x.grad.cpu().numpy()
    rel = []
    for v, ref in zip(dirs, arrays["lam_dot_jv"]):
        got = float((g * v).sum())
        rel.append(abs(got - ref) / abs(ref))
    rel = np.asarray(rel)
    print(f"rollout adjoint, {len(rel)} directions: max rel {rel.max():.2e}, median {np.median(rel):.2e}")
    assert rel.max() <= 1e-10, rel
