"""The batched path (many independent 2D Euler Q^2 meshes of uneven sizes,
one launch per phase over all of them): identical to per-instance launches of
the single-mesh kernels, identical under CUDA-graph capture, and in parity
with the oracle."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_12473_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [(8, 8), (20, 36), (40, 12), (33, 17), (64, 64), (24, 50)]


@pytest.fixture(scope="module")
def batch_setup():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2503_12473_gb300 import oecdg as G
    insts = W.batched_instances(seed=7, count=len(SIZES))
    descs, ics = [], []
    for (nx, ny), inst in zip(SIZES, insts):
        descs.append(G.MeshDesc(dim=2, nx=nx, ny=ny, system=G.EULER, bc=G.PERIODIC, cfl=0.1))
        ics.append(W.batched_ic(inst))
    return G, descs, ics


def _initial(G, descs, ics):
    out = []
    for d, f in zip(descs, ics):
        ctx = G.Context(d)
        out.append(ctx.project(f))
    return out


def test_batched_equals_per_instance(batch_setup):
    G, descs, ics = batch_setup
    u0 = _initial(G, descs, ics)
    ref = [u.clone() for u in u0]
    for d, u in zip(descs, ref):
        G.Context(d).cdg_step(u, 0.0, 0.0, 3)
    b = G.Batch(descs)
    assert b.cdg_batch_rows() == 4
    us = [u.clone() for u in u0]
    b.cdg_batch_step(us, 3)
    assert b.cdg_batch_check_status() == G.CDG_OK
    for u, r in zip(us, ref):
        assert torch.equal(u, r)
    # 11 launches per step whatever the number of instances
    assert b.cdg_batch_launch_count() == 33


def test_batched_graph_equals_direct(batch_setup):
    G, descs, ics = batch_setup
    u0 = _initial(G, descs, ics)
    b1 = G.Batch(descs)
    a = [u.clone() for u in u0]
    b1.cdg_batch_step(a, 4, use_graph=False)
    assert b1.cdg_batch_check_status() == G.CDG_OK
    stream = torch.cuda.Stream()
    b2 = G.Batch(descs, stream=stream)
    c = [u.clone() for u in u0]
    b2.cdg_batch_step(c, 2, use_graph=True)
    b2.cdg_batch_step(c, 2, use_graph=True)   # replays the captured graph
    stream.synchronize()
    torch.cuda.synchronize()
    for x, y in zip(a, c):
        assert torch.equal(x, y)
    np.testing.assert_allclose(b1.cdg_batch_get_time(), b2.cdg_batch_get_time(), rtol=0, atol=0)


@pytest.mark.parametrize("rows", [2, 8])
def test_tile_heights(batch_setup, rows):
    """Other tile heights sum the sigma partials in another order: one step
    agrees to round-off.  (Over several steps the 8 x 8 instance, far too
    coarse for its data, amplifies that round-off; equal tile heights stay
    bitwise equal, see test_batched_equals_per_instance.)"""
    G, descs, ics = batch_setup
    u0 = _initial(G, descs, ics)
    ref = [u.clone() for u in u0]
    G.Batch(descs).cdg_batch_step(ref, 1)
    b = G.Batch(descs)
    b.cdg_batch_set_rows(rows)
    us = [u.clone() for u in u0]
    b.cdg_batch_step(us, 1)
    assert b.cdg_batch_check_status() == G.CDG_OK  # synchronises the batch's stream
    for q, (u, r) in enumerate(zip(us, ref)):
        err = ((u - r).abs().sum() / r.abs().sum()).item()
        assert err <= 1e-13, (rows, q, descs[q].nx, descs[q].ny, err)


def test_tile_heights_and_autotune(batch_setup, tmp_path):
    G, descs, ics = batch_setup
    u0 = _initial(G, descs, ics)
    ref = [u.clone() for u in u0]
    G.Batch(descs).cdg_batch_step(ref, 1)
    cache = str(tmp_path / "tune.json")
    b = G.Batch(descs)
    rows = b.cdg_batch_autotune(u0, cache)
    assert rows in (2, 4, 8)
    bps, grid = b.cdg_batch_grid()
    assert bps >= 1 and grid >= 1
    data = json.load(open(cache))
    assert list(data.values()) == [rows * 100 + bps]  # tile height and persistent grid
    b2 = G.Batch(descs)
    assert b2.cdg_batch_autotune(u0, cache) == rows  # from the cache
    assert b2.cdg_batch_grid() == (bps, grid)
    for u, v in zip(u0, _initial(G, descs, ics)):  # the tuner only read the states
        assert torch.equal(u, v)
    us = [u.clone() for u in u0]
    b.cdg_batch_step(us, 1, persistent=True)
    assert b.cdg_batch_check_status() == G.CDG_OK  # synchronises the batch's stream
    for u, r in zip(us, ref):
        # other tile heights sum the sigma partials in another order
        err = ((u - r).abs().sum() / r.abs().sum()).item()
        assert err <= 1e-13


def test_batched_oracle_parity(batch_setup):
    G, descs, ics = batch_setup
    sel = [0, 3]
    d = [descs[q] for q in sel]
    f = [ics[q] for q in sel]
    us = _initial(G, d, f)
    b = G.Batch(d)
    b.cdg_batch_step(us, 3)
    assert b.cdg_batch_check_status() == G.CDG_OK  # synchronises the batch's stream
    for dq, fq, u in zip(d, f, us):
        p = O.Problem(dim=2, nx=dq.nx, ny=dq.ny, k=2, system=O.EULER, bc=O.PERIODIC, cfl=dq.cfl)
        ref, t, n, st = O.advance(p, O.project_fn(p, fq), 0.0, 0.0, 3)
        got = u.cpu().numpy()
        err = np.abs(got - ref).sum(axis=(0, 2, 3, 4)) / np.abs(ref).sum(axis=(0, 2, 3, 4))
        assert err.max() < 1e-9, err


@pytest.mark.parametrize("rows", [2, 4, 8])
def test_persistent_equals_per_phase_launches(batch_setup, rows):
    """One cooperative launch for all steps (grid-wide barriers between the
    phases) gives the per-phase launches' results bit for bit, directly and
    captured in a CUDA graph, for every tile height and for a persistent grid
    smaller than the tile count (blocks loop over several tiles)."""
    G, descs, ics = batch_setup
    u0 = _initial(G, descs, ics)
    b = G.Batch(descs)
    b.cdg_batch_set_rows(rows)
    ref = [u.clone() for u in u0]
    b.cdg_batch_step(ref, 3)
    assert b.cdg_batch_check_status() == G.CDG_OK
    t_ref = b.cdg_batch_get_time()
    for graph, bps in ((False, 0), (True, 0), (False, 1)):
        bp = G.Batch(descs, stream=torch.cuda.Stream())
        bp.cdg_batch_set_rows(rows)
        bp.cdg_batch_set_grid(bps)
        us = [u.clone() for u in u0]
        bp.cdg_batch_step(us, 3, use_graph=graph, persistent=True)
        assert bp.cdg_batch_check_status() == G.CDG_OK
        for u, r in zip(us, ref):
            assert torch.equal(u, r), (rows, graph, bps)
        np.testing.assert_array_equal(bp.cdg_batch_get_time(), t_ref)
        assert bp.cdg_batch_launch_count() == 1


def test_persistent_barrier_wait_runs_out_without_hanging(batch_setup):
    """The grid barriers' waits are bounded.  With the test hook that makes
    every barrier wait for one arrival that never comes, the launch ends by
    itself after about the limit and reports CDG_ETIMEOUT; nothing faults, and
    the same batch then steps normally again (from a restored state)."""
    import time
    G, descs, ics = batch_setup
    u0 = _initial(G, descs, ics)
    ref = [u.clone() for u in u0]
    G.Batch(descs).cdg_batch_step(ref, 2)
    torch.cuda.synchronize()
    b = G.Batch(descs)
    b.cdg_batch_set_wait(0.2, withheld=1)
    us = [u.clone() for u in u0]
    t0 = time.time()
    b.cdg_batch_step(us, 2, persistent=True)
    assert b.cdg_batch_check_status() == G.CDG_ETIMEOUT
    assert time.time() - t0 < 10.0
    b.cdg_batch_set_wait(5.0, withheld=0)
    us = [u.clone() for u in u0]
    b.cdg_batch_step(us, 2, persistent=True)
    assert b.cdg_batch_check_status() == G.CDG_OK
    for u, r in zip(us, ref):
        assert torch.equal(u, r)
