"""The stored oracle end states (tests/golden/*.npz) on the CPU: the storage
round trip keeps every value within its stated bound, and every golden file
decodes to a finite state of its workload's shape with the metadata the GPU
tests rely on (step counts, end time, mesh)."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import golden_io  # noqa: E402
import make_goldens as MG  # noqa: E402

from paper_2503_12473_gb300 import workloads as W  # noqa: E402


@pytest.mark.parametrize("keep", [8, 7, 6, 5])
def test_round_trip_within_the_stated_bound(tmp_path, keep):
    """keep bytes of each double survive: exact for 8, else within
    2^-(8 keep - 11) relative (round to nearest at the kept boundary), and the
    sign, zeros and the shape are kept."""
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, 3, 5, 7)) * np.exp(rng.uniform(-30, 30, (2, 3, 5, 7)))
    a[0, 0, 0, :3] = [0.0, -0.0, 1.0]
    path = str(tmp_path / "g.npz")
    golden_io.save(path, {"u": a}, {"note": "test"}, keep=keep)
    arrays, meta = golden_io.load(path)
    b = arrays["u"]
    assert b.shape == a.shape and meta["keep"] == keep and meta["note"] == "test"
    if keep == 8:
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    else:
        rel = np.abs(b - a) / np.abs(a).clip(1e-300)
        assert rel.max() <= 2.0 ** -(8 * keep - 11)
        assert np.array_equal(np.signbit(a), np.signbit(b))


def _state_shape(w):
    return tuple(w.state_shape)


def test_long_run_goldens_decode_to_their_workloads():
    cases = [(f"riemann_q2_{MG.RIEMANN_N}_{MG.RIEMANN_STEPS}steps.npz", MG.riemann_workload(), MG.RIEMANN_STEPS),
             ("shu_osher_p2_4000_T1.8.npz", MG.shu_workload(), None)]
    idx, ws = MG.smallest_batch_indices()
    for q in idx:
        cases.append((f"batched_seed0_{q}_{ws[q].nx}_{MG.BATCH_STEPS}steps.npz", ws[q], MG.BATCH_STEPS))
    for name, w, steps in cases:
        arrays, meta = golden_io.load(os.path.join(HERE, "golden", name))
        u = arrays["u"]
        assert u.shape == _state_shape(w), name
        assert np.isfinite(u).all(), name
        assert (meta["nx"], meta["ny"]) == (w.nx, w.ny), name
        if steps is not None:
            assert meta["steps"] == steps, name
        else:
            assert meta["t_final"] == w.T and meta["steps"] > 30000, name
        assert (u[:, 0, 0] > 0.0).all(), name  # density cell averages


def test_adjoint_golden_holds_its_inputs():
    """u0 is stored bit for bit; lam and the directions come from the
    counter-based generator, so they are the same values on any machine."""
    arrays, meta = golden_io.load(os.path.join(HERE, "golden", f"adjoint_vortex_{MG.ADJ_N}_{MG.ADJ_STEPS}steps.npz"))
    w, p, u0, lam, dirs = MG.adjoint_case()
    assert arrays["u0"].shape == u0.shape
    assert arrays["lam_dot_jv"].shape == (MG.ADJ_DIRS,)
    assert np.isfinite(arrays["lam_dot_jv"]).all()
    assert meta["steps"] == MG.ADJ_STEPS and meta["directions"] == MG.ADJ_DIRS
    assert "directions_generator" in meta
    np.testing.assert_array_equal(lam, W.counter_uniform(u0.shape, MG.ADJ_RNG_SEED))


def test_batched_goldens_conserve_every_field_on_each_mesh():
    """The periodic batched end states keep, on each mesh, the total of every
    conserved field of the oracle's projection of their initial data
    (Section 3.3: the scheme conserves the cell averages' sum on each mesh),
    to rounding: a stored state that was truncated or mixed up fails it."""
    from oracle import oracle as O
    idx, ws = MG.smallest_batch_indices()
    for q in idx[:3]:
        w = ws[q]
        arrays, _ = golden_io.load(os.path.join(HERE, "golden", f"batched_seed0_{q}_{w.nx}_{MG.BATCH_STEPS}steps.npz"))
        u0 = O.project_fn(MG.oracle_problem(w), w.u0)
        t0 = u0[:, :, 0].sum(axis=(2, 3))
        t1 = arrays["u"][:, :, 0].sum(axis=(2, 3))
        scale = np.abs(u0[:, :, 0]).sum(axis=(2, 3))
        assert (np.abs(t1 - t0) <= 1e-12 * scale).all(), (q, t0, t1)
