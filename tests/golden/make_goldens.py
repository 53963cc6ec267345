"""Write the oracle end states of the long discontinuous runs.

Runs ONLY the CPU oracle (oracle/) on the seeded initial data of
paper_2503_12473_gb300.workloads (point values of the physical initial data,
no arithmetic of the method) and stores the end states with golden_io:

  riemann   2D Euler four-quadrant Riemann data split at (0.8, 0.8), Q^2,
            transmissive [0,1]^2, 130 x 130 cells (130 = 4*32 + 2 = 32*4 + 2:
            ragged in both directions of the 32 x 4 cell tiles), SSP-RK3,
            CFL 0.1, OE, 200 steps with tau from the state (no end time).
  shu       1D Euler Shu-Osher data (Section 4), P^2, 4000 cells, transmissive
            [-5,5], SSP-RK3, CFL 0.1, OE, to T = 1.8.
  batched   the 8 smallest instances of the seed-0 batch of 256 periodic 2D
            Euler Q^2 problems (their own data and sizes), 100 SSP-RK3 steps.
  adjoint   directional derivatives of a 20-step rollout: on a 16 x 16 periodic
            isentropic vortex (the adjoint workload's data on a small mesh,
            CFL 0.1, OE) with a seeded 1e-3 perturbation and a 5% offset of the
            dual mesh's averages, <lam, J v_i> for a seeded lam and 16 seeded
            directions v_i, J the Jacobian of the 20 steps, from the
            complex-step build of the oracle (no difference quotient); lam and
            the v_i are counter-based uniform values in [-1, 1) (seeds 12,
            13..28), reproducible anywhere.

Each initial state is the oracle's projection (Section 3.3's projection-based
initialisation) of the point values.  The oracle runs with -ffp-contract=off
and fixed-order sums, so its results do not depend on the thread count.

Usage:  python tests/golden/make_goldens.py {riemann|shu|batched[:i,j,...]|adjoint} [--threads N]
Writes tests/golden/<name>.npz.  Hours of CPU time on 8 cores in all.
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

from oracle import oracle as O  # noqa: E402
from paper_2503_12473_gb300 import workloads as W  # noqa: E402
import golden_io  # noqa: E402

RIEMANN_N = 130
RIEMANN_STEPS = 200
BATCH_STEPS = 100
BATCH_COUNT = 8


def oracle_problem(w: W.Workload) -> O.Problem:
    return O.Problem(dim=w.dim, nx=w.nx, ny=w.ny, k=w.k, basis=w.basis, system=w.system, bc=w.bc, oe=w.oe,
                     rk=w.rk, ax=w.ax, bx=w.bx, ay=w.ay, by=w.by, gamma=w.gamma, adv_x=w.adv[0], adv_y=w.adv[1],
                     cfl=w.cfl)


def riemann_workload() -> W.Workload:
    return W.riemann_2d(RIEMANN_N, RIEMANN_STEPS)


def shu_workload() -> W.Workload:
    return W.shu_osher_1d(4000)


def smallest_batch_indices(count: int = BATCH_COUNT):
    """Indices of the `count` smallest meshes of the seed-0 batch (ties by index)."""
    ws = W.batch_workloads(seed=0, count=256, steps=BATCH_STEPS)
    order = sorted(range(len(ws)), key=lambda q: (ws[q].nx * ws[q].ny, q))
    return order[:count], ws


ADJ_N, ADJ_STEPS, ADJ_DIRS = 16, 20, 16
ADJ_PERTURB_SEED, ADJ_RNG_SEED = 5, 12


def adjoint_case():
    """(workload, oracle problem, u0, lam, directions) of the adjoint golden."""
    w = W.vortex_2d(n=ADJ_N, steps=ADJ_STEPS)
    p = oracle_problem(w)
    u0 = O.project_fn(p, w.u0) + W.perturbation(w.state_shape, ADJ_PERTURB_SEED, 1e-3)
    u0[1, :, 0] *= 1.05
    # lam and the directions from the counter-based generator (the same values
    # on every machine and numpy version; u0 itself is stored)
    lam = W.counter_uniform(u0.shape, ADJ_RNG_SEED)
    dirs = [W.counter_uniform(u0.shape, ADJ_RNG_SEED + 1 + i) for i in range(ADJ_DIRS)]
    return w, p, u0, lam, dirs


def _oracle_sha() -> str:
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "oracle", "oecdg_oracle.c"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def _run(w: W.Workload, path: str, keep: int, T_end: float, nsteps: int) -> None:
    p = oracle_problem(w)
    u0 = O.project_fn(p, w.u0)
    t0 = time.time()
    u, t, done, status = O.advance(p, u0, 0.0, T_end, nsteps)
    wall = time.time() - t0
    if status != O.OK:
        raise SystemExit(f"{w.name}: oracle status {status}")
    meta = {"workload": w.name, "nx": w.nx, "ny": w.ny, "steps": int(done), "t_final": float(t),
            "T_end": float(T_end), "oracle_sha256_16": _oracle_sha(), "oracle_wall_s": round(wall, 1),
            "oracle_threads": O.num_threads(),
            "u0_abs_sum": np.abs(u0).sum(axis=(0, 2, 3, 4)).tolist()}
    golden_io.save(path, {"u": u}, meta, keep=keep)
    print(f"{w.name}: {done} steps to t = {t!r} in {wall:.0f} s -> {path}", flush=True)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args(argv)
    if a.threads > 0:
        O.set_num_threads(a.threads)
    case, _, sel = a.case.partition(":")
    if case == "riemann":
        w = riemann_workload()
        _run(w, os.path.join(HERE, f"riemann_q2_{RIEMANN_N}_{RIEMANN_STEPS}steps.npz"), 8, 0.0, RIEMANN_STEPS)
    elif case == "shu":
        w = shu_workload()
        _run(w, os.path.join(HERE, "shu_osher_p2_4000_T1.8.npz"), 8, w.T, 1 << 30)
    elif case == "batched":
        idx, ws = smallest_batch_indices()
        pick = [int(s) for s in sel.split(",")] if sel else idx
        for q in pick:
            if q not in idx:
                raise SystemExit(f"instance {q} is not among the {BATCH_COUNT} smallest {idx}")
            _run(ws[q], os.path.join(HERE, f"batched_seed0_{q}_{ws[q].nx}_{BATCH_STEPS}steps.npz"), 6, 0.0,
                 BATCH_STEPS)
    elif case == "adjoint":
        w, p, u0, lam, dirs = adjoint_case()
        t0 = time.time()
        dots = []
        for v in dirs:
            _, jv, status = O.step_jvp(p, u0, v, nsteps=ADJ_STEPS)
            if status != O.OK:
                raise SystemExit(f"adjoint case: oracle status {status}")
            dots.append(float((lam * jv).sum()))
        meta = {"workload": w.name, "nx": w.nx, "ny": w.ny, "steps": ADJ_STEPS, "directions": ADJ_DIRS,
                "perturbation_seed": ADJ_PERTURB_SEED, "rng_seed": ADJ_RNG_SEED, "dual_average_offset": 0.05,
                "directions_generator": "counter_uniform(seed 12: lam; 13 + i: v_i)",
                "oracle_sha256_16": _oracle_sha(), "oracle_wall_s": round(time.time() - t0, 1)}
        path = os.path.join(HERE, f"adjoint_vortex_{ADJ_N}_{ADJ_STEPS}steps.npz")
        golden_io.save(path, {"u0": u0, "lam_dot_jv": np.asarray(dots)}, meta, keep=8)
        print(f"adjoint case: {len(dots)} directions -> {path}", flush=True)
    else:
        raise SystemExit(f"unknown case {case}")


if __name__ == "__main__":
    main()
