"""torch.autograd.Function over n OECDG time steps with sqrt(n) checkpoints.

Forward: cdg_step_async one step at a time, keeping the state every `segment`
steps (segment = ceil(sqrt(n)) by default); the steps of the last segment run
as cdg_step_record (same states) and keep their records.  Backward: for each
segment, last first, take or recompute its records (cdg_step_record from the
segment's checkpoint) and run cdg_step_adjoint_recorded through them in
reverse.  Peak memory: sqrt(n) checkpoints plus one segment of records (6
states and the OE maxima per step) plus the library's adjoint scratch; every
step outside the last segment is computed twice in all.  Every step and every adjoint runs in the
CUDA library; this module only orders the calls.
"""
from __future__ import annotations

import math

import torch


class OECDGRollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, u0, context, nsteps: int, segment: int):
        u = u0.detach().contiguous().clone()
        chk = [u.clone()]
        last_start = ((nsteps - 1) // segment) * segment if nsteps > 0 else 0
        rec_numel = context.cdg_record_numel()
        last_recs = []
        for s in range(nsteps):
            if s >= last_start:
                r = torch.empty(rec_numel, dtype=torch.float64, device=u.device)
                context.cdg_step_record(u, r)
                last_recs.append(r)
            else:
                context.cdg_step_async(u, 0.0, 0.0, 1)
            if (s + 1) % segment == 0 and s + 1 < nsteps:
                chk.append(u.clone())
        fctx.context = context
        fctx.nsteps = nsteps
        fctx.segment = segment
        fctx.chk = chk
        fctx.last_recs = last_recs
        return u

    @staticmethod
    def backward(fctx, lam_out):
        ctx, n, seg = fctx.context, fctx.nsteps, fctx.segment
        lam = lam_out.detach().contiguous().clone()
        nxt = torch.empty_like(lam)
        rec_numel = ctx.cdg_record_numel()
        for k in reversed(range(len(fctx.chk))):
            start = k * seg
            end = min(start + seg, n)
            if k == len(fctx.chk) - 1 and fctx.last_recs:
                recs, fctx.last_recs = fctx.last_recs, None  # recorded by the forward pass
            else:
                u = fctx.chk[k].clone()
                recs = []
                for _ in range(start, end):
                    r = torch.empty(rec_numel, dtype=torch.float64, device=u.device)
                    ctx.cdg_step_record(u, r)
                    recs.append(r)
                del u
            for q in reversed(range(end - start)):
                ctx.cdg_step_adjoint_recorded(recs[q], lam, nxt)
                lam, nxt = nxt, lam
            del recs
        fctx.chk = None
        fctx.last_recs = None
        return lam, None, None, None


def rollout(u0: torch.Tensor, context, nsteps: int, segment: int | None = None) -> torch.Tensor:
    """u(T) after nsteps steps, differentiable w.r.t. u0 (sqrt(n) checkpoints)."""
    seg = segment or max(1, math.ceil(math.sqrt(nsteps)))
    return OECDGRollout.apply(u0, context, nsteps, seg)
