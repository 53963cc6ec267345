"""The sqrt(n)-checkpoint schedule of the autograd wrapper, on the CPU.

The wrapper only orders calls to the library (steps, recorded steps and
recorded adjoints).  Here a fake context with the same four calls runs a
nonlinear elementwise step u <- u + h sin(u) on CPU tensors, whose adjoint is
lam <- (1 + h cos(u_n)) lam with u_n taken from the record.  The gradient the
wrapper returns must equal torch's own gradient of the plain loop for every
step count and segment length (segment boundaries, the last segment's records
kept from the forward pass, a segment longer than the run), and the wrapper
must recompute exactly the steps outside the last segment."""
import math

import pytest
import torch

from paper_2503_12473_gb300 import autograd as AG

H = 0.3


class FakeContext:
    def __init__(self, n):
        self.n = n
        self.steps = 0      # plain steps
        self.recorded = 0   # recorded steps (forward's last segment + recomputation)
        self.adjoints = 0

    def cdg_record_numel(self):
        return self.n

    def cdg_step_async(self, u, t, t_end, nsteps):
        for _ in range(nsteps):
            u.add_(H * torch.sin(u))
            self.steps += 1

    def cdg_step_record(self, u, rec):
        rec.copy_(u)
        u.add_(H * torch.sin(u))
        self.recorded += 1

    def cdg_step_adjoint_recorded(self, rec, lam_next, lam):
        torch.mul(1.0 + H * torch.cos(rec), lam_next, out=lam)
        self.adjoints += 1


def _reference_grad(u0, w, nsteps):
    u = u0.clone().requires_grad_(True)
    v = u
    for _ in range(nsteps):
        v = v + H * torch.sin(v)
    (v * w).sum().backward()
    return v.detach(), u.grad


@pytest.mark.parametrize("nsteps,segment", [(1, 1), (1, None), (7, 1), (7, 2), (7, 3), (7, 7), (7, 10),
                                            (9, None), (10, None), (16, 4), (17, 4), (400, None)])
def test_rollout_gradient_matches_the_plain_loop(nsteps, segment):
    g = torch.Generator().manual_seed(nsteps * 31 + (segment or 0))
    u0 = torch.randn(11, dtype=torch.float64, generator=g)
    w = torch.randn(11, dtype=torch.float64, generator=g)
    ctx = FakeContext(11)
    u = u0.clone().requires_grad_(True)
    uT = AG.rollout(u, ctx, nsteps, segment)
    (uT * w).sum().backward()
    ref_u, ref_g = _reference_grad(u0, w, nsteps)
    assert torch.allclose(uT.detach(), ref_u, rtol=1e-14, atol=1e-14)
    assert torch.allclose(u.grad, ref_g, rtol=1e-13, atol=1e-14)
    # schedule: every step once forward; the backward recomputes all but the last segment
    seg = segment or max(1, math.ceil(math.sqrt(nsteps)))
    last = nsteps - ((nsteps - 1) // seg) * seg
    assert ctx.steps + ctx.recorded == nsteps + (nsteps - last)
    assert ctx.adjoints == nsteps
