"""The FP64 reciprocal and square root of the kernels' hot loops (the Euler
flux's 1/rho, the norms of the damping coefficients of Eq. (OEstep2D)),
called through cdg_math_eval, against correctly rounded results: numpy's
IEEE division and square root on the host.  Bound: 1 ulp over the contract's
range 2^-1022 <= x <= 2^1022."""
import numpy as np
import pytest
import torch

from paper_2503_12473_gb300 import oecdg as G

pytestmark = pytest.mark.gpu


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    # uniform mantissas over the whole exponent range of the contract ...
    wide = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-1022, 1022, n))
    # ... and the ranges the kernels meet (densities, sums of squares)
    near = np.exp(rng.uniform(np.log(1e-30), np.log(1e20), n))
    edge = np.array([2.0**-1022, 2.0**1022, 1.0, 2.0, 4.0, 0.25, 9.0, 1.0 - 2.0**-53,
                     1.0 + 2.0**-52, 1e-300, 1e-300 + 1e-316, 3.0, 0.1, 1.5, 1.4142135623730951])
    # mantissas right below and above the seeds' 20-bit boundaries
    m20 = 1.0 + np.arange(1, 4097) * 2.0**-20
    bnd = np.concatenate([m20, m20 - 2.0**-52, np.nextafter(m20, 2.0)])
    return np.concatenate([wide, near, edge, bnd, 2.0 * bnd])


def _ulps(a, b):
    return np.abs(a.view(np.int64) - b.view(np.int64))


@pytest.mark.parametrize("op", [G.MATH_RCP, G.MATH_SQRT])
def test_math_eval_within_one_ulp(op):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    x = _inputs(1 << 21, 17 + op)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    G.cdg_math_eval(op, xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref = 1.0 / x if op == G.MATH_RCP else np.sqrt(x)
    assert np.isfinite(y).all()
    u = _ulps(y, ref)
    assert u.max() <= 1, (u.max(), x[np.argmax(u)])
    # in place (d_x aliasing d_y) gives the same values
    G.cdg_math_eval(op, xd, xd)
    torch.cuda.synchronize()
    assert torch.equal(xd, yd)


def test_reciprocal_of_negative_and_tiny_densities():
    """The Euler flux takes 1/rho at every quadrature point, and without a
    limiter point densities of discontinuous runs can be negative or tiny
    (cell averages stay positive).  The reciprocal keeps its 1-ulp bound
    there: negative inputs over the whole normal range, magnitudes down to
    2^-1022, and exact oddness rcp(-x) = -rcp(x)."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    rng = np.random.default_rng(23)
    pos = np.concatenate([_inputs(1 << 19, 29),
                          np.ldexp(rng.uniform(1.0, 2.0, 1 << 16), rng.integers(-1022, -1000, 1 << 16)),
                          np.exp(rng.uniform(np.log(1e-12), np.log(1e-3), 1 << 16))])
    x = np.concatenate([-pos, pos])
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    G.cdg_math_eval(G.MATH_RCP, xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    assert np.isfinite(y).all()
    u = _ulps(y, 1.0 / x)
    assert u.max() <= 1, (u.max(), x[np.argmax(u)])
    n = len(pos)
    assert np.array_equal(y[:n], -y[n:])


def test_math_eval_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(G.CdgError) as e:
        G.cdg_math_eval(7, x, x)
    assert e.value.status == G.CDG_EINVAL
    G.cdg_math_eval(G.MATH_SQRT, x[:0], x[:0])  # n = 0: nothing launched
