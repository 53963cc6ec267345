"""The synthetic inputs match their stated recipe (the workloads of the
benchmark and of the parity tests; all seeded where random)."""
import numpy as np

from paper_2503_12473_gb300 import workloads as W


def _prim(c):
    rho, mx, my, E = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    u, v = mx / rho, my / rho
    return np.stack([rho, u, v, (W.GAMMA - 1.0) * (E - 0.5 * rho * (u * u + v * v))], -1)


def test_riemann_quadrants_states():
    """Four constant states split at (0.8, 0.8), as (rho, u, v, p)."""
    f = W.riemann_quadrants()
    pts = np.array([[0.9, 0.9], [0.1, 0.9], [0.1, 0.1], [0.9, 0.1]])
    want = np.array([[1.5, 0.0, 0.0, 1.5], [0.5323, 1.206, 0.0, 0.3],
                     [0.138, 1.206, 1.206, 0.029], [0.5323, 0.0, 1.206, 0.3]])
    np.testing.assert_allclose(_prim(f(pts)), want, rtol=1e-14, atol=1e-15)
    w = W.riemann_2d()
    assert (w.nx, w.ny, w.k, w.system, w.bc) == (1024, 1024, 2, W.EULER, W.TRANSMISSIVE)


def test_vortex_far_field_and_centre():
    """rho = p = 1 and velocity (1, 1) far from the vortex; the centre at (5, 5)
    is the density minimum."""
    f = W.isentropic_vortex()
    far = _prim(f(np.array([[0.01, 0.01]])))[0]
    np.testing.assert_allclose(far, [1.0, 1.0, 1.0, 1.0], atol=2e-6)
    xs = np.linspace(4.0, 6.0, 41)
    X, Y = np.meshgrid(xs, xs)
    rho = f(np.stack([X.ravel(), Y.ravel()], 1))[:, 0]
    k = np.argmin(rho)
    assert abs(X.ravel()[k] - 5.0) < 1e-12 and abs(Y.ravel()[k] - 5.0) < 1e-12


def test_shu_osher_states():
    f = W.shu_osher()
    left = f(np.array([[-4.5]]))[0]
    rho, m, E = left
    v = m / rho
    assert abs(rho - 3.857143) < 1e-12 and abs(v - 2.629369) < 1e-12
    assert abs((W.GAMMA - 1.0) * (E - 0.5 * rho * v * v) - 10.33333) < 1e-9
    right = f(np.array([[1.0]]))[0]
    assert abs(right[0] - (1.0 + 0.2 * np.sin(5.0))) < 1e-15 and right[1] == 0.0


def test_batched_instances_follow_the_recipe():
    a = W.batched_instances(seed=0, count=256)
    b = W.batched_instances(seed=0, count=256)
    assert len(a) == 256
    for p, q in zip(a, b):  # seeded: the same instances every time
        assert p.n == q.n and np.array_equal(p.a, q.a) and np.array_equal(p.kv, q.kv)
    for inst in a:
        assert inst.n in W.BATCH_SIZES
        assert np.all(np.abs(inst.a) <= 1.0)
        assert inst.kv.dtype.kind == "i" and np.all(np.abs(inst.kv) <= 3)
        assert np.all(np.any(inst.kv != 0, axis=1))
        assert np.all((inst.centre >= 0.0) & (inst.centre <= 1.0))
        assert 0.1 <= inst.radius <= 0.25
        assert np.all(np.abs(inst.vel) <= 0.5)
    assert len({inst.n for inst in a}) == len(W.BATCH_SIZES)  # every size occurs
    # the initial data is periodic on [0, 1]^2 with p = 1
    f = W.batched_ic(a[0])
    pts = np.array([[0.13, 0.71], [0.42, 0.05]])
    np.testing.assert_allclose(f(pts), f(pts + 1.0), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(_prim(f(pts))[:, 3], 1.0, rtol=1e-13)


def test_random_modal_is_seeded_and_decays():
    u = W.random_modal((2, 4, 9, 3, 5), 7, 1.0, 0.5)
    v = W.random_modal((2, 4, 9, 3, 5), 7, 1.0, 0.5)
    assert np.array_equal(u, v)
    rms = np.sqrt((u ** 2).mean(axis=(0, 1, 3, 4)))
    assert rms[8] < rms[0] * 0.05  # mode m scaled by 0.5^m


def test_counter_uniform_is_splitmix64():
    """counter_uniform's element 0 for seed 0 is the first SplitMix64 output
    from state 0, 0xE220A8397B1DCDAF (the generator's published reference
    value), read as the fraction of its top 53 bits and mapped to [-1, 1);
    values are in range, seeds differ, and the mean and spread are uniform's."""
    from paper_2503_12473_gb300 import workloads as W
    top53 = 0xE220A8397B1DCDAF >> 11
    assert W.counter_uniform((1,), 0)[0] == 2.0 * (top53 / 2.0 ** 53) - 1.0
    a = W.counter_uniform((200000,), 7)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 0.01 and abs(a.std() - 1 / np.sqrt(3)) < 0.01
    assert not np.array_equal(W.counter_uniform((64,), 1), W.counter_uniform((64,), 2))
    np.testing.assert_array_equal(W.counter_uniform((4, 16), 3).ravel(), W.counter_uniform((64,), 3))
