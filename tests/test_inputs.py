"""Pins of the seeded input generator (no map-making arithmetic): the sweep with
finite-acceleration turnarounds and the batched-workload problem draws."""
import numpy as np

import gen
from gen.inputs import UNEVEN_MAP_SIZES, rng, sweep_offsets

F = 400.0


def test_sweep_instant_reversal_is_triangle():
    t = np.arange(0, 40, 1 / F)
    a = sweep_offsets(t, 120.0, 1200.0)
    period = 2 * 1200.0 / 120.0
    assert a.min() == -600.0 and a.max() == 600.0
    v = np.diff(a) * F
    assert np.all(np.isclose(np.abs(v), 120.0) | (np.abs(v) < 120.0))   # constant speed between reversals
    assert np.allclose(sweep_offsets(t + period, 120.0, 1200.0), a)     # periodic


def test_sweep_finite_acceleration_bounds():
    t = np.arange(0, 60, 1 / F)
    acc = 180.0
    a = sweep_offsets(t, 120.0, 1200.0, acc)
    v = np.diff(a) * F
    dv = np.diff(v) * F
    assert np.isclose(a.min(), -600.0) and np.isclose(a.max(), 600.0)   # full throw reached
    assert np.abs(v).max() <= 120.0 + 1e-6                            # cruise speed bound
    assert np.abs(dv).max() <= acc * (1 + 1e-6)                       # bounded acceleration
    # the braking distance v^2 / (2 acc) is spent at constant deceleration
    d = 120.0 ** 2 / (2 * acc)
    near_end = a > 600.0 - d + 1.0
    assert np.all(np.isclose(np.abs(dv[near_end[1:-1]]), acc, rtol=1e-6) | (np.abs(dv[near_end[1:-1]]) < acc))


def test_sweep_large_acceleration_approaches_triangle():
    t = np.arange(0, 30, 1 / F)
    tri = sweep_offsets(t, 120.0, 1200.0)
    fast = sweep_offsets(t, 120.0, 1200.0, 1e9)
    assert np.abs(fast - tri).max() < 1e-3


def test_uneven_problem_draws():
    seen = set()
    for k in range(64):
        g = rng(4, k, "misc")
        nd = int(g.choice([128, 256, 512, 1024]))
        nt = int(g.choice([1 << 18, 1 << 19, 1 << 20]))
        m = UNEVEN_MAP_SIZES[int(g.integers(len(UNEVEN_MAP_SIZES)))]
        seen.add((nd, nt, m))
        for n in m:   # 5-smooth map sides for the mixed-radix map FFT
            for p in (2, 3, 5):
                while n % p == 0:
                    n //= p
            assert n == 1
    assert len(seen) > 20
    scan, noise = gen.uneven_problem(1)
    assert (scan.n_det, scan.n_t) == (128, 1 << 18) and (scan.ny, scan.nx) == (450, 600)
    assert np.all(noise.sigma == 1.0) and np.all(noise.fknee == 2.0)
