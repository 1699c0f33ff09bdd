"""Pins of the tiled (locally varying) circulant preconditioner of the oracle (R15)."""
import math

import numpy as np
import pytest

import gen
from oracle import mapmaker as om


def test_windows_partition_of_unity():
    for n, t in ((64, 2), (45, 3), (900, 4)):
        w = om.tile_windows_1d(n, t)
        assert np.all(w >= 0) and np.allclose(w.sum(axis=0), 1.0, atol=1e-14)
        # smooth: no jump larger than the raised cosine's slope allows
        assert np.abs(np.diff(w, axis=1)).max() <= np.pi / 2 * t / n + 1e-12
    # centres at (i + 1/2) n / t, half height half a spacing away
    w = om.tile_windows_1d(16, 4)
    np.testing.assert_allclose(w[:, [2, 6, 10, 14]], np.eye(4), atol=1e-15)
    np.testing.assert_allclose([w[1, 4], w[1, 8], w[2, 8], w[2, 12]], 0.5, atol=1e-15)
    phi = om.tile_windows(30, 40, 2, 3)
    assert phi.shape == (6, 30, 40) and np.allclose(phi.sum(axis=0), 1.0)


@pytest.fixture(scope="module")
def cfg():
    scan = gen.small_scan(cfg=321, ny=24, nx=24, n_t=1 << 12, ncols=4, nrows=2, throw_px=30.0)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=321)
    return scan, noise, om.make_operator(scan, noise)


def test_one_tile_is_the_circulant(cfg):
    scan, noise, op = cfg
    r = np.random.default_rng(1).standard_normal(op.shape)
    r[:, ~op.mask.reshape(scan.ny, scan.nx)] = 0
    t = om.TiledCirculantPrecon(op, tiles=(1, 1), taper_sigma=4.0)
    c = om.CirculantPrecon(op, taper_sigma=4.0)
    np.testing.assert_allclose(t(r), c(r), rtol=0, atol=1e-12 * np.abs(c(r)).max())


def test_tiled_symmetric_positive_and_solves(cfg):
    scan, noise, op = cfg
    t = om.TiledCirculantPrecon(op, tiles=(2, 2), taper_sigma=4.0)
    g = np.random.default_rng(2)
    x, y = g.standard_normal((2,) + op.shape)
    msk = ~op.mask.reshape(scan.ny, scan.nx)
    x[:, msk] = 0
    y[:, msk] = 0
    assert np.vdot(y, t(x)) == pytest.approx(np.vdot(x, t(y)), rel=1e-10)
    assert np.vdot(x, t(x)) > 0
    # the four tiles' references differ, so the merge is not one circulant
    assert len({p.ref for p in t.parts}) == 4
    m = gen.sky_map(scan.ny, scan.nx, cfg=322)
    m[:, msk] = 0
    b = om.apply_A(op, m)
    xs, info = om.pcg(lambda v: om.apply_A(op, v), t, b, tol=1e-11, maxit=500)
    assert info.converged and np.linalg.norm(xs - m) <= 1e-8 * np.linalg.norm(m)
