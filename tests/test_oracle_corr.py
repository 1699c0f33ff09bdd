"""Pins of the oracle's N^-1 for noise correlated between detectors (reading R13:
N(f) = D(f) + V E(f) V^T per real-FFT bin)."""
import numpy as np
import pytest

import gen
from oracle import mapmaker as om

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def setup(n_t=1 << 10, r=3, amp=(3.0, 1.0, 1.0), scatter=0.3):
    scan = gen.small_scan(cfg=301, ny=12, nx=12, n_t=n_t, ncols=3, nrows=2, throw_px=14.0)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.0, scatter=scatter, cfg=301)
    corr = gen.corr_noise(scan.det_off, r=r, amp=amp)
    w = om.filter_weights(noise, scan.n_t, scan.f_samp)
    e = om.mode_psd(corr, scan.n_t, scan.f_samp)
    return scan, noise, corr, w, e


def test_woodbury_equals_definition():
    scan, noise, corr, w, e = setup()
    x = np.random.default_rng(1).standard_normal((scan.n_det, scan.n_t))
    a = om.apply_ninv_corr(w, corr, e, x)
    b = om.apply_ninv_corr_woodbury(w, corr, e, x)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)


def test_no_correlation_reduces_to_independent_filter():
    scan, noise, corr, w, e = setup(amp=(0.0, 0.0, 0.0))
    x = np.random.default_rng(2).standard_normal((scan.n_det, scan.n_t))
    np.testing.assert_allclose(om.apply_ninv_corr(w, corr, e, x), om.apply_ninv(w, x), rtol=0, atol=1e-12)


def test_symmetric_positive():
    scan, noise, corr, w, e = setup()
    g = np.random.default_rng(3)
    x, y = g.standard_normal((2, scan.n_det, scan.n_t))
    nx, ny = om.apply_ninv_corr(w, corr, e, x), om.apply_ninv_corr(w, corr, e, y)
    assert np.vdot(y, nx) == pytest.approx(np.vdot(x, ny), rel=1e-12)
    assert np.vdot(x, nx) > 0


def test_single_mode_closed_form():
    """One unit-norm mode v over detectors of equal weight w(f): N^-1 (v c) =
    v irfft(w / (1 + e w) rfft(c)) (the mode is down-weighted by 1 + e w)."""
    scan, noise, corr, w, e = setup(r=1, amp=(5.0,), scatter=None)
    c = np.random.default_rng(4).standard_normal(scan.n_t)
    v = corr.modes[:, 0]
    out = om.apply_ninv_corr(w, corr, e, np.outer(v, c))
    wk, ek = w[0], e[0]
    ref = np.outer(v, np.fft.irfft(wk / (1.0 + ek * wk) * np.fft.rfft(c), n=scan.n_t))
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_whitens_correlated_noise():
    """chi^2 = n^T N^-1 n of a simulated realisation has mean n_det n_t and standard
    deviation sqrt(2 n_det n_t) (the generator's covariance is the model's)."""
    scan, noise, corr, w, e = setup(n_t=1 << 12)
    chis = []
    for real in range(4):
        n = gen.corr_noise_tod(noise, corr, scan.n_t, scan.f_samp, cfg=302, real=real)
        chis.append(np.vdot(n, om.apply_ninv_corr(w, corr, e, n)))
    dim = scan.n_det * scan.n_t
    assert abs(np.mean(chis) - dim) < 5 * np.sqrt(2 * dim / len(chis))
    # the independent filter alone misses the correlated power
    n = gen.corr_noise_tod(noise, corr, scan.n_t, scan.f_samp, cfg=302, real=9)
    assert np.vdot(n, om.apply_ninv(w, n)) > dim + 10 * np.sqrt(2 * dim)


def test_operator_with_correlated_noise_symmetric_and_recovers_map():
    scan, noise, corr, w, e = setup()
    op = om.make_operator(scan, noise, corr=corr)
    g = np.random.default_rng(5)
    x, y = g.standard_normal((2,) + op.shape)
    x[:, ~op.mask.reshape(scan.ny, scan.nx)] = 0
    y[:, ~op.mask.reshape(scan.ny, scan.nx)] = 0
    assert np.vdot(y, om.apply_A(op, x)) == pytest.approx(np.vdot(x, om.apply_A(op, y)), rel=1e-10)
    m = gen.sky_map(scan.ny, scan.nx, cfg=303)
    m[:, ~op.mask.reshape(scan.ny, scan.nx)] = 0
    b = om.rhs(op, om.project(op, m))
    xs, info = om.pcg(lambda v: om.apply_A(op, v), om.BlockPrecon(op), b, tol=1e-12, maxit=2000)
    assert np.linalg.norm(xs - m) <= 1e-8 * np.linalg.norm(m)
