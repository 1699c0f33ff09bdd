"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it checks and is chosen so that a plausible slip
(a dropped term, a sign, an index, a transposed operand) fails it.  No test
here touches the CUDA path.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import gen
from oracle import mapmaker as om


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def one_sample_scan(bx_px, by_px, phi_deg, dx_px, dy_px, ny=8, nx=8, periodic=False, psi=0.0):
    """A scan of a single sample and a single detector, positions given in pixels."""
    phi = math.radians(phi_deg)
    bore = np.array([[round(bx_px * gen.QB), round(by_px * gen.QB),
                      round(math.cos(phi) * gen.QR), round(math.sin(phi) * gen.QR)]], np.int32)
    det = np.array([[round(dx_px * gen.QD), round(dy_px * gen.QD)]], np.int32)
    pol = np.array([[math.cos(2 * psi), math.sin(2 * psi)]])
    return gen.Scan(ny=ny, nx=nx, bore=bore, det_off=det, det_pol=pol, periodic=periodic)


def pix_of(scan):
    return int(om.sample_pixels(scan, np.array([0]))[0, 0])


@pytest.fixture(scope="module")
def tiny():
    """A small TQU scan with 1/f noise (8x8 map) and its operator."""
    scan = gen.small_scan(cfg=101, ny=8, nx=8, n_t=1 << 11, ncols=3, nrows=2,
                          spacing_px=1.0, throw_px=14.0, rot=20.0)
    noise = gen.noise_params(scan.n_det, sigma=1.0, fknee=2.0, alpha=3.5, scatter=0.2, cfg=101)
    op = om.make_operator(scan, noise)
    return op


@pytest.fixture(scope="module")
def tiny_dense(tiny):
    a, idx = om.dense_A(tiny)
    return a, idx


# ---------------------------------------------------------------------------
# pointing (R10)
# ---------------------------------------------------------------------------

def test_pointing_identity_and_axes():
    # boresight exactly on pixel (ix=5, iy=2), no offset, no rotation
    assert pix_of(one_sample_scan(5, 2, 0, 0, 0)) == 2 * 8 + 5
    # a pure x offset moves the column, a pure y offset moves the row
    assert pix_of(one_sample_scan(1, 1, 0, 3, 0)) == 1 * 8 + 4
    assert pix_of(one_sample_scan(1, 1, 0, 0, 3)) == 4 * 8 + 1


def test_pointing_rotation_sign():
    # R(phi) = [[c, -s], [s, c]]: a +90 deg rotation maps an x offset to +y,
    # and a y offset to -x
    assert pix_of(one_sample_scan(3, 3, 90, 2, 0)) == 5 * 8 + 3
    assert pix_of(one_sample_scan(3, 3, 90, 0, 2)) == 3 * 8 + 1
    assert pix_of(one_sample_scan(3, 3, -90, 2, 0)) == 1 * 8 + 3


def test_pointing_round_half_up_and_cut():
    assert pix_of(one_sample_scan(2.5, 0, 0, 0, 0)) == 3
    assert pix_of(one_sample_scan(2.5 - 2 ** -16, 0, 0, 0, 0)) == 2
    assert pix_of(one_sample_scan(-0.5, 0, 0, 0, 0)) == 0
    assert pix_of(one_sample_scan(-0.5 - 2 ** -16, 0, 0, 0, 0)) == -1
    assert pix_of(one_sample_scan(7.4, 7.49, 0, 0, 0)) == 63
    assert pix_of(one_sample_scan(7.5, 3, 0, 0, 0)) == -1
    assert pix_of(one_sample_scan(3, 7.5, 0, 0, 0)) == -1


def test_pointing_periodic_wrap():
    assert pix_of(one_sample_scan(9, -1, 0, 0, 0, periodic=True)) == 7 * 8 + 1
    assert pix_of(one_sample_scan(-3, 17, 0, 0, 0, periodic=True)) == 1 * 8 + 5


def test_pointing_is_nearest_pixel_of_exact_position():
    """The fixed-point rule picks the nearest pixel of the exact position
    B + R(phi) d (rational arithmetic, extreme-range random tables): the chosen pixel
    centre lies within half a pixel plus the 2^-16 flooring of the offset, and it is
    the nearest one whenever the exact position is not within 2^-16 px of a
    half-pixel boundary."""
    g = np.random.default_rng(7)
    n_t, n_det = 300, 6
    bore = np.stack([g.integers(-3 * gen.QB, 40 * gen.QB, n_t),
                     g.integers(-3 * gen.QB, 40 * gen.QB, n_t),
                     g.integers(-gen.QR, gen.QR + 1, n_t),
                     g.integers(-gen.QR, gen.QR + 1, n_t)], axis=1).astype(np.int32)
    det = g.integers(-(1 << 14) + 1, 1 << 14, (n_det, 2)).astype(np.int32)
    scan = gen.Scan(ny=37, nx=29, bore=bore, det_off=det, det_pol=np.zeros((n_det, 2)))
    pix = om.sample_pixels(scan, np.arange(n_det))
    tol = Fraction(1, 1 << 16)
    checked = 0
    for d in range(n_det):
        for t in range(n_t):
            bx, by, c, s = (int(v) for v in bore[t])
            dx, dy = int(det[d, 0]), int(det[d, 1])
            x = Fraction(bx, 1 << 16) + Fraction(c * dx - s * dy, 1 << 22)
            y = Fraction(by, 1 << 16) + Fraction(s * dx + c * dy, 1 << 22)
            p = pix[d, t]
            if p >= 0:
                iy, ix = divmod(int(p), 29)
                assert abs(x - ix) <= Fraction(1, 2) + tol and abs(y - iy) <= Fraction(1, 2) + tol
            fx, fy = x + Fraction(1, 2), y + Fraction(1, 2)
            if min(fx - math.floor(fx), math.ceil(fx) - fx) > tol and \
               min(fy - math.floor(fy), math.ceil(fy) - fy) > tol:
                ix, iy = math.floor(fx), math.floor(fy)
                want = iy * 29 + ix if (0 <= ix < 29 and 0 <= iy < 37) else -1
                assert p == want
                checked += 1
    assert checked > 0.9 * n_t * n_det


def test_polarisation_angle_is_psi_plus_phi():
    scan, _ = gen.tiny_patch()
    dets = np.arange(4)
    w = om.sample_weights(scan, dets)
    phi = np.arctan2(scan.bore[:, 3].astype(float), scan.bore[:, 2].astype(float))
    psi = 0.5 * np.arctan2(scan.det_pol[dets, 1], scan.det_pol[dets, 0])
    ang = 2 * (psi[:, None] + phi[None, :])
    np.testing.assert_allclose(w[0], 1.0)
    np.testing.assert_allclose(w[1], np.cos(ang), atol=1e-13)
    np.testing.assert_allclose(w[2], np.sin(ang), atol=1e-13)
    # the response row is the paper's unit row (1, cos 2a, sin 2a), although the
    # fixed-point rotation pairs are not exactly of unit length
    np.testing.assert_allclose(w[1] ** 2 + w[2] ** 2, 1.0, atol=1e-14)
    r2 = (scan.bore[:, 2].astype(float) ** 2 + scan.bore[:, 3].astype(float) ** 2) / 2.0 ** 30
    assert np.abs(r2 - 1.0).max() > 1e-6


# ---------------------------------------------------------------------------
# noise filter (R1-R3)
# ---------------------------------------------------------------------------

def test_filter_closed_forms():
    n_t, fs = 1024, 400.0
    noise = gen.Noise(np.array([1.3]), np.array([fs * 37 / n_t]), np.array([3.5]))
    w = om.filter_weights(noise, n_t, fs)
    # at f = f_knee the PSD is 2 sigma^2
    assert w[0, 37] == pytest.approx(1.0 / (2 * 1.3 ** 2), rel=1e-14)
    # far above the knee the filter tends to 1/sigma^2
    assert w[0, n_t // 2] == pytest.approx(1 / 1.3 ** 2 / (1 + (n_t / 2 / 37) ** -3.5), rel=1e-14)
    # DC takes the first bin (R2)
    assert w[0, 0] == w[0, 1]
    # a cosine at bin k is an eigenvector with eigenvalue w_k
    t = np.arange(n_t)
    for k in (0, 1, 5, 37, 200, n_t // 2):
        x = np.cos(2 * np.pi * k * t / n_t + (0.3 if 0 < k < n_t // 2 else 0.0))
        y = om.apply_ninv(w, x[None, :])[0]
        np.testing.assert_allclose(y, w[0, k] * x, atol=1e-12)


def test_ninv_is_inverse_of_covariance_and_diagonal():
    """N^-1 from the Fourier filter equals the inverse of the dense circulant
    covariance built from the PSD by the DFT definition; R3's diagonal is its
    diagonal entry."""
    n_t, fs = 128, 400.0
    noise = gen.Noise(np.array([0.7]), np.array([9.0]), np.array([2.5]))
    k = np.arange(n_t)
    f = np.minimum(k, n_t - k) * fs / n_t
    f[0] = fs / n_t
    psd = 0.7 ** 2 * (1 + (f / 9.0) ** -2.5)
    dft = np.exp(-2j * np.pi * np.outer(k, k) / n_t)
    cov = (np.conj(dft).T @ np.diag(psd) @ dft).real / n_t
    ninv = np.linalg.inv(cov)
    w = om.filter_weights(noise, n_t, fs)
    eye = np.eye(n_t)
    got = om.apply_ninv(np.repeat(w, n_t, axis=0), eye)
    np.testing.assert_allclose(got, ninv, atol=1e-10 * np.abs(ninv).max())
    assert om.ninv_diagonal(w, n_t)[0] == pytest.approx(ninv[0, 0], rel=1e-12)


# ---------------------------------------------------------------------------
# the operator A = P^T N^-1 P (Eq. 2)
# ---------------------------------------------------------------------------

def test_A_against_dense_matrices():
    """A built from an explicit dense P (one row per sample) and the inverse of the
    dense time-domain covariance equals the oracle's matrix-free A."""
    scan = gen.small_scan(cfg=102, ny=4, nx=5, n_t=256, ncols=2, nrows=1, spacing_px=1.0,
                          throw_px=8.0, rot=25.0)
    noise = gen.noise_params(scan.n_det, sigma=1.0, fknee=20.0, alpha=2.0, scatter=0.3, cfg=102)
    # two pixels that the scan hits are masked by hand: their samples leave P (R4)
    mask = om.pixel_mask(scan)
    hit = np.flatnonzero(om.hit_blocks(scan)[:, 0, 0] > 0)
    mask[hit[[1, 4]]] = False
    op = om.make_operator(scan, noise, mask=mask)
    nc, npix, n_t = 3, scan.npix, scan.n_t
    pix = om.sample_pixels(scan, np.arange(scan.n_det))
    wts = om.sample_weights(scan, np.arange(scan.n_det))
    k = np.arange(n_t)
    f = np.minimum(k, n_t - k) * scan.f_samp / n_t
    f[0] = scan.f_samp / n_t
    dft = np.exp(-2j * np.pi * np.outer(k, k) / n_t)
    a_ref = np.zeros((nc * npix, nc * npix))
    for d in range(scan.n_det):
        pm = np.zeros((n_t, nc * npix))
        for t in range(n_t):
            p = pix[d, t]
            if p >= 0 and op.mask[p]:
                for c in range(nc):
                    pm[t, c * npix + p] = wts[c, d, t]
        psd = noise.sigma[d] ** 2 * (1 + (f / noise.fknee[d]) ** -noise.alpha[d])
        cov = (np.conj(dft).T @ np.diag(psd) @ dft).real / n_t
        a_ref += pm.T @ np.linalg.solve(cov, pm)
    a, (comp, pixs) = om.dense_A(op)
    sel = comp * npix + pixs
    ref = a_ref[np.ix_(sel, sel)]
    np.testing.assert_allclose(a, ref, atol=1e-10 * np.abs(ref).max())
    # nothing outside the unmasked set
    rest = np.setdiff1d(np.arange(nc * npix), sel)
    assert rest.size >= 2 * nc and np.abs(a_ref[np.ix_(rest, rest)]).max() == 0.0
    # on every unknown, masked ones included: A e_p = 0 and (A m)_p = 0 for a masked
    # pixel p, whatever m holds there
    m = np.random.default_rng(7).standard_normal((nc, scan.ny, scan.nx))
    am = a_ref @ m.ravel()
    np.testing.assert_allclose(om.apply_A(op, m).ravel(), am, atol=1e-10 * np.abs(am).max())


def test_A_symmetric_positive(tiny, tiny_dense):
    a, _ = tiny_dense
    np.testing.assert_allclose(a, a.T, atol=1e-12 * np.abs(a).max())
    assert np.linalg.eigvalsh(a).min() > 0
    g = np.random.default_rng(3)
    x, y = g.standard_normal((2,) + tiny.shape)
    x[:, ~tiny.mask.reshape(8, 8)] = 0
    y[:, ~tiny.mask.reshape(8, 8)] = 0
    lhs = np.vdot(x, om.apply_A(tiny, y))
    rhs = np.vdot(y, om.apply_A(tiny, x))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_white_noise_T_only_is_hit_count():
    """With N = sigma^2 I and one pixel per sample, A is diagonal with the hit
    counts over sigma^2 (Eq. 3-5 become exact)."""
    scan = gen.small_scan(cfg=103, ny=6, nx=7, n_t=512, ncomp=1, throw_px=10.0)
    noise = gen.Noise(np.full(scan.n_det, 2.0), np.zeros(scan.n_det), np.full(scan.n_det, 3.5))
    op = om.make_operator(scan, noise)
    hits = np.zeros(scan.npix)
    pix = om.sample_pixels(scan, np.arange(scan.n_det))
    for p in pix.ravel():
        if p >= 0:
            hits[p] += 1
    m = np.random.default_rng(1).standard_normal((1, 6, 7))
    np.testing.assert_allclose(om.apply_A(op, m).ravel(), hits * m.ravel() / 4.0, atol=1e-12)
    # Jacobi (Eq. 5, a = 1): unit-weight blocks, the hit counts themselves
    mj = om.BlockPrecon(op, "jacobi")
    np.testing.assert_array_equal(mj.blocks[:, 0, 0], hits * op.mask)
    np.testing.assert_allclose(mj(m).ravel()[op.mask], m.ravel()[op.mask] / hits[op.mask], rtol=1e-14)
    # M_B = M_J * 4 = A^-1 there: PCG stops after one iteration
    mb = om.BlockPrecon(op, "binned")
    b = om.apply_A(op, m)
    x, info = om.pcg(lambda v: om.apply_A(op, v), mb, b, tol=1e-12)
    assert info.iterations == 1
    np.testing.assert_allclose(x.ravel()[op.mask], m.ravel()[op.mask], rtol=1e-12)


def test_binning_magnitude_bounds_A(tiny):
    """The binning-error scale S = P^T |N^-1 P m| with its hit counts: equal to A m
    and to the brute-force hit count where no term can cancel (white noise, T only,
    a positive map), above |A m| everywhere on a TQU scan with 1/f noise, and
    homogeneous of degree one in m."""
    scan = gen.small_scan(cfg=103, ny=6, nx=7, n_t=512, ncomp=1, throw_px=10.0)
    noise = gen.Noise(np.full(scan.n_det, 2.0), np.zeros(scan.n_det), np.full(scan.n_det, 3.5))
    op = om.make_operator(scan, noise)
    hits = np.zeros(scan.npix)
    for p in om.sample_pixels(scan, np.arange(scan.n_det)).ravel():
        if p >= 0:
            hits[p] += 1
    m = 1.0 + np.random.default_rng(2).random((1, 6, 7))
    s, h = om.binning_magnitude(op, m)
    np.testing.assert_array_equal(h.ravel(), hits)
    np.testing.assert_allclose(s, om.apply_A(op, m), rtol=1e-12)
    m3 = gen.random_maps(3, 8, 8, 1, cfg=5)[0]
    s3, h3 = om.binning_magnitude(tiny, m3)
    a3 = om.apply_A(tiny, m3)
    assert np.all(s3 >= np.abs(a3) * (1 - 1e-12))
    assert np.any(s3 > 2 * np.abs(a3))
    np.testing.assert_allclose(om.binning_magnitude(tiny, -2.0 * m3)[0], 2.0 * s3, rtol=1e-12)
    assert h3.sum() == (om._pix(tiny, np.arange(tiny.scan.n_det)) >= 0).sum()


def test_mask_removes_degenerate_pixels():
    # one detector at one angle hits pixels once: the TQU block is rank one
    scan = gen.small_scan(cfg=104, ny=6, nx=6, n_t=64, ncols=1, nrows=1, throw_px=30.0)
    mask = om.pixel_mask(scan)
    assert not mask.any()
    assert om.pixel_mask(gen.Scan(**{**scan.__dict__, "ncomp": 1})).any()


# ---------------------------------------------------------------------------
# solves (Eq. 2 by PCG; footnote on PCG)
# ---------------------------------------------------------------------------

def test_pcg_matches_dense_cholesky(tiny, tiny_dense):
    a, (comp, pixs) = tiny_dense
    g = np.random.default_rng(11)
    b = np.zeros(tiny.shape)
    b.reshape(3, -1)[comp, pixs] = g.standard_normal(comp.size)
    ref = np.linalg.solve(a, b.reshape(3, -1)[comp, pixs])
    for m in (om.BlockPrecon(tiny, "binned"), om.BlockPrecon(tiny, "jacobi"),
              om.CirculantPrecon(tiny, taper_sigma=3.0)):
        x, info = om.pcg(lambda v: om.apply_A(tiny, v), m, b, tol=1e-12, maxit=2000)
        assert info.converged
        np.testing.assert_allclose(x.reshape(3, -1)[comp, pixs], ref,
                                   atol=1e-8 * np.abs(ref).max())


def test_pcg_from_a_given_start(tiny, tiny_dense):
    """A start x0 enters through r0 = b - A x0: from the solution itself PCG stops
    at once, from any other start it reaches the same solution."""
    a, (comp, pixs) = tiny_dense
    g = np.random.default_rng(12)
    b = np.zeros(tiny.shape)
    b.reshape(3, -1)[comp, pixs] = g.standard_normal(comp.size)
    xs = np.zeros(tiny.shape)
    xs.reshape(3, -1)[comp, pixs] = np.linalg.solve(a, b.reshape(3, -1)[comp, pixs])
    mb = om.BlockPrecon(tiny)
    x, info = om.pcg(lambda v: om.apply_A(tiny, v), mb, b, tol=1e-9, x0=xs)
    assert info.iterations == 0 and info.rel_resid[0] <= 1e-9
    np.testing.assert_array_equal(x, xs)
    x0 = np.zeros(tiny.shape)
    x0.reshape(3, -1)[comp, pixs] = g.standard_normal(comp.size)
    for flexible, window in ((False, 1), (True, 1), (True, 4)):
        x, info = om.pcg(lambda v: om.apply_A(tiny, v), mb, b, tol=1e-12, maxit=2000, x0=x0,
                         flexible=flexible, window=window)
        assert info.converged
        assert info.rel_resid[0] == pytest.approx(
            np.linalg.norm(b - om.apply_A(tiny, x0)) / np.linalg.norm(b), rel=1e-12)
        np.testing.assert_allclose(x, xs, atol=1e-8 * np.abs(xs).max())


def test_noise_free_data_recover_input_map():
    """Sec. Test setup: noise-free TOD d = P m recover m (on the unmasked pixels)."""
    scan = gen.small_scan(cfg=105, ny=12, nx=12, n_t=1 << 12, ncols=4, nrows=2, throw_px=18.0)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=105)
    op = om.make_operator(scan, noise)
    m = gen.sky_map(12, 12, cfg=105)
    m[:, ~op.mask.reshape(12, 12)] = 0
    d = om.project(op, m)
    b = om.rhs(op, d)
    x, info = om.pcg(lambda v: om.apply_A(op, v), om.BlockPrecon(op), b, tol=1e-12, maxit=3000)
    assert info.converged
    np.testing.assert_allclose(x, m, atol=1e-8)


def test_anorm_error_identity(tiny, tiny_dense):
    """The error A-norm after i steps: sum over all remaining alpha_j r_j^T z_j equals
    ||x_i - x||_A^2 exactly (the Results footnote's estimate is its d-term truncation)."""
    a, (comp, pixs) = tiny_dense
    g = np.random.default_rng(5)
    b = np.zeros(tiny.shape)
    b.reshape(3, -1)[comp, pixs] = g.standard_normal(comp.size)
    xs = np.linalg.solve(a, b.reshape(3, -1)[comp, pixs])
    mb = om.BlockPrecon(tiny)
    x, info = om.pcg(lambda v: om.apply_A(tiny, v), mb, b, tol=1e-13, maxit=2000, keep_iterates=True)
    terms = np.array(info.anorm_terms)
    assert info.iterations >= 8
    for i in (0, 2, 5, info.iterations // 2):
        e = info.iterates[i].reshape(3, -1)[comp, pixs] - xs
        exact = e @ a @ e
        assert terms[i:].sum() == pytest.approx(exact, rel=1e-6)
    est = om.anorm_estimate(terms, d=4)
    assert np.all(est <= np.cumsum(terms[::-1])[::-1][:est.size] * (1 + 1e-12))
    # each term is the drop of the squared error A-norm over one step, so the d-term
    # estimate is ||x_i - x||_A^2 - ||x_{i+d} - x||_A^2
    err = [float((it.reshape(3, -1)[comp, pixs] - xs) @ a @ (it.reshape(3, -1)[comp, pixs] - xs))
           for it in info.iterates]
    assert est.size == info.iterations - 3
    for i in (0, 1, 3, est.size - 1):
        assert est[i] == pytest.approx(err[i] - err[i + 4], rel=1e-6, abs=1e-9 * err[0])


def test_flexible_cg_equals_pcg_for_fixed_preconditioner(tiny):
    b = om.apply_A(tiny, gen.sky_map(8, 8, cfg=106))
    mb = om.BlockPrecon(tiny)
    x1, i1 = om.pcg(lambda v: om.apply_A(tiny, v), mb, b, tol=1e-10)
    x2, i2 = om.pcg(lambda v: om.apply_A(tiny, v), mb, b, tol=1e-10, flexible=True)
    assert abs(i1.iterations - i2.iterations) <= 1
    np.testing.assert_allclose(x1, x2, atol=1e-8 * np.abs(x1).max())


def test_fcg_window_equals_pcg_for_fixed_preconditioner(tiny):
    """Truncated flexible CG with a fixed SPD preconditioner follows the PCG
    iterates (exact arithmetic): same residual history and solution."""
    b = om.apply_A(tiny, gen.sky_map(8, 8, cfg=107))
    mb = om.BlockPrecon(tiny)
    x1, i1 = om.pcg(lambda v: om.apply_A(tiny, v), mb, b, tol=1e-10)
    for m in (2, 5, 50):
        x2, i2 = om.pcg(lambda v: om.apply_A(tiny, v), mb, b, tol=1e-10, flexible=True, window=m)
        assert abs(i1.iterations - i2.iterations) <= 1
        np.testing.assert_allclose(i2.rel_resid[:12], i1.rel_resid[:12], rtol=1e-6)
        np.testing.assert_allclose(x1, x2, atol=1e-8 * np.abs(x1).max())


def test_fcg_keeps_window_directions_conjugate(tiny, tiny_dense):
    """With a preconditioner that changes every iteration (M_B plus a positive
    diagonal whose weight cycles), FCG(m) keeps each step direction d_i =
    x_{i+1} - x_i A-conjugate to the previous m ones and the new residual
    orthogonal to them, on the dense A; with m = 1 only to the last one."""
    a, idx = tiny_dense
    comp, pixs = idx
    mb = om.BlockPrecon(tiny)
    rng = np.random.default_rng(3)
    diag = rng.uniform(0.5, 2.0, size=tiny.shape)
    count = [0]

    def varying(r):
        count[0] += 1
        return mb(r) + (0.2 + 0.15 * math.sin(1.7 * count[0])) * np.where(tiny.mask.reshape(tiny.shape[1:]), diag * r, 0)

    b = om.apply_A(tiny, gen.sky_map(8, 8, cfg=108))
    flat = lambda v: v.reshape(tiny.scan.ncomp, -1)[comp, pixs]
    for m in (1, 4, 100):
        count[0] = 0
        _, info = om.pcg(lambda v: om.apply_A(tiny, v), varying, b, tol=1e-12, maxit=30, flexible=True,
                         window=m, keep_iterates=True)
        d = [flat(info.iterates[i + 1] - info.iterates[i]) for i in range(len(info.iterates) - 1)]
        assert len(d) >= 10
        for i in range(1, 10):
            r = flat(b) - a @ flat(info.iterates[i + 1])
            for j in range(max(0, i - m), i):
                c = abs(d[i] @ a @ d[j]) / math.sqrt((d[i] @ a @ d[i]) * (d[j] @ a @ d[j]))
                assert c < 1e-8, (m, i, j, c)
            assert abs(r @ d[i]) < 1e-9 * np.linalg.norm(r) * np.linalg.norm(d[i])
        # outside the window the conjugacy is lost (the preconditioner really varies)
        if m == 1:
            c02 = abs(d[3] @ a @ d[1]) / math.sqrt((d[3] @ a @ d[3]) * (d[1] @ a @ d[1]))
            assert c02 > 1e-6


# ---------------------------------------------------------------------------
# preconditioners (Eq. 3-5, 7-13)
# ---------------------------------------------------------------------------

def test_white_level_weights_alternative_of_R3(tiny):
    """R3's alternative weight 1/sigma_d^2 (Eq. 3): for the law R1 every bin weight is
    at most the white level, so the exact circulant diagonal lies below it, with
    equality for white noise, where both binned preconditioners coincide (and, the
    binned blocks being all of A there, equal A^-1)."""
    op = tiny
    exact = om.detector_weights(op)
    white = om.detector_weights(op, white=True)
    np.testing.assert_allclose(white, 1.0 / op.noise.sigma ** 2, rtol=0, atol=0)
    assert np.all(exact < white)
    wn = gen.noise_params(op.scan.n_det, sigma=1.0, fknee=0.0, alpha=3.5, scatter=0.2, cfg=101)
    wn.fknee[:] = 0.0
    opw = om.make_operator(op.scan, wn)
    np.testing.assert_allclose(om.detector_weights(opw), om.detector_weights(opw, white=True), rtol=1e-14)
    r = gen.random_maps(3, op.scan.ny, op.scan.nx, 1, cfg=102)[0] * opw.mask.reshape(op.scan.ny, op.scan.nx)
    z1 = om.BlockPrecon(opw)(r)
    z2 = om.BlockPrecon(opw, white=True)(r)
    np.testing.assert_allclose(z1, z2, rtol=1e-12, atol=1e-14)
    # 1/f noise: the blocks scale detector by detector, so the two differ
    assert not np.allclose(om.BlockPrecon(op)(r), om.BlockPrecon(op, white=True)(r))


def test_binned_blocks_are_block_diagonal_of_PtDP():
    """M_B^-1 (Eq. 4) is the per-pixel block of P^T diag(N^-1) P, with diag(N^-1) the
    diagonal of the dense inverse covariance."""
    scan = gen.small_scan(cfg=107, ny=4, nx=4, n_t=128, ncols=2, nrows=2, spacing_px=1.0,
                          throw_px=6.0, rot=30.0)
    noise = gen.noise_params(scan.n_det, fknee=10.0, alpha=3.0, scatter=0.3, cfg=107)
    op = om.make_operator(scan, noise)
    assert op.mask.sum() >= 8
    n_t = scan.n_t
    k = np.arange(n_t)
    f = np.minimum(k, n_t - k) * scan.f_samp / n_t
    f[0] = scan.f_samp / n_t
    dft = np.exp(-2j * np.pi * np.outer(k, k) / n_t)
    pix = om.sample_pixels(scan, np.arange(scan.n_det))
    wts = om.sample_weights(scan, np.arange(scan.n_det))
    ref = np.zeros((16, 3, 3))
    for d in range(scan.n_det):
        psd = noise.sigma[d] ** 2 * (1 + (f / noise.fknee[d]) ** -noise.alpha[d])
        cov = (np.conj(dft).T @ np.diag(psd) @ dft).real / n_t
        dd = np.linalg.inv(cov)[0, 0]
        for t in range(n_t):
            if pix[d, t] >= 0 and op.mask[pix[d, t]]:
                v = wts[:, d, t]
                ref[pix[d, t]] += dd * np.outer(v, v)
    mb = om.BlockPrecon(op, "binned")
    np.testing.assert_allclose(mb.blocks, ref, atol=1e-10 * np.abs(ref).max())


def test_eq11_fourier_convention_against_direct_convolution():
    """(Qx)_i = sum_j q_{j-i} x_j computed by loops equals F^-1 (Fq)* F x (Eq. 11),
    block-wise, on a non-square map with non-symmetric blocks."""
    g = np.random.default_rng(2)
    ny, nx = 5, 6
    q = g.standard_normal((3, 3, ny, nx))
    x = g.standard_normal((3, ny, nx))
    ref = np.zeros_like(x)
    for iy in range(ny):
        for ix in range(nx):
            for jy in range(ny):
                for jx in range(nx):
                    ref[:, iy, ix] += q[:, :, (jy - iy) % ny, (jx - ix) % nx] @ x[:, jy, jx]
    np.testing.assert_allclose(om.circulant_forward(q, x), ref, atol=1e-12)


@pytest.mark.parametrize("diagonal, ref", [(False, None), (True, None), (True, 1 * 8 + 2), (False, 5 * 8 + 7)])
def test_circulant_is_exact_inverse_on_bccb_scan(diagonal, ref):
    """On a periodic translation-invariant scan A is block circulant (footnotes of
    Sec. Implementation), so M_C = A^-1 and PCG converges in one iteration, whichever
    pixel the row is measured at (Eq. 10: offsets taken from the reference)."""
    ny, nx = 6, 8
    n_t = 16 * math.lcm(nx, ny)
    scan = gen.bccb_scan(ny, nx, n_t, diagonal=diagonal)
    noise = gen.Noise(np.ones(scan.n_det), np.full(scan.n_det, 30.0), np.full(scan.n_det, 2.0))
    op = om.make_operator(scan, noise)
    assert op.mask.all()
    mc = om.CirculantPrecon(op, ref=ref)
    assert mc.n_clamped == 0
    g = np.random.default_rng(4)
    x = g.standard_normal(op.shape)
    ax = om.apply_A(op, x)
    np.testing.assert_allclose(mc.approx_A(x), ax, atol=1e-10 * np.abs(ax).max())
    np.testing.assert_allclose(mc(ax), x, atol=1e-10 * np.abs(x).max())
    _, info = om.pcg(lambda v: om.apply_A(op, v), mc, ax, tol=1e-9)
    assert info.iterations == 1
    if diagonal:  # the diagonal sweep correlates rows: q has ky != 0 support
        assert np.abs(mc.q[:, :, 1:, :]).max() > 1e-6 * np.abs(mc.q).max()


def test_circulant_precon_symmetric_and_taper(tiny):
    mc = om.CirculantPrecon(tiny, taper_sigma=2.5)
    g = np.random.default_rng(8)
    x, y = g.standard_normal((2,) + tiny.shape)
    assert np.vdot(x, mc(y)) == pytest.approx(np.vdot(y, mc(x)), rel=1e-10)
    tp = om.taper(6, 7, 2.0)
    assert tp[0, 0] == 1.0
    assert tp[1, 0] == pytest.approx(math.exp(-1 / 8)) and tp[5, 0] == tp[1, 0]
    assert tp[0, 6] == tp[0, 1]
    # even in the offset on both sides, odd (7) and even (6): g(k) = g(-k)
    np.testing.assert_array_equal(tp[:, 1:], tp[:, :0:-1])
    np.testing.assert_array_equal(tp[1:, :], tp[:0:-1, :])
    assert np.all(om.taper(4, 4, math.inf) == 1.0)
    # R9 reference pixel and its fallback
    mask = np.ones(64, bool)
    assert om.reference_pixel(mask, 8, 8) == 4 * 8 + 4
    assert om.reference_pixel(np.ones(60, bool), 6, 10) == 3 * 10 + 5
    assert om.reference_pixel(np.ones(63, bool), 9, 7) == 4 * 7 + 3
    mask[4 * 8 + 4] = False
    assert om.reference_pixel(mask, 8, 8) == 3 * 8 + 4


def test_circulant_inverts_its_model_and_floors_relative(tiny):
    """Eq. 8 and Eq. 12 describe one matrix and its inverse: with no mode floored,
    M_C (Sigma^T Q Sigma x) = x on a TQU scan whose mode blocks are complex
    Hermitian, not real symmetric (so a dropped conjugate or a transposed block
    shows); the model Sigma^T Q Sigma is symmetric once q_k = q_{-k}^T (R5).  With a
    floor that bites, the smallest eigenvalue of the floored mode blocks is pd_eps
    times the largest (R6: relative to the largest over all modes)."""
    mc = om.CirculantPrecon(tiny)
    assert mc.n_clamped == 0
    h = np.conj(np.fft.fft2(mc.q, axes=(-2, -1))).transpose(2, 3, 0, 1)
    assert np.abs(h - h.transpose(0, 1, 3, 2)).max() > 1e-3 * np.abs(h).max()
    g = np.random.default_rng(9)
    x, y = g.standard_normal((2,) + tiny.shape)
    np.testing.assert_allclose(mc(mc.approx_A(x)), x, atol=1e-12 * np.abs(x).max())
    assert np.vdot(x, mc.approx_A(y)) == pytest.approx(np.vdot(y, mc.approx_A(x)), rel=1e-12)
    mf = om.CirculantPrecon(tiny, pd_eps=0.5)
    lam = np.linalg.eigvalsh(np.linalg.inv(mf.h_inv))
    assert mf.n_clamped > 0 and lam.max() > 1.05
    assert lam.min() == pytest.approx(0.5 * lam.max(), rel=1e-10)


def test_circulant_beats_binned_on_drift_scan():
    """Sec. Results (context): on a drift scan with correlated noise the circulant
    preconditioner needs fewer iterations than the binned one."""
    scan = gen.small_scan(cfg=108, ny=24, nx=24, n_t=1 << 13, ncols=4, nrows=2, throw_px=36.0,
                          rot=20.0)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, cfg=108)
    op = om.make_operator(scan, noise)
    b = om.apply_A(op, gen.sky_map(24, 24, cfg=108))
    _, ib = om.pcg(lambda v: om.apply_A(op, v), om.BlockPrecon(op), b, tol=1e-6, maxit=500)
    _, ic = om.pcg(lambda v: om.apply_A(op, v), om.CirculantPrecon(op, taper_sigma=4.0), b,
                   tol=1e-6, maxit=500)
    assert ib.converged and ic.converged
    assert ic.iterations < ib.iterations
