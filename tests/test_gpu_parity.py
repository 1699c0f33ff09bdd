"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.

Error measure (`rel`): the larger of the norm-wise relative error
||gpu - oracle|| / ||oracle|| and the element-wise one, max |gpu - oracle| over
max |oracle|, so that a few wrong pixels (a map edge, a masked-pixel boundary, a
cut sample) cannot hide in the norm.  Solutions are also compared per Stokes
component over the unmasked pixels (`stokes_errors`).
Tolerances:
  FP64 mode: 1e-10 per operator; solutions 1e-5 (the target relative map error).
  FP32 mode: 1e-5 per operator.  BF16 spectrum storage: 2e-2 per operator.
  Where a pixel's FP32 partial sum takes well over a thousand samples, the
  rounding of that sum is added per element (`within_summation_bound`).
Integer work (pixel masks) must agree exactly.
"""
import functools
import importlib.util
import math
import os

import numpy as np
import pytest

import gen
from oracle import mapmaker as om

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_7473_gb300 import build
    build.build()
    from paper_1309_7473_gb300 import cmm as c
    return c


@pytest.fixture(scope="module")
def ctx(cmm):
    return cmm.Context(0)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    norm = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    elem = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) if b.size else 0.0
    return max(norm, elem)


def stokes_errors(x, ref, mask):
    """||x_c - ref_c|| / ||ref_c|| over the unmasked pixels, per map component."""
    x = np.asarray(x).reshape(len(ref), -1)[:, mask]
    r = np.asarray(ref).reshape(len(ref), -1)[:, mask]
    return [float(np.linalg.norm(x[c] - r[c]) / np.linalg.norm(r[c])) for c in range(len(r))]


def within_summation_bound(y, oop, m, prec, lam=6.0):
    """Element-wise check of an FP32/BF16 A m against the oracle with the rounding
    of the binning sums accounted for: |y_p - (A m)_p| <= TOL * max|A m|
    + lam sqrt(h_p) u S_p, u = 2^-24, h_p the samples hitting element p and S_p the
    sum of their absolute contributions (`om.binning_magnitude`).  The second term
    is the probabilistic bound of recursive summation (Higham and Mary, SIAM J. Sci.
    Comput. 41, 2019): h rounding errors of at most u times a partial sum, which is
    at most S_p, add up like a random walk; lam = 6 leaves a failure probability of
    order h exp(-lam^2 / 2).  A dropped or misplaced sample moves y_p by about
    S_p / h_p, far above the bound for any h_p the tests use."""
    ref = om.apply_A(oop, m)
    s, h = om.binning_magnitude(oop, m)
    bound = TOL[prec] * np.abs(ref).max() + lam * np.sqrt(h)[None] * 2.0 ** -24 * s
    err = np.abs(np.asarray(y, np.float64) - ref)
    worst = np.unravel_index(np.argmax(err - bound), err.shape)
    assert np.all(err <= bound), (worst, err[worst], bound[worst], int(h[worst[1:]]))


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


TOL = {0: 1e-10, 1: 1e-5, 2: 2e-2}
# the same operator through two kernel paths (cached against on-the-fly pointing)
SAME = {1: 1e-6, 2: 1e-4}


def small(ncomp=3, periodic=False, cfg=201):
    if periodic:
        scan = gen.bccb_scan(8, 16, 1024, diagonal=True, ncomp=ncomp)
        noise = gen.Noise(np.ones(scan.n_det), np.full(scan.n_det, 30.0), np.full(scan.n_det, 2.0))
        return scan, noise
    scan = gen.small_scan(cfg=cfg, ny=24, nx=20, n_t=1 << 12, ncols=4, nrows=2, throw_px=30.0,
                          ncomp=ncomp)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=cfg)
    return scan, noise


# ---------------------------------------------------------------- pointing / noise setup

@pytest.mark.parametrize("ncomp", [1, 3])
def test_mask_bit_exact(cmm, ctx, ncomp):
    for scan in (small(ncomp)[0], gen.tiny_patch(ncomp=ncomp)[0],
                 gen.small_scan(cfg=202, ny=16, nx=16, n_t=1 << 10, ncols=2, nrows=1, ncomp=ncomp)):
        pt = cmm.Pointing(ctx, scan)
        mask, n_good = pt.mask()
        ref = om.pixel_mask(scan)
        assert np.array_equal(mask, ref)
        assert n_good == int(ref.sum())


def test_noise_diagonal(cmm, ctx):
    scan, noise = gen.tiny_patch()
    nz = cmm.Noise(ctx, noise, scan.n_t, scan.f_samp)
    w = om.filter_weights(noise, scan.n_t, scan.f_samp)
    assert rel(nz.diag(), om.ninv_diagonal(w, scan.n_t)) < 1e-13
    wn = gen.Noise(np.array([2.0]), np.array([0.0]), np.array([3.5]))
    assert cmm.Noise(ctx, wn, 1024, 400.0).diag()[0] == pytest.approx(0.25, rel=1e-14)


# ---------------------------------------------------------------- operators

@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("ncomp", [1, 3])
@pytest.mark.parametrize("chunk", [0, 3])
def test_apply_A_small(cmm, ctx, prec, ncomp, chunk):
    scan, noise = small(ncomp)
    op = cmm.Operator(ctx, scan, noise, precision=prec, det_chunk=chunk)
    oop = om.make_operator(scan, noise)
    m = gen.random_maps(ncomp, scan.ny, scan.nx, 1, cfg=203)[0]
    y = host(op.apply(dev(m)))
    assert rel(y, om.apply_A(oop, m)) < TOL[prec]


def test_handles_destroyed_out_of_order(cmm):
    """An operator and preconditioner stay usable after the context, pointing and
    noise handles they were made from are destroyed first."""
    scan, noise = small(3)
    c = cmm.Context(0)
    op = cmm.Operator(c, scan, noise, precision=0)
    pc = cmm.Precon(op, cmm.PRECON_BINNED)
    for owner in (c, op.pointing, op.noise):
        {cmm.Context: cmm.cmm_ctx_destroy, cmm.Pointing: cmm.cmm_pointing_destroy,
         cmm.Noise: cmm.cmm_noise_destroy}[type(owner)](owner.h)
        owner.h = None
    oop = om.make_operator(scan, noise)
    m = gen.random_maps(3, scan.ny, scan.nx, 1, cfg=203)[0]
    y = host(op.apply(dev(m)))
    assert rel(y, om.apply_A(oop, m)) < TOL[0]
    cmm.cmm_op_destroy(op.h)
    op.h = None
    z = host(pc.apply(dev(y)))
    assert np.isfinite(z).all()
    cmm.cmm_precon_destroy(pc.h)
    pc.h = None


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("ncomp", [1, 3])
def test_pixel_cache_same_result(cmm, ctx, prec, ncomp):
    """A with the cached pixel indices equals A with on-the-fly pointing (same pixels;
    the forward pass on the fly forms (cos 2phi, sin 2phi) from the boresight record
    in FP32 where the cached one reads the FP32 table, and the FP32 atomic additions
    into the partial map come in another order), including samples outside the map:
    agreement to FP32 rounding, or to BF16 rounding with BF16 spectrum storage (a
    last-bit FP32 difference can move a value to the neighbouring BF16 number)."""
    scan = gen.small_scan(cfg=211, ny=20, nx=18, n_t=1 << 13, ncols=4, nrows=2, throw_px=40.0, ncomp=ncomp)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=211)
    op = cmm.Operator(ctx, scan, noise, precision=prec, det_chunk=3)
    m = dev(gen.random_maps(ncomp, scan.ny, scan.nx, 1, cfg=212)[0])
    y0 = host(op.apply(m))
    op.set_pixel_cache(True)
    y1 = host(op.apply(m))
    assert rel(y1, y0) < SAME[prec]
    op.set_pixel_cache(False)
    assert rel(host(op.apply(m)), y0) < SAME[prec]
    oop = om.make_operator(scan, noise)
    assert rel(y1, om.apply_A(oop, gen.random_maps(ncomp, scan.ny, scan.nx, 1, cfg=212)[0])) < TOL[prec]


def test_pixel_cache_rejected_where_unsupported(cmm, ctx):
    scan, noise = small(3)
    with pytest.raises(cmm.CmmError):
        cmm.Operator(ctx, scan, noise, precision=0).set_pixel_cache(True)
    scan, noise = small(3, periodic=True)
    with pytest.raises(cmm.CmmError):
        cmm.Operator(ctx, scan, noise, precision=1).set_pixel_cache(True)


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_A_periodic(cmm, ctx, prec):
    scan, noise = small(3, periodic=True)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    oop = om.make_operator(scan, noise)
    m = gen.random_maps(3, scan.ny, scan.nx, 1, cfg=204)[0]
    assert rel(host(op.apply(dev(m))), om.apply_A(oop, m)) < TOL[prec]


@pytest.mark.parametrize("pair", [True, False])
@pytest.mark.parametrize("prec", [1, 2])
def test_apply_A_periodic_fast_path(cmm, ctx, prec, pair):
    """The periodic-boundary instances of the register-FFT kernels (2^13 samples on
    the wrapping scan), in both FFT packings, element-wise against the oracle.

    The 8x16 map takes 1536 samples per pixel, all in one FP32 partial sum (24
    detectors, one flush group), a deeper FP32 summation than anywhere else in
    these tests, so the bound is per element (`within_summation_bound`)."""
    scan = gen.bccb_scan(8, 16, 1 << 13, diagonal=True, ncomp=3)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=215)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    op.set_pair_packing(pair)
    oop = om.make_operator(scan, noise)
    m = gen.random_maps(3, scan.ny, scan.nx, 1, cfg=216)[0]
    within_summation_bound(host(op.apply(dev(m))), oop, m, prec)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_apply_A_tiny_patch(cmm, ctx, prec):
    scan, noise = gen.tiny_patch()
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=1)
    y = host(op.apply(dev(m)))
    ref = om.apply_A(oop, m)
    assert rel(y, ref) < TOL[prec]
    # host-buffer entry point gives the same numbers
    out = np.empty_like(m)
    cmm.cmm_apply_A_host(op.h, m, out)
    assert rel(out, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_project_and_rhs(cmm, ctx, prec):
    scan, noise = small(3)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=205)
    tod_ref = om.project(oop, m)
    tod = host(op.project(dev(m), dtype=torch.float64))
    assert rel(tod, tod_ref) < (1e-13 if prec == 0 else 1e-6)
    d = tod_ref + gen.noise_tod(noise, scan.n_t, scan.f_samp, cfg=205)
    for dt in (torch.float64, torch.float32):
        dd = torch.as_tensor(d, dtype=dt, device="cuda:0")
        b = host(op.rhs(dd))
        dref = d if dt == torch.float64 else d.astype(np.float32).astype(np.float64)
        assert rel(b, om.rhs(oop, dref)) < TOL[prec]


def test_A_symmetric_on_gpu(cmm, ctx):
    scan, noise = gen.tiny_patch()
    op = cmm.Operator(ctx, scan, noise, precision=0)
    x, y = gen.random_maps(3, scan.ny, scan.nx, 2, cfg=206)
    mask = op.pointing.mask()[0].reshape(scan.ny, scan.nx)
    x[:, ~mask] = 0
    y[:, ~mask] = 0
    ax = host(op.apply(dev(x)))
    ay = host(op.apply(dev(y)))
    assert np.vdot(x, ay) == pytest.approx(np.vdot(y, ax), rel=1e-12)


# ---------------------------------------------------------------- preconditioners

@pytest.mark.parametrize("kind", ["binned", "jacobi"])
@pytest.mark.parametrize("ncomp", [1, 3])
def test_block_precon(cmm, ctx, kind, ncomp):
    scan, noise = small(ncomp)
    op = cmm.Operator(ctx, scan, noise, precision=0)
    oop = om.make_operator(scan, noise)
    k = cmm.PRECON_BINNED if kind == "binned" else cmm.PRECON_JACOBI
    pc = cmm.Precon(op, k)
    r = gen.random_maps(ncomp, scan.ny, scan.nx, 1, cfg=207)[0]
    assert rel(host(pc.apply(dev(r))), om.BlockPrecon(oop, kind)(r)) < 1e-11


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("ncomp", [1, 3])
@pytest.mark.parametrize("taper", [math.inf, 3.0])
def test_circulant_precon(cmm, ctx, prec, ncomp, taper):
    scan, noise = small(ncomp)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    oop = om.make_operator(scan, noise)
    pc = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=taper if math.isfinite(taper) else 0.0)
    ref = om.CirculantPrecon(oop, taper_sigma=taper)
    r = gen.random_maps(ncomp, scan.ny, scan.nx, 1, cfg=208)[0]
    err = rel(host(pc.apply(dev(r))), ref(r))
    print(f"circulant apply, precision {prec}, ncomp {ncomp}, taper {taper}: error {err:.2e}")
    # FP32 operator: the map FFTs of the apply run in FP32 (measured 1.7e-7 to 1.9e-7)
    assert err < (1e-9 if prec == 0 else 1e-5)
    if prec == 0:
        assert pc.clamped() == ref.n_clamped


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", [(27, 25), (30, 45)])
def test_circulant_precon_odd_and_mixed_sides(cmm, ctx, prec, shape):
    """Maps whose sides are odd (27 x 25: radices 3 and 5 only, every Fourier mode but
    the zero one paired with a distinct mirror) or mixed (30 x 45): the line FFTs'
    radix passes and the TQU packing of the apply into two complex planes."""
    ny, nx = shape
    scan = gen.small_scan(cfg=231, ny=ny, nx=nx, n_t=1 << 12, ncols=4, nrows=2, throw_px=1.2 * nx, ncomp=3)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=231)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    oop = om.make_operator(scan, noise)
    pc = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=3.0)
    ref = om.CirculantPrecon(oop, taper_sigma=3.0)
    r = gen.random_maps(3, ny, nx, 1, cfg=232)[0]
    err = rel(host(pc.apply(dev(r))), ref(r))
    print(f"circulant apply {ny}x{nx}, precision {prec}: error {err:.2e}")
    assert err < (1e-9 if prec == 0 else 1e-5)


@pytest.mark.parametrize("ncomp", [1, 3])
def test_white_level_weights(cmm, ctx, ncomp):
    """The alternative reading of diag(N^-1) in Eq. 3 and Eq. 7 (white level
    1/sigma_d^2) against the oracle, binned and circulant, and unlike the default."""
    scan, noise = small(ncomp)
    op = cmm.Operator(ctx, scan, noise, precision=0)
    oop = om.make_operator(scan, noise)
    r = gen.random_maps(ncomp, scan.ny, scan.nx, 1, cfg=212)[0]
    zb = host(cmm.Precon(op, cmm.PRECON_BINNED, white_diag=True).apply(dev(r)))
    assert rel(zb, om.BlockPrecon(oop, "binned", white=True)(r)) < 1e-11
    assert rel(zb, host(cmm.Precon(op, cmm.PRECON_BINNED).apply(dev(r)))) > 1e-3
    zc = host(cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=3.0, white_diag=True).apply(dev(r)))
    assert rel(zc, om.CirculantPrecon(oop, taper_sigma=3.0, white=True)(r)) < 1e-9


def test_circulant_exact_on_bccb_gpu(cmm, ctx):
    scan, noise = small(3, periodic=True)
    op = cmm.Operator(ctx, scan, noise, precision=0)
    pc = cmm.Precon(op, cmm.PRECON_CIRCULANT)
    x = gen.random_maps(3, scan.ny, scan.nx, 1, cfg=209)[0]
    b = op.apply(dev(x))
    assert rel(host(pc.apply(b)), x) < 1e-10
    sol, info, _, _ = cmm.solve(op, pc, b, tol=1e-9, maxit=20)
    assert info.status == 0 and info.iterations == 1
    assert rel(host(sol), x) < 1e-9


# ---------------------------------------------------------------- solves

@pytest.mark.parametrize("graph", [True, False])
def test_pcg_binned_tiny_patch_matches_oracle(cmm, ctx, graph):
    scan, noise = gen.tiny_patch()
    op = cmm.Operator(ctx, scan, noise, precision=0)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=1)
    d = om.project(oop, m)
    b_ref = om.rhs(oop, d)
    b = op.rhs(torch.as_tensor(d, device="cuda:0"))
    assert rel(host(b), b_ref) < 1e-10
    pc = cmm.Precon(op, cmm.PRECON_BINNED)
    x, info, hist, terms = cmm.solve(op, pc, b, tol=1e-10, maxit=400, use_graph=graph, history=True)
    assert info.status == 0
    xo, io = om.pcg(lambda v: om.apply_A(oop, v), om.BlockPrecon(oop), b_ref, tol=1e-10, maxit=400)
    assert rel(host(x), xo) < 1e-5
    assert max(stokes_errors(host(x), xo, oop.mask)) < 1e-5
    assert abs(info.iterations - io.iterations) <= max(2, 0.1 * io.iterations)
    h = host(hist)[: info.iterations + 1]
    np.testing.assert_allclose(h[:10], io.rel_resid[:10], rtol=1e-6)
    t = host(terms)[: info.iterations]
    np.testing.assert_allclose(t[:10], io.anorm_terms[:10], rtol=1e-6)
    # noise-free data: the solution is the input map on unmasked pixels
    assert rel(host(x), m) < 1e-6
    # the exit check ||b - A x|| / ||b|| against the oracle's A on the returned x
    true_o = np.linalg.norm(b_ref - om.apply_A(oop, host(x))) / np.linalg.norm(b_ref)
    assert info.true_rel_resid < 1e-9
    assert info.true_rel_resid == pytest.approx(true_o, rel=0.2)


def test_pcg_circulant_tiny_patch(cmm, ctx):
    scan, noise = gen.tiny_patch()
    op = cmm.Operator(ctx, scan, noise, precision=0)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=1)
    b_ref = om.apply_A(oop, m)
    b = dev(b_ref)
    pc = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=8.0)
    x, info, _, _ = cmm.solve(op, pc, b, tol=1e-6, maxit=400)
    xo, io = om.pcg(lambda v: om.apply_A(oop, v), om.CirculantPrecon(oop, taper_sigma=8.0), b_ref,
                    tol=1e-6, maxit=400)
    assert info.status == 0 and io.converged
    assert abs(info.iterations - io.iterations) <= max(2, 0.1 * io.iterations)
    assert rel(host(x), xo) < 1e-5
    assert max(stokes_errors(host(x), xo, oop.mask)) < 1e-5
    assert info.rel_resid <= 1e-6 and info.true_rel_resid < 2e-6
    _, info2, _, _ = cmm.solve(op, pc, b, tol=1e-6, maxit=400, true_resid=False)
    assert info2.iterations == info.iterations and info2.true_rel_resid == -1.0


# ---------------------------------------------------------------- fast-path sizes
# The FP32 kernels with register-resident FFTs serve n_samp = 2^13 .. 2^20; these
# cases run them on the ACT-like focal plane at the bench's per-detector sizes
# (2^20 samples = the launch configuration of the 1024-detector bench) on a few
# detectors spread over the focal plane, which the oracle evaluates in seconds.

@pytest.mark.parametrize("pair", [True, False])
@pytest.mark.parametrize("log_nt", [13, 14, 15, 16, 17, 18, 19, 20])
@pytest.mark.parametrize("prec", [1, 2])
def test_apply_A_fast_path_sizes(cmm, ctx, log_nt, prec, pair):
    """Every size of the register-FFT kernels, with the two-detector packing (the
    default; the five detectors and chunks of two leave one detector alone in its
    last pair) and with the one-detector packing."""
    full, fnoise = gen.act_patch(n_t=1 << log_nt)
    dets = np.array([0, 300, 611, 1023, 17])
    scan, noise = full.subset(dets), fnoise.subset(dets)
    op = cmm.Operator(ctx, scan, noise, precision=prec, det_chunk=2)
    op.set_pair_packing(pair)
    oop = om.make_operator(scan, noise)
    assert np.array_equal(op.pointing.mask()[0], oop.mask)
    m = gen.sky_map(scan.ny, scan.nx, cfg=2)
    y = host(op.apply(dev(m)))
    assert rel(y, om.apply_A(oop, m)) < TOL[prec]
    op.set_pixel_cache(True)
    assert rel(host(op.apply(dev(m))), y) < SAME[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_A_turnaround_scan(cmm, ctx, prec):
    """ACT-like patch detectors on the scan with finite-acceleration turnarounds."""
    full, fnoise = gen.act_patch(n_t=1 << 18, accel_deg_s2=1.5)
    dets = np.array([3, 500, 1000])
    scan, noise = full.subset(dets), fnoise.subset(dets)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=2)
    assert rel(host(op.apply(dev(m))), om.apply_A(oop, m)) < TOL[prec]


@pytest.mark.parametrize("ncomp", [1, 3])
def test_apply_A_fast_small_ragged(cmm, ctx, ncomp):
    scan = gen.small_scan(cfg=210, ny=30, nx=22, n_t=1 << 13, ncols=5, nrows=1, throw_px=33.0, ncomp=ncomp)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=210)
    oop = om.make_operator(scan, noise)
    m = gen.random_maps(ncomp, scan.ny, scan.nx, 1, cfg=210)[0]
    ref = om.apply_A(oop, m)
    for chunk in (0, 2, 3):
        op = cmm.Operator(ctx, scan, noise, precision=1, det_chunk=chunk)
        assert rel(host(op.apply(dev(m))), ref) < TOL[1]
        op.set_pair_packing(False)
        assert rel(host(op.apply(dev(m))), ref) < TOL[1]


@functools.lru_cache(maxsize=None)
def _flush_case(log_nt):
    full, fnoise = gen.act_patch(n_t=1 << log_nt)
    dets = np.arange(0, 1024, 3)[:320]
    scan, noise = full.subset(dets), fnoise.subset(dets)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=2)
    return scan, noise, oop, m, om.apply_A(oop, m)


@pytest.mark.parametrize("pair", [True, False])
@pytest.mark.parametrize("log_nt", [13, 15, 18])
@pytest.mark.parametrize("prec", [1, 2])
def test_apply_A_flush_groups(cmm, ctx, log_nt, prec, pair):
    """320 ACT-like detectors in one chunk (det_chunk = 0), as the 1024-detector
    launch: the binning pass bins two groups (256 + 64 detectors) in one launch,
    each into its own FP32 partial map, and one flush adds both into the FP64
    accumulator.
    Element-wise against the oracle, on-the-fly and cached pointing; 2^18 samples
    use the 256-point column FFTs of the bench's size."""
    scan, noise, oop, m, ref = _flush_case(log_nt)
    op = cmm.Operator(ctx, scan, noise, precision=prec, det_chunk=0)
    op.set_pair_packing(pair)
    assert np.array_equal(op.pointing.mask()[0], oop.mask)
    assert rel(host(op.apply(dev(m))), ref) < TOL[prec]
    op.set_pixel_cache(True)
    assert rel(host(op.apply(dev(m))), ref) < TOL[prec]


def _golden_act_mask():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "act_patch_mask.py")
    spec = importlib.util.spec_from_file_location("act_patch_mask", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.load()


@pytest.mark.parametrize("pair", [True, False])
@pytest.mark.parametrize("prec", [1, 2])
def test_full_size_sampled_detectors_match_oracle(cmm, ctx, prec, pair):
    """The bench's workload in its launch configuration (1024 detectors x 2^20
    samples in one chunk, 1200x900 TQU, FP32 compute, on-the-fly and cached
    pointing) against the oracle on sampled detectors: every detector but four
    gets sigma = 1e25, whose weight 1/sigma^2 rounds to zero in FP32, so the full
    launch computes A restricted to the four, which the oracle evaluates with the
    full patch's pixel mask (tests/golden/act_patch_mask.json, written by the
    oracle).  The GPU's mask of all 1024 detectors must equal it bit for bit."""
    scan, noise = gen.act_patch()
    mask, doc = _golden_act_mask()
    keep = np.array([0, 341, 682, 1023])
    sigma = np.full(scan.n_det, 1e25)
    sigma[keep] = noise.sigma[keep]
    op = cmm.Operator(ctx, scan, gen.Noise(sigma, noise.fknee, noise.alpha), precision=prec)
    op.set_pair_packing(pair)
    gmask, n_good = op.pointing.mask()
    assert n_good == doc["n_good"] and np.array_equal(gmask, mask)
    oop = om.make_operator(scan.subset(keep), noise.subset(keep), mask=mask)
    m = gen.sky_map(scan.ny, scan.nx, cfg=2)
    ref = om.apply_A(oop, m)
    assert rel(host(op.apply(dev(m))), ref) < TOL[prec]
    op.set_pixel_cache(True)
    assert rel(host(op.apply(dev(m))), ref) < TOL[prec]


@pytest.fixture(scope="module")
def act_map_solution():
    """The ACT-like patch's 1200x900 map with 16 of its detectors at 2^18 samples,
    noise-free data: the oracle's binned-PCG solution converged to 1e-10."""
    full, fnoise = gen.act_patch(n_t=1 << 18)
    dets = np.linspace(0, 1023, 16).astype(int)
    scan, noise = full.subset(dets), fnoise.subset(dets)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=2)
    d = om.project(oop, m)
    b = om.rhs(oop, d)
    x, info = om.pcg(lambda v: om.apply_A(oop, v), om.BlockPrecon(oop), b, tol=1e-10, maxit=500)
    assert info.converged
    return scan, noise, oop, d, b, x, info


@pytest.mark.parametrize("kind", ["binned", "circulant"])
def test_full_map_solve_matches_oracle(cmm, ctx, act_map_solution, kind):
    """Solve on the full 1200x900 map (FP64 operator, PCG to 1e-10): the relative
    map error against the oracle's solution is below 1e-5 in each Stokes component
    over the unmasked pixels (the oracle's PCG used the binned preconditioner; the
    solution does not depend on the preconditioner)."""
    scan, noise, oop, d, b_ref, xo, io = act_map_solution
    op = cmm.Operator(ctx, scan, noise, precision=0)
    assert np.array_equal(op.pointing.mask()[0], oop.mask)
    b = op.rhs(torch.as_tensor(d, device="cuda:0"))
    assert rel(host(b), b_ref) < 1e-10
    pc = (cmm.Precon(op, cmm.PRECON_BINNED) if kind == "binned"
          else cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=10.0))
    x, info, _, _ = cmm.solve(op, pc, b, tol=1e-10, maxit=500)
    assert info.status == 0
    errs = stokes_errors(host(x), xo, oop.mask)
    print(f"full-map {kind} solve: {info.iterations} it (oracle binned {io.iterations}), "
          f"error per Stokes T/Q/U {errs[0]:.2e} {errs[1]:.2e} {errs[2]:.2e}")
    assert max(errs) < 1e-5
    if kind == "binned":
        assert abs(info.iterations - io.iterations) <= max(2, 0.1 * io.iterations)


def test_full_map_solve_f32_operator(cmm, ctx, act_map_solution):
    """The same solve with the FP32 operator (FP64 CG) stopped at a residual of 1e-6:
    its error per Stokes component against the oracle's tightly converged solution
    is that of the FP64 operator stopped at the same residual (the CG truncation,
    larger in Q and U, whose maps are ten times weaker than T) plus at most 2e-5,
    and below 1e-4 (measured: FP64 3.3e-6 / 4.5e-5 / 3.4e-5 in T / Q / U, the FP32
    operator 1.1e-5 more in Q)."""
    scan, noise, oop, d, b_ref, xo, io = act_map_solution
    errs = {}
    for prec in (0, 1):
        op = cmm.Operator(ctx, scan, noise, precision=prec)
        dt = torch.float64 if prec == 0 else torch.float32
        b = op.rhs(torch.as_tensor(d, dtype=dt, device="cuda:0"))
        pc = cmm.Precon(op, cmm.PRECON_BINNED)
        x, info, _, _ = cmm.solve(op, pc, b, tol=1e-6, maxit=500)
        assert info.status == 0
        errs[prec] = stokes_errors(host(x), xo, oop.mask)
        print(f"full-map solve to 1e-6, precision {prec}: {info.iterations} it, error per Stokes T/Q/U "
              f"{errs[prec][0]:.2e} {errs[prec][1]:.2e} {errs[prec][2]:.2e}")
    assert max(errs[1]) < 1e-4
    for c in range(3):
        assert errs[1][c] <= errs[0][c] + 2e-5


def test_full_size_symmetry_and_rhs(cmm, ctx):
    """At the bench's full size (1024 x 2^20, 1200x900): x^T A y = y^T A x, and the
    right-hand side of noise-free data P m equals A m."""
    scan, noise = gen.act_patch()
    op = cmm.Operator(ctx, scan, noise, precision=1)
    x, y = gen.random_maps(3, scan.ny, scan.nx, 2, cfg=211)
    mask = op.pointing.mask()[0].reshape(scan.ny, scan.nx)
    x[:, ~mask] = 0
    y[:, ~mask] = 0
    xd, yd = dev(x), dev(y)
    ax, ay = host(op.apply(xd)), host(op.apply(yd))
    assert np.vdot(x, ay) == pytest.approx(np.vdot(y, ax), rel=1e-5)
    m = dev(gen.sky_map(scan.ny, scan.nx, cfg=2))
    b1 = host(op.rhs(op.project(m, dtype=torch.float32)))
    b2 = host(op.apply(m))
    assert rel(b1, b2) < 1e-5
    op.set_pixel_cache(True)
    assert rel(host(op.apply(m)), b2) < 1e-6


# ---------------------------------------------------------------- precision modes (tiny patch)

@pytest.fixture(scope="module")
def tiny_solution():
    """Tiny patch, noise-free data: the FP64 oracle's tightly converged solution."""
    scan, noise = gen.tiny_patch()
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=1)
    d = om.project(oop, m)
    b = om.rhs(oop, d)
    x, info = om.pcg(lambda v: om.apply_A(oop, v), om.BlockPrecon(oop), b, tol=1e-11, maxit=2000)
    assert info.converged
    return scan, noise, d, b, x, info


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("cg_f32", [False, True])
def test_precision_grid_tiny_patch(cmm, ctx, tiny_solution, prec, cg_f32):
    """TOD/filter in FP32 or BF16 storage x CG in FP64 or FP32 with residual
    replacement every 50 iterations: converges to 1e-6 with the stated errors."""
    scan, noise, d, b_ref, x_ref, info_ref = tiny_solution
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    b = op.rhs(torch.as_tensor(d, dtype=torch.float32, device="cuda:0"))
    pc = cmm.Precon(op, cmm.PRECON_BINNED)
    x, info, _, _ = cmm.solve(op, pc, b, tol=1e-6, maxit=600, cg_f32=cg_f32,
                              resid_replace=50 if cg_f32 else 0)
    assert info.status == 0
    err = rel(host(x), x_ref)
    _, io = om.pcg(lambda v: om.apply_A(om.make_operator(scan, noise), v), om.BlockPrecon(om.make_operator(scan, noise)),
                   b_ref, tol=1e-6, maxit=600)
    assert abs(info.iterations - io.iterations) <= 0.2 * io.iterations + 2
    assert err < (2e-5 if prec == 1 else 2e-2)


def test_flexible_cg_matches_pcg_gpu(cmm, ctx, tiny_solution):
    scan, noise, d, b_ref, x_ref, _ = tiny_solution
    op = cmm.Operator(ctx, scan, noise, precision=0)
    pc = cmm.Precon(op, cmm.PRECON_BINNED)
    b = dev(b_ref)
    x1, i1, _, _ = cmm.solve(op, pc, b, tol=1e-9, maxit=600)
    x2, i2, _, _ = cmm.solve(op, pc, b, tol=1e-9, maxit=600, flexible=True)
    assert i1.status == 0 and i2.status == 0
    assert abs(i1.iterations - i2.iterations) <= 1
    assert rel(host(x2), host(x1)) < 1e-7
    assert rel(host(x1), x_ref) < 1e-6


@pytest.mark.parametrize("window", [2, 8])
def test_fcg_window_matches_oracle(cmm, ctx, tiny_solution, window):
    """Truncated flexible CG, FCG(m), with a fixed preconditioner (binned, FP64): the
    same residual history and solution as the oracle's FCG(m), which itself follows
    PCG for a fixed preconditioner."""
    scan, noise, d, b_ref, x_ref, _ = tiny_solution
    op = cmm.Operator(ctx, scan, noise, precision=0)
    oop = om.make_operator(scan, noise)
    pc = cmm.Precon(op, cmm.PRECON_BINNED)
    x, info, hist, _ = cmm.solve(op, pc, dev(b_ref), tol=1e-9, maxit=600, flexible=True, window=window,
                                 history=True)
    xo, io = om.pcg(lambda v: om.apply_A(oop, v), om.BlockPrecon(oop), b_ref, tol=1e-9, maxit=600,
                    flexible=True, window=window)
    assert info.status == 0 and io.converged
    assert abs(info.iterations - io.iterations) <= 1
    np.testing.assert_allclose(host(hist)[:15], io.rel_resid[:15], rtol=1e-6)
    assert rel(host(x), xo) < 1e-7
    assert max(stokes_errors(host(x), x_ref, oop.mask)) < 1e-5
    with pytest.raises(cmm.CmmError):
        cmm.solve(op, pc, dev(b_ref), tol=1e-9, maxit=10, flexible=True, window=9)


# ---------------------------------------------------------------- batched solves and tuning (uneven problems)

def test_batch_solve_matches_individual_solves(cmm):
    """Uneven problems solved together in one graph per check interval give the same
    iterates as solving each alone (FP64), and the oracle's solutions."""
    probs = []
    for k, (ny, nx, log_nt, ncols) in enumerate([(16, 20, 12, 3), (24, 18, 13, 4), (12, 12, 11, 2)]):
        scan = gen.small_scan(cfg=220 + k, ny=ny, nx=nx, n_t=1 << log_nt, ncols=ncols, nrows=2,
                              throw_px=1.5 * nx)
        noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=220 + k)
        probs.append((scan, noise))
    ops, pcs, bs, xs, refs = [], [], [], [], []
    for k, (scan, noise) in enumerate(probs):
        ctx = cmm.Context(0)
        op = cmm.Operator(ctx, scan, noise, precision=0)
        oop = om.make_operator(scan, noise)
        b_ref = om.apply_A(oop, gen.sky_map(scan.ny, scan.nx, cfg=230 + k))
        kind = cmm.PRECON_CIRCULANT if k != 1 else cmm.PRECON_BINNED
        pc = cmm.Precon(op, kind, taper_sigma_px=4.0)
        ops.append(op)
        pcs.append(pc)
        bs.append(dev(b_ref))
        xs.append(op.new_map())
        mo = om.CirculantPrecon(oop, taper_sigma=4.0) if k != 1 else om.BlockPrecon(oop)
        refs.append(om.pcg(lambda v, oop=oop: om.apply_A(oop, v), mo, b_ref, tol=1e-9, maxit=500))
    infos = cmm.cmm_batch_solve([o.h for o in ops], [p.h for p in pcs], bs, xs, tol=1e-9, maxit=500,
                                check_every=7)
    # the same with two lanes (one solve after another inside a lane)
    xs2 = [op.new_map() for op in ops]
    infos2 = cmm.cmm_batch_solve([o.h for o in ops], [p.h for p in pcs], bs, xs2, tol=1e-9, maxit=500,
                                 check_every=5, width=2)
    for k in range(len(ops)):
        assert infos2[k].iterations == infos[k].iterations
        assert rel(host(xs2[k]), host(xs[k])) < 1e-12
    for k in range(len(ops)):
        xi, ii, _, _ = cmm.solve(ops[k], pcs[k], bs[k], tol=1e-9, maxit=500)
        assert infos[k].status == 0 and ii.status == 0
        assert infos[k].iterations == ii.iterations
        assert rel(host(xs[k]), host(xi)) < 1e-12
        xo, io = refs[k]
        assert abs(infos[k].iterations - io.iterations) <= max(2, 0.1 * io.iterations)
        assert rel(host(xs[k]), xo) < 1e-6
        assert infos[k].true_rel_resid < 1e-8
        assert infos[k].true_rel_resid == pytest.approx(ii.true_rel_resid, rel=0.05, abs=1e-11)


def test_autotune_keeps_parity(cmm, ctx, tmp_path):
    """The tuner times the two-detector packing and the one-detector splits, keeps the
    fastest (parity holds either way) and remembers it in its file cache."""
    scan, noise = gen.tiny_patch()
    op = cmm.Operator(ctx, scan, noise, precision=1)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=1)
    ref = om.apply_A(oop, m)
    cache = str(tmp_path / "tune.txt")
    lr, pair, ms = cmm.cmm_autotune(op.h, 3, cache)
    assert 6 <= lr <= 8 and ms > 0
    assert rel(host(op.apply(dev(m))), ref) < TOL[1]
    op2 = cmm.Operator(ctx, scan, noise, precision=1)
    lr2, pair2, ms2 = cmm.cmm_autotune(op2.h, 3, cache)
    assert (lr2, pair2) == (lr, pair) and ms2 == -1.0
    assert rel(host(op2.apply(dev(m))), ref) < TOL[1]
    assert open(cache).read().split()[-1] == ("0" if pair else str(lr))


# ---------------------------------------------------------------- tiled circulant (next row 3)

@pytest.mark.parametrize("prec", [0, 1])
def test_tiled_circulant_matches_oracle(cmm, ctx, prec):
    scan, noise = small(3)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    oop = om.make_operator(scan, noise)
    r = gen.random_maps(3, scan.ny, scan.nx, 1, cfg=331)[0]
    r[:, ~oop.mask.reshape(scan.ny, scan.nx)] = 0
    ref = om.TiledCirculantPrecon(oop, tiles=(2, 3), taper_sigma=4.0)(r)
    pc = cmm.Precon(op, cmm.PRECON_CIRC_TILED, taper_sigma_px=4.0, tiles=(2, 3))
    assert rel(host(pc.apply(dev(r))), ref) < (1e-9 if prec == 0 else 2e-5)
    one = cmm.Precon(op, cmm.PRECON_CIRC_TILED, taper_sigma_px=4.0, tiles=(1, 1))
    circ = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=4.0)
    assert rel(host(one.apply(dev(r))), host(circ.apply(dev(r)))) < 1e-12


def test_tiled_circulant_pcg_tiny_patch(cmm, ctx):
    scan, noise = gen.tiny_patch()
    op = cmm.Operator(ctx, scan, noise, precision=0)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=332)
    b_ref = om.apply_A(oop, m)
    pc = cmm.Precon(op, cmm.PRECON_CIRC_TILED, taper_sigma_px=8.0, tiles=(2, 2))
    x, info, _, _ = cmm.solve(op, pc, dev(b_ref), tol=1e-10, maxit=500)
    assert info.status == 0
    xo, io = om.pcg(lambda v: om.apply_A(oop, v), om.TiledCirculantPrecon(oop, tiles=(2, 2), taper_sigma=8.0),
                    b_ref, tol=1e-10, maxit=500)
    assert abs(info.iterations - io.iterations) <= 2
    assert rel(host(x), xo) < 1e-8
