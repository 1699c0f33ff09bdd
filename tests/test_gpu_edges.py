"""Edge and degenerate cases of the GPU path: white noise with T-only pointing
(A is the hit count), the generic kernels beyond the fast-path sizes, a single
detector, and inputs the library must reject."""
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


@pytest.mark.parametrize("prec,cached", [(0, False), (1, False), (1, True)])
def test_white_noise_T_only_is_hit_count(cmm, ctx, prec, cached):
    scan = gen.small_scan(cfg=341, ny=20, nx=22, n_t=1 << 13, ncomp=1, throw_px=30.0)
    noise = gen.Noise(np.full(scan.n_det, 2.0), np.zeros(scan.n_det), np.full(scan.n_det, 3.5))
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    if cached:
        op.set_pixel_cache(True)
    mask = op.pointing.mask()[0]
    pix = om.sample_pixels(scan, np.arange(scan.n_det)).ravel()
    pix = pix[(pix >= 0)]
    pix = pix[mask[pix]]
    hits = np.bincount(pix, minlength=scan.npix).astype(float)
    m = np.random.default_rng(1).standard_normal((1, scan.ny, scan.nx))
    y = op.apply(dev(m)).cpu().numpy().ravel()
    np.testing.assert_allclose(y, hits * m.ravel() / 4.0, rtol=0, atol=(1e-10 if prec == 0 else 1e-5) * hits.max())


def test_beyond_fast_path_sizes(cmm, ctx):
    """n_samp = 2^21 runs the generic FP32 kernels; parity with the oracle."""
    full, fnoise = gen.act_patch(n_t=1 << 21)
    dets = np.array([5, 700])
    scan, noise = full.subset(dets), fnoise.subset(dets)
    op = cmm.Operator(ctx, scan, noise, precision=1)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=2)
    assert rel(op.apply(dev(m)).cpu().numpy(), om.apply_A(oop, m)) < 1e-5


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_single_detector(cmm, ctx, prec):
    """One detector constrains T; with TQU its per-pixel blocks are rank one, every
    pixel fails the conditioning test and A is exactly zero (on both sides)."""
    full, fnoise = gen.tiny_patch(ncomp=1)
    scan, noise = full.subset(np.array([7])), fnoise.subset(np.array([7]))
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    oop = om.make_operator(scan, noise)
    m = gen.sky_map(scan.ny, scan.nx, cfg=3, ncomp=1)
    assert rel(op.apply(dev(m)).cpu().numpy(), om.apply_A(oop, m)) < {0: 1e-10, 1: 1e-5, 2: 2e-2}[prec]
    full3, _ = gen.tiny_patch()
    scan3 = full3.subset(np.array([7]))
    op3 = cmm.Operator(ctx, scan3, noise, precision=prec)
    assert op3.pointing.mask()[1] == 0 and not om.pixel_mask(scan3).any()
    assert not op3.apply(dev(gen.sky_map(scan3.ny, scan3.nx, cfg=3))).any()


def test_rejected_inputs(cmm, ctx):
    scan, noise = gen.tiny_patch()
    bad_nt = gen.small_scan(cfg=342, ny=8, nx=8, n_t=1000, ncols=2, nrows=1)   # not a power of two
    with pytest.raises(cmm.CmmError):
        cmm.Operator(ctx, bad_nt, gen.noise_params(bad_nt.n_det))
    far = scan.det_off.copy()
    far[0, 0] = 1 << 15   # detector offset beyond the exact fixed-point range
    with pytest.raises(cmm.CmmError):
        cmm.cmm_pointing_create(ctx.h, scan.ny, scan.nx, 3, False, far, scan.det_pol, scan.bore)
    with pytest.raises(cmm.CmmError):
        cmm.cmm_pointing_create(ctx.h, scan.ny, scan.nx, 2, False, scan.det_off, scan.det_pol, scan.bore)
    with pytest.raises(cmm.CmmError, match="map size"):   # beyond 2^28 pixels, before any allocation
        cmm.cmm_pointing_create(ctx.h, 1 << 14, (1 << 14) + 1, 3, False, scan.det_off, scan.det_pol, scan.bore)
    with pytest.raises(cmm.CmmError):
        cmm.cmm_noise_create(ctx.h, scan.n_t, scan.f_samp, np.array([-1.0]), np.array([1.0]), np.array([3.5]))
    op = cmm.Operator(ctx, scan, noise, precision=1)
    m = dev(np.zeros((3, scan.ny, scan.nx)))
    with pytest.raises(cmm.CmmError):
        cmm.cmm_apply_A(op.h, m, m)   # aliasing input and output


@pytest.mark.parametrize("prec", [0, 1])
def test_smallest_sample_count(cmm, ctx, prec):
    """n_samp = 64: the generic kernels at the bottom of the supported range."""
    scan = gen.small_scan(cfg=343, ny=6, nx=6, n_t=64, ncols=2, nrows=2, spacing_px=1.0, throw_px=5.0,
                          speed_px_s=120.0)
    noise = gen.noise_params(scan.n_det, fknee=20.0, alpha=2.0, scatter=0.2, cfg=343)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    oop = om.make_operator(scan, noise)
    m = gen.random_maps(3, scan.ny, scan.nx, 1, cfg=344)[0]
    ref = om.apply_A(oop, m)
    if np.linalg.norm(ref) > 0:
        assert rel(op.apply(dev(m)).cpu().numpy(), ref) < (1e-10 if prec == 0 else 1e-5)


def test_zero_rhs_solves_to_zero(cmm, ctx):
    scan, noise = gen.tiny_patch()
    op = cmm.Operator(ctx, scan, noise, precision=1)
    pc = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=8.0)
    b = dev(np.zeros((3, scan.ny, scan.nx)))
    x, info, _, _ = cmm.solve(op, pc, b, tol=1e-6, maxit=50)
    assert info.status == 0 and not x.any()
