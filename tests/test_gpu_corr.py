"""Noise correlated between detectors on the GPU (split filter pass, cross-detector
Woodbury solve, merge) against the FP64 oracle's per-bin definition."""
import numpy as np
import pytest

import gen
from oracle import mapmaker as om

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {1: 1e-5, 2: 2e-2}


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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def small(n_t=1 << 13, r=3):
    scan = gen.small_scan(cfg=311, ny=20, nx=18, n_t=n_t, ncols=4, nrows=2, throw_px=30.0)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=311)
    return scan, noise, gen.corr_noise(scan.det_off, r=r)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("r", [1, 3])
def test_apply_A_correlated_small(cmm, ctx, prec, r):
    scan, noise, corr = small(r=r)
    op = cmm.Operator(ctx, scan, noise, precision=prec, corr=corr)
    oop = om.make_operator(scan, noise, corr=corr)
    m = gen.random_maps(3, scan.ny, scan.nx, 1, cfg=312)[0]
    ref = om.apply_A(oop, m)
    assert rel(host(op.apply(dev(m))), ref) < TOL[prec]
    # the correlation matters at this tolerance, and removing it restores the independent operator
    assert rel(om.apply_A(om.make_operator(scan, noise), m), ref) > 0.05
    op.noise.set_correlated(None)
    assert rel(host(op.apply(dev(m))), om.apply_A(om.make_operator(scan, noise), m)) < TOL[prec]


def test_apply_A_correlated_act_patch_subset(cmm, ctx):
    full, fnoise = gen.act_patch(n_t=1 << 18)
    dets = np.array([0, 301, 602, 903, 17, 1023])
    scan, noise = full.subset(dets), fnoise.subset(dets)
    corr = gen.corr_noise(scan.det_off)
    op = cmm.Operator(ctx, scan, noise, precision=1, corr=corr)
    op.set_pixel_cache(True)
    oop = om.make_operator(scan, noise, corr=corr)
    m = gen.sky_map(scan.ny, scan.nx, cfg=2)
    assert rel(host(op.apply(dev(m))), om.apply_A(oop, m)) < TOL[1]


def test_correlated_symmetry_rhs_and_pcg(cmm, ctx):
    scan, noise = gen.tiny_patch()
    corr = gen.corr_noise(scan.det_off)
    op = cmm.Operator(ctx, scan, noise, precision=1, corr=corr)
    oop = om.make_operator(scan, noise, corr=corr)
    mask = op.pointing.mask()[0].reshape(scan.ny, scan.nx)
    x, y = gen.random_maps(3, scan.ny, scan.nx, 2, cfg=313)
    x[:, ~mask] = 0
    y[:, ~mask] = 0
    assert np.vdot(x, host(op.apply(dev(y)))) == pytest.approx(np.vdot(y, host(op.apply(dev(x)))), rel=1e-5)
    m = gen.sky_map(scan.ny, scan.nx, cfg=5)
    d = om.project(oop, m) + gen.corr_noise_tod(noise, corr, scan.n_t, scan.f_samp, cfg=314)
    b_ref = om.rhs(oop, d)
    b = op.rhs(torch.as_tensor(d, device="cuda:0"))
    assert rel(host(b), b_ref) < 1e-5
    pc = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=8.0)
    xs, info, _, _ = cmm.solve(op, pc, b, tol=1e-8, maxit=500)
    assert info.status == 0
    xo, io = om.pcg(lambda v: om.apply_A(oop, v), om.BlockPrecon(oop), b_ref, tol=1e-10, maxit=3000)
    assert rel(host(xs), xo) < 1e-4


def test_correlated_unsupported_cases(cmm, ctx):
    scan, noise, corr = small()
    with pytest.raises(cmm.CmmError):
        cmm.Operator(ctx, scan, noise, precision=0, corr=corr).apply(dev(np.zeros((3, scan.ny, scan.nx))))
    with pytest.raises(cmm.CmmError):
        cmm.Operator(ctx, scan, noise, precision=1, det_chunk=3, corr=corr).apply(
            dev(np.zeros((3, scan.ny, scan.nx))))
