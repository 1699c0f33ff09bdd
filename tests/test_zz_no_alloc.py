"""cmm_apply_A_noalloc (A with its temporaries in the library's static scratch
array) against the FP64 oracle, and against cmm_apply_A on the same operator and
map over consecutive calls that leave the shared array holding another operator's
data in between.

Collected last so it also runs after every other GPU test in one process; it
builds its own context and passes alone in a fresh process too.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# same tolerances as the A-application parity tests: F64 1e-10, F32 1e-5
TOL = {0: 1e-10, 1: 1e-5}


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
    return float((a - b).norm() / b.norm())


def operator(cmm, ctx, prec, ncomp, cfg, ny, nx, n_t, chunk=0):
    scan = gen.small_scan(cfg=cfg, ny=ny, nx=nx, n_t=n_t, ncols=4, nrows=2, throw_px=30.0, ncomp=ncomp)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=cfg)
    return cmm.Operator(ctx, scan, noise, precision=prec, det_chunk=chunk), scan


def maps(scan, cfg):
    m = gen.random_maps(scan.ncomp, scan.ny, scan.nx, 1, cfg=cfg)[0]
    return torch.as_tensor(np.ascontiguousarray(m), dtype=torch.float64, device="cuda:0")


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_apply_A_on_consecutive_calls(cmm, ctx, prec):
    op1, s1 = operator(cmm, ctx, prec, 3, 301, 24, 20, 1 << 12, chunk=3)
    op2, s2 = operator(cmm, ctx, prec, 1, 302, 40, 36, 1 << 13)
    m1, m2 = maps(s1, 303), maps(s2, 304)
    ref1, ref2 = op1.apply(m1), op2.apply(m2)
    for _ in range(2):
        for op, m, ref in ((op1, m1, ref1), (op2, m2, ref2)):
            out = torch.full_like(ref, float("nan"))
            cmm.cmm_apply_A_noalloc(op.h, m, out)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert rel(out, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_oracle(cmm, ctx, prec):
    """Against the FP64 oracle itself, on the scan and map of the small A-application
    parity test, with its error measure (the larger of the norm-wise and the
    element-wise relative error)."""
    from oracle import mapmaker as om
    scan = gen.small_scan(cfg=201, ny=24, nx=20, n_t=1 << 12, ncols=4, nrows=2, throw_px=30.0, ncomp=3)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=201)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    m = gen.random_maps(3, scan.ny, scan.nx, 1, cfg=203)[0]
    out = torch.full((3, scan.ny, scan.nx), float("nan"), dtype=torch.float64, device="cuda:0")
    cmm.cmm_apply_A_noalloc(op.h, torch.as_tensor(np.ascontiguousarray(m), dtype=torch.float64, device="cuda:0"),
                            out)
    torch.cuda.synchronize()
    y, ref = out.cpu().numpy(), om.apply_A(om.make_operator(scan, noise), m)
    err = max(np.linalg.norm(y - ref) / np.linalg.norm(ref), np.abs(y - ref).max() / np.abs(ref).max())
    assert err < TOL[prec]


def test_noalloc_tiny_patch(cmm, ctx):
    scan, noise = gen.tiny_patch()
    op = cmm.Operator(ctx, scan, noise, precision=1)
    m = maps(scan, 305)
    ref = op.apply(m)
    for _ in range(2):
        out = torch.zeros_like(ref)
        cmm.cmm_apply_A_noalloc(op.h, m, out)
        torch.cuda.synchronize()
        assert rel(out, ref) < TOL[1]


def test_noalloc_rejects_oversize(cmm, ctx):
    # a 1024 x 1024 TQU map needs 64 MiB of map buffers alone
    op, scan = operator(cmm, ctx, 1, 3, 306, 1024, 1024, 1 << 10)
    m = torch.zeros((3, 1024, 1024), dtype=torch.float64, device="cuda:0")
    out = torch.zeros_like(m)
    with pytest.raises(cmm.CmmError, match="static scratch"):
        cmm.cmm_apply_A_noalloc(op.h, m, out)


def test_noalloc_detectors_in_several_passes(cmm, ctx):
    """A 512x512 TQU map leaves room in the static array for the spectra of only
    three of the eight detectors at 2^20 samples (F32): the detectors go through
    it in passes of three, three and two, reusing the spectrum region."""
    op, scan = operator(cmm, ctx, 1, 3, 307, 512, 512, 1 << 20)
    assert scan.n_det == 8
    m = maps(scan, 308)
    ref = op.apply(m)
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        cmm.cmm_apply_A_noalloc(op.h, m, out)
        torch.cuda.synchronize()
        assert rel(out, ref) < TOL[1]


def test_noalloc_bf16_storage(cmm, ctx):
    """BF16 spectrum storage (4 bytes per complex value in the array): the same
    numbers as cmm_apply_A up to the order of the FP32 reductions."""
    op, scan = operator(cmm, ctx, 2, 3, 309, 64, 48, 1 << 16, chunk=2)
    m = maps(scan, 310)
    ref = op.apply(m)
    for _ in range(2):
        out = torch.zeros_like(ref)
        cmm.cmm_apply_A_noalloc(op.h, m, out)
        torch.cuda.synchronize()
        assert rel(out, ref) < TOL[1]


def test_noalloc_rejects_correlated_noise(cmm, ctx):
    op, scan = operator(cmm, ctx, 1, 3, 311, 24, 20, 1 << 12)
    op.noise.set_correlated(gen.corr_noise(scan.det_off, r=1))
    m = maps(scan, 312)
    out = torch.zeros_like(m)
    with pytest.raises(cmm.CmmError, match="correlated"):
        cmm.cmm_apply_A_noalloc(op.h, m, out)
