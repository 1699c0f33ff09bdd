"""Tabulated noise weights (cmm_noise_set_table) against the oracle."""
import numpy as np
import pytest

import gen
from oracle import mapmaker as om

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {0: 1e-10, 1: 1e-5, 2: 2e-2}


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


def setup():
    scan = gen.small_scan(cfg=351, ny=20, nx=18, n_t=1 << 13, ncols=4, nrows=2, throw_px=30.0)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=351)
    return scan, noise


def measured_like_table(scan, noise):
    """A positive table unlike the law: the law times a smooth ripple and a bump."""
    w = om.filter_weights(noise, scan.n_t, scan.f_samp)
    k = np.arange(w.shape[1])
    ripple = 1.0 + 0.3 * np.sin(k / 37.0)[None] * np.linspace(0.5, 1.0, w.shape[0])[:, None]
    return w * ripple


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_table_equal_to_law_gives_same_operator(cmm, ctx, prec):
    scan, noise = setup()
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    m = dev(gen.random_maps(3, scan.ny, scan.nx, 1, cfg=352)[0])
    y0 = op.apply(m).cpu().numpy()
    d0 = op.noise.diag()
    op.noise.set_table(om.filter_weights(noise, scan.n_t, scan.f_samp))
    assert rel(op.apply(m).cpu().numpy(), y0) < {0: 1e-12, 1: 1e-5, 2: 2e-2}[prec]
    assert rel(op.noise.diag(), d0) < 1e-12


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_table_matches_oracle(cmm, ctx, prec):
    scan, noise = setup()
    w = measured_like_table(scan, noise)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    op.noise.set_table(w)
    oop = om.make_operator(scan, noise, w=w)
    m = gen.random_maps(3, scan.ny, scan.nx, 1, cfg=353)[0]
    assert rel(op.apply(dev(m)).cpu().numpy(), om.apply_A(oop, m)) < TOL[prec]
    assert rel(op.noise.diag(), om.ninv_diagonal(w, scan.n_t)) < 1e-13
    if prec == 0:
        b = om.apply_A(oop, gen.sky_map(scan.ny, scan.nx, cfg=354))
        pc = cmm.Precon(op, cmm.PRECON_BINNED)
        x, info, _, _ = cmm.solve(op, pc, dev(b), tol=1e-10, maxit=1000)
        xo, io = om.pcg(lambda v: om.apply_A(oop, v), om.BlockPrecon(oop), b, tol=1e-10, maxit=1000)
        assert info.status == 0 and abs(info.iterations - io.iterations) <= 2
        assert rel(x.cpu().numpy(), xo) < 1e-8


def test_table_rejects_bad_values(cmm, ctx):
    scan, noise = setup()
    op = cmm.Operator(ctx, scan, noise, precision=1)
    w = measured_like_table(scan, noise)
    w[0, 5] = -1.0
    with pytest.raises(cmm.CmmError):
        op.noise.set_table(w)
