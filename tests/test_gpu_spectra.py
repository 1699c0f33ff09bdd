"""cmm_spectra (flat-sky binned TT, EE, BB on the GPU) against the oracle."""
import numpy as np
import pytest

import gen
from oracle import spectra as osp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PIX = np.deg2rad(0.5 / 60)


@pytest.fixture(scope="module")
def cmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_7473_gb300 import build
    build.build()
    from paper_1309_7473_gb300 import cmm as c
    return c


@pytest.mark.parametrize("ny,nx,nbins", [(48, 60, 12), (900, 1200, 40)])
def test_spectra_match_oracle(cmm, ny, nx, nbins):
    ctx = cmm.Context(0)
    maps = np.stack([gen.sky_map(ny, nx, cfg=9, real=k) for k in range(2)])
    lmax = np.pi / PIX
    cls, n = cmm.cmm_spectra(ctx.h, torch.as_tensor(maps, device="cuda:0"), PIX, nbins, lmax)
    for k in range(2):
        ref, nref = osp.flat_spectra(maps[k], PIX, nbins, lmax)
        assert np.array_equal(n, nref)
        np.testing.assert_allclose(cls[k], ref, rtol=1e-10, atol=1e-30)
