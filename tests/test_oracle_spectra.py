"""Pins of the flat-sky spectrum oracle (reading R14)."""
import numpy as np

from oracle import spectra as osp

PIX = np.deg2rad(0.5 / 60)


def test_plane_wave_closed_form():
    ny, nx, A = 48, 60, 2.5
    y, x = np.mgrid[0:ny, 0:nx]
    m = np.zeros((3, ny, nx))
    m[0] = A * np.cos(2 * np.pi * (5 * y / ny + 7 * x / nx))
    l0 = 2 * np.pi * np.hypot(5 / (ny * PIX), 7 / (nx * PIX))
    nbins, lmax = 30, 2 * np.pi / PIX
    cls, n = osp.flat_spectra(m, PIX, nbins, lmax)
    b = int(l0 // (lmax / nbins))
    # two modes (+k, -k) of |X| = A N / 2 in bin b, nothing elsewhere
    expect = PIX ** 2 / (ny * nx) * 2 * (A * ny * nx / 2) ** 2 / n[b]
    assert np.isclose(cls[0, b], expect, rtol=1e-12)
    assert np.all(np.delete(cls[0], b) < 1e-20 * expect)
    assert np.all(cls[1:] == 0)
    # in bins 1/20 as wide the wave still lands at |l| = l0, the wavenumbers scaled
    # by the map's own side in each direction
    fine, _ = osp.flat_spectra(m, PIX, 20 * nbins, lmax)
    bf = int(l0 // (lmax / (20 * nbins)))
    assert fine[0, bf] > 0 and np.all(np.delete(fine[0], bf) < 1e-20 * fine[0, bf])


def test_pure_e_has_no_b_and_rotation_swaps():
    ny, nx = 40, 50
    g = np.random.default_rng(1)
    e = np.fft.fft2(g.standard_normal((ny, nx)))
    e[ny // 2, :] = 0   # Nyquist modes are their own mirror: no Hermitian rotation there
    e[:, nx // 2] = 0
    ly, lx = osp.mode_grid(ny, nx, PIX)
    phi = np.arctan2(ly, lx)
    q = np.fft.ifft2(e * np.cos(2 * phi)).real
    u = np.fft.ifft2(e * np.sin(2 * phi)).real
    t = np.fft.ifft2(e).real
    m = np.stack([t, q, u])
    cls, _ = osp.flat_spectra(m, PIX, 20, 2 * np.pi / PIX)
    assert np.all(cls[2] <= 1e-20 * cls[1].max())
    # the pure-E map's EE is the T spectrum of the map made from e alone
    assert np.allclose(cls[1], cls[0], rtol=1e-10)
    rot, _ = osp.flat_spectra(np.stack([t, u, -q]), PIX, 20, 2 * np.pi / PIX)
    assert np.allclose(rot[2], cls[1], rtol=1e-10) and np.all(rot[1] <= 1e-20 * cls[1].max())


def test_parseval():
    g = np.random.default_rng(2)
    m = g.standard_normal((3, 30, 36))
    ny, nx = 30, 36
    cls, n = osp.flat_spectra(m, PIX, 50, 1e9)
    total = (cls[0] * n).sum() * ny * nx / PIX ** 2
    assert np.isclose(total, ny * nx * (m[0] ** 2).sum() - m[0].sum() ** 2, rtol=1e-12)
