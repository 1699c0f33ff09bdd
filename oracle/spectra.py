"""Flat-sky binned TT, EE, BB power spectra of TQU maps: the oracle of the
convergence diagnostic of the Results section (spectra of PCG iterates compared
with the input map's, in units of cosmic variance).

TEST INFRASTRUCTURE ONLY (see oracle/mapmaker.py).

Reading R14 (the paper uses a curved-sky estimator it only cites): on the flat
ny x nx map with square pixels of side pix (radians), the 2-D DFT X of each
component gives modes l = 2 pi (ky / (ny pix), kx / (nx pix)) with signed
frequencies; E = Q cos 2 phi + U sin 2 phi, B = -Q sin 2 phi + U cos 2 phi with
phi = atan2(ly, lx); C_b = pix^2 / (ny nx) times the mean of |X|^2 over the modes
of bin b = floor(|l| / (lmax / nbins)) < nbins, l = 0 excluded.  The cosmic
variance of a bin with n_b modes is C_b sqrt(2 / n_b).
"""
from __future__ import annotations

import numpy as np


def mode_grid(ny, nx, pix):
    ky = np.fft.fftfreq(ny, d=1.0 / ny)
    kx = np.fft.fftfreq(nx, d=1.0 / nx)
    ly = 2 * np.pi * ky[:, None] / (ny * pix) * np.ones((1, nx))
    lx = 2 * np.pi * kx[None, :] / (nx * pix) * np.ones((ny, 1))
    return ly, lx


def flat_spectra(m, pix, nbins, lmax):
    """(cls [3, nbins] TT EE BB, modes per bin [nbins]) of a TQU map [3, ny, nx]."""
    _, ny, nx = m.shape
    T, Q, U = (np.fft.fft2(m[c]) for c in range(3))
    ly, lx = mode_grid(ny, nx, pix)
    ell = np.hypot(ly, lx)
    phi = np.arctan2(ly, lx)
    c2, s2 = np.cos(2 * phi), np.sin(2 * phi)
    E = Q * c2 + U * s2
    B = -Q * s2 + U * c2
    b = np.floor(ell / (lmax / nbins)).astype(np.int64)
    ok = (ell > 0) & (b < nbins)
    counts = np.bincount(b[ok], minlength=nbins)
    norm = pix * pix / (ny * nx)
    cls = np.zeros((3, nbins))
    for c, X in enumerate((T, E, B)):
        sums = np.bincount(b[ok], weights=(np.abs(X) ** 2)[ok], minlength=nbins)
        cls[c] = np.where(counts > 0, norm * sums / np.maximum(counts, 1), 0.0)
    return cls, counts
