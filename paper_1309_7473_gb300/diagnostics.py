"""Convergence diagnostics of the Results section on spectra computed by the
library (``cmm.cmm_spectra``): when each multipole bin of TT, EE and BB comes
within a fraction of cosmic variance of the input map's spectrum."""
from __future__ import annotations

import numpy as np


def cosmic_variance(cls_true, nmodes):
    """sigma_cv of each bin: C_b sqrt(2 / n_b)."""
    return cls_true * np.sqrt(2.0 / np.maximum(nmodes, 1))


def steps_to_converge(cls_iter, iters, cls_true, nmodes, level=0.1):
    """Per spectrum and bin, the first sampled iteration after which
    |C_b(x_k) - C_b(x_true)| stays below level * sigma_cv; -1 if it never does.
    cls_iter [n_snap, 3, nbins] at the iterations ``iters``; cls_true [3, nbins]."""
    sigma = cosmic_variance(cls_true, nmodes)
    err = np.abs(cls_iter - cls_true[None]) / np.where(sigma > 0, sigma, np.inf)
    out = np.full(cls_true.shape, -1, dtype=np.int64)
    for c in range(cls_true.shape[0]):
        for b in range(cls_true.shape[1]):
            above = np.flatnonzero(err[:, c, b] >= level)
            if above.size == 0:
                out[c, b] = iters[0]
            elif above[-1] + 1 < len(iters):
                out[c, b] = iters[above[-1] + 1]
    return out
