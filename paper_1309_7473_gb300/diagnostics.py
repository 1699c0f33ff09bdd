"""Convergence diagnostics of the Results section on spectra computed by the
library (``cmm.cmm_spectra``): when each multipole bin of TT, EE and BB comes
within a fraction of cosmic variance of the input map's spectrum.  The count
itself is the library's (``cmm_spectra_converged_at``); this module only
marshals arguments."""
from __future__ import annotations

from . import cmm


def steps_to_converge(cls_iter, iters, cls_true, nmodes, level=0.1):
    """Per spectrum and bin, the first sampled iteration after which
    |C_b(x_k) - C_b(x_true)| stays below level * sigma_cv; -1 if it never does.
    cls_iter [n_snap, 3, nbins] at the iterations ``iters``; cls_true [3, nbins]."""
    return cmm.cmm_spectra_converged_at(cls_iter, iters, cls_true, nmodes, level)
