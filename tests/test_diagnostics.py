"""The spectrum convergence count of the Results section (host code of the C-ABI
library; no device call), on a sequence worked by hand."""
import numpy as np
import pytest

from paper_1309_7473_gb300 import diagnostics


def test_steps_to_converge():
    # three bins with a true spectrum of 1, 1 and 2 over 200 modes each: sigma_cv =
    # C sqrt(2 / 200).  Bin 0 is within 0.1 sigma from the snapshot at iteration 20
    # on, bin 1 only at the last snapshot (iteration 30), bin 2 never (its last
    # snapshot is still 0.25 sigma_cv = 0.05 off).
    iters = np.array([0, 10, 20, 30])
    true = np.array([[1.0, 1.0, 2.0]])
    n = np.array([200, 200, 200])
    sig = np.sqrt(2 / 200)
    c = np.array([[[5.0, 1.0, 2.0]], [[1 + 0.5 * sig, 1 + 0.3 * sig, 2.5]],
                  [[1 + 0.05 * sig, 1 + 0.2 * sig, 2.0]], [[1.0, 1.0, 2 + 0.25 * 2 * sig]]])
    out = diagnostics.steps_to_converge(c, iters, true, n)
    assert out.tolist() == [[20, 30, -1]]
    # already converged at the first snapshot
    assert diagnostics.steps_to_converge(c[3:], iters[3:], true, n)[0, 0] == 30
    # the level sets the threshold: at 0.6 sigma bin 0 has converged from iteration 10
    assert diagnostics.steps_to_converge(c, iters, true, n, level=0.6)[0, 0] == 10


def test_steps_to_converge_zero_spectrum_and_empty_bin():
    # a bin without true power has no cosmic-variance scale (converged at the first
    # snapshot); a bin without modes counts as one mode
    iters = np.array([0, 5])
    true = np.array([[0.0, 4.0]])
    n = np.array([10, 0])
    c = np.array([[[3.0, 4.0 + 0.2 * 4.0 * np.sqrt(2.0)]], [[3.0, 4.0]]])
    assert diagnostics.steps_to_converge(c, iters, true, n).tolist() == [[0, 5]]


def test_steps_to_converge_rejects_bad_arguments():
    from paper_1309_7473_gb300 import cmm
    c = np.ones((2, 3, 4))
    with pytest.raises(ValueError):
        diagnostics.steps_to_converge(c, np.array([0]), np.ones((3, 4)), np.ones(4))
    with pytest.raises(cmm.CmmError):
        diagnostics.steps_to_converge(c, np.array([0, 1]), np.ones((3, 4)), np.ones(4), level=0.0)
