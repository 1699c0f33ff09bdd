"""Host logic of the spectrum convergence diagnostic."""
import numpy as np

from paper_1309_7473_gb300 import diagnostics


def test_steps_to_converge():
    iters = np.array([0, 10, 20, 30])
    true = np.ones((1, 3))
    n = np.array([200, 200, 200])
    sig = np.sqrt(2 / 200)
    c = np.array([[[5.0, 1.0, 2.0]], [[1 + 0.5 * sig, 1.0, 2.0]], [[1 + 0.05 * sig, 1 + 0.2 * sig, 2.0]],
                  [[1.0, 1.0, 2.0]]])
    out = diagnostics.steps_to_converge(c, iters, true, n)
    assert out.tolist() == [[20, 30, -1]]
    assert np.allclose(diagnostics.cosmic_variance(true, n), sig)
