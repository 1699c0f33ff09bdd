"""The oracle against the hand-worked examples of ``tests/golden/`` (Eq. 1-4):
A m under white, DC-removed, Nyquist-doubled and quarter-bin-doubled filters,
polarised blocks at two sky angles, the binned preconditioner as the exact
inverse of A for white noise, and the pointing of a rotated off-axis detector.
Each example is taken at its 64-sample period and repeated (K = 16), where every
A m scales by K."""
import numpy as np
import pytest

import golden_cases as gc
from oracle import mapmaker as om

CASES = list(gc.cases())
IDS = [f"{name}-{case['name']}" for name, _, case in CASES]


def operator(fx, case, K):
    scan = gc.scan_of(fx, K)
    noise = gc.noise_of(case, scan.n_det)
    return om.make_operator(scan, noise, w=gc.table_of(case, scan.n_det, scan.n_t), corr=gc.corr_of(case)), scan


@pytest.mark.parametrize("K", [1, 16])
@pytest.mark.parametrize("name,fx,case", CASES, ids=IDS)
def test_A_m_matches_worked_example(name, fx, case, K):
    op, scan = operator(fx, case, K)
    got = om.apply_A(op, gc.map_of(fx))
    want = K * np.array(case["expected_A_m"], np.float64)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * K * np.abs(want).max())


@pytest.mark.parametrize("K", [1, 16])
def test_binned_preconditioner_inverts_white_A(K):
    fx = gc.load("two_angle_blocks_TQU")
    case = next(c for c in fx["cases"] if c["name"] == "white")
    op, _ = operator(fx, case, K)
    z = om.BlockPrecon(op)(om.apply_A(op, gc.map_of(fx)))
    np.testing.assert_allclose(z, np.array(case["expected_binned_of_A_m"], np.float64), rtol=0, atol=1e-12)


def test_projection_of_rotated_offset():
    fx = gc.load("rotated_offset_pointing")
    op, scan = operator(fx, fx["cases"][0], 2)
    tod = om.project(op, gc.map_of(fx))
    period = np.array(fx["expected_tod_period"], np.float64)
    np.testing.assert_array_equal(tod[0], np.tile(period, scan.n_t // period.size))


def test_fixtures_are_what_their_derivations_say():
    """The expanded scans have the hit counts the derivations state."""
    fx = gc.load("runs_T_filters")
    scan = gc.scan_of(fx, 1)
    hits = np.bincount(om.sample_pixels(scan, np.arange(1))[0], minlength=scan.npix)
    assert hits.tolist() == [10, 20, 6, 15, 13, 0]
    fx = gc.load("two_angle_blocks_TQU")
    scan = gc.scan_of(fx, 1)
    blocks = om.hit_blocks(scan)   # [npix, 3, 3]
    np.testing.assert_array_equal(blocks[0], np.diag([64.0, 32.0, 32.0]))
    np.testing.assert_array_equal(blocks[1], np.diag([64.0, 32.0, 32.0]))
    assert not blocks[2:].any()
