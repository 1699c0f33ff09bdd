"""The CUDA path, through the C-ABI, on the hand-worked examples of
``tests/golden/`` (Eq. 1-4; correlated noise per reading R13), at the examples'
64-sample period (generic kernels), repeated to 2^13 samples (the smallest size
of the register-resident FFT kernels) and to 2^20 samples (the per-detector
length of the 1024-detector workload, the four-step split 256 x 2048).  Every
A m scales by the number of repeats K."""
import numpy as np
import pytest

import golden_cases as gc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# relative to the largest expected value: F64 1e-10, F32 1e-5 (the parity tolerances)
TOL = {0: 1e-10, 1: 1e-5}
CASES = list(gc.cases())
IDS = [f"{name}-{case['name']}" for name, _, case in CASES]


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


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def operator(cmm, ctx, fx, case, K, prec):
    scan = gc.scan_of(fx, K)
    op = cmm.Operator(ctx, scan, gc.noise_of(case, scan.n_det), precision=prec, corr=gc.corr_of(case))
    w = gc.table_of(case, scan.n_det, scan.n_t)
    if w is not None:
        op.noise.set_table(w)
    return op


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("K", [1, 128, 16384])
@pytest.mark.parametrize("name,fx,case", CASES, ids=IDS)
def test_A_m_matches_worked_example(cmm, ctx, name, fx, case, K, prec):
    if "corr" in case and (prec == 0 or K == 1):
        pytest.skip("correlated noise runs on the FP32 kernels at 2^13 samples and up")
    op = operator(cmm, ctx, fx, case, K, prec)
    want = K * np.array(case["expected_A_m"], np.float64)
    atol = TOL[prec] * np.abs(want).max()
    m = dev(gc.map_of(fx))
    np.testing.assert_allclose(op.apply(m).cpu().numpy(), want, rtol=0, atol=atol)
    if prec == 1 and K > 1:
        op.set_pixel_cache(True)
        np.testing.assert_allclose(op.apply(m).cpu().numpy(), want, rtol=0, atol=atol)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("K", [1, 16384])
def test_binned_preconditioner_inverts_white_A(cmm, ctx, K, prec):
    fx = gc.load("two_angle_blocks_TQU")
    case = next(c for c in fx["cases"] if c["name"] == "white")
    op = operator(cmm, ctx, fx, case, K, prec)
    pc = cmm.Precon(op, cmm.PRECON_BINNED)
    z = pc.apply(op.apply(dev(gc.map_of(fx)))).cpu().numpy()
    np.testing.assert_allclose(z, np.array(case["expected_binned_of_A_m"], np.float64), rtol=0, atol=TOL[prec] * 6)


@pytest.mark.parametrize("K", [1, 16384])
def test_projection_of_rotated_offset(cmm, ctx, K):
    fx = gc.load("rotated_offset_pointing")
    op = operator(cmm, ctx, fx, fx["cases"][0], K, 0)
    tod = op.project(dev(gc.map_of(fx)), dtype=torch.float64).cpu().numpy()
    period = np.array(fx["expected_tod_period"], np.float64)
    np.testing.assert_array_equal(tod[0], np.tile(period, op.n_t // period.size))
