"""Failure detection and checkpoint / resume of the solver, tested on the host side
only: the failures are made in the inputs (a non-finite right-hand side or
starting guess, an operator whose noise weights are all zero), never by faulting
the GPU.  Each must end the solve with CMM_ERR_BREAKDOWN, finite reported
scalars and no hang.  A solve stopped after k iterations and resumed from its
saved state continues the iterates of the uninterrupted solve."""
import math

import numpy as np
import pytest

import gen
from oracle import mapmaker as om

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BREAKDOWN = 4
NOT_CONVERGED = 5


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


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def problem(cmm, ctx, prec=0):
    scan = gen.small_scan(cfg=371, ny=20, nx=18, n_t=1 << 12, ncols=4, nrows=2, throw_px=30.0)
    noise = gen.noise_params(scan.n_det, fknee=2.0, alpha=3.5, scatter=0.2, cfg=371)
    op = cmm.Operator(ctx, scan, noise, precision=prec)
    oop = om.make_operator(scan, noise)
    b = om.apply_A(oop, gen.sky_map(scan.ny, scan.nx, cfg=371))
    return scan, noise, op, oop, b


def finite_info(info):
    return (math.isfinite(info.rel_resid) and math.isfinite(info.true_rel_resid)
            and math.isfinite(info.seconds) and info.iterations >= 0)


@pytest.mark.parametrize("graph", [True, False])
def test_nan_in_rhs_is_breakdown(cmm, ctx, graph):
    scan, noise, op, oop, b = problem(cmm, ctx)
    b[1, 3, 4] = np.nan
    pc = cmm.Precon(op, cmm.PRECON_BINNED)
    x = op.new_map()
    x.fill_(7.0)
    info = cmm.cmm_solve(op.h, pc.h, dev(b), x, 1e-8, 200, 10, graph)
    assert info.status == BREAKDOWN
    assert info.iterations == 0 and info.rel_resid == -1.0
    assert finite_info(info)
    assert bool(torch.all(x == 7.0))      # nothing was iterated: x is left as given
    # the operator and preconditioner stay usable: the same solve with a clean b converges
    b[1, 3, 4] = 0.0
    x2, info2, _, _ = cmm.solve(op, pc, dev(b), tol=1e-8, maxit=400)
    assert info2.status == 0 and np.isfinite(host(x2)).all()


def test_inf_in_starting_guess_is_breakdown(cmm, ctx):
    scan, noise, op, oop, b = problem(cmm, ctx)
    pc = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=4.0)
    x0 = np.zeros_like(b)
    x0[0, 5, 5] = np.inf
    x = dev(x0)
    info = cmm.cmm_solve(op.h, pc.h, dev(b), x, 1e-8, 200, 10, True, True, true_resid=False)
    assert info.status == BREAKDOWN
    assert info.iterations == 0
    assert info.rel_resid == -1.0 and info.true_rel_resid == -1.0
    assert finite_info(info)


@pytest.mark.parametrize("kind", ["binned", "jacobi"])
def test_zero_noise_weights_is_breakdown(cmm, ctx, kind):
    """A tabulated noise filter of zeros makes A = 0, so p^T A p = 0 (Jacobi, whose
    weights do not depend on the noise) or M itself is not finite (binned, whose
    blocks are weighted by diag(N^-1) = 0): both are breakdowns, not garbage."""
    scan, noise, op, oop, b = problem(cmm, ctx)
    op.noise.set_table(np.zeros((scan.n_det, scan.n_t // 2 + 1)))
    m = gen.sky_map(scan.ny, scan.nx, cfg=372)
    assert np.abs(host(op.apply(dev(m)))).max() == 0.0
    pc = cmm.Precon(op, cmm.PRECON_BINNED if kind == "binned" else cmm.PRECON_JACOBI)
    x = op.new_map()
    info = cmm.cmm_solve(op.h, pc.h, dev(b), x, 1e-8, 200, 10, True)
    assert info.status == BREAKDOWN
    assert info.iterations == 0
    assert finite_info(info)
    assert info.rel_resid == pytest.approx(1.0)
    assert np.isfinite(host(x)).all()
    with pytest.raises(cmm.CmmError):
        cmm.cmm_solve_state_save(op.h, torch.zeros(cmm.cmm_solve_state_size(op.h), dtype=torch.float64,
                                                   device="cuda:0"))


@pytest.mark.parametrize("flexible", [False, True])
@pytest.mark.parametrize("via_host", [False, True])
def test_resume_continues_the_iterates(cmm, ctx, flexible, via_host):
    """Stop after k iterations, save the state (optionally through host memory),
    load it into a fresh operator, resume: same iteration count, residual history
    and solution as the solve that was never stopped, to the rounding of the
    FP64 atomic sums (the oracle's solution is the reference for the rest)."""
    scan, noise, op, oop, b = problem(cmm, ctx)
    pc = cmm.Precon(op, cmm.PRECON_CIRCULANT, taper_sigma_px=4.0)
    bd = dev(b)
    tol, k = 1e-10, 9
    n = 3 * scan.npix
    hist0 = torch.zeros(401, dtype=torch.float64, device="cuda:0")
    x_full = op.new_map()
    i_full = cmm.cmm_solve(op.h, pc.h, bd, x_full, tol, 400, 4, True, False, hist0, None, flexible=flexible)
    assert i_full.status == 0 and i_full.iterations > k + 5
    # stopped after k iterations
    hist1 = torch.zeros(401, dtype=torch.float64, device="cuda:0")
    x = op.new_map()
    i1 = cmm.cmm_solve(op.h, pc.h, bd, x, tol, k, 4, True, False, hist1, None, flexible=flexible)
    assert i1.status == NOT_CONVERGED and i1.iterations == k
    state = torch.zeros(cmm.cmm_solve_state_size(op.h), dtype=torch.float64, device="cuda:0")
    assert state.numel() == 3 * n + 8
    cmm.cmm_solve_state_save(op.h, state)
    xk = host(x).copy()
    if via_host:
        saved, xk_saved = host(state).copy(), xk.copy()
        state = dev(saved)
        x = dev(xk_saved)
    # a fresh operator and preconditioner on the same inputs
    op2 = cmm.Operator(ctx, scan, noise, precision=0)
    pc2 = cmm.Precon(op2, cmm.PRECON_CIRCULANT, taper_sigma_px=4.0)
    with pytest.raises(cmm.CmmError):
        cmm.cmm_solve(op2.h, pc2.h, bd, x, tol, 400, 4, True, False, resume=True)
    cmm.cmm_solve_state_load(op2.h, state)
    i2 = cmm.cmm_solve(op2.h, pc2.h, bd, x, tol, 400, 4, True, False, hist1, None, flexible=flexible,
                       resume=True)
    assert i2.status == 0
    assert i2.iterations == i_full.iterations
    h0, h1 = host(hist0)[: i_full.iterations + 1], host(hist1)[: i2.iterations + 1]
    np.testing.assert_allclose(h1, h0, rtol=1e-8)
    assert rel(host(x), host(x_full)) < 1e-10
    xo, io = om.pcg(lambda v: om.apply_A(oop, v), om.CirculantPrecon(oop, taper_sigma=4.0), b, tol=tol,
                    maxit=400)
    assert rel(host(x), xo) < 1e-6
    # a garbage buffer is refused
    with pytest.raises(cmm.CmmError):
        cmm.cmm_solve_state_load(op2.h, torch.zeros_like(state))
