"""Thin Python binding of the map-maker's C ABI (``include/cmm.h``).

The functions ``cmm_*`` below marshal arguments to the entry points of the same
name in ``libcmm.so``: torch tensors are passed as raw device pointers, numpy
arrays as host pointers.  No map-making arithmetic happens here; every step runs
in the library's CUDA kernels.  There is no CPU fallback: importing this module
without the built library raises.

The small classes (Context, Pointing, Noise, Operator, Precon) own the library
handles and free them when garbage-collected.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcmm.so")

PREC_F64, PREC_F32, PREC_BF16 = 0, 1, 2
PRECON_BINNED, PRECON_JACOBI, PRECON_CIRCULANT, PRECON_IDENTITY, PRECON_CIRC_LEARNED = 0, 1, 2, 3, 4
PRECON_CIRC_TILED = 5
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_BREAKDOWN",
          5: "ERR_NOT_CONVERGED", 6: "ERR_TIMEOUT", 7: "ERR_UNSUPPORTED"}


class CmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class MapGeom(C.Structure):
    _fields_ = [("ny", C.c_int32), ("nx", C.c_int32), ("ncomp", C.c_int32), ("periodic", C.c_int32)]


class PreconOpts(C.Structure):
    _fields_ = [("taper_sigma_px", C.c_double), ("ref_pixel", C.c_int64), ("pd_eps", C.c_double),
                ("tiles_y", C.c_int32), ("tiles_x", C.c_int32), ("white_diag", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int32), ("check_every", C.c_int32),
                ("use_graph", C.c_int32), ("x0_given", C.c_int32), ("cg_f32", C.c_int32),
                ("resid_replace", C.c_int32), ("flexible", C.c_int32), ("snapshot_every", C.c_int32),
                ("snapshot_max", C.c_int32), ("batch_width", C.c_int32), ("skip_true_resid", C.c_int32),
                ("resume", C.c_int32), ("fcg_window", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("rel_resid", C.c_double),
                ("seconds", C.c_double), ("true_rel_resid", C.c_double)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run paper_1309_7473_gb300/build.py "
                      "(or __graft_entry__.build()) first")
_lib = C.CDLL(LIB_PATH)

_vp, _i32, _i64, _d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_PP = C.POINTER(C.c_void_p)
_SIGS = {
    "cmm_ctx_create": [C.c_int, _vp, _PP],
    "cmm_ctx_destroy": [_vp],
    "cmm_pointing_create": [_vp, C.POINTER(MapGeom), _i32, _vp, _vp, _i64, _vp, _PP],
    "cmm_pointing_destroy": [_vp],
    "cmm_pointing_mask": [_vp, _vp, C.POINTER(_i64)],
    "cmm_noise_create": [_vp, _i32, _i64, _d, _vp, _vp, _vp, _PP],
    "cmm_noise_destroy": [_vp],
    "cmm_noise_set_correlated": [_vp, _i32, _vp, _vp, _vp, _vp],
    "cmm_noise_set_table": [_vp, _vp],
    "cmm_spectra": [_vp, _i32, _i32, C.c_double, _i32, _vp, _i32, C.c_double, _vp, _vp],
    "cmm_spectra_converged_at": [_i32, _vp, _i32, _i32, _vp, _vp, _vp, C.c_double, _vp],
    "cmm_noise_diag": [_vp, _vp],
    "cmm_op_create": [_vp, _vp, _vp, _i32, _i32, _PP],
    "cmm_op_destroy": [_vp],
    "cmm_op_set_pixel_cache": [_vp, _i32],
    "cmm_op_set_pair_packing": [_vp, _i32],
    "cmm_apply_A": [_vp, _vp, _vp],
    "cmm_apply_A_host": [_vp, _vp, _vp],
    "cmm_apply_A_noalloc": [_vp, _vp, _vp],
    "cmm_profile_apply": [_vp, _vp, _vp, _i32, _vp],
    "cmm_project": [_vp, _vp, _vp, _i32],
    "cmm_rhs": [_vp, _vp, _i32, _vp],
    "cmm_dot": [_vp, _vp, _vp, _i64, C.POINTER(_d)],
    "cmm_precon_create": [_vp, _i32, C.POINTER(PreconOpts), _PP],
    "cmm_precon_destroy": [_vp],
    "cmm_precon_apply": [_vp, _vp, _vp],
    "cmm_precon_clamped": [_vp, C.POINTER(_i64)],
    "cmm_solve": [_vp, _vp, _vp, _vp, C.POINTER(SolveOpts), _vp, _vp, _vp, C.POINTER(SolveInfo)],
    "cmm_solve_host": [_vp, _vp, _vp, _vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo)],
    "cmm_solve_state_size": [_vp, C.POINTER(_i64)],
    "cmm_solve_state_save": [_vp, _vp],
    "cmm_solve_state_load": [_vp, _vp],
    "cmm_precon_set_correction": [_vp, _vp],
    "cmm_harvest_pairs": [_vp, _vp, _i32, _vp, _vp, _vp],
    "cmm_unet_create": [_vp, _i32, _i32, _i32, _vp, _i32, _PP],
    "cmm_unet_destroy": [_vp],
    "cmm_unet_set_tensor_cores": [_vp, _i32],
    "cmm_unet_param_count": [_vp, C.POINTER(_i64)],
    "cmm_unet_set_params": [_vp, _vp],
    "cmm_unet_get_params": [_vp, _vp],
    "cmm_unet_init": [_vp, C.c_uint64],
    "cmm_unet_forward": [_vp, _i32, _vp, _vp],
    "cmm_unet_loss_grad": [_vp, _i32, _vp, _vp, _vp, C.POINTER(_d)],
    "cmm_unet_train_step": [_vp, _i32, _vp, _vp, C.c_float, C.POINTER(_d)],
    "cmm_batch_solve": [_i32, _vp, _vp, _vp, _vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo)],
    "cmm_autotune": [_vp, _i32, C.c_char_p, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_d)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.cmm_last_error.restype = C.c_char_p
_lib.cmm_last_error.argtypes = []
_lib.cmm_version.restype = C.c_char_p
_lib.cmm_version.argtypes = []

EXPORTED = sorted(list(_SIGS) + ["cmm_last_error", "cmm_version"])


def _check(code):
    if code != 0:
        raise CmmError(code, _lib.cmm_last_error().decode())


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


def _dev(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (checked)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- raw entry points

def cmm_version() -> str:
    return _lib.cmm_version().decode()


def cmm_last_error() -> str:
    return _lib.cmm_last_error().decode()


def cmm_ctx_create(device: int, stream: int):
    h = C.c_void_p()
    _check(_lib.cmm_ctx_create(device, C.c_void_p(stream), C.byref(h)))
    return h


def cmm_ctx_destroy(h):
    _check(_lib.cmm_ctx_destroy(h))


def cmm_pointing_create(ctx, ny, nx, ncomp, periodic, det_off, det_pol, bore):
    geom = MapGeom(ny, nx, ncomp, 1 if periodic else 0)
    det_off, p_off = _host(det_off, np.int32)
    det_pol, p_pol = _host(det_pol, np.float64)
    bore, p_bore = _host(bore, np.int32)
    n_det = det_off.shape[0]
    if det_off.shape != (n_det, 2) or det_pol.shape != (n_det, 2) or bore.ndim != 2 or bore.shape[1] != 4:
        raise ValueError("bad pointing table shapes")
    h = C.c_void_p()
    _check(_lib.cmm_pointing_create(ctx, C.byref(geom), n_det, p_off, p_pol, bore.shape[0], p_bore, C.byref(h)))
    return h


def cmm_pointing_destroy(h):
    _check(_lib.cmm_pointing_destroy(h))


def cmm_pointing_mask(h, npix):
    out = np.empty(npix, np.uint8)
    n = C.c_int64()
    _check(_lib.cmm_pointing_mask(h, out.ctypes.data_as(C.c_void_p), C.byref(n)))
    return out.astype(bool), int(n.value)


def cmm_noise_create(ctx, n_samp, f_samp, sigma, fknee, alpha):
    sigma, ps = _host(sigma, np.float64)
    fknee, pf = _host(fknee, np.float64)
    alpha, pa = _host(alpha, np.float64)
    h = C.c_void_p()
    _check(_lib.cmm_noise_create(ctx, sigma.size, n_samp, f_samp, ps, pf, pa, C.byref(h)))
    return h


def cmm_noise_set_correlated(h, corr=None):
    """corr: gen.CorrNoise-like (modes [n_det, r], amp, fknee, alpha) or None to remove."""
    if corr is None:
        _check(_lib.cmm_noise_set_correlated(h, 0, None, None, None, None))
        return
    v = np.ascontiguousarray(corr.modes, dtype=np.float64)
    amp, fk, al = (np.ascontiguousarray(a, dtype=np.float64) for a in (corr.amp, corr.fknee, corr.alpha))
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(_lib.cmm_noise_set_correlated(h, int(v.shape[1]), p(v), p(amp), p(fk), p(al)))


def cmm_spectra(ctx, maps, pix_rad, nbins, lmax):
    """Binned flat-sky TT, EE, BB of device maps [nmaps, 3, ny, nx] (float64);
    returns (cls [nmaps, 3, nbins], modes per bin [nbins])."""
    if maps.dim() == 3:
        maps = maps.unsqueeze(0)
    nm, _, ny, nx = maps.shape
    cls = np.zeros((nm, 3, nbins))
    nmodes = np.zeros(nbins, dtype=np.int64)
    _check(_lib.cmm_spectra(ctx, ny, nx, float(pix_rad), nm, _dev(maps, name="maps"), int(nbins), float(lmax),
                            cls.ctypes.data_as(C.c_void_p), nmodes.ctypes.data_as(C.c_void_p)))
    return cls, nmodes


def cmm_spectra_converged_at(cls_iter, iters, cls_true, nmodes, level=0.1):
    """cls_iter [n_snap, nspec, nbins] at the iterations ``iters``, cls_true [nspec,
    nbins], nmodes [nbins]; returns int32 [nspec, nbins] (see include/cmm.h)."""
    ci, pci = _host(cls_iter, np.float64)
    ct, pct = _host(cls_true, np.float64)
    it, pit = _host(iters, np.int32)
    nm, pnm = _host(nmodes, np.int64)
    if ci.ndim != 3 or ct.shape != ci.shape[1:] or it.shape != (ci.shape[0],) or nm.shape != (ci.shape[2],):
        raise ValueError("shapes: cls_iter [n_snap, nspec, nbins], iters [n_snap], cls_true [nspec, nbins], "
                         "nmodes [nbins]")
    out = np.zeros(ct.shape, dtype=np.int32)
    _check(_lib.cmm_spectra_converged_at(ci.shape[0], pit, ci.shape[1], ci.shape[2], pci, pct, pnm, float(level),
                                         out.ctypes.data_as(C.c_void_p)))
    return out


def cmm_noise_set_table(h, w=None):
    """w: float64 [n_det, n_samp/2 + 1] of w_d(f_k) = 1 / PSD_d(f_k), or None for the law."""
    if w is None:
        _check(_lib.cmm_noise_set_table(h, None))
        return
    w = np.ascontiguousarray(w, dtype=np.float64)
    _check(_lib.cmm_noise_set_table(h, w.ctypes.data_as(C.c_void_p)))


def cmm_noise_destroy(h):
    _check(_lib.cmm_noise_destroy(h))


def cmm_noise_diag(h, n_det):
    out = np.empty(n_det)
    _check(_lib.cmm_noise_diag(h, out.ctypes.data_as(C.c_void_p)))
    return out


def cmm_op_create(ctx, pointing, noise, precision=PREC_F32, det_chunk=0):
    h = C.c_void_p()
    _check(_lib.cmm_op_create(ctx, pointing, noise, precision, det_chunk, C.byref(h)))
    return h


def cmm_op_destroy(h):
    _check(_lib.cmm_op_destroy(h))


def cmm_op_set_pixel_cache(op, enable=True):
    _check(_lib.cmm_op_set_pixel_cache(op, 1 if enable else 0))


def cmm_op_set_pair_packing(h, enable):
    _check(_lib.cmm_op_set_pair_packing(h, 1 if enable else 0))


def cmm_apply_A(op, m_in, m_out):
    _check(_lib.cmm_apply_A(op, _dev(m_in, name="m_in"), _dev(m_out, name="m_out")))


def cmm_apply_A_noalloc(op, m_in, m_out):
    """As cmm_apply_A, with the temporaries in the library's static scratch array."""
    _check(_lib.cmm_apply_A_noalloc(op, _dev(m_in, name="m_in"), _dev(m_out, name="m_out")))


def cmm_apply_A_host(op, m_in: np.ndarray, m_out: np.ndarray):
    if m_in.dtype != np.float64 or m_out.dtype != np.float64 or not m_out.flags.c_contiguous:
        raise ValueError("host maps must be contiguous float64")
    m_in = np.ascontiguousarray(m_in)
    _check(_lib.cmm_apply_A_host(op, m_in.ctypes.data_as(C.c_void_p), m_out.ctypes.data_as(C.c_void_p)))


def cmm_profile_apply(op, m_in, m_out, reps):
    """Mean ms per launch: [forward pass, filter pass, inverse+binning pass, map copies, whole apply]."""
    out = np.zeros(5)
    _check(_lib.cmm_profile_apply(op, _dev(m_in, name="m_in"), _dev(m_out, name="m_out"), int(reps),
                                  out.ctypes.data_as(C.c_void_p)))
    return out


def cmm_project(op, m, tod):
    import torch
    _check(_lib.cmm_project(op, _dev(m, torch.float64, name="m"), _dev(tod, name="tod"),
                            1 if tod.dtype == torch.float64 else 0))


def cmm_rhs(op, tod, b):
    import torch
    if tod.dtype not in (torch.float32, torch.float64):
        raise ValueError("tod must be float32 or float64")
    _check(_lib.cmm_rhs(op, _dev(tod, name="tod"), 1 if tod.dtype == torch.float64 else 0,
                        _dev(b, torch.float64, name="b")))


def cmm_dot(op, x, y):
    out = C.c_double()
    _check(_lib.cmm_dot(op, _dev(x), _dev(y), x.numel(), C.byref(out)))
    return out.value


def cmm_precon_create(op, kind, taper_sigma_px=0.0, ref_pixel=-1, pd_eps=0.0, tiles=(0, 0), white_diag=False):
    opts = PreconOpts(float(taper_sigma_px), int(ref_pixel), float(pd_eps), int(tiles[0]), int(tiles[1]),
                      1 if white_diag else 0)
    h = C.c_void_p()
    _check(_lib.cmm_precon_create(op, kind, C.byref(opts), C.byref(h)))
    return h


def cmm_precon_destroy(h):
    _check(_lib.cmm_precon_destroy(h))


def cmm_precon_apply(pc, r, z):
    _check(_lib.cmm_precon_apply(pc, _dev(r, name="r"), _dev(z, name="z")))


def cmm_precon_clamped(pc):
    n = C.c_int64()
    _check(_lib.cmm_precon_clamped(pc, C.byref(n)))
    return int(n.value)


def cmm_solve(op, pc, b, x, tol=1e-6, maxit=500, check_every=10, use_graph=True, x0_given=False,
              resid_hist=None, anorm_terms=None, cg_f32=False, resid_replace=0, flexible=False,
              snapshots=None, snapshot_every=1, true_resid=True, resume=False, window=1):
    snap_max = 0 if snapshots is None else snapshots.shape[0]
    opts = SolveOpts(float(tol), int(maxit), int(check_every), 1 if use_graph else 0, 1 if x0_given else 0,
                     1 if cg_f32 else 0, int(resid_replace), 1 if flexible else 0, int(snapshot_every),
                     int(snap_max), 0, 0 if true_resid else 1, 1 if resume else 0, int(window))
    info = SolveInfo()
    _check(_lib.cmm_solve(op, pc, _dev(b, name="b"), _dev(x, name="x"), C.byref(opts),
                          _dev(resid_hist, numel=None, name="resid_hist"),
                          _dev(anorm_terms, numel=None, name="anorm_terms"),
                          _dev(snapshots, name="snapshots"), C.byref(info)))
    return info


def cmm_solve_host(op, pc, b_host, x_host, tol=1e-6, maxit=500, check_every=10, x0_given=False,
                   true_resid=True, resume=False):
    """cmm_solve on host float64 arrays (numpy, or pinned CPU torch tensors via .numpy())."""
    import numpy as np
    for name, a in (("b", b_host), ("x", x_host)):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise TypeError(f"{name} must be a C-contiguous float64 numpy array")
    opts = SolveOpts(float(tol), int(maxit), int(check_every), 1, 1 if x0_given else 0, 0, 0, 0, 0, 0, 0,
                     0 if true_resid else 1, 1 if resume else 0, 1)
    info = SolveInfo()
    _check(_lib.cmm_solve_host(op, pc, b_host.ctypes.data, x_host.ctypes.data, C.byref(opts), C.byref(info)))
    return info


def cmm_solve_state_size(op):
    n = C.c_int64()
    _check(_lib.cmm_solve_state_size(op, C.byref(n)))
    return int(n.value)


def cmm_solve_state_save(op, state):
    import torch
    _check(_lib.cmm_solve_state_save(op, _dev(state, torch.float64, name="state")))


def cmm_solve_state_load(op, state):
    import torch
    _check(_lib.cmm_solve_state_load(op, _dev(state, torch.float64, name="state")))


def cmm_harvest_pairs(pc, snapshots, count, x_star, inputs, targets):
    import torch
    _check(_lib.cmm_harvest_pairs(pc, _dev(snapshots, torch.float64, name="snapshots"), int(count),
                                  _dev(x_star, torch.float64, name="x_star"), _dev(inputs, torch.float32, name="inputs"),
                                  _dev(targets, torch.float32, name="targets")))


def cmm_precon_set_correction(pc, net):
    _check(_lib.cmm_precon_set_correction(pc, net))


def cmm_unet_create(ctx, ny, nx, widths, batch_max):
    w = (C.c_int32 * len(widths))(*widths)
    h = C.c_void_p()
    _check(_lib.cmm_unet_create(ctx, ny, nx, len(widths), w, batch_max, C.byref(h)))
    return h


def cmm_unet_destroy(h):
    _check(_lib.cmm_unet_destroy(h))


def cmm_unet_set_tensor_cores(h, enable=True):
    _check(_lib.cmm_unet_set_tensor_cores(h, 1 if enable else 0))


def cmm_unet_param_count(h):
    n = C.c_int64()
    _check(_lib.cmm_unet_param_count(h, C.byref(n)))
    return int(n.value)


def cmm_unet_set_params(h, params):
    import torch
    _check(_lib.cmm_unet_set_params(h, _dev(params, torch.float32, name="params")))


def cmm_unet_init(h, seed=0):
    _check(_lib.cmm_unet_init(h, int(seed)))


def cmm_unet_get_params(h, params):
    import torch
    _check(_lib.cmm_unet_get_params(h, _dev(params, torch.float32, name="params")))


def cmm_unet_forward(h, x, out):
    import torch
    _check(_lib.cmm_unet_forward(h, x.shape[0], _dev(x, torch.float32, name="in"), _dev(out, torch.float32, name="out")))


def cmm_unet_loss_grad(h, x, target, grad=None):
    import torch
    loss = C.c_double()
    _check(_lib.cmm_unet_loss_grad(h, x.shape[0], _dev(x, torch.float32, name="in"),
                                   _dev(target, torch.float32, name="target"),
                                   _dev(grad, torch.float32, name="grad"), C.byref(loss)))
    return loss.value


def cmm_unet_train_step(h, x, target, lr):
    import torch
    loss = C.c_double()
    _check(_lib.cmm_unet_train_step(h, x.shape[0], _dev(x, torch.float32, name="in"),
                                    _dev(target, torch.float32, name="target"), float(lr), C.byref(loss)))
    return loss.value


def cmm_batch_solve(ops, pcs, bs, xs, tol=1e-6, maxit=500, check_every=10, cg_f32=False, flexible=False,
                    width=0, true_resid=True):
    """Batched PCG over parallel lists of operator / preconditioner handles and
    device maps; returns the list of SolveInfo."""
    n = len(ops)
    arr = lambda items: (C.c_void_p * n)(*[C.c_void_p(v if isinstance(v, int) else v.value) for v in items])
    opts = SolveOpts(float(tol), int(maxit), int(check_every), 1, 0, 1 if cg_f32 else 0, 0, 1 if flexible else 0,
                     0, 0, int(width), 0 if true_resid else 1, 0, 1)
    infos = (SolveInfo * n)()
    _check(_lib.cmm_batch_solve(n, arr(ops), arr(pcs), arr([t.data_ptr() for t in bs]),
                                arr([t.data_ptr() for t in xs]), C.byref(opts), infos))
    return list(infos)


def cmm_autotune(op, reps=3, cache_path=None):
    """Returns (log2 R, two-detector packing chosen, ms per application or -1 from a cache)."""
    lr = C.c_int32()
    pair = C.c_int32()
    ms = C.c_double()
    _check(_lib.cmm_autotune(op, int(reps), cache_path.encode() if cache_path else None, C.byref(lr),
                             C.byref(pair), C.byref(ms)))
    return int(lr.value), bool(pair.value), float(ms.value)


# ---------------------------------------------------------------- handle owners

class Context:
    def __init__(self, device=0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.device = device
        self.h = cmm_ctx_create(device, stream)

    def __del__(self):
        if getattr(self, "h", None):
            cmm_ctx_destroy(self.h)
            self.h = None


class Pointing:
    def __init__(self, ctx: Context, scan):
        self.ctx = ctx
        self.scan = scan
        self.shape = (scan.ncomp, scan.ny, scan.nx)
        self.h = cmm_pointing_create(ctx.h, scan.ny, scan.nx, scan.ncomp, scan.periodic,
                                     scan.det_off, scan.det_pol, scan.bore)

    def mask(self):
        return cmm_pointing_mask(self.h, self.scan.npix)

    def __del__(self):
        if getattr(self, "h", None):
            cmm_pointing_destroy(self.h)
            self.h = None


class Noise:
    def __init__(self, ctx: Context, noise, n_samp, f_samp):
        self.ctx = ctx
        self.n_det = noise.sigma.size
        self.h = cmm_noise_create(ctx.h, n_samp, f_samp, noise.sigma, noise.fknee, noise.alpha)

    def diag(self):
        return cmm_noise_diag(self.h, self.n_det)

    def set_correlated(self, corr):
        cmm_noise_set_correlated(self.h, corr)

    def set_table(self, w):
        cmm_noise_set_table(self.h, w)

    def __del__(self):
        if getattr(self, "h", None):
            cmm_noise_destroy(self.h)
            self.h = None


class Operator:
    """A = P^T N^-1 P for one scan and noise model."""

    def __init__(self, ctx: Context, scan, noise, precision=PREC_F32, det_chunk=0, corr=None):
        self.ctx = ctx
        self.pointing = Pointing(ctx, scan)
        self.noise = Noise(ctx, noise, scan.n_t, scan.f_samp)
        if corr is not None:
            self.noise.set_correlated(corr)
        self.shape = self.pointing.shape
        self.n_det, self.n_t = scan.n_det, scan.n_t
        self.h = cmm_op_create(ctx.h, self.pointing.h, self.noise.h, precision, det_chunk)

    def set_pixel_cache(self, enable=True):
        cmm_op_set_pixel_cache(self.h, enable)

    def set_pair_packing(self, enable=True):
        cmm_op_set_pair_packing(self.h, enable)

    def new_map(self):
        import torch
        return torch.zeros(self.shape, dtype=torch.float64, device=f"cuda:{self.ctx.device}")

    def apply(self, m, out=None):
        out = self.new_map() if out is None else out
        cmm_apply_A(self.h, m, out)
        return out

    def project(self, m, dtype=None):
        import torch
        tod = torch.empty((self.n_det, self.n_t), dtype=dtype or torch.float32, device=m.device)
        cmm_project(self.h, m, tod)
        return tod

    def rhs(self, tod, out=None):
        out = self.new_map() if out is None else out
        cmm_rhs(self.h, tod, out)
        return out

    def __del__(self):
        if getattr(self, "h", None):
            cmm_op_destroy(self.h)
            self.h = None


class Precon:
    """A preconditioner of an operator: PRECON_BINNED / _JACOBI (per-pixel blocks),
    _CIRCULANT (taper_sigma_px, ref_pixel, pd_eps), _CIRC_TILED (tiles = (ty, tx));
    white_diag weights the detectors by 1/sigma^2 instead of the exact diagonal of
    N^-1 (binned and circulant kinds)."""

    def __init__(self, op: Operator, kind, taper_sigma_px=0.0, ref_pixel=-1, pd_eps=0.0, tiles=(0, 0),
                 white_diag=False):
        self.op = op
        self.kind = kind
        self.h = cmm_precon_create(op.h, kind, taper_sigma_px, ref_pixel, pd_eps, tiles, white_diag)

    def apply(self, r, out=None):
        out = self.op.new_map() if out is None else out
        cmm_precon_apply(self.h, r, out)
        return out

    def clamped(self):
        return cmm_precon_clamped(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            cmm_precon_destroy(self.h)
            self.h = None


class UNet:
    """Owner of a cmm_unet handle (the learned correction of the circulant preconditioner)."""

    def __init__(self, ctx: Context, ny, nx, widths=(16, 32, 48, 96), batch_max=32):
        self.ctx = ctx
        self.shape = (3, ny, nx)
        self.widths = tuple(widths)
        self.h = cmm_unet_create(ctx.h, ny, nx, widths, batch_max)
        self.n_params = cmm_unet_param_count(self.h)

    def set_params(self, params):
        cmm_unet_set_params(self.h, params)

    def init(self, seed=0):
        cmm_unet_init(self.h, seed)

    def params(self):
        import torch
        p = torch.empty(self.n_params, dtype=torch.float32, device=f"cuda:{self.ctx.device}")
        cmm_unet_get_params(self.h, p)
        return p

    def __call__(self, x):
        import torch
        out = torch.empty_like(x, dtype=torch.float32)
        cmm_unet_forward(self.h, x, out)
        return out

    def __del__(self):
        if getattr(self, "h", None):
            cmm_unet_destroy(self.h)
            self.h = None


def solve(op: Operator, pc: Precon, b, x=None, tol=1e-6, maxit=500, check_every=10, use_graph=True,
          history=False, cg_f32=False, resid_replace=0, flexible=False, true_resid=True, window=1):
    """PCG on A x = b; returns (x, info, resid_hist, anorm_terms).  info.rel_resid is
    the recursive ||r|| / ||b||; info.true_rel_resid recomputes ||b - A x|| / ||b||
    from the returned x (one more application of A; -1 with true_resid=False)."""
    import torch
    x0_given = x is not None
    x = op.new_map() if x is None else x
    hist = torch.zeros(maxit + 1, dtype=torch.float64, device=b.device) if history else None
    terms = torch.zeros(max(maxit, 1), dtype=torch.float64, device=b.device) if history else None
    info = cmm_solve(op.h, pc.h, b, x, tol, maxit, check_every, use_graph, x0_given, hist, terms,
                     cg_f32, resid_replace, flexible, true_resid=true_resid, window=window)
    return x, info, hist, terms
