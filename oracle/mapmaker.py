"""Plain FP64 CPU oracle of the maximum-likelihood map-maker and its
preconditioners (Naess & Louis, "A fast map-making preconditioner for regular
scanning patterns").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA path; its only inputs are the seeded tables of the ``gen`` package.

Each function states the passage it follows.  Steps the paper leaves open are
taken as follows (the numbered readings):

R1  noise filter w_d(f) = 1 / (sigma_d^2 (1 + (f/f_knee)^-alpha)), f_k = k f_s / n_t,
    with f_knee = 0 meaning white noise.
R2  the DC bin, where the law diverges, takes the first non-zero bin's value.
R3  diag(N^-1) in Eq. 3 / Eq. 7 is the exact diagonal of the circulant filter,
    the mean of w over the two-sided DFT grid (option: the white level 1/sigma_d^2).
R4  Sigma in Eq. 7 is the symmetric positive square root of each block; a pixel
    whose unit-weight hit block has reciprocal condition < RCOND_MIN (or no hits)
    is masked: its samples are cut from P everywhere.
R5  the measured row is made symmetric, q_k <- (q_k + q_{-k}^T) / 2.
R6  each Hermitian mode block (Fq)*_f is inverted through its eigen-decomposition
    with eigenvalues floored at PD_EPS * (largest eigenvalue over all modes).
R7  Eq. 11 is applied block-wise with the element-wise conjugate, F unnormalised
    forward and 1/(ny nx) on the inverse.
R8  the regularising Gaussian (Sec. Regularization) is g(k) = exp(-|k|^2 / (2 s^2))
    over wrapped pixel offsets k in [-n/2, n/2); s = inf switches it off.
R9  the reference pixel is (ny // 2, nx // 2), else the nearest unmasked pixel
    (ties: smallest linear index).
R10 pointing is the integer fixed-point rule below; polarisation angle on the sky
    is psi_d + phi_t, phi_t the angle of the fixed-point rotation pair (the pair
    normalised for the response; positions use the integer pair as it is).
R11 PCG starts from x0 = 0 and stops when ||r_k|| / ||b|| <= tol.
R12 the A-norm error estimate of the Results footnote estimates the SQUARE of
    the error A-norm: ||x_i - x||_A^2 ~ sum_{j=i}^{i+d-1} alpha_j r_j^T z_j.
R13 noise correlated between detectors (the Test setup section's noise model had
    inter-detector correlations but the paper states no model): per real-FFT bin
    N(f) = D(f) + V E(f) V^T, D from R1, V fixed mode templates, E diagonal red mode
    spectra (DC at the first bin); N^-1 acts on the detectors' Fourier coefficients
    bin by bin.
R15 tiled circulant (the Summary's locally varying variant, not specified): tiles
    on a regular ty x tx grid, each with the circulant preconditioner measured at
    the unmasked pixel nearest its centre, merged as sum_t D_t M_t D_t with D_t the
    square roots of a raised-cosine partition of unity.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

RCOND_MIN = 1e-3
PD_EPS = 1e-6
DET_CHUNK = 16


# ---------------------------------------------------------------------------
# Pointing (Eq. 1: the sparse P; Sec. Test setup: response T + cos2psi Q + sin2psi U)
# ---------------------------------------------------------------------------

def sample_pixels(scan, dets):
    """Nearest pixel of every sample of detectors ``dets`` (R10).

    The rotated offset (ox, oy) = R(phi) (dx, dy) = (cphi dx - sphi dy, sphi dx + cphi dy)
    is exact in units of 2^-22 pixel; it is floored to 2^-16 pixel and added to the
    boresight: x = bx + floor(ox / 64); ix = floor((x + 2^15) / 2^16) (round half up),
    same for y.  Samples outside the map are -1 (cut) unless the scan is periodic,
    where the indices wrap.
    """
    bore = scan.bore.astype(np.int64)
    bx, by, cp, sp = bore[:, 0], bore[:, 1], bore[:, 2], bore[:, 3]
    dx = scan.det_off[dets, 0].astype(np.int64)[:, None]
    dy = scan.det_off[dets, 1].astype(np.int64)[:, None]
    ox = cp[None, :] * dx - sp[None, :] * dy
    oy = sp[None, :] * dx + cp[None, :] * dy
    x = bx[None, :] + np.floor_divide(ox, 64)
    y = by[None, :] + np.floor_divide(oy, 64)
    ix = np.floor_divide(x + (1 << 15), 1 << 16)
    iy = np.floor_divide(y + (1 << 15), 1 << 16)
    if scan.periodic:
        ix = np.mod(ix, scan.nx)
        iy = np.mod(iy, scan.ny)
        return iy * scan.nx + ix
    inside = (ix >= 0) & (ix < scan.nx) & (iy >= 0) & (iy < scan.ny)
    return np.where(inside, iy * scan.nx + ix, -1)


def sample_weights(scan, dets):
    """Rows of P: (1,) for T-only maps, (1, cos 2a, sin 2a) with a = psi_d + phi_t for
    TQU maps (Sec. Test setup), by angle addition from the tabulated cos/sin.

    phi_t is the angle of the fixed-point pair (cphi, sphi), whose length differs
    from one by the table's rounding (up to ~2^-16): the double angle is therefore
    formed from the normalised pair, cos 2phi = (c^2 - s^2) / (c^2 + s^2) and
    sin 2phi = 2 c s / (c^2 + s^2) (R10), so the row is the paper's unit response."""
    nd = len(np.atleast_1d(dets))
    if scan.ncomp == 1:
        return np.ones((1, nd, scan.n_t))
    cf = scan.bore[:, 2].astype(np.float64) * 2.0 ** -15
    sf = scan.bore[:, 3].astype(np.float64) * 2.0 ** -15
    r2 = cf * cf + sf * sf
    c2f = (cf * cf - sf * sf) / r2
    s2f = 2.0 * cf * sf / r2
    c2p = scan.det_pol[dets, 0][:, None]
    s2p = scan.det_pol[dets, 1][:, None]
    c = c2p * c2f[None, :] - s2p * s2f[None, :]
    s = s2p * c2f[None, :] + c2p * s2f[None, :]
    return np.stack([np.ones_like(c), c, s])


def hit_blocks(scan, det_weight=None, mask=None):
    """Per-pixel blocks sum_t u_d P_t P_t^T over the samples hitting each pixel
    (Eq. 3-5); u_d = 1 (Jacobi / hit matrix) unless ``det_weight`` is given.
    Samples of masked pixels are skipped when ``mask`` is given."""
    nc, npix = scan.ncomp, scan.npix
    out = np.zeros((nc, nc, npix))
    for d0 in range(0, scan.n_det, DET_CHUNK):
        dets = np.arange(d0, min(scan.n_det, d0 + DET_CHUNK))
        pix = sample_pixels(scan, dets)
        if mask is not None:
            pix = np.where((pix >= 0) & mask[np.maximum(pix, 0)], pix, -1)
        wts = sample_weights(scan, dets)
        u = np.ones(dets.size) if det_weight is None else det_weight[dets]
        ok = pix >= 0
        for a in range(nc):
            for b in range(nc):
                vals = (wts[a] * wts[b] * u[:, None])[ok]
                out[a, b] += np.bincount(pix[ok], weights=vals, minlength=npix)
    return out.transpose(2, 0, 1)          # [npix, nc, nc]


def pixel_mask(scan):
    """R4: keep pixels whose unit-weight hit block is well conditioned."""
    h = hit_blocks(scan)
    if scan.ncomp == 1:
        return h[:, 0, 0] > 0
    ev = np.linalg.eigvalsh(h)
    return (ev[:, -1] > 0) & (ev[:, 0] >= RCOND_MIN * ev[:, -1])


# ---------------------------------------------------------------------------
# Noise model (Eq. 1: gaussian n with covariance N; Fig. 3: a noise PSD)
# ---------------------------------------------------------------------------

def filter_weights(noise, n_t, f_samp):
    """w_d(f_k) = 1 / PSD_d(f_k), k = 0 .. n_t/2 (R1, R2): the eigenvalues of the
    circulant N_d^-1."""
    k = np.arange(n_t // 2 + 1)
    f = k * (f_samp / n_t)
    f[0] = f[1]
    out = np.empty((noise.sigma.size, k.size))
    for d in range(noise.sigma.size):
        if noise.fknee[d] > 0:
            psd = noise.sigma[d] ** 2 * (1.0 + (f / noise.fknee[d]) ** (-noise.alpha[d]))
        else:
            psd = np.full(f.shape, noise.sigma[d] ** 2)
        out[d] = 1.0 / psd
    return out


def white_weights(noise):
    """R3's alternative detector weight: the white level 1 / sigma_d^2 of the law R1."""
    return 1.0 / noise.sigma ** 2


def detector_weights(op, white=False):
    """The per-detector diag(N^-1) of Eq. 3 and Eq. 7: R3 (exact circulant diagonal),
    or with ``white`` its alternative 1 / sigma_d^2."""
    return white_weights(op.noise) if white else ninv_diagonal(op.w, op.scan.n_t)


def ninv_diagonal(w, n_t):
    """R3: diagonal of the circulant N_d^-1 = mean of w over the full DFT grid."""
    inner = w[:, 1:n_t // 2].sum(axis=1)
    return (w[:, 0] + 2.0 * inner + w[:, n_t // 2]) / n_t


def apply_ninv(w, tod):
    """N^-1 applied per detector as a Fourier-diagonal filter: irfft(w * rfft(tod))."""
    n_t = tod.shape[-1]
    return np.fft.irfft(w * np.fft.rfft(tod, axis=-1), n=n_t, axis=-1)


# ---------------------------------------------------------------------------
# Noise correlated between detectors (extension: the paper's test noise model had
# inter-detector correlations, Sec. Test setup, without stating the model)
# ---------------------------------------------------------------------------
#
# Reading R13: per real-FFT bin k, the detectors' noise covariance is
#   N(f_k) = D(f_k) + V E(f_k) V^T,
# D = diag(PSD_d(f_k)) the per-detector law of R1, V [n_det, r] fixed mode templates
# (common mode, focal-plane gradients), E = diag(e_j(f_k)) with
# e_j(f) = amp_j^2 (1 + (f / fknee_j)^-alpha_j), DC at the first bin as in R2.
# N^-1 acts on the vector of the detectors' Fourier coefficients at each bin (the
# same real matrix at k and n_t - k, so the filtered TOD stays real).  The model's
# parameters come in a gen.CorrNoise (modes V, amp, fknee, alpha).

def mode_psd(corr, n_t, f_samp):
    """e_j(f_k), k = 0 .. n_t/2 (R13); [r, n_t/2 + 1]."""
    k = np.arange(n_t // 2 + 1)
    f = k * (f_samp / n_t)
    f[0] = f[1]
    return np.stack([corr.amp[j] ** 2 * (1.0 + (f / corr.fknee[j]) ** (-corr.alpha[j]))
                     for j in range(corr.amp.size)])


def corr_covariance(w, corr, e):
    """N(f_k) for every bin: [K, n_det, n_det] = diag(1 / w[:, k]) + V diag(e[:, k]) V^T."""
    V = corr.modes
    cov = np.einsum("dj,jk,ej->kde", V, e, V)
    idx = np.arange(V.shape[0])
    cov[:, idx, idx] += (1.0 / w).T
    return cov


def apply_ninv_corr(w, corr, e, tod):
    """N^-1 applied by its definition: per bin k, solve N(f_k) y = x for the vector
    x of the detectors' rfft coefficients, then irfft (R13)."""
    n_t = tod.shape[-1]
    X = np.fft.rfft(tod, axis=-1)
    cov = corr_covariance(w, corr, e)
    Y = np.linalg.solve(cov, X.T[:, :, None])[:, :, 0].T
    return np.fft.irfft(Y, n=n_t, axis=-1)


def apply_ninv_corr_woodbury(w, corr, e, tod):
    """The same by the Woodbury identity, N^-1 = D^-1 - D^-1 V (E^-1 + V^T D^-1 V)^-1
    V^T D^-1 (r x r solves per bin): the form the GPU path evaluates."""
    n_t = tod.shape[-1]
    V = corr.modes
    X = np.fft.rfft(tod, axis=-1)
    WX = w * X                                            # D^-1 x
    t = np.einsum("dj,dk->kj", V, WX)                    # V^T D^-1 x
    M = np.einsum("dj,dk,dl->kjl", V, w, V)              # V^T D^-1 V
    r = V.shape[1]
    M[:, np.arange(r), np.arange(r)] += (1.0 / e).T      # + E^-1
    s = np.linalg.solve(M, t[:, :, None])[:, :, 0]        # [K, r]
    Y = WX - w * np.einsum("dj,kj->dk", V, s)
    return np.fft.irfft(Y, n=n_t, axis=-1)


# ---------------------------------------------------------------------------
# The operator A = P^T N^-1 P (Eq. 2)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Operator:
    scan: object
    noise: object
    mask: np.ndarray
    w: np.ndarray
    corr: object = None          # CorrNoise or None (independent detectors)
    e: np.ndarray = None         # mode PSDs of corr

    @property
    def shape(self):
        return (self.scan.ncomp, self.scan.ny, self.scan.nx)


def make_operator(scan, noise, mask=None, corr=None, w=None):
    """w: tabulated weights w_d(f_k) [n_det, n_t/2 + 1] replacing the law of R1."""
    if mask is None:
        mask = pixel_mask(scan)
    e = None if corr is None else mode_psd(corr, scan.n_t, scan.f_samp)
    if w is None:
        w = filter_weights(noise, scan.n_t, scan.f_samp)
    return Operator(scan, noise, np.asarray(mask, bool), np.asarray(w, np.float64), corr, e)


def _ninv(op, tod, dets):
    if op.corr is None:
        return apply_ninv(op.w[dets], tod)
    return apply_ninv_corr(op.w, op.corr, op.e, tod)


def _pix(op, dets):
    pix = sample_pixels(op.scan, dets)
    return np.where((pix >= 0) & op.mask[np.maximum(pix, 0)], pix, -1)


def project(op, m, dets=None):
    """P m (Eq. 1): tod[d, t] = sum_c P_{dt,c} m[c, pix(d, t)], 0 for cut samples."""
    if dets is None:
        dets = np.arange(op.scan.n_det)
    pix = _pix(op, dets)
    wts = sample_weights(op.scan, dets)
    flat = m.reshape(op.scan.ncomp, -1)
    safe = np.maximum(pix, 0)
    tod = np.zeros(pix.shape)
    for c in range(op.scan.ncomp):
        tod += wts[c] * flat[c][safe]
    return np.where(pix >= 0, tod, 0.0)


def bin_tod(op, tod, dets=None):
    """P^T tod (Eq. 2): out[c, p] = sum over samples hitting p of P_{dt,c} tod[d, t]."""
    if dets is None:
        dets = np.arange(op.scan.n_det)
    pix = _pix(op, dets)
    wts = sample_weights(op.scan, dets)
    ok = pix >= 0
    out = np.empty((op.scan.ncomp, op.scan.npix))
    for c in range(op.scan.ncomp):
        out[c] = np.bincount(pix[ok], weights=(wts[c] * tod)[ok], minlength=op.scan.npix)
    return out.reshape(op.shape)


def binning_magnitude(op, m):
    """Scale of the rounding error of the binning sums of A m = P^T N^-1 P m (Eq. 2),
    for error bounds in tests: S[c, p] = sum over the samples hitting p of
    |P_{dt,c} (N^-1 P m)_{dt}| (no cancellation), and h[p], the number of those
    samples.  Not a step of the method."""
    dets = np.arange(op.scan.n_det)
    y = _ninv(op, project(op, m, dets), dets)
    pix = _pix(op, dets)
    wts = sample_weights(op.scan, dets)
    ok = pix >= 0
    s = np.empty((op.scan.ncomp, op.scan.npix))
    for c in range(op.scan.ncomp):
        s[c] = np.bincount(pix[ok], weights=np.abs(wts[c] * y)[ok], minlength=op.scan.npix)
    h = np.bincount(pix[ok], minlength=op.scan.npix)
    return s.reshape(op.shape), h.reshape(op.shape[1:])


def _chunks(op):
    # correlated noise couples the detectors: one chunk holding all of them
    step = DET_CHUNK if op.corr is None else op.scan.n_det
    for d0 in range(0, op.scan.n_det, step):
        yield np.arange(d0, min(op.scan.n_det, d0 + step))


def apply_A(op, m):
    """A m = P^T N^-1 P m (Eq. 2), accumulated over detector chunks."""
    out = np.zeros(op.shape)
    for dets in _chunks(op):
        tod = project(op, m, dets)
        out += bin_tod(op, _ninv(op, tod, dets), dets)
    return out


def rhs(op, d):
    """b = P^T N^-1 d (right-hand side of Eq. 2)."""
    out = np.zeros(op.shape)
    for dets in _chunks(op):
        out += bin_tod(op, _ninv(op, d[dets], dets), dets)
    return out


def dense_A(op):
    """Every row of A by one operator application each (Eq. 6), over unmasked pixels.
    Returns (A [n, n], index arrays (comp, pixel) of the n unknowns)."""
    nc = op.scan.ncomp
    pix = np.flatnonzero(op.mask)
    comp = np.repeat(np.arange(nc), pix.size)
    pixs = np.tile(pix, nc)
    n = comp.size
    a = np.empty((n, n))
    for i in range(n):
        e = np.zeros(op.shape)
        e.reshape(nc, -1)[comp[i], pixs[i]] = 1.0
        a[:, i] = apply_A(op, e).reshape(nc, -1)[comp, pixs]
    return a, (comp, pixs)


# ---------------------------------------------------------------------------
# Binned and Jacobi preconditioners (Eq. 3-5)
# ---------------------------------------------------------------------------

def _block_inverse(blocks, mask):
    out = np.zeros_like(blocks)
    out[mask] = np.linalg.inv(blocks[mask])
    return out


def _apply_blocks(blocks, x):
    nc = x.shape[0]
    flat = x.reshape(nc, -1)
    return np.einsum("pab,bp->ap", blocks, flat).reshape(x.shape)


class BlockPrecon:
    """M = (per-pixel block of P^T D P)^-1 with D = diag(N^-1) (binned, Eq. 3-4)
    or D = I (Jacobi, Eq. 5, a = 1)."""

    def __init__(self, op, kind="binned", white=False):
        u = detector_weights(op, white) if kind == "binned" else None
        self.blocks = hit_blocks(op.scan, u, op.mask)
        self.inv = _block_inverse(self.blocks, op.mask)

    def __call__(self, r):
        return _apply_blocks(self.inv, r)


# ---------------------------------------------------------------------------
# Circulant (constant-correlation) preconditioner (Sec. Implementation,
# Regularization, Polarization; Eq. 7-13)
# ---------------------------------------------------------------------------

def _sym_sqrt(blocks, mask):
    """R4: Sigma = B^(1/2) and Sigma^-1 = B^(-1/2), symmetric, per unmasked pixel."""
    sig = np.zeros_like(blocks)
    sig_inv = np.zeros_like(blocks)
    lam, vec = np.linalg.eigh(blocks[mask])
    sig[mask] = np.einsum("pak,pk,pbk->pab", vec, np.sqrt(lam), vec)
    sig_inv[mask] = np.einsum("pak,pk,pbk->pab", vec, 1.0 / np.sqrt(lam), vec)
    return sig, sig_inv


def reference_pixel(mask, ny, nx):
    """R9."""
    p0 = (ny // 2) * nx + nx // 2
    if mask[p0]:
        return p0
    iy, ix = np.divmod(np.flatnonzero(mask), nx)
    cand = np.flatnonzero(mask)
    d2 = (iy - ny // 2) ** 2 + (ix - nx // 2) ** 2
    best = d2.min()
    return int(cand[d2 == best].min())


def wrapped_offsets(n):
    """Offsets 0..n-1 wrapped into [-n/2, n/2) (even n) or [-(n-1)/2, (n-1)/2] (odd n)."""
    k = np.arange(n)
    return np.where(k < (n + 1) // 2, k, k - n)


def taper(ny, nx, sigma):
    """R8: g(k) over wrapped offsets; sigma = inf gives g = 1."""
    if not np.isfinite(sigma):
        return np.ones((ny, nx))
    ky = wrapped_offsets(ny)[:, None].astype(np.float64)
    kx = wrapped_offsets(nx)[None, :].astype(np.float64)
    return np.exp(-(ky ** 2 + kx ** 2) / (2.0 * sigma ** 2))


def tile_windows_1d(n, t):
    """R15: t raised-cosine windows on n pixels, centres c_i = (i + 1/2) n / t, spacing
    h = n / t: w_i(y) = cos^2(pi (y - c_i) / (2 h)) within h of c_i, the outermost
    windows held at 1 beyond their centres; sum_i w_i = 1 everywhere."""
    y = np.arange(n, dtype=np.float64)
    h = n / t
    out = np.zeros((t, n))
    for i in range(t):
        c = (i + 0.5) * h
        u = (y - c) / h
        w = np.where(np.abs(u) <= 1.0, np.cos(0.5 * np.pi * u) ** 2, 0.0)
        if i == 0:
            w = np.where(y <= c, 1.0, w)
        if i == t - 1:
            w = np.where(y >= c, 1.0, w)
        out[i] = w
    return out


def tile_windows(ny, nx, ty, tx):
    """phi_t(y, x) = w_i(y) w_j(x), t = i tx + j: a partition of unity over the map."""
    wy, wx = tile_windows_1d(ny, ty), tile_windows_1d(nx, tx)
    return np.einsum("iy,jx->ijyx", wy, wx).reshape(ty * tx, ny, nx)


def tile_reference(mask, ny, nx, cy, cx):
    """The unmasked pixel nearest (cy, cx), ties to the lowest index (R9 at a tile centre)."""
    cand = np.flatnonzero(mask)
    iy, ix = np.divmod(cand, nx)
    d2 = (iy - cy) ** 2 + (ix - cx) ** 2
    return int(cand[d2 == d2.min()].min())


class TiledCirculantPrecon:
    """Locally varying circulant preconditioner (Summary section: tiles with their
    own constant-correlation model), reading R15: a circulant M_t measured at each
    tile's centre, merged with the partition of unity phi_t,
    M = sum_t D_t M_t D_t, D_t = diag(sqrt(phi_t)) on every Stokes component
    (symmetric positive definite whenever every M_t is)."""

    def __init__(self, op, tiles=(2, 2), taper_sigma=math.inf, pd_eps=PD_EPS, white=False):
        nc, ny, nx = op.shape
        ty, tx = tiles
        self.shape = op.shape
        self.sqrt_phi = np.sqrt(tile_windows(ny, nx, ty, tx))
        self.parts = []
        for i in range(ty):
            for j in range(tx):
                ref = tile_reference(op.mask, ny, nx, int((i + 0.5) * ny / ty), int((j + 0.5) * nx / tx))
                self.parts.append(CirculantPrecon(op, taper_sigma=taper_sigma, ref=ref, pd_eps=pd_eps,
                                                  white=white))

    def __call__(self, r):
        z = np.zeros(self.shape)
        for d, m in zip(self.sqrt_phi, self.parts):
            z += d[None] * m(d[None] * r)
        return z


def circulant_forward(q, x):
    """Q x for the circulant Q_ij = q_{j-i} through Eq. 11 (R7):
    F^-1 (Fq)* F x, block-wise.  q: [nc, nc, ny, nx] real, x: [nc, ny, nx]."""
    h = np.conj(np.fft.fft2(q, axes=(-2, -1)))
    xf = np.fft.fft2(x, axes=(-2, -1))
    yf = np.einsum("abyx,byx->ayx", h, xf)
    return np.fft.ifft2(yf, axes=(-2, -1)).real


class CirculantPrecon:
    """M_C = Sigma^-1 F^-1 ((Fq)*)^-1 F Sigma^-T (Eq. 12), built from the rows
    A e_{ref,gamma} (Eq. 6, Eq. 13)."""

    def __init__(self, op, taper_sigma=math.inf, ref=None, pd_eps=PD_EPS, white=False):
        scan = op.scan
        nc, ny, nx = op.shape
        self.nc, self.ny, self.nx = nc, ny, nx
        # Eq. 7: Sigma^T Sigma = binned block
        u = detector_weights(op, white)
        blocks = hit_blocks(scan, u, op.mask)
        self.sigma, self.sigma_inv = _sym_sqrt(blocks, op.mask)
        self.ref = reference_pixel(op.mask, ny, nx) if ref is None else int(ref)
        # Eq. 6: one row of A per Stokes component of the reference pixel
        rows = np.empty((nc, nc, scan.npix))            # rows[gamma, delta, j]
        for g in range(nc):
            e = np.zeros(op.shape)
            e.reshape(nc, -1)[g, self.ref] = 1.0
            rows[g] = apply_A(op, e).reshape(nc, -1)
        self.rows = rows
        # Eq. 13: Q_{ref a, j b} = Sigma^-T_{ref a g} (A e_{ref g})_{j d} Sigma^-1_{j d b}
        s_ref = self.sigma_inv[self.ref]
        t = np.einsum("ga,gdj->adj", s_ref, rows)        # Sigma^-T = (Sigma^-1)^T
        qrow = np.einsum("adj,jdb->abj", t, self.sigma_inv).reshape(nc, nc, ny, nx)
        # Eq. 10: Q_ij = q_{j-i}: offsets relative to the reference pixel
        ry, rx = divmod(self.ref, nx)
        q = np.roll(qrow, shift=(-ry, -rx), axis=(-2, -1))
        # R5: symmetrise, q_k <- (q_k + q_{-k}^T) / 2
        qneg = np.roll(q[:, :, ::-1, ::-1], shift=(1, 1), axis=(-2, -1))
        q = 0.5 * (q + qneg.transpose(1, 0, 2, 3))
        # Sec. Regularization: multiply q by a Gaussian
        q = q * taper(ny, nx, taper_sigma)[None, None]
        self.q = q
        # Eq. 11: (F Q F^-1)_ff = (Fq)*_f
        h = np.conj(np.fft.fft2(q, axes=(-2, -1)))       # [a, b, y, x]
        hm = h.transpose(2, 3, 0, 1)                      # [y, x, a, b], Hermitian
        lam, vec = np.linalg.eigh(hm)
        floor = pd_eps * lam.max()
        self.n_clamped = int((lam < floor).sum())
        lam = np.maximum(lam, floor)
        self.h_inv = np.einsum("yxak,yxk,yxbk->yxab", vec, 1.0 / lam, np.conj(vec))

    def __call__(self, r):
        """Eq. 12: z = Sigma^-1 F^-1 ((Fq)*)^-1 F Sigma^-T r."""
        y = _apply_blocks(self.sigma_inv, r)             # Sigma symmetric: Sigma^-T = Sigma^-1
        yf = np.fft.fft2(y, axes=(-2, -1))
        zf = np.einsum("yxab,byx->ayx", self.h_inv, yf)
        z = np.fft.ifft2(zf, axes=(-2, -1)).real
        return _apply_blocks(self.sigma_inv, z)

    def approx_A(self, x):
        """M_C^-1 x = Sigma^T Q Sigma x (Eq. 8), through Eq. 11."""
        y = _apply_blocks(self.sigma, x)
        return _apply_blocks(self.sigma, circulant_forward(self.q, y))


# ---------------------------------------------------------------------------
# Preconditioned conjugate gradients (Introduction, footnote on PCG; Results
# footnote on the A-norm error)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class SolveInfo:
    iterations: int
    converged: bool
    rel_resid: list
    anorm_terms: list       # alpha_j * r_j^T z_j
    iterates: list | None = None


def pcg(apply_a, apply_m, b, tol=1e-6, maxit=1000, x0=None, flexible=False, keep_iterates=False, window=1):
    """PCG on A x = b with preconditioner M (R11); with ``flexible`` the
    Polak-Ribiere beta = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k) (flexible CG) is used.
    With ``flexible`` and ``window`` m > 1: truncated flexible CG, FCG(m) (Notay 2000),
    see fcg().  Returns (x, SolveInfo)."""
    if flexible and window > 1:
        return fcg(apply_a, apply_m, b, window, tol=tol, maxit=maxit, x0=x0, keep_iterates=keep_iterates)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_a(x) if x0 is not None else b.copy()
    bnorm = math.sqrt(float(np.vdot(b, b)))
    z = apply_m(r)
    p = z.copy()
    rho = float(np.vdot(r, z))
    hist = [math.sqrt(float(np.vdot(r, r))) / bnorm]
    terms = []
    iters = [x.copy()] if keep_iterates else None
    converged = hist[0] <= tol
    k = 0
    while not converged and k < maxit:
        q = apply_a(p)
        alpha = rho / float(np.vdot(p, q))
        terms.append(alpha * rho)
        x = x + alpha * p
        r_old = r
        r = r - alpha * q
        k += 1
        hist.append(math.sqrt(float(np.vdot(r, r))) / bnorm)
        if keep_iterates:
            iters.append(x.copy())
        if hist[-1] <= tol:
            converged = True
            break
        z_new = apply_m(r)
        rho_new = float(np.vdot(r, z_new))
        if flexible:
            beta = float(np.vdot(z_new, r - r_old)) / rho
        else:
            beta = rho_new / rho
        p = z_new + beta * p
        z, rho = z_new, rho_new
    return x, SolveInfo(k, converged, hist, terms, iters)


def fcg(apply_a, apply_m, b, window, tol=1e-6, maxit=1000, x0=None, keep_iterates=False):
    """Truncated flexible conjugate gradients FCG(m), m = ``window`` (Notay 2000, for a
    preconditioner that changes from one iteration to the next, such as M_C followed
    by a nonlinear learned correction).  Each new direction is the preconditioned
    residual made A-conjugate to the previous m directions,
        p_i = z_i - sum_{j = i-m}^{i-1} (z_i^T A p_j / p_j^T A p_j) p_j,
    and the step is alpha_i = p_i^T r_i / p_i^T A p_i.  For a fixed symmetric positive
    definite M it produces the PCG iterates (exact arithmetic).  SolveInfo.terms
    holds alpha_i p_i^T r_i.  Returns (x, SolveInfo)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_a(x) if x0 is not None else b.copy()
    bnorm = math.sqrt(float(np.vdot(b, b)))
    hist = [math.sqrt(float(np.vdot(r, r))) / bnorm]
    terms = []
    iters = [x.copy()] if keep_iterates else None
    converged = hist[0] <= tol
    kept = []   # (p_j, A p_j, p_j^T A p_j) of the last `window` steps
    k = 0
    p = apply_m(r)
    while not converged and k < maxit:
        q = apply_a(p)
        pq = float(np.vdot(p, q))
        alpha = float(np.vdot(p, r)) / pq
        terms.append(alpha * float(np.vdot(p, r)))
        x = x + alpha * p
        r = r - alpha * q
        kept.append((p, q, pq))
        if len(kept) > window:
            kept.pop(0)
        k += 1
        hist.append(math.sqrt(float(np.vdot(r, r))) / bnorm)
        if keep_iterates:
            iters.append(x.copy())
        if hist[-1] <= tol:
            converged = True
            break
        z = apply_m(r)
        p = z.copy()
        for pj, qj, pqj in kept:
            p = p - (float(np.vdot(z, qj)) / pqj) * pj
    return x, SolveInfo(k, converged, hist, terms, iters)


def anorm_estimate(terms, d=4):
    """R12: estimate of ||x_i - x||_A^2 from the next d terms alpha_j r_j^T z_j."""
    terms = np.asarray(terms)
    n = terms.size
    return np.array([terms[i:i + d].sum() for i in range(max(0, n - d + 1))])
