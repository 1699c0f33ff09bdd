"""Seeded synthetic inputs for the map-maker: scan tables, focal planes, noise
parameters, skies and noise time streams.

This module holds no map-making arithmetic.  It draws the numbers that the
paper's test setup (Sec. "Test setup") takes from ACT scans and noise models,
which are not available here, and quantises the pointing into the integer
fixed-point tables that both the oracle and the CUDA path take as input.

Conventions shared with the consumers (they are input formats, not method):

* map: ``ny x nx`` pixels, pixel ``(iy, ix)`` centred at coordinate
  ``(x, y) = (ix, iy)`` in pixel units; linear index ``p = iy * nx + ix``;
  Stokes-major storage ``[ncomp][ny][nx]`` (ncomp 1 = T, 3 = T, Q, U).
* boresight table ``bore``: int32 ``[n_t, 4]`` = (bx, by, cphi, sphi) with
  bx, by in units of 2^-16 pixel and (cphi, sphi) = (cos phi, sin phi) of the
  sky rotation in units of 2^-15 (|cphi|, |sphi| <= 2^15).
* detector table ``det_off``: int32 ``[n_det, 2]`` = (dx, dy) in units of 2^-7
  pixel (|dx|, |dy| < 2^14);
  ``det_pol``: float64 ``[n_det, 2]`` = (cos 2psi, sin 2psi).
* noise: per detector (sigma, f_knee, alpha) of PSD(f) = sigma^2 (1 + (f/f_knee)^-alpha).

Every random draw comes from ``np.random.default_rng(SeedSequence([cfg, realisation, kind]))``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

QB = 1 << 16   # boresight position units per pixel
QR = 1 << 15   # rotation cos/sin units
QD = 1 << 7    # detector offset units per pixel

KIND = {"sky": 0, "noise": 1, "psi": 2, "sigma": 3, "fknee": 4, "vec": 5, "misc": 6}


def rng(cfg: int, real: int, kind: str) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(cfg), int(real), KIND[kind]]))


@dataclasses.dataclass
class Scan:
    ny: int
    nx: int
    bore: np.ndarray        # int32 [n_t, 4]
    det_off: np.ndarray     # int32 [n_det, 2]
    det_pol: np.ndarray     # float64 [n_det, 2]
    f_samp: float = 400.0
    periodic: bool = False
    ncomp: int = 3

    @property
    def n_t(self) -> int:
        return int(self.bore.shape[0])

    @property
    def n_det(self) -> int:
        return int(self.det_off.shape[0])

    @property
    def npix(self) -> int:
        return self.ny * self.nx

    def subset(self, dets) -> "Scan":
        dets = np.asarray(dets)
        return dataclasses.replace(self, det_off=np.ascontiguousarray(self.det_off[dets]),
                                   det_pol=np.ascontiguousarray(self.det_pol[dets]))


@dataclasses.dataclass
class Noise:
    sigma: np.ndarray   # float64 [n_det]
    fknee: np.ndarray   # float64 [n_det]; 0 means white noise
    alpha: np.ndarray   # float64 [n_det]

    def subset(self, dets) -> "Noise":
        dets = np.asarray(dets)
        return Noise(self.sigma[dets].copy(), self.fknee[dets].copy(), self.alpha[dets].copy())


# ---------------------------------------------------------------------------
# focal planes
# ---------------------------------------------------------------------------

def grid_focal_plane(ncols: int, nrows: int, spacing_px: float) -> np.ndarray:
    """Rectangular grid of offsets (float pixels), x fastest, centred on 0."""
    ix = (np.arange(ncols) - (ncols - 1) / 2.0) * spacing_px
    iy = (np.arange(nrows) - (nrows - 1) / 2.0) * spacing_px
    yy, xx = np.meshgrid(iy, ix, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def hex_focal_plane(n_det: int, rings: int, spacing_px: float) -> np.ndarray:
    """The n_det sites of a hexagonal lattice (``rings`` rings) nearest the centre,
    ties broken by polar angle."""
    pts = []
    for a in range(-rings, rings + 1):
        for b in range(-rings, rings + 1):
            c = -a - b
            if max(abs(a), abs(b), abs(c)) <= rings:
                x = spacing_px * (a + 0.5 * b)
                y = spacing_px * (math.sqrt(3.0) / 2.0) * b
                pts.append((x, y))
    pts = np.array(pts)
    r = np.round(np.hypot(pts[:, 0], pts[:, 1]), 9)
    ang = np.round(np.mod(np.arctan2(pts[:, 1], pts[:, 0]), 2 * np.pi), 9)
    order = np.lexsort((ang, r))
    if n_det > len(pts):
        raise ValueError("not enough lattice sites")
    return pts[order[:n_det]]


# ---------------------------------------------------------------------------
# scan law
# ---------------------------------------------------------------------------

def _quantise_bore(bx, by, phi):
    bore = np.empty((bx.shape[0], 4), np.int32)
    bore[:, 0] = np.round(bx * QB).astype(np.int64)
    bore[:, 1] = np.round(by * QB).astype(np.int64)
    bore[:, 2] = np.round(np.cos(phi) * QR).astype(np.int64)
    bore[:, 3] = np.round(np.sin(phi) * QR).astype(np.int64)
    return bore


def sweep_offsets(t, speed, throw, accel=None):
    """Azimuth offset a(t) of a back-and-forth sweep of peak-to-peak ``throw`` at
    cruise ``speed``.  accel None: instant reversal (a triangle wave).  Otherwise the
    sweep brakes and reverses at constant ``accel`` over the last speed^2/(2 accel)
    of each end, as a telescope must."""
    A = 0.5 * throw
    if accel is None:
        period = 2.0 * throw / speed
        ph = np.mod(t / period, 1.0)
        return A * np.where(ph < 0.5, -1.0 + 4.0 * ph, 3.0 - 4.0 * ph)
    d = speed * speed / (2.0 * accel)          # braking distance
    if d > A:
        raise ValueError("acceleration too low for this throw and speed")
    tc = (2.0 * A - 2.0 * d) / speed            # cruise time of one leg
    tr = 2.0 * speed / accel                    # time of one reversal
    tau = np.mod(t, 2.0 * (tc + tr))
    a = np.empty_like(tau)
    s1 = tau < tc
    s2 = (tau >= tc) & (tau < tc + tr)
    s3 = (tau >= tc + tr) & (tau < 2 * tc + tr)
    s4 = tau >= 2 * tc + tr
    u = tau - tc
    w = tau - 2 * tc - tr
    a[s1] = -A + d + speed * tau[s1]
    a[s2] = (A - d) + speed * u[s2] - 0.5 * accel * u[s2] ** 2
    a[s3] = (A - d) - speed * (tau[s3] - tc - tr)
    a[s4] = (-A + d) - speed * w[s4] + 0.5 * accel * w[s4] ** 2
    return a


def drift_scan_positions(n_t, ny, nx, f_samp, speed_px_s, throw_px, segments, margin_px, accel_px_s2=None):
    """Boresight of constant-elevation drift scans in map-pixel coordinates.

    B(t) = C + R(phi(t)) (a(t), 0) + (0, y(t)): a(t) is the sweep of
    ``sweep_offsets`` (peak-to-peak ``throw_px`` at ``speed_px_s``, reversals at
    ``accel_px_s2`` or instant); the sky rotation phi(t) and the drift y(t) are
    linear within each segment.  ``segments`` is a list of (fraction of samples,
    phi_start_deg, phi_end_deg, rising) tuples; a rising segment drifts from below
    the map to above it, a setting one back down.
    """
    t = np.arange(n_t, dtype=np.float64) / f_samp
    a = sweep_offsets(t, speed_px_s, throw_px, accel_px_s2)
    phi = np.empty(n_t)
    yd = np.empty(n_t)
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    half = ny / 2.0 + margin_px
    start = 0
    for k, (frac, p0, p1, rising) in enumerate(segments):
        stop = n_t if k == len(segments) - 1 else start + int(round(frac * n_t))
        n = stop - start
        u = (np.arange(n) + 0.5) / n
        phi[start:stop] = np.deg2rad(p0 + (p1 - p0) * u)
        yd[start:stop] = (-half + 2 * half * u) if rising else (half - 2 * half * u)
        start = stop
    bx = cx + np.cos(phi) * a
    by = cy + np.sin(phi) * a + yd
    return bx, by, phi


def make_scan(*, cfg, real=0, ny, nx, n_t, focal_px, f_samp=400.0, speed_px_s=120.0,
              throw_px=240.0, segments=((1.0, -15.0, 15.0, True),), ncomp=3,
              margin_px=None, accel_px_s2=None):
    focal_px = np.asarray(focal_px, np.float64)
    if margin_px is None:
        margin_px = float(np.abs(focal_px).max()) + 2.0
    bx, by, phi = drift_scan_positions(n_t, ny, nx, f_samp, speed_px_s, throw_px,
                                       list(segments), margin_px, accel_px_s2)
    bore = _quantise_bore(bx, by, phi)
    det_off = np.round(focal_px * QD).astype(np.int32)
    psi = rng(cfg, real, "psi").uniform(0.0, np.pi, size=focal_px.shape[0])
    det_pol = np.stack([np.cos(2 * psi), np.sin(2 * psi)], axis=1)
    return Scan(ny=ny, nx=nx, bore=bore, det_off=det_off, det_pol=det_pol,
                f_samp=f_samp, periodic=False, ncomp=ncomp)


def bccb_scan(ny, nx, n_t, diagonal=False, ncomp=3):
    """Periodic, translation-invariant scan: one detector row per map row, three
    detectors per row at psi = 0, pi/6, pi/3, each sweeping x = t mod nx (one pixel
    per sample), no sky rotation.  With ``diagonal`` the sweep also advances y by
    one pixel per sample, which correlates neighbouring rows.  A = P^T N^-1 P is
    then block circulant with circulant blocks whenever every detector has the
    same noise."""
    per = math.lcm(nx, ny) if diagonal else nx
    if n_t % per:
        raise ValueError("n_t must be a multiple of the scan period")
    t = np.arange(n_t, dtype=np.int64)
    bore = np.zeros((n_t, 4), np.int32)
    bore[:, 0] = (t % nx) * QB
    if diagonal:
        bore[:, 1] = (t % ny) * QB
    bore[:, 2] = QR
    psis = np.array([0.0, np.pi / 6, np.pi / 3]) if ncomp == 3 else np.array([0.0])
    rows = np.repeat(np.arange(ny), len(psis))
    det_off = np.zeros((rows.size, 2), np.int32)
    det_off[:, 1] = rows * QD
    psi = np.tile(psis, ny)
    det_pol = np.stack([np.cos(2 * psi), np.sin(2 * psi)], axis=1)
    return Scan(ny=ny, nx=nx, bore=bore, det_off=det_off, det_pol=det_pol,
                periodic=True, ncomp=ncomp)


# ---------------------------------------------------------------------------
# the workloads: the tiny patch (32 detectors x 2^16 samples, 64x64 map), the
# ACT-like patch (1024 detectors x 2^20 samples, 1200x900 map) and the uneven
# problems of the batched solves; the precision study and the learned-correction
# data use the tiny patch
# ---------------------------------------------------------------------------

PIX_ARCMIN = 0.5


def tiny_patch(real=0, ncomp=3):
    """32 detectors on a 4x8 grid at 1', 2^16 samples at 400 Hz, 1 deg/s, 2 deg throw,
    30 deg sky rotation, 64x64 map at 0.5'; sigma=1, f_knee=2 Hz, alpha=3.5."""
    px_per_deg = 60.0 / PIX_ARCMIN
    focal = grid_focal_plane(8, 4, 1.0 / PIX_ARCMIN)
    scan = make_scan(cfg=1, real=real, ny=64, nx=64, n_t=1 << 16, focal_px=focal,
                     speed_px_s=1.0 * px_per_deg, throw_px=2.0 * px_per_deg,
                     segments=((1.0, -15.0, 15.0, True),), ncomp=ncomp)
    n = scan.n_det
    noise = Noise(np.ones(n), np.full(n, 2.0), np.full(n, 3.5))
    return scan, noise


def act_patch(real=0, n_det=1024, n_t=1 << 20, ny=900, nx=1200, ncomp=3, accel_deg_s2=None):
    """1024 detectors on a hex focal plane 1 deg across, 2^20 samples at 400 Hz,
    10 deg throw, a rising half at phi = 25 +- 15 deg and a setting half at
    phi = -25 -+ 15 deg, 1200x900 map at 0.5'; sigma lognormal (mean 1, 20 %),
    f_knee uniform in [1, 5] Hz, alpha = 3.5.  accel_deg_s2: finite-acceleration
    turnarounds (None: instant reversal)."""
    px_per_deg = 60.0 / PIX_ARCMIN
    focal = hex_focal_plane(n_det, 18, (60.0 / 36.0) / PIX_ARCMIN)
    scan = make_scan(cfg=2, real=real, ny=ny, nx=nx, n_t=n_t, focal_px=focal,
                     speed_px_s=1.0 * px_per_deg, throw_px=10.0 * px_per_deg,
                     segments=((0.5, 10.0, 40.0, True), (0.5, -10.0, -40.0, False)),
                     ncomp=ncomp, accel_px_s2=None if accel_deg_s2 is None else accel_deg_s2 * px_per_deg)
    return scan, act_patch_noise(real, n_det)


@dataclasses.dataclass
class CorrNoise:
    """Noise correlated between detectors: per frequency N(f) = D(f) + V E(f) V^T with
    templates V [n_det, r] and mode spectra e_j(f) = amp_j^2 (1 + (f/fknee_j)^-alpha_j)."""
    modes: np.ndarray    # float64 [n_det, r]
    amp: np.ndarray      # float64 [r]
    fknee: np.ndarray    # float64 [r]
    alpha: np.ndarray    # float64 [r]

    @property
    def r(self) -> int:
        return int(self.modes.shape[1])

    def subset(self, dets):
        return CorrNoise(self.modes[dets].copy(), self.amp.copy(), self.fknee.copy(), self.alpha.copy())


def focal_modes(det_off, r=3):
    """Atmosphere-like templates over the focal plane: the common mode and the x and y
    offset gradients (each column unit norm), the first r of them."""
    off = np.asarray(det_off, np.float64) / QD
    n = off.shape[0]
    cols = [np.ones(n)]
    for ax in (0, 1):
        g = off[:, ax] - off[:, ax].mean()
        cols.append(g if np.any(g) else np.zeros(n))
    V = np.stack(cols[:r], axis=1)
    norms = np.linalg.norm(V, axis=0)
    return V / np.where(norms > 0, norms, 1.0)


def corr_noise(det_off, r=3, amp=(3.0, 1.0, 1.0), fknee=(2.0, 1.0, 1.0), alpha=(3.0, 2.5, 2.5)):
    """Correlated modes with red spectra, the common mode strongest."""
    return CorrNoise(focal_modes(det_off, r), np.asarray(amp[:r], float), np.asarray(fknee[:r], float),
                     np.asarray(alpha[:r], float))


UNEVEN_MAP_SIZES = ((256, 256), (240, 320), (360, 480), (450, 600), (600, 800), (750, 1000), (900, 1200))


def uneven_problem(k, real=0, ncomp=3, sizes=None):
    """Problem k of the batched Monte-Carlo workload: seeded n_det from
    {128, 256, 512, 1024}, n_t from {2^18, 2^19, 2^20} and a 5-smooth map size from
    256x256 to 1200x900 (ny x nx) at 0.5'; hex focal plane at 1.667', the scan law of
    the ACT-like patch (rising and setting halves) with a throw of 0.8 of the map
    width; the noise law of the tiny patch (sigma 1, f_knee 2 Hz, alpha 3.5).
    sizes = (n_det, n_t, ny, nx) fixes the sizes (e.g. the smallest corner of the
    distribution, 128 detectors x 2^18 samples on 256x256) and keeps the rest."""
    g = rng(4, 1000 * real + k, "misc")
    n_det = int(g.choice([128, 256, 512, 1024]))
    n_t = int(g.choice([1 << 18, 1 << 19, 1 << 20]))
    ny, nx = UNEVEN_MAP_SIZES[int(g.integers(len(UNEVEN_MAP_SIZES)))]
    if sizes is not None:
        n_det, n_t, ny, nx = (int(v) for v in sizes)
    rings = 1
    while 3 * rings * (rings + 1) + 1 < n_det:
        rings += 1
    focal = hex_focal_plane(n_det, rings, (60.0 / 36.0) / PIX_ARCMIN)
    px_per_deg = 60.0 / PIX_ARCMIN
    scan = make_scan(cfg=4, real=1000 * real + k, ny=ny, nx=nx, n_t=n_t, focal_px=focal,
                     speed_px_s=1.0 * px_per_deg, throw_px=0.8 * nx,
                     segments=((0.5, 10.0, 40.0, True), (0.5, -10.0, -40.0, False)), ncomp=ncomp)
    noise = Noise(np.ones(n_det), np.full(n_det, 2.0), np.full(n_det, 3.5))
    return scan, noise


def act_patch_noise(real, n_det):
    s = math.sqrt(math.log(1.04))
    mu = -0.5 * math.log(1.04)
    sigma = np.exp(rng(2, real, "sigma").normal(mu, s, size=n_det))
    fknee = rng(2, real, "fknee").uniform(1.0, 5.0, size=n_det)
    return Noise(sigma, fknee, np.full(n_det, 3.5))


def small_scan(*, cfg=100, real=0, ny=16, nx=16, n_t=1 << 12, ncols=4, nrows=2,
               spacing_px=1.5, throw_px=None, speed_px_s=None, rot=15.0, ncomp=3,
               f_samp=400.0):
    """A scaled-down tiny-patch scan for fast tests; speed defaults to 0.3 px/sample."""
    focal = grid_focal_plane(ncols, nrows, spacing_px)
    if throw_px is None:
        throw_px = 1.5 * nx
    if speed_px_s is None:
        speed_px_s = 0.3 * f_samp
    return make_scan(cfg=cfg, real=real, ny=ny, nx=nx, n_t=n_t, focal_px=focal,
                     f_samp=f_samp, speed_px_s=speed_px_s, throw_px=throw_px,
                     segments=((0.5, rot, 2 * rot, True), (0.5, -rot, -2 * rot, False)),
                     ncomp=ncomp)


def noise_params(n_det, sigma=1.0, fknee=2.0, alpha=3.5, scatter=None, cfg=100, real=0):
    if scatter is None:
        return Noise(np.full(n_det, float(sigma)), np.full(n_det, float(fknee)),
                     np.full(n_det, float(alpha)))
    sig = sigma * np.exp(rng(cfg, real, "sigma").normal(0.0, scatter, size=n_det))
    fk = rng(cfg, real, "fknee").uniform(0.5 * fknee, 1.5 * fknee, size=n_det)
    return Noise(sig, fk, np.full(n_det, float(alpha)))


# ---------------------------------------------------------------------------
# sky and noise realisations
# ---------------------------------------------------------------------------

def sky_map(ny, nx, *, cfg=1, real=0, ncomp=3, pix_arcmin=PIX_ARCMIN, pol_rms=0.1):
    """Gaussian random field with C_l proportional to l^-2 (C_0 = 0); T scaled to unit
    rms and Q, U (independent fields) to ``pol_rms``.  Returns float64 [ncomp, ny, nx]."""
    g = rng(cfg, real, "sky")
    dpix = np.deg2rad(pix_arcmin / 60.0)
    fy = np.fft.fftfreq(ny, d=dpix)
    fx = np.fft.fftfreq(nx, d=dpix)
    ell = 2 * np.pi * np.hypot(fy[:, None], fx[None, :])
    amp = np.zeros_like(ell)
    nz = ell > 0
    amp[nz] = 1.0 / ell[nz]           # sqrt(C_l), C_l = l^-2
    out = np.empty((ncomp, ny, nx))
    for c in range(ncomp):
        white = g.standard_normal((ny, nx))
        f = np.fft.ifft2(np.fft.fft2(white) * amp).real
        f -= f.mean()
        f /= f.std()
        out[c] = f * (1.0 if c == 0 else pol_rms)
    return out


def noise_tod(noise: Noise, n_t: int, f_samp: float, *, cfg=1, real=0):
    """Stationary gaussian noise with PSD sigma^2 (1 + (f/f_knee)^-alpha): Fourier
    amplitudes sqrt(n_t PSD(f_k)) (g1 + i g2)/sqrt 2 for 0 < k < n_t/2, real bins at
    k = 0 and n_t/2 with variance n_t PSD; the DC bin uses PSD(f_1)."""
    g = rng(cfg, real, "noise")
    n_det = noise.sigma.size
    k = np.arange(n_t // 2 + 1)
    f = k * f_samp / n_t
    f[0] = f[1]
    out = np.empty((n_det, n_t))
    for d in range(n_det):
        if noise.fknee[d] > 0:
            psd = noise.sigma[d] ** 2 * (1.0 + (f / noise.fknee[d]) ** (-noise.alpha[d]))
        else:
            psd = np.full(f.shape, noise.sigma[d] ** 2)
        amp = np.sqrt(n_t * psd)
        re = g.standard_normal(k.size)
        im = g.standard_normal(k.size)
        spec = amp * (re + 1j * im) / np.sqrt(2.0)
        spec[0] = amp[0] * re[0]
        spec[-1] = amp[-1] * re[-1]
        out[d] = np.fft.irfft(spec, n=n_t)
    return out


def corr_noise_tod(noise: Noise, corr: CorrNoise, n_t: int, f_samp: float, *, cfg=1, real=0):
    """Noise with covariance D + V E V^T per frequency: the independent streams of
    noise_tod plus sum_j V[:, j] m_j(t), m_j independent streams with PSD e_j."""
    out = noise_tod(noise, n_t, f_samp, cfg=cfg, real=real)
    modes = Noise(corr.amp.copy(), corr.fknee.copy(), corr.alpha.copy())
    m = noise_tod(modes, n_t, f_samp, cfg=cfg, real=real + 7919)
    return out + corr.modes @ m


def random_maps(ncomp, ny, nx, count, *, cfg=1, real=0):
    return rng(cfg, real, "vec").standard_normal((count, ncomp, ny, nx))
