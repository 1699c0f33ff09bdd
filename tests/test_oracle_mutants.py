"""Planted mistakes in the oracle are caught by its pins.

Each case copies ``oracle/`` into a scratch directory, turns one expression of the
copy into a plausible slip (a sign, an index, a dropped factor or conjugate, a
transposed operand, a wrong window or normalisation) and runs the CPU pin tests of
that module against the copy: at least one of them must fail.  The repository's
own oracle is never modified; nothing here touches the CUDA path.

Slips that give the same result in exact arithmetic are not listed, because no pin
can tell them apart: in FCG(m) orthogonalising against the running direction
instead of z_i (the kept directions are mutually A-conjugate, so the two
Gram-Schmidt orders agree), and the Fletcher-Reeves for the Polak-Ribiere beta
under a fixed preconditioner (z_{k+1}^T r_k = 0 there).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PINS = {
    "mapmaker": ["test_oracle.py", "test_oracle_corr.py", "test_oracle_tiled.py", "test_golden.py"],
    "spectra": ["test_oracle_spectra.py"],
    "unet": ["test_oracle_unet.py"],
}

# (module, slip, expression, planted replacement): the first occurrence is replaced
MUTANTS = [
    # pointing, R10 (Eq. 1)
    ("mapmaker", "rotation sign in x", "ox = cp[None, :] * dx - sp[None, :] * dy",
     "ox = cp[None, :] * dx + sp[None, :] * dy"),
    ("mapmaker", "rotation sign in y", "oy = sp[None, :] * dx + cp[None, :] * dy",
     "oy = -sp[None, :] * dx + cp[None, :] * dy"),
    ("mapmaker", "offset scale", "x = bx[None, :] + np.floor_divide(ox, 64)",
     "x = bx[None, :] + np.floor_divide(ox, 32)"),
    ("mapmaker", "floor instead of round", "ix = np.floor_divide(x + (1 << 15), 1 << 16)",
     "ix = np.floor_divide(x, 1 << 16)"),
    ("mapmaker", "periodic wrap by ny", "ix = np.mod(ix, scan.nx)", "ix = np.mod(ix, scan.ny)"),
    ("mapmaker", "first column cut", "inside = (ix >= 0) & (ix < scan.nx)", "inside = (ix > 0) & (ix < scan.nx)"),
    ("mapmaker", "column nx kept", "inside = (ix >= 0) & (ix < scan.nx)", "inside = (ix >= 0) & (ix <= scan.nx)"),
    ("mapmaker", "transposed pixel index", "return np.where(inside, iy * scan.nx + ix, -1)",
     "return np.where(inside, ix * scan.ny + iy, -1)"),
    # response (1, cos 2a, sin 2a), Sec. Test setup
    ("mapmaker", "cos 2phi not normalised", "c2f = (cf * cf - sf * sf) / r2", "c2f = (cf * cf - sf * sf)"),
    ("mapmaker", "double angle not normalised", "    c2f = (cf * cf - sf * sf) / r2\n    s2f = 2.0 * cf * sf / r2",
     "    c2f = (cf * cf - sf * sf)\n    s2f = 2.0 * cf * sf"),
    ("mapmaker", "sin 2phi without the 2", "s2f = 2.0 * cf * sf / r2", "s2f = cf * sf / r2"),
    ("mapmaker", "angle addition sign", "c = c2p * c2f[None, :] - s2p * s2f[None, :]",
     "c = c2p * c2f[None, :] + s2p * s2f[None, :]"),
    ("mapmaker", "psi - phi", "s = s2p * c2f[None, :] + c2p * s2f[None, :]",
     "s = s2p * c2f[None, :] - c2p * s2f[None, :]"),
    ("mapmaker", "Q and U swapped", "np.stack([np.ones_like(c), c, s])", "np.stack([np.ones_like(c), s, c])"),
    ("mapmaker", "sign of U", "np.stack([np.ones_like(c), c, s])", "np.stack([np.ones_like(c), c, -s])"),
    # hit blocks and mask, Eq. 3-5 and R4
    ("mapmaker", "hit blocks unweighted", "vals = (wts[a] * wts[b] * u[:, None])[ok]", "vals = (wts[a] * wts[b])[ok]"),
    ("mapmaker", "mask without the condition test", "(ev[:, 0] >= RCOND_MIN * ev[:, -1])", "(ev[:, 0] >= 0)"),
    # noise filter, R1-R3
    ("mapmaker", "frequency grid", "    f = k * (f_samp / n_t)\n    f[0] = f[1]\n    out = np.empty",
     "    f = k * (f_samp / (2 * n_t))\n    f[0] = f[1]\n    out = np.empty"),
    ("mapmaker", "DC bin", "    f[0] = f[1]\n    out = np.empty", "    f[0] = f[2]\n    out = np.empty"),
    ("mapmaker", "sign of alpha", "(f / noise.fknee[d]) ** (-noise.alpha[d])", "(f / noise.fknee[d]) ** (noise.alpha[d])"),
    ("mapmaker", "sigma not squared", "psd = noise.sigma[d] ** 2 * (1.0", "psd = noise.sigma[d] * (1.0"),
    ("mapmaker", "white sigma not squared", "psd = np.full(f.shape, noise.sigma[d] ** 2)",
     "psd = np.full(f.shape, noise.sigma[d])"),
    ("mapmaker", "diagonal without the mirror bins", "(w[:, 0] + 2.0 * inner + w[:, n_t // 2]) / n_t",
     "(w[:, 0] + inner + w[:, n_t // 2]) / n_t"),
    ("mapmaker", "diagonal counts Nyquist twice", "inner = w[:, 1:n_t // 2].sum(axis=1)",
     "inner = w[:, 1:n_t // 2 + 1].sum(axis=1)"),
    ("mapmaker", "diagonal normalisation", "(w[:, 0] + 2.0 * inner + w[:, n_t // 2]) / n_t",
     "(w[:, 0] + 2.0 * inner + w[:, n_t // 2]) / (n_t // 2 + 1)"),
    ("mapmaker", "filter bins reversed", "return np.fft.irfft(w * np.fft.rfft(tod, axis=-1), n=n_t, axis=-1)",
     "return np.fft.irfft(w[..., ::-1] * np.fft.rfft(tod, axis=-1), n=n_t, axis=-1)"),
    ("mapmaker", "filter square root", "return np.fft.irfft(w * np.fft.rfft(tod, axis=-1), n=n_t, axis=-1)",
     "return np.fft.irfft(np.sqrt(w) * np.fft.rfft(tod, axis=-1), n=n_t, axis=-1)"),
    # correlated noise, R13
    ("mapmaker", "mode spectrum alpha", "(f / corr.fknee[j]) ** (-corr.alpha[j])", "(f / corr.fknee[j]) ** (corr.alpha[j])"),
    ("mapmaker", "mode amplitude not squared", "corr.amp[j] ** 2 * (1.0", "corr.amp[j] * (1.0"),
    ("mapmaker", "covariance diagonal inverted", "cov[:, idx, idx] += (1.0 / w).T", "cov[:, idx, idx] += w.T"),
    ("mapmaker", "mode spectra squared", 'cov = np.einsum("dj,jk,ej->kde", V, e, V)',
     'cov = np.einsum("dj,jk,ej->kde", V, e ** 2, V)'),
    ("mapmaker", "Woodbury E not inverted", "M[:, np.arange(r), np.arange(r)] += (1.0 / e).T",
     "M[:, np.arange(r), np.arange(r)] += e.T"),
    ("mapmaker", "Woodbury sign", "Y = WX - w * np.einsum", "Y = WX + w * np.einsum"),
    # P, P^T and A, Eq. 1-2
    ("mapmaker", "projection reads component 0", "tod += wts[c] * flat[c][safe]", "tod += wts[0] * flat[c][safe]"),
    ("mapmaker", "binning without the response", "weights=(wts[c] * tod)[ok]", "weights=tod[ok]"),
    ("mapmaker", "cut samples read pixel 0", "    return np.where(pix >= 0, tod, 0.0)", "    return tod"),
    ("mapmaker", "masked pixels kept in P", "return np.where((pix >= 0) & op.mask[np.maximum(pix, 0)], pix, -1)",
     "return np.where(pix >= 0, pix, -1)"),
    ("mapmaker", "A keeps the last chunk only", "        out += bin_tod(op, _ninv(op, tod, dets), dets)",
     "        out = bin_tod(op, _ninv(op, tod, dets), dets)"),
    ("mapmaker", "right-hand side with other detectors' filters",
     "out += bin_tod(op, _ninv(op, d[dets], dets), dets)", "out += bin_tod(op, _ninv(op, d[dets], dets[::-1]), dets)"),
    # binned and Jacobi preconditioners, Eq. 3-5
    ("mapmaker", "binned without the noise weights", 'u = detector_weights(op, white) if kind == "binned" else None',
     "u = None"),
    ("mapmaker", "Jacobi with the noise weights", 'u = detector_weights(op, white) if kind == "binned" else None',
     "u = detector_weights(op, white)"),
    ("mapmaker", "blocks ignore the mask", "self.blocks = hit_blocks(op.scan, u, op.mask)",
     "self.blocks = hit_blocks(op.scan, u)"),
    # circulant preconditioner, Eq. 6-13 and R5-R9
    ("mapmaker", "Sigma = B", 'sig[mask] = np.einsum("pak,pk,pbk->pab", vec, np.sqrt(lam), vec)',
     'sig[mask] = np.einsum("pak,pk,pbk->pab", vec, lam, vec)'),
    ("mapmaker", "Sigma^-1 = B^-1", 'sig_inv[mask] = np.einsum("pak,pk,pbk->pab", vec, 1.0 / np.sqrt(lam), vec)',
     'sig_inv[mask] = np.einsum("pak,pk,pbk->pab", vec, 1.0 / lam, vec)'),
    ("mapmaker", "reference column from ny", "p0 = (ny // 2) * nx + nx // 2", "p0 = (ny // 2) * nx + ny // 2"),
    ("mapmaker", "reference tie to the largest index", "return int(cand[d2 == best].min())",
     "return int(cand[d2 == best].max())"),
    ("mapmaker", "odd-side offsets", "return np.where(k < (n + 1) // 2, k, k - n)", "return np.where(k < n // 2, k, k - n)"),
    ("mapmaker", "taper width", "np.exp(-(ky ** 2 + kx ** 2) / (2.0 * sigma ** 2))",
     "np.exp(-(ky ** 2 + kx ** 2) / (sigma ** 2))"),
    ("mapmaker", "Eq. 11 without the conjugate", "    h = np.conj(np.fft.fft2(q, axes=(-2, -1)))\n    xf",
     "    h = np.fft.fft2(q, axes=(-2, -1))\n    xf"),
    ("mapmaker", "Eq. 11 block transposed", 'yf = np.einsum("abyx,byx->ayx", h, xf)', 'yf = np.einsum("bayx,byx->ayx", h, xf)'),
    ("mapmaker", "Eq. 13 without the left Sigma", 't = np.einsum("ga,gdj->adj", s_ref, rows)', "t = rows"),
    ("mapmaker", "Eq. 13 with Sigma on the right", 'qrow = np.einsum("adj,jdb->abj", t, self.sigma_inv)',
     'qrow = np.einsum("adj,jdb->abj", t, self.sigma)'),
    ("mapmaker", "Eq. 10 offsets of the wrong sign", "q = np.roll(qrow, shift=(-ry, -rx), axis=(-2, -1))",
     "q = np.roll(qrow, shift=(ry, rx), axis=(-2, -1))"),
    ("mapmaker", "Eq. 10 offsets swapped", "q = np.roll(qrow, shift=(-ry, -rx), axis=(-2, -1))",
     "q = np.roll(qrow, shift=(-rx, -ry), axis=(-2, -1))"),
    ("mapmaker", "R5 mirror off by one", "qneg = np.roll(q[:, :, ::-1, ::-1], shift=(1, 1), axis=(-2, -1))",
     "qneg = q[:, :, ::-1, ::-1]"),
    ("mapmaker", "R5 without the block transpose", "q = 0.5 * (q + qneg.transpose(1, 0, 2, 3))", "q = 0.5 * (q + qneg)"),
    ("mapmaker", "R5 not applied", "q = 0.5 * (q + qneg.transpose(1, 0, 2, 3))", "q = q"),
    ("mapmaker", "mode blocks without the conjugate", "        h = np.conj(np.fft.fft2(q, axes=(-2, -1)))       # [a, b",
     "        h = np.fft.fft2(q, axes=(-2, -1))       # [a, b"),
    ("mapmaker", "R6 absolute floor", "floor = pd_eps * lam.max()", "floor = pd_eps"),
    ("mapmaker", "mode inverse without the conjugate", "vec, 1.0 / lam, np.conj(vec))", "vec, 1.0 / lam, vec)"),
    ("mapmaker", "mode inverse transposed", 'zf = np.einsum("yxab,byx->ayx", self.h_inv, yf)',
     'zf = np.einsum("yxba,byx->ayx", self.h_inv, yf)'),
    ("mapmaker", "Eq. 12 with Sigma on the left", "        return _apply_blocks(self.sigma_inv, z)",
     "        return _apply_blocks(self.sigma, z)"),
    ("mapmaker", "Eq. 8 with one Sigma", "        return _apply_blocks(self.sigma, circulant_forward(self.q, y))",
     "        return circulant_forward(self.q, y)"),
    # tiled circulant, R15
    ("mapmaker", "window frequency", "np.cos(0.5 * np.pi * u) ** 2", "np.cos(np.pi * u) ** 2"),
    ("mapmaker", "window centres", "        c = (i + 0.5) * h\n", "        c = i * h\n"),
    ("mapmaker", "one-sided window", "z += d[None] * m(d[None] * r)", "z += d[None] * m(r)"),
    ("mapmaker", "tile reference at the corner", "int((i + 0.5) * ny / ty)", "int(i * ny / ty)"),
    # PCG, FCG(m) and the A-norm estimate, R11, R12, R16
    ("mapmaker", "alpha from r", "alpha = rho / float(np.vdot(p, q))", "alpha = rho / float(np.vdot(r, q))"),
    ("mapmaker", "beta inverted", "            beta = rho_new / rho\n", "            beta = rho / rho_new\n"),
    ("mapmaker", "direction sign", "p = z_new + beta * p", "p = z_new - beta * p"),
    ("mapmaker", "A-norm terms without alpha", "terms.append(alpha * rho)", "terms.append(rho)"),
    ("mapmaker", "start ignored in the residual",
     "    r = b - apply_a(x) if x0 is not None else b.copy()\n    bnorm = math.sqrt(float(np.vdot(b, b)))\n    z = apply_m(r)",
     "    r = b.copy()\n    bnorm = math.sqrt(float(np.vdot(b, b)))\n    z = apply_m(r)"),
    ("mapmaker", "Polak-Ribiere sign", "beta = float(np.vdot(z_new, r - r_old)) / rho",
     "beta = float(np.vdot(z_new, r + r_old)) / rho"),
    ("mapmaker", "FCG step from r", "alpha = float(np.vdot(p, r)) / pq", "alpha = float(np.vdot(r, r)) / pq"),
    ("mapmaker", "FCG orthogonalisation sign", "p = p - (float(np.vdot(z, qj)) / pqj) * pj",
     "p = p + (float(np.vdot(z, qj)) / pqj) * pj"),
    ("mapmaker", "FCG drops the newest direction", "        if len(kept) > window:\n            kept.pop(0)",
     "        if len(kept) > window:\n            kept.pop()"),
    ("mapmaker", "A-norm window d - 1", "terms[i:i + d].sum()", "terms[i:i + d - 1].sum()"),
    # flat-sky spectra, R14
    ("spectra", "unsigned frequencies", "ky = np.fft.fftfreq(ny, d=1.0 / ny)", "ky = np.arange(ny)"),
    ("spectra", "l_y scaled by nx", "ly = 2 * np.pi * ky[:, None] / (ny * pix)", "ly = 2 * np.pi * ky[:, None] / (nx * pix)"),
    ("spectra", "angle arguments swapped", "phi = np.arctan2(ly, lx)", "phi = np.arctan2(lx, ly)"),
    ("spectra", "sign in E", "E = Q * c2 + U * s2", "E = Q * c2 - U * s2"),
    ("spectra", "sign in B", "B = -Q * s2 + U * c2", "B = Q * s2 + U * c2"),
    ("spectra", "l = 0 kept", "ok = (ell > 0) & (b < nbins)", "ok = b < nbins"),
    ("spectra", "normalisation pix", "norm = pix * pix / (ny * nx)", "norm = pix / (ny * nx)"),
    ("spectra", "amplitude not squared", "(np.abs(X) ** 2)[ok]", "np.abs(X)[ok]"),
    ("spectra", "bins rounded", "b = np.floor(ell / (lmax / nbins))", "b = np.round(ell / (lmax / nbins))"),
    # U-Net
    ("unet", "convolution instead of cross-correlation",
     'y += np.einsum("oc,bcyx->boyx", w[:, :, dy, dx], xp[:, :, dy:dy + H, dx:dx + W])',
     'y += np.einsum("oc,bcyx->boyx", w[:, :, 2 - dy, 2 - dx], xp[:, :, dy:dy + H, dx:dx + W])'),
    ("unet", "max pooling", "return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))",
     "return x.reshape(B, C, H // 2, 2, W // 2, 2).max(axis=(3, 5))"),
    ("unet", "loss summed", "    g = diff / diff.size\n", "    g = diff\n"),
    ("unet", "ReLU on the output", "    y = conv1(h, w, b)\n", "    y = np.maximum(conv1(h, w, b), 0.0)\n"),
    ("unet", "bias before weights", "        w = params[o:o + n].reshape(shp)\n        o += n\n        b = params[o:o + co]\n        o += co\n",
     "        b = params[o:o + co]\n        o += co\n        w = params[o:o + n].reshape(shp)\n        o += n\n"),
    ("unet", "transposed-conv taps swapped", "y[:, :, dy::2, dx::2] = np.einsum", "y[:, :, dx::2, dy::2] = np.einsum"),
    ("unet", "ReLU gradient dropped", "            g = g * (hout > 0)\n", ""),
    ("unet", "weight gradient transposed", 'gw[:, :, dy, dx] = np.einsum("boyx,bcyx->oc", g, xp[:, :, dy:dy + H, dx:dx + W])',
     'gw[:, :, 2 - dy, 2 - dx] = np.einsum("boyx,bcyx->oc", g, xp[:, :, dy:dy + H, dx:dx + W])'),
    ("unet", "pool gradient not averaged", "return np.repeat(np.repeat(g, 2, axis=2), 2, axis=3) * 0.25",
     "return np.repeat(np.repeat(g, 2, axis=2), 2, axis=3)"),
]


def _workspace(base, module, old, new):
    """A copy of oracle/, gen/ and the pin tests with one expression of ``module`` replaced."""
    os.makedirs(os.path.join(base, "tests"))
    for d in ("oracle", "gen"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(base, d), ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(base, "tests", "golden"))
    for f in PINS[module] + ["conftest.py", "golden_cases.py"]:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(base, "tests", f))
    if old is not None:
        path = os.path.join(base, "oracle", module + ".py")
        src = open(path).read()
        assert old in src, f"the expression to replace is no longer in oracle/{module}.py: {old!r}"
        open(path, "w").write(src.replace(old, new, 1))
    return base


def _pins_pass(base, module):
    # one BLAS thread per run: the runs themselves go in parallel
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    env.pop("PYTHONPATH", None)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
                       + [os.path.join("tests", f) for f in PINS[module]],
                       cwd=base, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-400:]


def test_pins_pass_on_an_unchanged_copy(tmp_path):
    for module in PINS:
        rc, out = _pins_pass(_workspace(str(tmp_path / module), module, None, None), module)
        assert rc == 0, out


def test_every_planted_mistake_is_caught(tmp_path):
    def one(k):
        module, _, old, new = MUTANTS[k]
        return _pins_pass(_workspace(str(tmp_path / f"m{k}"), module, old, new), module)[0]

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        codes = list(ex.map(one, range(len(MUTANTS))))
    # exit code 1: a pin failed (an exception inside a test counts as a failure)
    survived = [f"{m[0]}: {m[1]} (pytest exit {c})" for m, c in zip(MUTANTS, codes) if c != 1]
    assert not survived, survived
