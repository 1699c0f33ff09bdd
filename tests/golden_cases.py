"""Loader of the worked examples under ``tests/golden/``.

Each fixture is a hand-derived example of the paper's definitions (its
``cite`` and ``derivation`` fields give the passage and the arithmetic): a
small scan written as runs of samples on pixel centres, a cycle of boresight
angles that are exact in the fixed-point tables, detectors, a map, and for
each noise case the expected A m (and where given P m or M_B A m).  The
64-sample period can be repeated K times; every expected A m then scales by K.

This module only expands the compact description into the input tables of
``gen`` (the same tables the oracle and the CUDA path read); it holds no
map-making arithmetic.
"""
from __future__ import annotations

import json
import os

import numpy as np

import gen
from gen.inputs import QB, QD, QR

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = ("runs_T_filters", "two_angle_blocks_TQU", "rotated_offset_pointing", "common_mode_pair_T")

# (cos phi, sin phi) in rotation units for the angles the fixtures use: exact
_ROT = {0: (QR, 0), 90: (0, QR), 180: (-QR, 0), 270: (0, -QR)}


def load(name: str) -> dict:
    with open(os.path.join(HERE, name + ".json")) as f:
        return json.load(f)


def scan_of(fx: dict, K: int) -> gen.Scan:
    """The fixture's scan with its period repeated K times."""
    period = int(fx["period"])
    pix = []
    for ix, iy, length in fx["runs"]:
        pix += [(ix, iy)] * int(length)
    assert len(pix) == period, "runs must fill one period"
    n_t = period * K
    bore = np.zeros((n_t, 4), np.int32)
    t = np.arange(n_t)
    cells = np.array(pix, np.int64)[t % period]
    bore[:, 0] = cells[:, 0] * QB
    bore[:, 1] = cells[:, 1] * QB
    phis = fx["phi_deg"]
    rot = np.array([_ROT[int(phis[q % len(phis)])] for q in range(len(phis))], np.int64)
    bore[:, 2] = rot[t % len(phis), 0]
    bore[:, 3] = rot[t % len(phis), 1]
    det_off = np.round(np.array(fx["det_off_px"], np.float64) * QD).astype(np.int32)
    det_pol = np.array(fx["det_pol"], np.float64)
    return gen.Scan(ny=int(fx["ny"]), nx=int(fx["nx"]), bore=bore, det_off=det_off, det_pol=det_pol,
                    ncomp=int(fx["ncomp"]))


def noise_of(case: dict, n_det: int) -> gen.Noise:
    """The law's parameters of a case (a table case keeps sigma 1, no knee: the
    table replaces the law)."""
    s = float(case.get("sigma", 1.0))
    return gen.Noise(np.full(n_det, s), np.full(n_det, float(case.get("fknee", 0.0))),
                     np.full(n_det, float(case.get("alpha", 1.0))))


def table_of(case: dict, n_det: int, n_t: int):
    """Weights w[d, k], k = 0 .. n_t/2, of a table case; None for a law case."""
    spec = case.get("table")
    if spec is None:
        return None
    w = np.full((n_det, n_t // 2 + 1), float(spec["default"]))
    for key, k in (("dc", 0), ("nyquist", n_t // 2), ("quarter", n_t // 4)):
        if key in spec:
            w[:, k] = float(spec[key])
    return w


def corr_of(case: dict):
    """The case's noise correlated between detectors (templates and mode spectra),
    or None."""
    c = case.get("corr")
    if c is None:
        return None
    return gen.CorrNoise(np.array(c["modes"], np.float64), np.array(c["amp"], np.float64),
                         np.array(c["fknee"], np.float64), np.array(c["alpha"], np.float64))


def map_of(fx: dict) -> np.ndarray:
    return np.array(fx["map"], np.float64)


def cases(names=NAMES):
    """(fixture name, fixture, case) for every case of every fixture."""
    for name in names:
        fx = load(name)
        for case in fx["cases"]:
            yield name, fx, case
