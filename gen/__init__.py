"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

No map-making arithmetic lives here: only scan tables, focal planes, noise
parameters and random skies / noise streams (see ``gen.inputs``).
"""
from .inputs import (QB, QD, QR, CorrNoise, Noise, Scan, bccb_scan, tiny_patch, act_patch, act_patch_noise, uneven_problem,
                     corr_noise, corr_noise_tod, focal_modes,
                     grid_focal_plane, hex_focal_plane, make_scan, noise_params, noise_tod,
                     random_maps, rng, sky_map, small_scan)

__all__ = ["QB", "QD", "QR", "CorrNoise", "Noise", "Scan", "bccb_scan", "tiny_patch", "act_patch", "act_patch_noise",
           "uneven_problem", "corr_noise", "corr_noise_tod", "focal_modes",
           "grid_focal_plane", "hex_focal_plane", "make_scan", "noise_params", "noise_tod",
           "random_maps", "rng", "sky_map", "small_scan"]
