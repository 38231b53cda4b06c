"""Seeded synthetic workloads of the pCT simulator: phantoms, angle sets,
path models and seeds.

This module holds input descriptions only (numbers, no arithmetic of the
method), so that the CUDA library, the CPU oracle, the tests and the
benchmark all read the same inputs.

Phantoms are NEO head phantoms (Sec. II-A): nested ellipses (2D) or
ellipsoids (3D) in painter's order, region 0 being the outer boundary.  The
paper gives the outer axes (180 x 140 mm) and the RSP values (skull 1.6,
brain 1.04, ventricles 0.9, sinus 0.0, NEO 2 adds skin); the inner
positions and sizes below are our reading of its Fig. 1.

Workloads (sizes of the paper's 2D and head-size 3D examples):
  neo1_2d_straight   200x200 px of 1 mm, 180 angles x 500 straight paths
  neo2_2d_spline     512x512 px of 0.4 mm, 360 angles x 10,000 spline paths,
                     MCS sigmas 15 mrad / 1 mm, 1% WEPL noise
  head_3d_spline     200x200x160 voxels of 1 mm, 90 angles x 200,000 spline
                     paths, 1% WEPL noise
  head_3d_large      256x256x160 voxels of 1 mm, spline paths (matrix-free)
"""
from __future__ import annotations

import math

import numpy as np

ELLIPSOID, EXTRUDED = 0, 1
CENTER, CORNER, AREA = 0, 1, 2
STRAIGHT, STRAIGHT_MCS, SPLINE = 0, 1, 2
CHORD_EXACT, CHORD_CONSTANT = 0, 1
NOISE_NONE, NOISE_GAUSS_REL = 0, 1
MCS_FIXED, MCS_HIGHLAND = 0, 1
X0_WATER_MM = 360.8  # radiation length of water (PDG)

BASE_SEED = 210812369


def _region(c, a, rsp):
    return {"c": tuple(float(v) for v in c), "a": tuple(float(v) for v in a), "rsp": float(rsp)}


def neo_regions(skin: bool, scale: float = 1.0):
    """NEO 1 (skin=False) or NEO 2 (skin=True) regions, 3D semi-axes.

    2D users ignore the z entries.  `scale` shrinks every axis and centre."""
    s = float(scale)
    regs = []
    if skin:
        regs.append(_region((0, 0, 0), (93 * s, 73 * s, 83 * s), 1.1))
    regs += [
        _region((0, 0, 0), (90 * s, 70 * s, 80 * s), 1.6),        # skull (outer)
        _region((0, 0, 0), (85 * s, 65 * s, 75 * s), 1.04),       # brain (5 mm shell)
        _region((-10 * s, 0, 0), (15 * s, 6 * s, 12 * s), 0.9),   # left ventricle
        _region((10 * s, 0, 0), (15 * s, 6 * s, 12 * s), 0.9),    # right ventricle
        _region((0, 60 * s, 0), (8 * s, 5 * s, 6 * s), 0.0),      # frontal sinus
    ]
    return regs


def phantom(dim: int, n, h, skin: bool, kind: int = ELLIPSOID, raster: int = CORNER,
            scale: float = 1.0, area_samples: int = 4):
    """area_samples: sub-samples per axis of the weighted-area raster (AREA)."""
    n = tuple(int(v) for v in n)
    h = tuple(float(v) for v in h)
    return {"dim": int(dim), "kind": int(kind), "raster": int(raster),
            "n": n + (1,) * (3 - len(n)), "h": h + (1.0,) * (3 - len(h)),
            "regions": neo_regions(skin, scale), "area_samples": int(area_samples)}


def angles(n_angles: int) -> np.ndarray:
    """n_angles projection angles uniform over the full circle (Sec. II-B)."""
    return np.array([2.0 * math.pi * k / n_angles for k in range(n_angles)], dtype=np.float64)


def model(kind: int, t_range, v_range=(0.0, 0.0), sigma_lat=0.0, sigma_in=0.0, sigma_out=0.0,
          rho=0.0, spline_segments=32, chord=CHORD_EXACT, noise_rel=0.0, mcs=MCS_FIXED,
          beam_mev=200.0, x0_mm=X0_WATER_MM):
    """Path model.  mcs = MCS_HIGHLAND replaces sigma_lat, sigma_out and rho
    per proton by the Highland / PDG widths for its chord through the hull
    (beam kinetic energy beam_mev, radiation length x0_mm)."""
    return {"model": int(kind), "chord": int(chord), "spline_segments": int(spline_segments),
            "noise": NOISE_GAUSS_REL if noise_rel > 0 else NOISE_NONE,
            "t_range": (float(t_range[0]), float(t_range[1])),
            "v_range": (float(v_range[0]), float(v_range[1])),
            "sigma_lat": float(sigma_lat), "sigma_in": float(sigma_in),
            "sigma_out": float(sigma_out), "rho": float(rho), "noise_rel": float(noise_rel),
            "mcs": int(mcs), "beam_mev": float(beam_mev), "x0_mm": float(x0_mm)}


def neo1_2d_straight(n_angles: int = 180, paths_per_angle: int = 500):
    """NEO 1, 200x200 px of 1 mm, straight parallel-beam paths, t in +-100 mm."""
    return {"name": "neo1_2d_straight",
            "phantom": phantom(2, (200, 200), (1.0, 1.0), skin=False),
            "angles": angles(n_angles), "paths_per_angle": int(paths_per_angle),
            "model": model(STRAIGHT, (-100.0, 100.0)), "seed": BASE_SEED + 0}


def neo2_2d_spline(n_angles: int = 360, paths_per_angle: int = 10000, n: int = 512,
                   h: float = 0.4, spline_segments: int = 32, noise_rel: float = 0.01):
    """NEO 2 (skin), n x n px of h mm, cubic Hermite spline paths with entry /
    exit slopes ~ N(0, 15 mrad), exit displacement ~ N(0, 1 mm), 1% noise."""
    half = 0.5 * n * h
    return {"name": "neo2_2d_spline",
            "phantom": phantom(2, (n, n), (h, h), skin=True),
            "angles": angles(n_angles), "paths_per_angle": int(paths_per_angle),
            "model": model(SPLINE, (-half, half), sigma_lat=1.0, sigma_in=0.015,
                           sigma_out=0.015, spline_segments=spline_segments,
                           noise_rel=noise_rel),
            "seed": BASE_SEED + 1}


def head_3d_spline(n_angles: int = 90, paths_per_angle: int = 200000, n=(200, 200, 160),
                   h=(1.0, 1.0, 1.0), spline_segments: int = 32, noise_rel: float = 0.01,
                   seed_offset: int = 2):
    """3D NEO head of ellipsoids, n voxels of h mm, spline paths, 1% noise."""
    half_t = 0.5 * n[0] * h[0]
    half_v = 0.5 * n[2] * h[2]
    return {"name": "head_3d_spline",
            "phantom": phantom(3, n, h, skin=False, kind=ELLIPSOID),
            "angles": angles(n_angles), "paths_per_angle": int(paths_per_angle),
            "model": model(SPLINE, (-half_t, half_t), (-half_v, half_v), sigma_lat=1.0,
                           sigma_in=0.015, sigma_out=0.015, spline_segments=spline_segments,
                           noise_rel=noise_rel),
            "seed": BASE_SEED + seed_offset}


def head_3d_large(n_angles: int = 500, paths_per_angle: int = 200000):
    """256x256x160 voxels of 1 mm, 100M spline paths (matrix-free projector)."""
    w = head_3d_spline(n_angles, paths_per_angle, n=(256, 256, 160), seed_offset=4)
    w["name"] = "head_3d_large"
    return w


def n_rows(w) -> int:
    return len(w["angles"]) * int(w["paths_per_angle"])


def n_vox(w) -> int:
    p = w["phantom"]
    return int(np.prod(p["n"][: p["dim"]]))


def batch_instances(count: int = 64, seed: int = BASE_SEED + 3, max_paths: int = 2_000_000):
    """Heterogeneous instances: 2D grids of 128^2-512^2 and 3D grids of
    64^3-160^3, 10k-2M paths, straight or spline, axes scaled 0.7-1.0."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        three_d = bool(rng.integers(0, 2))
        scale = float(rng.uniform(0.7, 1.0))
        straight = bool(rng.integers(0, 2))
        paths = int(rng.integers(10_000, max_paths + 1))
        if three_d:
            nn = int(rng.integers(64, 161))
            hh = 200.0 / nn
            ph = phantom(3, (nn, nn, nn), (hh, hh, hh), skin=False, scale=scale)
            half = 0.5 * nn * hh
            v_rng = (-half, half)
        else:
            nn = int(rng.integers(128, 513))
            hh = 200.0 / nn
            ph = phantom(2, (nn, nn), (hh, hh), skin=False, scale=scale)
            half = 0.5 * nn * hh
            v_rng = (0.0, 0.0)
        n_ang = int(rng.integers(8, 65))
        ppa = max(1, paths // n_ang)
        md = model(STRAIGHT if straight else SPLINE, (-half, half), v_rng,
                   sigma_lat=0.0 if straight else 1.0, sigma_in=0.0 if straight else 0.015,
                   sigma_out=0.0 if straight else 0.015, noise_rel=0.01)
        out.append({"name": f"batch_{i}", "phantom": ph, "angles": angles(n_ang),
                    "paths_per_angle": ppa, "model": md, "seed": seed * 1000 + i})
    return out
