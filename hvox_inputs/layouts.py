"""Synthetic interferometer layouts and their baselines.

Antenna positions are in a local East-North-Up frame (metres). A baseline is
(a_j - a_i) / lambda for i < j, in wavelengths, so no pair appears twice and no
conjugate pair is present. Earth rotation is modelled by rotating the ENU
antenna vectors about the celestial polar axis a = (0, cos(lat), sin(lat)) by the
hour angle H (Rodrigues' rotation formula); the sky frame stays fixed with the
field centre at +z.
"""
from __future__ import annotations

import math

import numpy as np


def disk_uniform(rng: np.random.Generator, n: int, radius_m: float, sigma_z_m: float) -> np.ndarray:
    r = radius_m * np.sqrt(rng.uniform(0.0, 1.0, n))
    t = rng.uniform(0.0, 2.0 * math.pi, n)
    z = rng.normal(0.0, sigma_z_m, n)
    return np.stack([r * np.cos(t), r * np.sin(t), z], axis=1)


def log_radial(rng: np.random.Generator, n: int, r_min_m: float, r_max_m: float,
               sigma_z_m: float) -> np.ndarray:
    r = np.exp(rng.uniform(math.log(r_min_m), math.log(r_max_m), n))
    t = rng.uniform(0.0, 2.0 * math.pi, n)
    z = rng.normal(0.0, sigma_z_m, n)
    return np.stack([r * np.cos(t), r * np.sin(t), z], axis=1)


def core_plus_arms(rng: np.random.Generator, n: int, core_frac: float, core_sigma_m: float,
                   r_min_m: float, r_max_m: float, sigma_z_m: float) -> np.ndarray:
    n_core = int(round(core_frac * n))
    core = np.stack([rng.normal(0.0, core_sigma_m, n_core), rng.normal(0.0, core_sigma_m, n_core),
                     rng.normal(0.0, sigma_z_m, n_core)], axis=1)
    outer = log_radial(rng, n - n_core, r_min_m, r_max_m, sigma_z_m)
    return np.concatenate([core, outer], axis=0)


def annuli(rng: np.random.Generator, edges_m, counts, sigma_z_m: float) -> np.ndarray:
    """counts[k] antennas uniform in area in the annulus edges_m[k] <= r < edges_m[k + 1]."""
    parts = []
    for k, n in enumerate(counts):
        r0, r1 = edges_m[k], edges_m[k + 1]
        r = np.sqrt(rng.uniform(r0 * r0, r1 * r1, n))
        t = rng.uniform(0.0, 2.0 * math.pi, n)
        z = rng.normal(0.0, sigma_z_m, n)
        parts.append(np.stack([r * np.cos(t), r * np.sin(t), z], axis=1))
    return np.concatenate(parts, axis=0)


def rotate_about_axis(v: np.ndarray, axis: np.ndarray, angle_rad: float) -> np.ndarray:
    a = axis / np.linalg.norm(axis)
    c, s = math.cos(angle_rad), math.sin(angle_rad)
    return v * c + np.cross(a, v) * s + np.outer(v @ a, a) * (1.0 - c)


def pair_differences(ant: np.ndarray) -> np.ndarray:
    i, j = np.triu_indices(len(ant), k=1)
    return ant[j] - ant[i]


def baselines(ant: np.ndarray, hour_angles_deg, latitude_deg: float, wavelengths_m) -> np.ndarray:
    """(n_pairs * n_times * n_channels, 3) float64 baselines in wavelengths.

    Ordering: time-major, then channel, then pair (i < j, row-major upper triangle).
    """
    axis = np.array([0.0, math.cos(math.radians(latitude_deg)), math.sin(math.radians(latitude_deg))])
    d = pair_differences(ant)
    out = []
    for h in hour_angles_deg:
        dr = rotate_about_axis(d, axis, math.radians(h)) if h != 0.0 else d
        for lam in wavelengths_m:
            out.append(dr / lam)
    return np.ascontiguousarray(np.concatenate(out, axis=0))


def centred_steps(n: int, step_deg: float) -> list[float]:
    """n hour angles step_deg apart, symmetric about transit."""
    return [(k - (n - 1) / 2.0) * step_deg for k in range(n)]
