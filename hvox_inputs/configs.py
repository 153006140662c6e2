"""Seeded synthetic workloads with the shapes of the paper's experiments.

The paper's own datasets (SKA-Low simulations, a LOFAR measurement set) are not
available; these inputs stand in for them with the sizes, layouts and value
distributions of its setups (Tables 2-3, the LOFAR/SKA layouts it plots).

Seeds: master 20230609; stream = master + 1000 * config + purpose, numpy PCG64.
purpose: 1 antennas, 2 sky, 3 point sources, 4 visibilities, 5 samples.

Configs (sizes are exact for the stated seeds and rules):
  1  nside 32, 45 deg cap (1,740 px), I ~ U[0,1] + 1.0 at 10 pixels; 200 antennas
     uniform in a 1 km disk, sigma_z 10 m, all 19,900 pairs, lambda 2 m.
  2  nside 256, 30 deg cap (52,812 px), I ~ lognormal(0,1); 300 antennas log-radial
     50 m - 100 km, sigma_z 20 m, 4 hour angles 15 deg apart at lat +52.9 deg,
     8 channels lambda = 1.8..2.2 m (1,435,200 baselines).
  3  nside 1024, 40 deg cap (1,470,612 px), I ~ lognormal(0,1.5) + 10.0 at 1,000
     pixels; 512 antennas (60 % Gaussian core sigma 0.5 km, rest log-radial 1-65 km),
     sigma_z 5 m, lambda 2 m, 32 hour angles 3.75 deg apart at lat -26.7 deg
     (4,186,112 baselines).
  4  nside 4096 hemisphere (100,671,488 px), I ~ lognormal(0,1); 1,024 antennas
     log-radial 50 m - 100 km, sigma_z 10 m, lambda 2 m, 40 hour angles 3 deg apart
     at lat -26.7 deg (20,951,040 baselines).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import healpix, layouts

MASTER_SEED = 20230609


def rng_for(config: int, purpose: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(MASTER_SEED + 1000 * config + purpose))


@dataclass
class Workload:
    name: str
    pix: np.ndarray       # (N_pix, 3) float64 unit vectors
    uvw: np.ndarray       # (N_vis, 3) float64 baselines in wavelengths
    sky: np.ndarray       # (N_pix,) float64 intensities
    eps: tuple            # tolerances the workload is run at

    @property
    def n_pix(self) -> int:
        return len(self.pix)

    @property
    def n_vis(self) -> int:
        return len(self.uvw)


def _point_sources(rng, sky, count, amp):
    idx = rng.choice(len(sky), size=count, replace=False)
    sky[idx] += amp
    return sky


def config1() -> Workload:
    pix = healpix.cap_pixels(32, 45.0)
    sky = rng_for(1, 2).uniform(0.0, 1.0, len(pix))
    sky = _point_sources(rng_for(1, 3), sky, 10, 1.0)
    ant = layouts.disk_uniform(rng_for(1, 1), 200, 1000.0, 10.0)
    uvw = layouts.baselines(ant, [0.0], 52.9, [2.0])
    return Workload("healpix nside=32 45deg cap x 200-antenna 1 km disk", pix, uvw, sky, (1e-9, 1e-6, 1e-4))


def config2_antennas() -> np.ndarray:
    return layouts.log_radial(rng_for(2, 1), 300, 50.0, 100e3, 20.0)


def config2() -> Workload:
    pix = healpix.cap_pixels(256, 30.0)
    sky = rng_for(2, 2).lognormal(0.0, 1.0, len(pix))
    uvw = layouts.baselines(config2_antennas(), layouts.centred_steps(4, 15.0), 52.9,
                            np.linspace(1.8, 2.2, 8))
    return Workload("healpix nside=256 30deg cap x LOFAR-like 300 antennas 4 times 8 channels",
                    pix, uvw, sky, (1e-9, 1e-5))


def config3_antennas() -> np.ndarray:
    return layouts.core_plus_arms(rng_for(3, 1), 512, 0.6, 500.0, 1e3, 65e3, 5.0)


def config3() -> Workload:
    pix = healpix.cap_pixels(1024, 40.0)
    sky = rng_for(3, 2).lognormal(0.0, 1.5, len(pix))
    sky = _point_sources(rng_for(3, 3), sky, 1000, 10.0)
    uvw = layouts.baselines(config3_antennas(), layouts.centred_steps(32, 3.75), -26.7, [2.0])
    return Workload("healpix nside=1024 40deg cap x SKA-Low-like 512 antennas 32 times",
                    pix, uvw, sky, (1e-6,))


def config4() -> Workload:
    pix = healpix.cap_pixels(4096, 90.0)
    sky = rng_for(4, 2).lognormal(0.0, 1.0, len(pix)).astype(np.float32).astype(np.float64)
    ant = layouts.log_radial(rng_for(4, 1), 1024, 50.0, 100e3, 10.0)
    uvw = layouts.baselines(ant, layouts.centred_steps(40, 3.0), -26.7, [2.0])
    return Workload("healpix nside=4096 hemisphere x 1024 antennas 40 times", pix, uvw, sky, (1e-5, 1e-9))


def visibilities_cn(config: int, n: int) -> np.ndarray:
    """Complex Gaussian CN(0,1) visibilities (input of vis->sky timing runs)."""
    rng = rng_for(config, 4)
    return (rng.normal(0.0, math.sqrt(0.5), n) + 1j * rng.normal(0.0, math.sqrt(0.5), n)).astype(np.complex128)


def sample_indices(config: int, n_total: int, count: int, purpose_offset: int = 0) -> np.ndarray:
    """Sorted, distinct seeded output indices for sampled oracle checks."""
    rng = rng_for(config, 5 + 10 * purpose_offset)
    count = min(count, n_total)
    return np.sort(rng.choice(n_total, size=count, replace=False)).astype(np.int64)


def small_case(seed: int, n_pix: int, n_vis: int, cap_deg: float = 30.0, radius_m: float = 300.0,
               sigma_z_m: float = 10.0, lam: float = 2.0, nside: int | None = None) -> Workload:
    """A seeded small case: a cap of HEALPix pixels and a random disk layout.

    The pixel count is the first n_pix pixels (RING order) of the smallest nside
    whose cap holds at least n_pix pixels; visibilities are the first n_vis pairs
    of enough antennas.
    """
    if nside is None:
        nside = 1
        while healpix.cap_count(nside, cap_deg) < n_pix:
            nside += 1
    pix = healpix.cap_pixels(nside, cap_deg, max_pixels=n_pix)
    rng = np.random.Generator(np.random.PCG64(MASTER_SEED + 7919 * seed))
    n_ant = 2
    while n_ant * (n_ant - 1) // 2 < n_vis:
        n_ant += 1
    ant = layouts.disk_uniform(rng, n_ant, radius_m, sigma_z_m)
    uvw = layouts.pair_differences(ant)[:n_vis] / lam
    sky = rng.lognormal(0.0, 1.0, len(pix))
    return Workload(f"small seed={seed}", pix, np.ascontiguousarray(uvw), sky, ())


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4}


# Telescope-radius sweep (the paper's Table 3 setups): radius (km) -> (N_vis, N_pix). One
# SKA-Low-like layout of 888 antennas in annuli whose cumulative counts (24, 162, 437, 545,
# 690, 826, 888 within 0.1 .. 100 km) give the table's visibility counts as all pairs
# within the radius; one snapshot at transit, lambda 2 m. The sky is the first N_pix RING
# pixels around +z at the HEALPix resolution that puts two pixels in the finest fringe
# (nside = ceil(4.1 R / lambda)), I ~ lognormal(0, 1).
RADIUS_TABLE = {0.1: (273, 6_400), 0.3: (13_000, 25_600), 1.0: (95_000, 130_000), 3.0: (148_000, 810_000),
                10.0: (238_000, 10_240_000), 30.0: (341_000, 74_650_000), 100.0: (394_000, 182_250_000)}
SWEEP_EDGES_KM = (0.0, 0.1, 0.3, 1.0, 3.0, 10.0, 30.0, 100.0)
SWEEP_COUNTS = (24, 138, 275, 108, 145, 136, 62)


def sweep_antennas() -> np.ndarray:
    return layouts.annuli(rng_for(6, 1), [e * 1e3 for e in SWEEP_EDGES_KM], SWEEP_COUNTS, 5.0)


def radius_sweep(radius_km: float, lam: float = 2.0, sparse_pixels: int = 0) -> Workload:
    """Radius-sweep workload; sparse_pixels > 0 keeps only that many pixels of interest,
    in 5 compact groups around seeded directions of the field (the sparse-sky setup)."""
    radius_km = float(radius_km)
    if radius_km not in RADIUS_TABLE:
        raise ValueError(f"radius must be one of {sorted(RADIUS_TABLE)} km")
    ant = sweep_antennas()
    ant = ant[np.hypot(ant[:, 0], ant[:, 1]) <= radius_km * 1e3]
    uvw = layouts.baselines(ant, [0.0], -26.7, [lam])
    n_pix = RADIUS_TABLE[radius_km][1]
    nside = int(math.ceil(4.1 * radius_km * 1e3 / lam))
    pix = healpix.cap_pixels(nside, 90.0, max_pixels=n_pix)
    name = f"radius {radius_km:g} km: {len(ant)} antennas, HEALPix nside={nside} first {len(pix)} RING pixels"
    if sparse_pixels > 0:
        rng = rng_for(6, 3)
        centres = pix[rng.choice(len(pix), 5, replace=False)]
        per = -(-sparse_pixels // 5)
        keep = []
        for c in centres:
            d = np.einsum("ij,j->i", pix, c)
            keep.append(np.argpartition(-d, per)[:per])
        idx = np.unique(np.concatenate(keep))[:sparse_pixels]
        pix = np.ascontiguousarray(pix[idx])
        name += f", sparse: {len(pix)} pixels in 5 groups"
    sky = rng_for(6, 2).lognormal(0.0, 1.0, len(pix))
    return Workload(name, pix, uvw, sky, (1e-6,))


def _cap_for(n_pix: int, cap_deg: float = 40.0) -> np.ndarray:
    """The first n_pix RING pixels of the smallest nside whose cap_deg cap holds n_pix."""
    nside = 1
    while healpix.cap_count(nside, cap_deg) < n_pix:
        nside *= 2
    lo = nside // 2 if nside > 1 else 1
    while lo < nside and healpix.cap_count(lo, cap_deg) < n_pix:
        lo += max(1, (nside - lo) // 8)
    if healpix.cap_count(lo, cap_deg) >= n_pix:
        nside = lo
    return healpix.cap_pixels(nside, cap_deg, max_pixels=n_pix)


def _baselines_for(n_vis: int, layout: int) -> np.ndarray:
    """n_vis baselines from the config-2 (LOFAR-like) or config-3 (SKA-like) layout, with
    as many earth-rotation steps as needed, truncated."""
    if layout == 2:
        ant, lat, step, lams = config2_antennas(), 52.9, 15.0, [2.0]
    else:
        ant, lat, step, lams = config3_antennas(), -26.7, 3.75, [2.0]
    pairs = len(ant) * (len(ant) - 1) // 2
    n_steps = max(1, -(-n_vis // pairs))
    uvw = layouts.baselines(ant, layouts.centred_steps(n_steps, step), lat, lams)
    return np.ascontiguousarray(uvw[:n_vis])


@dataclass
class Request:
    rid: int
    arrival: float        # seconds after the start of the stream
    pix: np.ndarray
    uvw: np.ndarray
    eps: float
    direction: str        # "s2v" (sky -> vis) or "v2s" (vis -> sky)
    data: np.ndarray      # sky (float64) or visibilities (complex128)


def config5_requests(n_requests: int = 2000, rate_hz: float = 50.0, n_min: float = 1e4, n_max: float = 1e7,
                     eps_choices=(1e-4, 1e-6, 1e-9), seed_offset: int = 0):
    """Served mixed stream: Poisson arrivals; per request log-uniform pixel and baseline
    counts in [n_min, n_max], a HEALPix cap (<= 40 deg) and the config-2 or config-3
    layout (p = 1/2), eps uniform over eps_choices, direction S or A (p = 1/2).
    Seeds: master + 5000 + request id."""
    out = []
    t = 0.0
    arr = rng_for(5, 9 + seed_offset)
    for rid in range(n_requests):
        t += arr.exponential(1.0 / rate_hz)
        rng = np.random.Generator(np.random.PCG64(MASTER_SEED + 5000 + 100003 * seed_offset + rid))
        n_pix = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        n_vis = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        layout = 2 if rng.uniform() < 0.5 else 3
        eps = float(eps_choices[int(rng.integers(len(eps_choices)))])
        direction = "s2v" if rng.uniform() < 0.5 else "v2s"
        pix = _cap_for(n_pix)
        uvw = _baselines_for(n_vis, layout)
        if direction == "s2v":
            data = rng.lognormal(0.0, 1.0, n_pix)
        else:
            data = (rng.normal(0.0, math.sqrt(0.5), n_vis) + 1j * rng.normal(0.0, math.sqrt(0.5), n_vis))
        out.append(Request(rid, t, pix, uvw, eps, direction, data))
    return out
