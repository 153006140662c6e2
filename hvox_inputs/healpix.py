"""HEALPix RING-scheme pixel centres (Gorski et al. 2005, ApJ 622:759, Sect. 4).

Synthetic sky geometry for the workloads. Pixel centres lie on iso-latitude rings:

* north polar cap, ring i = 1 .. nside-1: z = 1 - i^2 / (3 nside^2), 4 i pixels at
  phi = (pi / (2 i)) (j - 1/2), j = 1 .. 4 i;
* equatorial belt, ring i = nside .. 3 nside: z = 4/3 - 2 i / (3 nside), 4 nside pixels at
  phi = (pi / (2 nside)) (j - s/2), s = (i - nside + 1) mod 2;
* south polar cap mirrors the north cap.

RING order numbers pixels ring by ring from the north pole, so a polar cap
z >= cos(theta_cap) is a prefix of the RING order.
"""
from __future__ import annotations

import math

import numpy as np


def ring_z(nside: int, i: int) -> float:
    """z = cos(colatitude) of RING ring i (1-based, 1 .. 4 nside - 1)."""
    if i < nside:
        return 1.0 - i * i / (3.0 * nside * nside)
    if i <= 3 * nside:
        return 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
    ii = 4 * nside - i
    return -(1.0 - ii * ii / (3.0 * nside * nside))


def ring_npix(nside: int, i: int) -> int:
    if i < nside:
        return 4 * i
    if i <= 3 * nside:
        return 4 * nside
    return 4 * (4 * nside - i)


def _rings_in_cap(nside: int, zmin: float):
    # A tolerance keeps rings that sit exactly on the boundary (z = 0 for a hemisphere).
    tol = 1e-12
    i = 1
    while i <= 4 * nside - 1 and ring_z(nside, i) >= zmin - tol:
        yield i
        i += 1


def cap_count(nside: int, cap_deg: float) -> int:
    """Number of RING pixels with z >= cos(cap_deg), by summing ring sizes."""
    zmin = math.cos(math.radians(cap_deg))
    return sum(ring_npix(nside, i) for i in _rings_in_cap(nside, zmin))


def ring_pixels(nside: int, i: int) -> np.ndarray:
    """(4 i or 4 nside, 3) float64 unit vectors of RING ring i."""
    z = ring_z(nside, i)
    n = ring_npix(nside, i)
    j = np.arange(1, n + 1, dtype=np.float64)
    if i < nside or i > 3 * nside:
        ii = i if i < nside else 4 * nside - i
        phi = (math.pi / (2.0 * ii)) * (j - 0.5)
    else:
        s = (i - nside + 1) % 2
        phi = (math.pi / (2.0 * nside)) * (j - 0.5 * s)
    # sin(theta) from (1 - z)(1 + z) keeps precision near the poles.
    st = math.sqrt(max(0.0, (1.0 - z) * (1.0 + z)))
    out = np.empty((n, 3), dtype=np.float64)
    out[:, 0] = st * np.cos(phi)
    out[:, 1] = st * np.sin(phi)
    out[:, 2] = z
    return out


def cap_pixels(nside: int, cap_deg: float, max_pixels: int | None = None) -> np.ndarray:
    """RING-ordered pixel centres with z >= cos(cap_deg), as (N, 3) float64.

    With ``max_pixels`` the result is the first ``max_pixels`` pixels of that cap
    in RING order (the most polar ones).
    """
    zmin = math.cos(math.radians(cap_deg))
    total = cap_count(nside, cap_deg)
    n = total if max_pixels is None else min(total, int(max_pixels))
    out = np.empty((n, 3), dtype=np.float64)
    pos = 0
    for i in _rings_in_cap(nside, zmin):
        if pos >= n:
            break
        r = ring_pixels(nside, i)
        take = min(len(r), n - pos)
        out[pos:pos + take] = r[:take]
        pos += take
    return out


def full_sphere(nside: int) -> np.ndarray:
    return np.concatenate([ring_pixels(nside, i) for i in range(1, 4 * nside)], axis=0)
