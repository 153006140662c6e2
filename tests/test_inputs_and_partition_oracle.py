"""Pins for the synthetic inputs (HEALPix, Gorski et al. 2005) and the planner oracle
(Algorithm 1 box dimensions, Algorithm 2 lattice chunking; Sect. 3.2)."""
import json
import math
import os

import numpy as np
import pytest

from hvox_inputs import healpix, layouts, configs
from oracle import partition

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ HEALPix

def test_healpix_cap_counts_golden():
    with open(os.path.join(GOLDEN, "healpix_cap_counts.json")) as f:
        g = json.load(f)
    for row in g["cases"]:
        assert healpix.cap_count(row["nside"], row["cap_deg"]) == row["count"]


@pytest.mark.parametrize("nside", [1, 2, 3, 8, 13])
def test_healpix_full_sphere(nside):
    v = healpix.full_sphere(nside)
    assert len(v) == 12 * nside * nside
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    # Equal area: the mean of z and of x, y over the sphere vanishes.
    assert np.all(np.abs(v.mean(axis=0)) < 1e-12)
    # No two pixel centres coincide.
    assert len(np.unique(np.round(v, 12), axis=0)) == len(v)


def test_healpix_equal_area_bands():
    # Pixels are equal-area, so a polar cap z >= z0 holds ~ Npix (1 - z0) / 2 of them.
    nside = 64
    v = healpix.full_sphere(nside)
    for z0 in (0.9, 0.5, 0.0, -0.4):
        frac = np.mean(v[:, 2] >= z0)
        assert abs(frac - (1.0 - z0) / 2.0) < 4.0 / nside


def test_cap_prefix_of_ring_order():
    full = healpix.full_sphere(16)
    cap = healpix.cap_pixels(16, 40.0)
    assert np.array_equal(cap, full[:len(cap)])
    assert np.all(cap[:, 2] >= math.cos(math.radians(40.0)) - 1e-12)
    assert full[len(cap), 2] < math.cos(math.radians(40.0))


def test_layout_sizes():
    ant = layouts.disk_uniform(np.random.default_rng(0), 10, 100.0, 1.0)
    b = layouts.baselines(ant, [0.0, 10.0], 45.0, [1.0, 2.0])
    assert b.shape == (45 * 4, 3)
    # Rotation about the polar axis preserves baseline lengths.
    axis = np.array([0.0, math.cos(math.radians(45.0)), math.sin(math.radians(45.0))])
    d = layouts.pair_differences(ant)
    r = layouts.rotate_about_axis(d, axis, 0.3)
    assert np.allclose(np.linalg.norm(r, axis=1), np.linalg.norm(d, axis=1))


def test_config1_shapes():
    w = configs.config1()
    assert (w.n_pix, w.n_vis) == (1740, 19900)
    assert np.all(np.abs(w.uvw[:, :2]) <= 1000.0)


# ------------------------------------------------------------------ Algorithm 1

def test_box_dims_fits_whole():
    eta, h, t = partition.box_dims([1.0, 1.0, 0.1], [10.0, 10.0, 2.0], 1e9, 2.0, 7, 8)
    assert t == 1.0


def test_box_dims_maximal_under_budget():
    P, B = [1.0, 0.9, 0.13], [2e5, 1.9e5, 4.5e4]
    for budget in (16e6, 500e6):
        eta, h, t = partition.box_dims(P, B, budget, 2.0, 10, 16)
        assert 0.0 < t < 1.0
        assert partition.grid_bytes(eta, h, 2.0, 10, 16) <= budget
        bigger = t * (1.0 + 1e-6)
        assert partition.grid_bytes([bigger * x for x in P], [bigger * x for x in B], 2.0, 10, 16) > budget
        # Isotropic: every ratio h_k/B_k and eta_k/P_k equals t.
        assert np.allclose(np.array(h) / B, t) and np.allclose(np.array(eta) / P, t)


@pytest.mark.parametrize("alpha", [1.0, 1.5, 4.0])
def test_box_dims_lp_isotropic_optimum(alpha):
    # The paper's LP in log variables (scipy linprog): at alpha=1 it returns the
    # isotropic point; for alpha>1 the isotropic point attains the same optimum.
    P, B = [1.0, 0.8, 0.2], [3e3, 2e3, 80.0]
    log_budget = math.log(1e4)
    eta, h, obj = partition.box_dims_lp(P, B, log_budget, alpha)
    const = sum(math.log(P[k] * B[k]) for k in range(3))
    t = math.exp((log_budget - const) / 6.0)
    assert abs(obj - 6.0 * math.log(t)) < 1e-7
    assert abs(sum(math.log(eta[k] * h[k]) for k in range(3)) - log_budget) < 1e-7
    if alpha == 1.0:
        assert np.allclose(np.array(h) / B, t, rtol=1e-6) and np.allclose(np.array(eta) / P, t, rtol=1e-6)


def test_smooth_even():
    assert [partition.smooth_even(n) for n in (1, 2, 11, 13, 22, 23, 97)] == [2, 2, 12, 14, 24, 24, 98]
    for n in range(2, 500):
        m = partition.smooth_even(n)
        assert m >= n and m % 2 == 0


# Grid sizes worked by hand from Eq. 5-7 (one grid dimension ~ sigma x pixel extent x
# baseline extent) with the sizing reading: n1 = even >= sigma P B + w + 2 (spread grid,
# kernel margin), n2 = smallest even 2,3,5,7-smooth number >= max(sigma n1, 2 w) (FFT
# grid: the second upsampling of the two-stage type-3), bytes = elem (prod n1 + prod n2).
# Each value below was derived on paper, not by running the code:
#   P=0.5, B=100, sigma=2, w=7: need 2*50+9 = 109 -> n1 110; sigma n1 = 220 = 2^2 5 11,
#       222 = 2 3 37 are not 7-smooth, 224 = 2^5 7 is -> n2 224.
#   same with sigma=1.5, w=9: need 75+11 = 86 -> n1 86; 1.5*86 = 129 -> even 130 = 2 5 13
#       no, 132 = 2^2 3 11 no, 134 no, 136 = 2^3 17 no, 138 = 2 3 23 no, 140 = 2^2 5 7 -> 140.
#   sigma=1.5, w=7: need 75+9 = 84 -> n1 84; 126 = 2 3^2 7 -> n2 126.
#   degenerate extent (P=0): need w+2 = 9 -> n1 10; sigma=2: max(20, 14) -> 20;
#       sigma=1.25: max(ceil 12.5 = 13, 2w = 14) -> 14.
#   degenerate, w=16, sigma=1.25: need 18 -> n1 18; sigma n1 = 22.5 -> 23 -> even 24 = 2^3 3,
#       but the 2w floor is 32 -> n2 32 (the floor decides).
GRID_SIZE_CASES = [
    (0.5, 100.0, 2.0, 7, 110, 224),
    (0.5, 100.0, 1.5, 9, 86, 140),
    (0.5, 100.0, 1.5, 7, 84, 126),
    (0.0, 100.0, 2.0, 7, 10, 20),
    (0.7, 0.0, 1.25, 7, 10, 14),
    (0.0, 5.0, 1.25, 16, 18, 32),
]


@pytest.mark.parametrize("P,B,sigma,w,n1,n2", GRID_SIZE_CASES)
def test_grid_sizes_hand_worked(P, B, sigma, w, n1, n2):
    assert partition.grid_sizes(P, B, sigma, w) == (n1, n2)


def test_grid_bytes_hand_worked():
    # x, y: as the first case above (110, 224); z: P 0.1, B 10: need 2+9 = 11 -> n1 12,
    # max(24, 14) = 24 = 2^3 3 -> n2 24. Bytes (complex64) = 8 (110^2 12 + 224^2 24)
    # = 8 (145,200 + 1,204,224) = 10,795,392.
    assert partition.grid_bytes([0.5, 0.5, 0.1], [100.0, 100.0, 10.0], 2.0, 7, 8) == 10_795_392
    # complex128 doubles it.
    assert partition.grid_bytes([0.5, 0.5, 0.1], [100.0, 100.0, 10.0], 2.0, 7, 16) == 21_590_784


# Algorithm 1 at a budget worked by hand: P = (1,1,1), B = (100,100,100), sigma 2, w 7,
# complex64. At scale t every dimension needs 200 t^2 + 9 cells. The budget is the bytes
# of n1 = 110, n2 = 224 per dimension: 8 (110^3 + 224^3) = 100,563,392. The grids fit
# while 200 t^2 + 9 <= 110, i.e. t <= sqrt(101/200); just above, n1 = 112 and n2 =
# smooth(224) = 224 exceed it. So t* = sqrt(101/200) = 0.71063352...
# Counting sigma once (n2 = smooth(n1)) or dropping the w + 2 margin would let t grow past it.
def test_box_dims_hand_worked_budget():
    budget = 8 * (110 ** 3 + 224 ** 3)
    assert budget == 100_563_392
    eta, h, t = partition.box_dims([1.0, 1.0, 1.0], [100.0, 100.0, 100.0], budget, 2.0, 7, 8)
    assert abs(t - math.sqrt(101.0 / 200.0)) < 1e-12
    assert np.allclose(h, 100.0 * t) and np.allclose(eta, t)


def test_grid_pins_catch_planted_mistakes(monkeypatch):
    """Mistakes planted in a copy of the oracle's sizing (on the CPU) fail the pins above."""
    good = partition.grid_sizes

    def sigma_once(P, B, sigma, w):  # FFT grid not upsampled a second time
        n1, _ = good(P, B, sigma, w)
        return n1, partition.smooth_even(max(n1, 2 * w))

    def no_margin(P, B, sigma, w):  # kernel margin w + 2 dropped
        n1 = 2 * int(math.ceil(sigma * P * B / 2.0))
        return n1, partition.smooth_even(max(int(math.ceil(sigma * n1)), 2 * w))

    def no_floor(P, B, sigma, w):  # 2w floor of the FFT grid dropped
        n1, _ = good(P, B, sigma, w)
        return n1, partition.smooth_even(int(math.ceil(sigma * n1)))

    budget = 8 * (110 ** 3 + 224 ** 3)
    for bad in (sigma_once, no_margin, no_floor):
        monkeypatch.setattr(partition, "grid_sizes", bad)
        size_fail = any(bad(P, B, s, w) != (n1, n2) for P, B, s, w, n1, n2 in GRID_SIZE_CASES)
        _, _, t = partition.box_dims([1.0, 1.0, 1.0], [100.0, 100.0, 100.0], budget, 2.0, 7, 8)
        assert size_fail, bad.__name__
        if bad is not no_floor:  # the floor never binds at this budget
            assert abs(t - math.sqrt(101.0 / 200.0)) > 1e-3, bad.__name__
    monkeypatch.setattr(partition, "grid_sizes", good)


# ------------------------------------------------------------------ Algorithm 2

def _check_partition(pts, h, labels, nc):
    assert labels.min() == 0 and labels.max() == nc - 1
    assert len(np.unique(labels)) == nc  # no empty chunk
    lo, hi = partition.chunk_boxes(pts, labels, nc)
    assert np.all(hi - lo <= np.asarray(h) + 0.0)
    cells = partition.lattice_cells(pts, h)
    for c in range(nc):
        cc = cells[labels == c]
        assert np.all(cc.max(axis=0) - cc.min(axis=0) <= 1)  # inside a 2x2x2 window


def test_chunk_invariants_random():
    rng = np.random.default_rng(7)
    pts = np.concatenate([rng.normal(0, 1, (400, 3)), rng.normal(0, 10, (100, 3)) * [1, 1, 0.1]])
    h = [0.7, 0.9, 0.5]
    labels, nc = partition.chunk(pts, h)
    _check_partition(pts, h, labels, nc)


def test_chunk_hand_case():
    # 1-D layout along x with h = 1: cells 0,0,1,2,5 -> points at x=0.1,0.5 (cell 0),
    # 1.05 (cell 1), 2.7 (cell 2), 5.2 (cell 5). Cell 0 absorbs cell 1 (extent 0.95 <= 1);
    # cell 2 alone (absorbing nothing at cell 3); cell 5 alone.
    x = np.array([0.1, 0.5, 1.05, 2.7, 5.2])
    pts = np.stack([x, np.zeros(5), np.zeros(5)], axis=1)
    labels, nc = partition.chunk(pts, [1.0, 1.0, 1.0])
    assert nc == 3
    assert labels.tolist() == [0, 0, 0, 1, 2]
    # Refusal of fusion when the joint box would exceed h: 1.15 - 0.1 > 1.
    pts[2, 0] = 1.15
    labels, nc = partition.chunk(pts, [1.0, 1.0, 1.0])
    assert labels.tolist() == [0, 0, 1, 2, 3]


def test_chunk_degenerate_dims():
    # All points share z, and h_z = 0: one cell along z.
    rng = np.random.default_rng(3)
    pts = np.concatenate([rng.uniform(0, 3, (50, 2)), np.zeros((50, 1))], axis=1)
    labels, nc = partition.chunk(pts, [1.0, 1.0, 0.0])
    _check_partition(pts, [1.0, 1.0, 0.0], labels, nc)
    labels, nc = partition.chunk(pts[:1], [1.0, 1.0, 0.0])
    assert nc == 1
