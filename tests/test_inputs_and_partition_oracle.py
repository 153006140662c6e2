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
