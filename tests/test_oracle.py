"""Pins of the direct-sum oracle against facts that do not come from the oracle itself:
the DFT special case (numpy.fft), the Dirichlet-kernel closed form, exact rational
phase reduction, symmetries of the Fourier sum, and adjointness. Sect. 2, Eq. 2-3."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(12345)


def grid_points(shape):
    nx, ny, nz = shape
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)


@pytest.mark.parametrize("isign", [-1, 1])
def test_dft_special_case_sky2vis(isign):
    # Pixels on a regular (4,5,3) lattice r = (i/4, j/5, k/3) and integer baselines:
    # the sum is the 3-D DFT, i.e. numpy.fft.fftn (isign=-1) or N*ifftn (isign=+1).
    shape = (4, 5, 3)
    idx = grid_points(shape)
    pix = idx / np.array(shape, dtype=np.float64)
    uvw = grid_points(shape)
    sky = RNG.uniform(0.0, 1.0, len(pix))
    wgt = RNG.uniform(0.5, 1.5, len(pix))
    v = oracle.sky2vis(pix, uvw, sky, weight=wgt, isign=isign)
    cube = (sky * wgt).reshape(shape)
    ref = np.fft.fftn(cube) if isign < 0 else np.fft.ifftn(cube) * cube.size
    assert np.max(np.abs(v - ref.ravel())) < 1e-12 * cube.size


@pytest.mark.parametrize("isign", [-1, 1])
def test_dft_special_case_vis2sky(isign):
    shape = (3, 4, 5)
    idx = grid_points(shape)
    pix = idx / np.array(shape, dtype=np.float64)
    uvw = grid_points(shape)
    vis = RNG.normal(size=len(uvw)) + 1j * RNG.normal(size=len(uvw))
    wgt = RNG.uniform(0.5, 1.5, len(pix))
    img = oracle.vis2sky(pix, uvw, vis, weight=wgt, isign=isign)
    cube = vis.reshape(shape)
    # sum_k V_k exp(-isign j 2pi p.r): isign=-1 -> N*ifftn, isign=+1 -> fftn
    ref = (np.fft.ifftn(cube) * cube.size) if isign < 0 else np.fft.fftn(cube)
    assert np.max(np.abs(img - wgt * ref.real.ravel())) < 1e-11 * cube.size


def test_dirichlet_closed_form():
    # Pixels equispaced on a line, one non-integer baseline: a geometric series.
    n, d = 257, 0.0137
    pix = np.zeros((n, 3))
    pix[:, 0] = np.arange(n) * d
    for q in (0.37, 11.91, 250.123):
        uvw = np.array([[q, 0.0, 0.0]])
        v = oracle.sky2vis(pix, uvw, np.ones(n), isign=-1)[0]
        th = 2 * math.pi * q * d
        ref = np.exp(-1j * th * (n - 1) / 2) * math.sin(n * th / 2) / math.sin(th / 2)
        assert abs(v - ref) < 1e-11 * n


def test_phase_reduction_exact_rational():
    # Large arguments (|p| ~ 1e5 wavelengths): compare the turn fraction with exact
    # rational arithmetic on the same binary64 inputs.
    m = 200
    uvw = RNG.uniform(-1.2e5, 1.2e5, (m, 3))
    pix = RNG.normal(size=(m, 3))
    pix /= np.linalg.norm(pix, axis=1, keepdims=True)
    got = oracle.phase_turns(uvw, pix)
    for i in range(m):
        t = sum(Fraction(float(uvw[i, d])) * Fraction(float(pix[i, d])) for d in range(3))
        f = t - round(t)
        ref = float(f)
        diff = abs(got[i] - ref)
        diff = min(diff, abs(abs(diff) - 1.0))  # +-0.5 ties are the same angle
        assert diff < 2e-16, (i, got[i], ref)


def _case(n_pix=60, n_vis=70, scale=300.0):
    pix = RNG.normal(size=(n_pix, 3))
    pix /= np.linalg.norm(pix, axis=1, keepdims=True)
    uvw = RNG.uniform(-scale, scale, (n_vis, 3))
    sky = RNG.lognormal(size=n_pix)
    wgt = RNG.uniform(0.5, 2.0, n_pix)
    return pix, uvw, sky, wgt


def test_conjugate_symmetry():
    pix, uvw, sky, wgt = _case()
    a = oracle.sky2vis(pix, uvw, sky, weight=wgt)
    b = oracle.sky2vis(pix, -uvw, sky, weight=wgt)
    assert np.max(np.abs(b - np.conj(a))) < 1e-11 * np.sum(sky * wgt)


def test_rotation_invariance():
    pix, uvw, sky, wgt = _case()
    q, _ = np.linalg.qr(RNG.normal(size=(3, 3)))
    a = oracle.sky2vis(pix, uvw, sky, weight=wgt)
    b = oracle.sky2vis(pix @ q.T, uvw @ q.T, sky, weight=wgt)
    assert oracle.rel_l2(b, a) < 1e-11


def test_shift_theorem():
    pix, uvw, sky, wgt = _case()
    r0 = np.array([0.013, -0.021, 0.0077])
    for isign in (-1, 1):
        a = oracle.sky2vis(pix, uvw, sky, weight=wgt, isign=isign)
        b = oracle.sky2vis(pix + r0, uvw, sky, weight=wgt, isign=isign)
        ramp = np.exp(isign * 2j * math.pi * (uvw @ r0))
        assert oracle.rel_l2(b, a * ramp) < 1e-11


def test_zero_baseline_is_total_flux():
    pix, uvw, sky, wgt = _case()
    uvw[5] = 0.0
    v = oracle.sky2vis(pix, uvw, sky, weight=wgt)
    assert abs(v[5] - np.sum(sky * wgt)) < 1e-12 * np.sum(sky * wgt)


def test_point_source_phase_ramp_is_character():
    # One unit source: V(p) is a character of the baseline group, |V| = 1 and
    # V(p1 + p2) = V(p1) V(p2).
    pix, uvw, _, _ = _case(n_pix=1, n_vis=50, scale=2e4)
    sky = np.ones(1)
    p1, p2 = uvw[:25], uvw[25:]
    v1 = oracle.sky2vis(pix, p1, sky)
    v2 = oracle.sky2vis(pix, p2, sky)
    v12 = oracle.sky2vis(pix, p1 + p2, sky)
    assert np.max(np.abs(np.abs(v1) - 1.0)) < 1e-14
    assert np.max(np.abs(v12 - v1 * v2)) < 1e-10


def test_adjointness_and_linearity():
    pix, uvw, sky, wgt = _case(80, 90, 2e3)
    y = RNG.normal(size=len(uvw)) + 1j * RNG.normal(size=len(uvw))
    for isign in (-1, 1):
        ax = oracle.sky2vis(pix, uvw, sky, weight=wgt, isign=isign)
        ahy = oracle.vis2sky(pix, uvw, y, weight=wgt, isign=isign)
        lhs = np.real(np.vdot(y, ax))
        rhs = float(np.dot(sky, ahy))
        assert abs(lhs - rhs) < 1e-11 * np.linalg.norm(ax) * np.linalg.norm(y)
    x2 = RNG.lognormal(size=len(pix))
    a = oracle.sky2vis(pix, uvw, 2.0 * sky - 3.0 * x2, weight=wgt)
    b = 2.0 * oracle.sky2vis(pix, uvw, sky, weight=wgt) - 3.0 * oracle.sky2vis(pix, uvw, x2, weight=wgt)
    assert oracle.rel_l2(a, b) < 1e-12


def test_sample_mode_matches_full():
    pix, uvw, sky, wgt = _case()
    full = oracle.sky2vis(pix, uvw, sky, weight=wgt)
    idx = np.array([0, 3, 17, 69])
    assert np.array_equal(oracle.sky2vis(pix, uvw, sky, weight=wgt, sample=idx), full[idx])
    y = RNG.normal(size=len(uvw)) + 1j * RNG.normal(size=len(uvw))
    img = oracle.vis2sky(pix, uvw, y, weight=wgt)
    idx = np.array([1, 2, 59])
    assert np.array_equal(oracle.vis2sky(pix, uvw, y, weight=wgt, sample=idx), img[idx])


def test_pins_catch_planted_mistakes():
    """The DFT pin fails for plausible oracle mistakes planted on the CPU side:
    a flipped sign, swapped coordinate axes, or a dropped 2*pi."""
    shape = (4, 5, 3)
    pix = grid_points(shape) / np.array(shape, dtype=np.float64)
    uvw = grid_points(shape)
    sky = RNG.uniform(0.0, 1.0, len(pix))
    ref = np.fft.fftn(sky.reshape(shape)).ravel()
    good = oracle.sky2vis(pix, uvw, sky, isign=-1)
    assert np.max(np.abs(good - ref)) < 1e-10
    flipped = oracle.sky2vis(pix, uvw, sky, isign=+1)
    swapped = oracle.sky2vis(pix[:, [1, 0, 2]], uvw, sky, isign=-1)
    no2pi = oracle.sky2vis(pix / (2 * math.pi), uvw, sky, isign=-1)
    for bad in (flipped, swapped, no2pi):
        assert np.max(np.abs(bad - ref)) > 1e-3
