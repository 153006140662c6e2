"""GPU: the double-float FFT of FP64 NUFFT grids against cuFFT's Z2Z transform of the same
grids, and against the oracle.

Both plans of a comparison share the partition, kernel, grids and every other stage; only the
uniform FFT of step 2 of the type-3 transform (Sect. 3) differs, so the outputs agree to the
rounding of a ~48-bit FFT (relative l2 far below eps), in both directions and for both signs
of the exponent."""
import numpy as np
import pytest
import torch

import oracle
from hvox_inputs import configs

pytestmark = pytest.mark.gpu


def _pair(hvox, w, eps, isign, monkeypatch, **kw):
    out = []
    vis = configs.visibilities_cn(8, w.n_vis)
    for df in ("1", "0"):
        monkeypatch.setenv("HVOX_DF_FFT", df)
        plan = hvox.Plan(w.pix, w.uvw, eps, isign=isign, **kw)
        info = plan.info()
        V = plan.synthesize(torch.as_tensor(w.sky, dtype=plan.real_dtype, device="cuda")).cpu().numpy()
        img = plan.analyze(torch.as_tensor(vis, dtype=plan.complex_dtype, device="cuda")).cpu().numpy()
        plan.close()
        out.append((V, img, info))
    monkeypatch.delenv("HVOX_DF_FFT")
    return out, vis


@pytest.mark.parametrize("isign", [-1, 1])
def test_df_fft_matches_z2z_small(gpu_lib, isign, monkeypatch):
    w = configs.small_case(seed=3, n_pix=1333, n_vis=2777, cap_deg=35.0, radius_m=400.0)
    (a, b), vis = _pair(gpu_lib, w, 1e-9, isign, monkeypatch, mode="nufft")
    (Va, Ia, ia), (Vb, Ib, ib) = a, b
    assert ia["precision"] == 2 and ia["fft_batches"] > 0
    assert ia["fft_batches_df"] == ia["fft_batches"] and ib["fft_batches_df"] == 0
    d_v, d_i = oracle.rel_l2(Va, Vb), oracle.rel_l2(Ia, Ib)
    print(f"isign={isign}: df vs z2z rel_l2 sky->vis {d_v:.3e} vis->sky {d_i:.3e}")
    assert d_v <= 1e-11 and d_i <= 1e-11
    assert oracle.rel_l2(Va, oracle.sky2vis(w.pix, w.uvw, w.sky, isign=isign)) <= 1e-8
    assert oracle.rel_l2(Ia, oracle.vis2sky(w.pix, w.uvw, vis, isign=isign)) <= 1e-8


def test_df_fft_matches_z2z_1km(gpu_lib, monkeypatch):
    # 130,000 pixels x 95,266 baselines: several waves of FP64 NUFFT sub-problems, grids of
    # every shape the planner picks there (ragged column tiles, odd radices 3, 5, 7).
    w = configs.radius_sweep(1.0)
    (a, b), _ = _pair(gpu_lib, w, 1e-9, -1, monkeypatch)
    (Va, Ia, ia), (Vb, Ib, ib) = a, b
    assert ia["n_nufft_blocks"] > 0 and ia["fft_batches_df"] > 0 and ib["fft_batches_df"] == 0
    d_v, d_i = oracle.rel_l2(Va, Vb), oracle.rel_l2(Ia, Ib)
    print(f"1 km: {ia['fft_batches_df']} df batches; df vs z2z rel_l2 sky->vis {d_v:.3e} vis->sky {d_i:.3e}")
    assert d_v <= 1e-11 and d_i <= 1e-11


def test_df_fft_off_where_it_does_not_apply(gpu_lib):
    w = configs.small_case(seed=3, n_pix=1333, n_vis=2777, cap_deg=35.0, radius_m=400.0)
    for kw in ({"eps": 1e-12}, {"eps": 1e-9, "plain": True}, {"eps": 1e-6}):
        eps = kw.pop("eps")
        plan = gpu_lib.Plan(w.pix, w.uvw, eps, mode="nufft", **kw)
        info = plan.info()
        plan.close()
        assert info["fft_batches"] > 0 and info["fft_batches_df"] == 0, (eps, kw)
