"""The entry point that allocates nothing (hvox_direct_synthesize_noalloc).

It exists for callers that cannot call cudaMalloc, such as code running inside a
framework that owns the device's memory pool, or a per-iteration loop where an
allocation is not allowed. This file is collected last so that a run stopping at the
first failure has already run every other test; it passes alone or after the others.

Checks, through the C ABI, that two calls in a row match the planned path
(hvox_plan + hvox_synthesize, direct mode, FP32) within the FP32 tolerance the other
tests use (relative l2 <= 10 eps at eps = 1e-6), and that sizes beyond the static
limit are refused."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from hvox_inputs import configs

pytestmark = pytest.mark.gpu


def _call(lib, pix, uvw, I, V, isign=-1):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.hvox_direct_synthesize_noalloc(pix.data_ptr(), pix.shape[0], uvw.data_ptr(), uvw.shape[0],
                                              I.data_ptr(), V.data_ptr(), isign, ctypes.c_void_p(stream))


def test_noalloc_matches_planned_path_twice(gpu_lib):
    lib = gpu_lib.load()
    w = configs.small_case(seed=21, n_pix=3001, n_vis=7001, cap_deg=35.0, radius_m=2000.0)
    plan = gpu_lib.Plan(w.pix, w.uvw, 1e-6, mode="direct", precision="fp32")
    I = torch.as_tensor(w.sky, dtype=torch.float32, device="cuda")
    ref = plan.synthesize(I).cpu().numpy()
    plan.close()
    pix = torch.as_tensor(w.pix, dtype=torch.float64, device="cuda")
    uvw = torch.as_tensor(w.uvw, dtype=torch.float64, device="cuda")
    for _ in range(2):
        V = torch.full((w.n_vis,), float("nan"), dtype=torch.complex64, device="cuda")
        code = _call(lib, pix, uvw, I, V)
        assert code == 0, lib.hvox_last_error().decode()
        torch.cuda.synchronize()
        got = V.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert oracle.rel_l2(got, ref) <= 1e-5


def test_noalloc_rejects_sizes_beyond_limit(gpu_lib):
    lib = gpu_lib.load()
    n_pix, n_vis = 300000, 300000  # 600,000 points > 524,288
    pix = torch.zeros((n_pix, 3), dtype=torch.float64, device="cuda")
    uvw = torch.zeros((n_vis, 3), dtype=torch.float64, device="cuda")
    I = torch.zeros(n_pix, dtype=torch.float32, device="cuda")
    V = torch.zeros(n_vis, dtype=torch.complex64, device="cuda")
    code = _call(lib, pix, uvw, I, V)
    assert code == 1
    assert "exceeds the static limit" in lib.hvox_last_error().decode()
