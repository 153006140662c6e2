"""The entry point that allocates nothing (hvox_direct_synthesize_noalloc).

It exists for callers that cannot call cudaMalloc, such as code running inside a
framework that owns the device's memory pool, or a per-iteration loop where an
allocation is not allowed. This file is collected last so that a run stopping at the
first failure has already run every other test; it passes alone or after the others.

Checks, through the C ABI, for both signs of the exponent: two calls in a row agree with
the FP64 oracle (relative l2 <= 10 eps at eps = 1e-6, the FP32 bound the other tests use)
and with the planned path (hvox_plan + hvox_synthesize, direct mode, FP32); the second
call leaves the device's free memory and torch's allocation unchanged; sizes beyond the
static limit are refused."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from hvox_inputs import configs

pytestmark = pytest.mark.gpu

EPS = 1e-6


def _call(lib, pix, uvw, I, V, isign):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.hvox_direct_synthesize_noalloc(pix.data_ptr(), pix.shape[0], uvw.data_ptr(), uvw.shape[0],
                                              I.data_ptr(), V.data_ptr(), isign, ctypes.c_void_p(stream))


@pytest.mark.parametrize("isign", [-1, 1])
def test_noalloc_matches_oracle_and_planned_path_twice(gpu_lib, isign):
    lib = gpu_lib.load()
    w = configs.small_case(seed=21, n_pix=3001, n_vis=7001, cap_deg=35.0, radius_m=2000.0)
    ref = oracle.sky2vis(w.pix, w.uvw, w.sky, isign=isign)
    plan = gpu_lib.Plan(w.pix, w.uvw, EPS, isign=isign, mode="direct", precision="fp32")
    I = torch.as_tensor(w.sky, dtype=torch.float32, device="cuda")
    planned = plan.synthesize(I).cpu().numpy()
    plan.close()
    pix = torch.as_tensor(w.pix, dtype=torch.float64, device="cuda")
    uvw = torch.as_tensor(w.uvw, dtype=torch.float64, device="cuda")
    outs = [torch.full((w.n_vis,), float("nan"), dtype=torch.complex64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for i, V in enumerate(outs):
        if i == 1:  # warmed up: the second call must take no device memory at all
            free0, _ = torch.cuda.mem_get_info()
            torch_bytes0 = torch.cuda.memory_allocated()
        code = _call(lib, pix, uvw, I, V, isign)
        assert code == 0, lib.hvox_last_error().decode()
        torch.cuda.synchronize()
        if i == 1:
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == torch_bytes0
    for V in outs:
        got = V.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert oracle.rel_l2(got, ref) <= 10 * EPS
        assert oracle.rel_l2(got, planned) <= 10 * EPS


def test_noalloc_rejects_sizes_beyond_limit(gpu_lib):
    lib = gpu_lib.load()
    n_pix, n_vis = 300000, 300000  # 600,000 points > 524,288
    pix = torch.zeros((n_pix, 3), dtype=torch.float64, device="cuda")
    uvw = torch.zeros((n_vis, 3), dtype=torch.float64, device="cuda")
    I = torch.zeros(n_pix, dtype=torch.float32, device="cuda")
    V = torch.zeros(n_vis, dtype=torch.complex64, device="cuda")
    code = _call(lib, pix, uvw, I, V, -1)
    assert code == 1
    assert "exceeds the static limit" in lib.hvox_last_error().decode()
