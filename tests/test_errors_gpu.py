"""Error paths on the GPU without any fault: an allocation the device cannot satisfy is
reported as HVOX_ENOMEM with nothing created, and the library keeps working after it."""
import numpy as np
import pytest
import torch

import oracle
from hvox_inputs import configs

pytestmark = pytest.mark.gpu


def test_out_of_memory_plan_is_reported_and_recoverable(gpu_lib):
    rng = np.random.default_rng(17)
    # Hemisphere of pixels x baselines spanning 12,000 wavelengths: one NUFFT sub-problem
    # whose spread grid alone needs ~1.5 TB (36,000 x 36,000 x 150 cells at sigma 1.5).
    v = rng.normal(size=(2000, 3))
    v[:, 2] = np.abs(v[:, 2])
    pix = v / np.linalg.norm(v, axis=1, keepdims=True)
    uvw = np.column_stack([rng.uniform(-6000, 6000, 2000), rng.uniform(-6000, 6000, 2000),
                           rng.uniform(-50, 50, 2000)])
    with pytest.raises(gpu_lib.HvoxError) as e:
        gpu_lib.Plan(pix, uvw, 1e-6, mode="nufft", upsampfac=1.5, chunk_budget_bytes=1e14)
    assert e.value.code == 2  # HVOX_ENOMEM
    # The failed plan left nothing behind: a normal plan runs and matches the oracle.
    w = configs.small_case(seed=2, n_pix=500, n_vis=700)
    plan = gpu_lib.Plan(w.pix, w.uvw, 1e-6, mode="nufft")
    V = plan.synthesize(torch.as_tensor(w.sky, dtype=plan.real_dtype, device="cuda")).cpu().numpy()
    plan.close()
    assert oracle.rel_l2(V, oracle.sky2vis(w.pix, w.uvw, w.sky)) <= 1e-5
