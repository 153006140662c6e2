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


# ---------------------------------------------------------------------------------------
# Host-side fault injection (HVOX_FAULT, read by the library at every injection site):
# each failure is raised or prepared on the host; no kernel faults, traps or waits.

@pytest.fixture
def fault(monkeypatch):
    def set_(spec):
        if spec:
            monkeypatch.setenv("HVOX_FAULT", spec)
        else:
            monkeypatch.delenv("HVOX_FAULT", raising=False)
    yield set_
    monkeypatch.delenv("HVOX_FAULT", raising=False)


def _case():
    return configs.small_case(seed=5, n_pix=900, n_vis=1300)


def _check_clean_plan(gpu_lib, w, **kw):
    plan = gpu_lib.Plan(w.pix, w.uvw, 1e-6, **kw)
    V = plan.synthesize(torch.as_tensor(w.sky, dtype=plan.real_dtype, device="cuda")).cpu().numpy()
    plan.close()
    assert oracle.rel_l2(V, oracle.sky2vis(w.pix, w.uvw, w.sky)) <= 1e-5


def test_every_failed_allocation_of_a_plan_is_clean(gpu_lib, fault):
    # The n-th device allocation of hvox_plan fails for n = 1, 2, ...: each attempt returns
    # HVOX_ENOMEM and frees what it had allocated (device free memory back where it was),
    # until n passes the plan's last allocation and the plan succeeds.
    w = _case()
    # A complete plan first, so that CUDA has loaded the library's device code and cuFFT
    # its own state (both hold device memory for the life of the process).
    _check_clean_plan(gpu_lib, w, mode="nufft")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n_failed = 0
    for n in range(1, 200):
        fault(f"alloc:{n}")
        try:
            plan = gpu_lib.Plan(w.pix, w.uvw, 1e-6, mode="nufft")
        except gpu_lib.HvoxError as e:
            assert e.code == 2 and "injected" in str(e), str(e)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0, f"allocation {n}: device memory not returned"
            n_failed += 1
            continue
        plan.close()
        break
    else:
        pytest.fail("the plan never got past its injected allocation failures")
    assert n_failed >= 10  # coordinates, splits, permutations, tables, lanes' grids, call buffers
    fault(None)
    _check_clean_plan(gpu_lib, w, mode="nufft")


def test_failed_cufft_plan_is_reported(gpu_lib, fault):
    w = _case()
    fault("cufft:1")
    with pytest.raises(gpu_lib.HvoxError) as e:
        gpu_lib.Plan(w.pix, w.uvw, 1e-6, mode="nufft")
    assert e.value.code == 3 and "injected" in str(e.value)  # HVOX_ECUDA
    fault(None)
    _check_clean_plan(gpu_lib, w, mode="nufft")


def test_failed_staging_allocation_in_a_call(gpu_lib, fault):
    # A host-pointer call allocates its staging buffers on first use: if that fails the call
    # reports HVOX_ENOMEM and the plan stays usable.
    w = _case()
    plan = gpu_lib.Plan(w.pix, w.uvw, 1e-6, mode="nufft")
    I_host = torch.as_tensor(w.sky, dtype=plan.real_dtype)
    fault("alloc:1")
    with pytest.raises(gpu_lib.HvoxError) as e:
        plan.synthesize(I_host)
    assert e.value.code == 2
    fault(None)
    V = plan.synthesize(I_host).numpy()
    plan.close()
    assert oracle.rel_l2(V, oracle.sky2vis(w.pix, w.uvw, w.sky)) <= 1e-5


def test_failed_graph_capture_falls_back_to_eager(gpu_lib, fault):
    w = _case()
    fault("capture:1")
    plan = gpu_lib.Plan(w.pix, w.uvw, 1e-6, mode="nufft", graphs=1)
    I = torch.as_tensor(w.sky, dtype=plan.real_dtype, device="cuda")
    outs = [plan.synthesize(I).cpu().numpy() for _ in range(3)]  # eager, failed capture, eager
    assert plan.info()["graph_state"] == -1
    plan.close()
    for V in outs:
        assert oracle.rel_l2(V, oracle.sky2vis(w.pix, w.uvw, w.sky)) <= 1e-5


@pytest.mark.parametrize("eps", [1e-6, 1e-9])
def test_device_error_word_reports_clamped_windows(gpu_lib, fault, eps):
    # One sub-problem's pixel scale is multiplied by 4 on the host: its pixels' windows fall
    # outside the n1 grid, the kernels clamp them into it (every access stays in bounds) and
    # set the plan's device error word, which hvox_sync reports once as HVOX_EINTERNAL.
    w = _case()
    fault("window:1")
    plan = gpu_lib.Plan(w.pix, w.uvw, eps, mode="nufft", upsampfac=2.0, chunk_budget_bytes=1e6)
    fault(None)
    assert plan.info()["n_nufft_blocks"] >= 2
    I = torch.as_tensor(w.sky, dtype=plan.real_dtype, device="cuda")
    plan.synthesize(I)
    with pytest.raises(gpu_lib.HvoxError) as e:
        plan.sync()
    assert e.value.code == 6 and "pixel window" in str(e.value)
    plan.sync()  # the report cleared the word
    plan.close()
    _check_clean_plan(gpu_lib, w, mode="nufft")
