"""CPU checks of the host planner's search (Algorithm 1 budgets, upsampling, box ratios)
through host-only planning: infeasible budgets are skipped or rejected, FP64 plans take
NUFFT sub-problems where the cost model prices them below direct sums, and a dense core
inside a long-baseline array is met by elongated boxes (one pixel box over the whole
sky, small baseline boxes)."""
import pytest

import paper_2306_06007_gb300 as hvox
from hvox_inputs import configs


@pytest.fixture(scope="module")
def lib():
    hvox.build()
    return hvox.load()


def test_forced_nufft_search_skips_infeasible_budgets(lib):
    # At the smallest budgets forced NUFFT mode would cut the 1 km case into ~1e10
    # candidate sub-problems; those budgets are skipped, not enumerated.
    w = configs.radius_sweep(1.0)
    info = hvox.plan_dry(w.pix, w.uvw, 1e-9, mode="nufft")
    assert info["n_nufft_blocks"] >= 1 and info["direct_pairs"] == 0.0
    assert 0 < info["max_grid_bytes"] <= info["budget_bytes"]


def test_budget_below_the_smallest_grid_is_rejected(lib):
    # A grid needs at least 2w cells per dimension (w = 10 at 1e-9): 10 kB holds none.
    w = configs.small_case(seed=3, n_pix=500, n_vis=500)
    with pytest.raises(hvox.HvoxError) as e:
        hvox.plan_dry(w.pix, w.uvw, 1e-9, mode="nufft", chunk_budget_bytes=1e4)
    assert e.value.code == 1  # HVOX_EINVAL
    assert "chunk budget" in str(e.value)


@pytest.mark.parametrize("radius_km", [1.0, 3.0])
def test_fp64_plans_choose_nufft_where_cheaper(lib, radius_km):
    w = configs.radius_sweep(radius_km)
    auto = hvox.plan_dry(w.pix, w.uvw, 1e-9)
    direct = hvox.plan_dry(w.pix, w.uvw, 1e-9, mode="direct")
    assert auto["precision"] == 2 and auto["n_nufft_blocks"] >= 1
    assert auto["model_seconds"] < 0.5 * direct["model_seconds"]


def test_dense_core_in_long_array_gets_elongated_boxes(lib):
    # LOFAR-like layout (log-radial 50 m .. 100 km): isotropic boxes cut the sky into
    # chunks too small for any grid to pay; the ratio search finds pixel boxes that span
    # the sky and NUFFT sub-problems for the short baselines.
    w = configs.config2()
    auto = hvox.plan_dry(w.pix, w.uvw, 1e-6)
    direct = hvox.plan_dry(w.pix, w.uvw, 1e-6, mode="direct")
    assert auto["n_nufft_blocks"] >= 1 and auto["box_ratio"] > 1.0
    assert auto["n_pix_chunks"] <= 4
    assert auto["direct_pairs"] < direct["direct_pairs"]
    assert auto["model_seconds"] < direct["model_seconds"]


@pytest.mark.parametrize("eps,sigma_ok", [(1e-10, (1.5, 2.0)), (1e-12, (2.0,)), (1e-14, (2.0,))])
def test_tolerances_below_1e9_are_planned(lib, eps, sigma_ok):
    # Upsamplings whose kernel would exceed 16 cells are dropped from the search instead
    # of failing the plan; the remaining candidates keep w <= 16.
    w = configs.radius_sweep(1.0)
    info = hvox.plan_dry(w.pix, w.uvw, eps)
    assert info["precision"] == 2 and info["upsampfac"] in sigma_ok and info["w"] <= 16


def test_tolerance_beyond_the_widest_kernel_is_unsupported(lib):
    w = configs.small_case(seed=3, n_pix=500, n_vis=500)
    with pytest.raises(hvox.HvoxError) as e:
        hvox.plan_dry(w.pix, w.uvw, 1e-16)
    assert e.value.code == 5  # HVOX_EUNSUPPORTED


def test_fp64_plans_widen_the_kernel(lib):
    # FP64 NUFFT sub-problems take the width rule at eps / 10: at 1e-9, w = 11 for
    # sigma 2 (the bare rule gives 10) and 13 for sigma 1.5 (bare: 12).
    w = configs.small_case(seed=3, n_pix=500, n_vis=500)
    assert hvox.plan_dry(w.pix, w.uvw, 1e-9, mode="nufft", upsampfac=2.0)["w"] == 11
    assert hvox.plan_dry(w.pix, w.uvw, 1e-9, mode="nufft", upsampfac=1.5)["w"] == 13
    assert hvox.es_params(1e-10, 2.0)[0] == 11 and hvox.es_params(1e-9, 2.0)[0] == 10
    # A caller-fixed sigma 1.25 would need 17 cells with the margin: it keeps the widest
    # kernel, 16 cells (the bare rule's 15 still fits).
    assert hvox.plan_dry(w.pix, w.uvw, 1e-9, mode="nufft", upsampfac=1.25)["w"] == 16
    # FP32 plans keep the bare rule.
    assert hvox.plan_dry(w.pix, w.uvw, 1e-6, mode="nufft", upsampfac=2.0)["w"] == 7


def test_direct_sums_below_1e9_are_priced_as_fp64(lib):
    # Below 1e-9 the direct sums run on the FP64 kernels (~1/100 of the double-float
    # rate), so the same job's all-direct model cost rises ~100x.
    w = configs.small_case(seed=3, n_pix=1333, n_vis=2777)
    a = hvox.plan_dry(w.pix, w.uvw, 1e-9, mode="direct")["model_seconds"]
    b = hvox.plan_dry(w.pix, w.uvw, 1e-11, mode="direct")["model_seconds"]
    assert 50 < b / a < 200


@pytest.mark.parametrize("factor,which", [("pixels", "n_vis_chunks"), ("baselines", "n_pix_chunks")])
def test_factored_plans_span_the_other_set(lib, factor, which):
    # A factored evaluation shares one set's spreading across sub-problems only when one box
    # spans the other set: forcing it leaves a single chunk of that set, at a budget where
    # Algorithm 1's own boxes would cut both sets.
    w = configs.radius_sweep(1.0)
    base = hvox.plan_dry(w.pix, w.uvw, 1e-6, mode="nufft", chunk_budget_bytes=4e6)
    assert base["n_pix_chunks"] > 1 and base["n_vis_chunks"] > 1 and base["t"] < 1.0
    f = hvox.plan_dry(w.pix, w.uvw, 1e-6, mode="nufft", chunk_budget_bytes=4e6, factor=factor)
    assert f[which] == 1
    assert abs(f["t"] - base["t"]) < 1e-12  # the same grid budget per sub-problem
    assert (f["box_ratio"] < 1.0) == (factor == "pixels")


def test_caller_fixed_kernel_width(lib):
    # hvox_opts.kernel_width fixes the width for every upsampling the search tries (the
    # shape parameter from the same rule); the rule's own width is reported beside it.
    w = configs.radius_sweep(1.0)
    rule = hvox.plan_dry(w.pix, w.uvw, 1e-6, mode="nufft")
    fixed = hvox.plan_dry(w.pix, w.uvw, 1e-6, mode="nufft", kernel_width=rule["w"] - 1)
    assert fixed["w"] == rule["w"] - 1
    assert fixed["kernel_width_rule"] == rule["w"] or fixed["upsampfac"] != rule["upsampfac"]
    with pytest.raises(hvox.HvoxError):
        hvox.plan_dry(w.pix, w.uvw, 1e-6, kernel_width=17)
