"""GPU: transforms of several plans in one call (hvox_synthesize_batch / hvox_analyze_batch),
the direct sums of the FP32 plans and of the double-float plans each merged into one
launch, against the same plans called one by one and against the FP64 oracle (Eq. 2 /
Eq. 3, relative l2 <= 10 eps)."""
import numpy as np
import pytest
import torch

import oracle
from hvox_inputs import configs

pytestmark = pytest.mark.gpu


PLAIN = [False, False, False, False, False, True]


@pytest.fixture(scope="module")
def jobs(gpu_lib):
    hv = gpu_lib
    cases = [
        # (seed, n_pix, n_vis, cap, radius, eps, isign, kwargs)
        (11, 700, 1500, 30.0, 300.0, 1e-6, -1, {"mode": "direct"}),
        (12, 1333, 911, 20.0, 500.0, 1e-4, 1, {"mode": "direct"}),
        (13, 900, 2100, 35.0, 400.0, 1e-9, -1, {"mode": "direct"}),
        (14, 1200, 1700, 25.0, 350.0, 1e-9, 1, {"mode": "auto"}),
        (15, 1500, 2500, 35.0, 400.0, 1e-6, -1, {"mode": "nufft"}),
        (16, 400, 600, 30.0, 300.0, 1e-9, -1, {"mode": "direct", "plain": True}),
    ]
    assert [bool(c[7].get("plain")) for c in cases] == PLAIN
    out = []
    for seed, npix, nvis, cap, rad, eps, isign, kw in cases:
        w = configs.small_case(seed=seed, n_pix=npix, n_vis=nvis, cap_deg=cap, radius_m=rad)
        plan = hv.Plan(w.pix, w.uvw, eps, isign=isign, **kw)
        vis = configs.visibilities_cn(seed, w.n_vis)
        out.append((w, plan, eps, isign, vis))
    yield out
    for _, plan, *_ in out:
        plan.close()


def _tol(eps):
    return 2e-6 if eps >= 1e-6 else 1e-12


def test_batch_matches_single_calls_and_oracle(gpu_lib, jobs):
    hv = gpu_lib
    plans = [j[1] for j in jobs]
    skies = [torch.as_tensor(w.sky, dtype=p.real_dtype, device="cuda") for w, p, *_ in jobs]
    vises = [torch.as_tensor(v, dtype=p.complex_dtype, device="cuda") for w, p, _, _, v in jobs]
    Vb, ls = hv.synthesize_batch(plans, skies, return_launches=True)
    Ib, la = hv.analyze_batch(plans, vises, return_launches=True)
    torch.cuda.synchronize()
    # FP32 direct plans (2) share a launch, double-float ones (2 with direct work) another,
    # the plain FP64 plan launches alone; the NUFFT-only plan has no direct work.
    n_direct = {"f32": 0, "df": 0, "f64": 0}
    for (w, p, eps, isign, v), plain in zip(jobs, PLAIN):
        if p.info()["direct_pairs"] > 0:
            n_direct["f64" if plain else ("f32" if p.precision == 1 else "df")] += 1
    print("direct launches", ls, la, n_direct)
    expect = sum(1 for k, c in n_direct.items() if c > 0)
    assert ls == expect and la == expect
    for (w, p, eps, isign, v), Vbatch, Ibatch in zip(jobs, Vb, Ib):
        Vs = p.synthesize(torch.as_tensor(w.sky, dtype=p.real_dtype, device="cuda")).cpu().numpy()
        Is = p.analyze(torch.as_tensor(v, dtype=p.complex_dtype, device="cuda")).cpu().numpy()
        Vbatch, Ibatch = Vbatch.cpu().numpy(), Ibatch.cpu().numpy()
        assert oracle.rel_l2(Vbatch, Vs) <= _tol(eps), (eps, oracle.rel_l2(Vbatch, Vs))
        assert oracle.rel_l2(Ibatch, Is) <= _tol(eps), (eps, oracle.rel_l2(Ibatch, Is))
        e_v = oracle.rel_l2(Vbatch, oracle.sky2vis(w.pix, w.uvw, w.sky, isign=isign))
        e_i = oracle.rel_l2(Ibatch, oracle.vis2sky(w.pix, w.uvw, v, isign=isign))
        assert e_v <= 10 * eps and e_i <= 10 * eps, (eps, e_v, e_i)


def test_batch_on_a_side_stream_is_ordered_with_the_plans(gpu_lib, jobs):
    # The call waits for each plan's queued work and each plan's stream waits for the call:
    # batch, then the plans' own calls, then batch again, on another stream, same results.
    hv = gpu_lib
    plans = [j[1] for j in jobs[:4]]
    skies = [torch.as_tensor(w.sky, dtype=p.real_dtype, device="cuda") for w, p, *_ in jobs[:4]]
    side = torch.cuda.Stream()
    a = hv.synthesize_batch(plans, skies, stream=side)
    singles = [p.synthesize(x) for p, x in zip(plans, skies)]
    b = hv.synthesize_batch(plans, skies, stream=side)
    torch.cuda.synchronize()
    for (w, p, eps, *_), x, y, z in zip(jobs, a, singles, b):
        assert oracle.rel_l2(x.cpu().numpy(), y.cpu().numpy()) <= _tol(eps)
        assert oracle.rel_l2(z.cpu().numpy(), y.cpu().numpy()) <= _tol(eps)


def test_batch_arguments(gpu_lib, jobs):
    hv = gpu_lib
    w, p = jobs[0][0], jobs[0][1]
    x = torch.as_tensor(w.sky, dtype=p.real_dtype, device="cuda")
    with pytest.raises(hv.HvoxError):
        hv.synthesize_batch([p, p], [x, x])          # a plan twice
    assert hv.synthesize_batch([], []) == []
