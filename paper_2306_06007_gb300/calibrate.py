"""Per-stage calibration of the planner's cost model.

The paper fits its CPU build's runtime by regressing measured stage times on stage work
(spread, FFT, interpolation). This does the same for the GPU stages: each workload runs
in the library's serial profiling mode (every stage alone on the plan's stream, so the
CUDA-event stage times are the stages' own device times and add up to the step), over a
few steps, and each rate is fitted by least squares through the origin across the
workloads:

    spread ms         ~ taps         * c_spread     taps = (pix + vis points) * w^3
    interp ms         ~ taps         * c_interp
    fft ms            ~ 2 sum M2 log2 M2 * c_fft    (one FFT per direction)
    deconv + zero ms  ~ 2 (2 M1 + 2 M2)  * c_grid   (grid passes per direction)
    direct ms         ~ 2 direct_pairs   * c_direct

The fitted rates are printed beside the model's so that the constants of the planner can
be replaced by measured ones. Runs on the GPU through the public binding only. At
eps <= 1e-9 the sub-problems run in FP64; `--mode nufft` forces NUFFT sub-problems where
the model would choose direct sums, so that their rates can be measured at all.

    python -m paper_2306_06007_gb300.calibrate [--eps 1e-6] [--steps 3] [--mode nufft]
"""
from __future__ import annotations

import argparse
import json

STAGE_WORK = {
    "spread": lambda i: (i["nufft_pix_points"] + i["nufft_vis_points"]) * i["w"] ** 3,
    "interp": lambda i: (i["nufft_pix_points"] + i["nufft_vis_points"]) * i["w"] ** 3,
    "fft": lambda i: 2.0 * i["fft_work"],
    "grid": lambda i: 2.0 * (2.0 * i["spread_cells"] + 2.0 * i["nufft_cells"]),
    "direct": lambda i: 2.0 * i["direct_pairs"],
}

# Plan-info fields the stage work is computed from (kept with each measured row).
INFO_KEYS = ("precision", "w", "n_nufft_blocks", "nufft_pix_points", "nufft_vis_points", "spread_cells",
             "nufft_cells", "fft_work", "direct_pairs", "upsampfac")



def model_rates(precision: str) -> dict:
    """The planner's rates in the stage units above (from the library, FP32 or FP64 plans)."""
    from . import cost_model
    m = cost_model("fp32" if precision == "f32" else "fp64")
    return {"spread": m["scatter_smem"], "interp": m["gather_tap"], "fft": m["fft_cell"], "grid": m["grid_cell"],
            "direct": m["direct_pair"]}


def _workloads():
    import numpy as np

    from hvox_inputs import configs
    out = []
    for r in (1.0, 3.0, 10.0):
        out.append((f"radius {r:g} km", configs.radius_sweep(r)))
    w = configs.config3()
    w.uvw = np.ascontiguousarray(w.uvw[np.hypot(w.uvw[:, 0], w.uvw[:, 1]) <= 500.0])
    out.append(("config-3 dense core", w))
    return out


def measure(w, eps: float, steps: int, mode: str = "auto"):
    import torch

    from . import Plan
    plan = Plan(w.pix, w.uvw, eps, graphs=-1, mode=mode)
    info = plan.info()
    I = torch.as_tensor(w.sky, dtype=plan.real_dtype, device="cuda")
    V = torch.zeros(w.n_vis, dtype=plan.complex_dtype, device="cuda")
    plan.synthesize(I)
    plan.analyze(V)
    torch.cuda.synchronize()
    plan.profile("serial")
    for _ in range(steps):
        plan.synthesize(I, out=V)
        plan.analyze(V)
    st = plan.stats()
    plan.close()
    ms = {k: v / steps for k, v in st["ms"].items()}
    ms["grid"] = ms.pop("deconv") + ms.pop("zero")
    return info, ms


def fit(rows):
    """Least squares through the origin per stage: rate = sum(x t) / sum(x x)."""
    rates = {}
    for stage in STAGE_WORK:
        xs = [(STAGE_WORK[stage](info), ms[stage] * 1e-3) for info, ms in rows]
        sxx = sum(x * x for x, _ in xs)
        sxt = sum(x * t for x, t in xs)
        rates[stage] = sxt / sxx if sxx > 0 else None
    return rates


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--mode", default="auto", choices=["auto", "nufft"])
    ap.add_argument("--out", default="", help="also write the JSON report to this file")
    args = ap.parse_args(argv)
    rows, report = [], []
    for name, w in _workloads():
        info, ms = measure(w, args.eps, args.steps, args.mode)
        rows.append((info, ms))
        report.append({"workload": name, "n_pix": w.n_pix, "n_vis": w.n_vis, "blocks": info["n_nufft_blocks"],
                       "w": info["w"], "upsampfac": info["upsampfac"], "stage_ms": ms,
                       "work": {k: f(info) for k, f in STAGE_WORK.items()}})
    rates = fit(rows)
    model = model_rates("f64" if rows and rows[0][0]["precision"] == 2 else "f32")
    for r, (info, ms) in zip(report, rows):
        r["model_ms"] = {k: 1e3 * model[k] * f(info) for k, f in STAGE_WORK.items()}
        r["fitted_ms"] = {k: (1e3 * rates[k] * f(info) if rates[k] else None) for k, f in STAGE_WORK.items()}
    out = {"eps": args.eps, "mode": args.mode, "steps": args.steps, "fitted_seconds_per_unit": rates,
           "model_seconds_per_unit": model, "workloads": report,
           "rows": [{"info": {k: info[k] for k in INFO_KEYS}, "stage_ms": ms} for info, ms in rows]}
    text = json.dumps(out, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
