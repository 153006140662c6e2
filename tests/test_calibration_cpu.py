"""The planner's cost model against measured stage times (CPU; the measurements are stored).

The paper fits its runtime model by regressing measured spread, FFT and interpolation
times on their work (appendix). calibrate.py does the same for this library's GPU stages.
The fixtures under tests/golden/ are its reports from one GB300 run each:

    python -m paper_2306_06007_gb300.calibrate --eps 1e-6 --steps 3 --out calibration_f32_eps1e-6.json
    python -m paper_2306_06007_gb300.calibrate --eps 1e-9 --steps 2 --mode nufft --out calibration_f64_eps1e-9.json

(the 1, 3 and 10 km sweep cases and the dense core of the SKA-Low-like workload, serial
profiling mode). The tests check that the fit in calibrate.py reproduces the report's own
fitted rates from its rows, that the planner's constants are those fits (stages with
enough work in every workload: spreading, interpolation, FFT and grid passes), and that
the model predicts each measured step within 20 %."""
import json
import os

import pytest

import paper_2306_06007_gb300 as hvox
from paper_2306_06007_gb300 import calibrate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FIXTURES = {"fp32": "calibration_f32_eps1e-6.json", "fp64": "calibration_f64_eps1e-9.json"}
STAGES = ("spread", "interp", "fft", "grid")


def _load(prec):
    with open(os.path.join(GOLDEN, FIXTURES[prec])) as f:
        rep = json.load(f)
    rows = [(r["info"], r["stage_ms"]) for r in rep["rows"]]
    return rep, rows


@pytest.fixture(scope="module")
def lib():
    hvox.build()
    return hvox.load()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fit_reproduces_the_report(lib, prec):
    rep, rows = _load(prec)
    fitted = calibrate.fit(rows)
    for stage, v in rep["fitted_seconds_per_unit"].items():
        if v is None:
            assert fitted[stage] is None
        else:
            assert abs(fitted[stage] - v) <= 1e-12 * abs(v) + 1e-30, stage


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_planner_constants_are_the_fit(lib, prec):
    _, rows = _load(prec)
    fitted = calibrate.fit(rows)
    model = calibrate.model_rates("f32" if prec == "fp32" else "f64")
    for stage in STAGES:
        assert abs(model[stage] / fitted[stage] - 1.0) < 0.05, (stage, model[stage], fitted[stage])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_model_predicts_measured_steps(lib, prec):
    _, rows = _load(prec)
    model = calibrate.model_rates("f32" if prec == "fp32" else "f64")
    for info, ms in rows:
        measured = sum(ms[s] for s in STAGES + ("direct",))
        predicted = 1e3 * sum(model[s] * calibrate.STAGE_WORK[s](info) for s in STAGES + ("direct",))
        assert abs(predicted / measured - 1.0) < 0.20, (info, predicted, measured)
