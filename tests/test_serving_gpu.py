"""Serving (continuous batching): each request's result is the same whether it runs alone
or in a mix of concurrent requests of different sizes and tolerances, and agrees with
the oracle within 10 eps. Admission keeps the device memory in use under the budget."""
import numpy as np
import pytest

import oracle
from hvox_inputs import configs

pytestmark = pytest.mark.gpu


def _stream(n=14, seed=0):
    reqs = configs.config5_requests(n, rate_hz=200.0, n_min=500, n_max=20000, seed_offset=seed)
    # repeat a few geometries so that several requests share a resident plan
    rng = np.random.default_rng(77 + seed)
    for i in (5, 9, 12):
        if i < n:
            src = reqs[i - 4]
            reqs[i].pix, reqs[i].uvw, reqs[i].eps, reqs[i].direction = src.pix, src.uvw, src.eps, src.direction
            n_in = len(src.pix) if src.direction == "s2v" else len(src.uvw)
            if src.direction == "s2v":
                reqs[i].data = rng.lognormal(0.0, 1.0, n_in)
            else:
                reqs[i].data = rng.normal(size=n_in) + 1j * rng.normal(size=n_in)
    return reqs


def _tol(eps, r_alone):
    return 1e-11 if eps < 1e-6 else 1e-5


def test_alone_equals_mix_and_oracle(gpu_lib):
    from paper_2306_06007_gb300.serve import Server
    reqs = _stream()
    alone = Server(max_inflight=1)
    rep_a = alone.run(reqs, realtime=False)
    alone.close()
    mix = Server(max_inflight=8)
    rep_m = mix.run(reqs, realtime=True)
    mix.close()
    assert set(rep_a.results) == set(rep_m.results) == {r.rid for r in reqs}
    for r in reqs:
        a, m = rep_a.results[r.rid], rep_m.results[r.rid]
        assert oracle.rel_l2(m, a) <= _tol(r.eps, a), (r.rid, r.eps)
        if r.direction == "s2v":
            ref = oracle.sky2vis(r.pix, r.uvw, r.data)
        else:
            ref = oracle.vis2sky(r.pix, r.uvw, r.data)
        assert oracle.rel_l2(m, ref) <= 10 * r.eps, (r.rid, r.eps, r.direction)
    s = rep_m.summary()
    assert s["requests"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0


def test_admission_respects_budget(gpu_lib):
    from paper_2306_06007_gb300.serve import Server
    reqs = _stream(8, seed=1)
    budget = 600e6
    srv = Server(hbm_budget_bytes=budget, max_inflight=8, keep_plans=False)
    rep = srv.run(reqs, realtime=False)
    srv.close()
    assert len(rep.results) == len(reqs)
    assert rep.peak_bytes <= budget


def test_failed_request_does_not_stop_the_server(gpu_lib):
    # A request whose geometry the library rejects (a non-finite coordinate) fails alone;
    # every other request of the stream completes and matches the oracle.
    from paper_2306_06007_gb300.serve import Server
    reqs = _stream(6, seed=2)
    bad = reqs[2]
    bad.pix = bad.pix.copy()
    bad.pix[0, 0] = np.nan
    srv = Server(max_inflight=4)
    rep = srv.run(reqs, realtime=False)
    srv.close()
    assert set(rep.errors) == {bad.rid}
    assert set(rep.results) == {r.rid for r in reqs} - {bad.rid}
    for r in reqs:
        if r.rid == bad.rid:
            continue
        ref = oracle.sky2vis(r.pix, r.uvw, r.data) if r.direction == "s2v" else oracle.vis2sky(r.pix, r.uvw, r.data)
        assert oracle.rel_l2(rep.results[r.rid], ref) <= 10 * r.eps


def test_batched_admission_matches_alone(gpu_lib):
    # With every plan resident (a second pass over the same stream), the requests admitted
    # together go through batched calls whose direct sums share launches; each result
    # still equals the request run alone and the oracle.
    from paper_2306_06007_gb300.serve import Server
    reqs = _stream(10, seed=3)
    alone = Server(max_inflight=1)
    rep_a = alone.run(reqs, realtime=False)
    alone.close()
    srv = Server(max_inflight=8)
    srv.run(reqs, realtime=False)
    rep = srv.run(reqs, realtime=False)
    srv.close()
    assert rep.batches and max(rep.batches) >= 2, rep.batches
    assert set(rep.results) == {r.rid for r in reqs}
    for r in reqs:
        a, m = rep_a.results[r.rid], rep.results[r.rid]
        assert oracle.rel_l2(m, a) <= _tol(r.eps, a), (r.rid, r.eps)
        ref = oracle.sky2vis(r.pix, r.uvw, r.data) if r.direction == "s2v" else oracle.vis2sky(r.pix, r.uvw, r.data)
        assert oracle.rel_l2(m, ref) <= 10 * r.eps, (r.rid, r.eps, r.direction)
    s = rep.summary()
    assert s["batch_calls"] == len(rep.batches) and s["batched_requests"] == sum(rep.batches)
