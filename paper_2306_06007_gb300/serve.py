"""Continuous-batching request server for HVOX transforms on one GPU.

Requests (sky -> vis or vis -> sky, any geometry and tolerance) arrive over time. The
server keeps plans resident on the device (one per geometry and tolerance, each bound
to its own CUDA stream), plans new geometries on worker threads while the GPU works,
admits a request as soon as a slot is free, its plan is idle and the HBM budget has
room for the plan and the request's buffers, and overlaps the admitted requests on the
device through their streams. Requests of one direction admitted in the same pass go
through one batched call (hvox_synthesize_batch / hvox_analyze_batch), so that their
direct sums share kernel launches and one dynamic schedule, not only the device. Completion is detected by polling a CUDA event recorded
after each request's device-to-host copy; latency = completion - arrival.

`plain=True` gives the comparison form: one request at a time in arrival order, plans
in the plain FP64 form (hvox_opts.plain).

This module is scheduling and bookkeeping only; every transform step runs in libhvox.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import statistics
import time
from dataclasses import dataclass, field

import numpy as np

from . import HvoxError, Plan, estimate_bytes


def geometry_key(pix: np.ndarray, uvw: np.ndarray, eps: float, plain: bool) -> str:
    h = hashlib.blake2b(digest_size=16)
    h.update(np.ascontiguousarray(pix, dtype=np.float64).tobytes())
    h.update(np.ascontiguousarray(uvw, dtype=np.float64).tobytes())
    h.update(repr((float(eps), bool(plain))).encode())
    return h.hexdigest()


@dataclass
class _Resident:
    plan: Plan
    stream: object
    bytes: float
    busy: bool = False
    last_used: float = 0.0


@dataclass
class _Inflight:
    req: object
    key: str
    event: object
    out: object
    io_bytes: float
    start: float          # admission time (seconds after the start of the run)


@dataclass
class ServeReport:
    results: dict = field(default_factory=dict)      # rid -> numpy output
    latency_s: dict = field(default_factory=dict)    # rid -> completion - arrival
    plan_s: dict = field(default_factory=dict)       # key -> planning seconds
    makespan_s: float = 0.0
    units: float = 0.0                               # sum of (n_pix + n_vis) over requests
    peak_bytes: float = 0.0
    errors: dict = field(default_factory=dict)       # rid -> message of a request that failed
    # rid -> (seconds waiting for its plan, waiting for a slot after that, on the device)
    phases: dict = field(default_factory=dict)
    # sizes of the batched calls (requests admitted together whose direct sums shared launches)
    batches: list = field(default_factory=list)

    def summary(self) -> dict:
        lat = sorted(self.latency_s.values())
        q = (lambda f: lat[min(len(lat) - 1, int(round(f * (len(lat) - 1))))] * 1e3) if lat else (lambda f: None)
        out = {"requests": len(lat), "p50_ms": q(0.50), "p99_ms": q(0.99), "max_ms": q(1.0),
               "mean_ms": statistics.mean(lat) * 1e3 if lat else None,
               "throughput_units_per_s": self.units / self.makespan_s if self.makespan_s > 0 else None,
               "makespan_s": self.makespan_s, "plans": len(self.plan_s),
               "plan_s_total": sum(self.plan_s.values()), "peak_bytes": self.peak_bytes,
               "errors": len(self.errors), "batch_calls": len(self.batches),
               "batched_requests": sum(self.batches)}
        if lat and self.phases:
            # Where the time of the slowest 1 % of requests went (mean over them, ms).
            by_lat = sorted(self.latency_s, key=self.latency_s.get)
            tail = by_lat[int(0.99 * (len(by_lat) - 1)):]
            ph = [self.phases[r] for r in tail if r in self.phases]
            if ph:
                out["tail_ms"] = {"plan_wait": 1e3 * statistics.mean(p[0] for p in ph),
                                  "slot_wait": 1e3 * statistics.mean(p[1] for p in ph),
                                  "device": 1e3 * statistics.mean(p[2] for p in ph), "requests": len(ph)}
        return out


class Server:
    """Request loop over libhvox plans (see the module docstring)."""

    def __init__(self, hbm_budget_bytes: float = 150e9, max_inflight: int = 8, planner_threads: int = 0,
                 plain: bool = False, keep_plans: bool = True, search_threshold: float | None = None):
        import os
        if planner_threads <= 0:
            planner_threads = max(2, (os.cpu_count() or 4) // 2)
        self.budget = float(hbm_budget_bytes)
        self.max_inflight = 1 if plain else int(max_inflight)
        self.plain = plain
        self.keep_plans = keep_plans
        # A request's plan is usually used once: skip the partition search for jobs whose
        # direct evaluation is modelled below this many seconds, or below the search's own
        # cost (~2 us a point, see _threshold).
        # The plain form's direct sums are ~100x slower, but a one-shot plan with NUFFT
        # sub-problems also pays for the search, its grids and cuFFT plans: on the
        # benchmark's stream (N up to 3e4) planning plain requests with a 0.1 s threshold
        # gave p50 / p99 286 / 1,524 ms against 78 / 200 ms with direct sums, so the plain
        # form searches only above 1 s of direct work.
        if search_threshold is None:
            search_threshold = 1.0 if plain else 0.1
        self.search_threshold = float(search_threshold)
        self.pool = cf.ThreadPoolExecutor(max_workers=max(1, planner_threads))
        self.resident: dict[str, _Resident] = {}
        self.used = 0.0

    # ------------------------------------------------------------------ plans
    # Seconds of partition search per point (both point sets; measured on a 16-core host):
    # a one-shot plan searches only when its direct work could repay that.
    SEARCH_SECONDS_PER_POINT = 2e-6

    def _threshold(self, req) -> float:
        return max(self.search_threshold, self.SEARCH_SECONDS_PER_POINT * (len(req.pix) + len(req.uvw)))

    def _make_plan(self, req):
        import torch
        t0 = time.perf_counter()
        stream = torch.cuda.Stream()
        plan = Plan(req.pix, req.uvw, req.eps, plain=self.plain, stream=stream,
                    search_threshold=self._threshold(req))
        info = plan.info()
        return plan, stream, info["workspace_bytes"], time.perf_counter() - t0

    def _estimate_plan_bytes(self, req) -> float:
        # Upper bound of what planning may allocate (the plan's own figure replaces it).
        return estimate_bytes(len(req.pix), len(req.uvw), req.eps, plain=self.plain,
                              search_threshold=self._threshold(req))

    def _evict_idle(self, need: float, protect: set):
        for key, r in sorted(self.resident.items(), key=lambda kv: kv[1].last_used):
            if self.used + need <= self.budget:
                return
            if r.busy or key in protect:
                continue
            r.plan.close()
            self.used -= r.bytes
            del self.resident[key]

    # ------------------------------------------------------------------ loop
    def run(self, requests, realtime: bool = True, time_scale: float = 1.0) -> ServeReport:
        """Serve `requests` (objects with rid, arrival, pix, uvw, eps, direction, data).
        realtime: arrivals happen at their timestamps (times time_scale); otherwise all
        requests are present at t = 0."""
        import torch
        rep = ServeReport()
        pending = sorted(requests, key=lambda r: r.arrival)
        arrived: list = []
        planning: dict[str, cf.Future] = {}
        reserved: dict[str, float] = {}
        inflight: list[_Inflight] = []
        ready: dict[str, float] = {}   # key -> time its plan became resident
        t0 = time.perf_counter()
        first_arrival = None
        rep.units = float(sum(len(r.pix) + len(r.uvw) for r in requests))
        nxt = 0
        while nxt < len(pending) or arrived or inflight or planning:
            now = time.perf_counter() - t0
            progressed = False
            # arrivals
            while nxt < len(pending) and (not realtime or pending[nxt].arrival * time_scale <= now):
                r = pending[nxt]
                r._key = geometry_key(r.pix, r.uvw, r.eps, self.plain)
                arrived.append(r)
                nxt += 1
                progressed = True
                if first_arrival is None:
                    first_arrival = (r.arrival * time_scale) if realtime else 0.0
            # planning (admitted against the budget with an estimate)
            for r in arrived:
                k = r._key
                if k in self.resident or k in planning:
                    continue
                if self.plain and (inflight or planning):
                    break
                est = self._estimate_plan_bytes(r)
                if self.used + est > self.budget:
                    self._evict_idle(est, {x._key for x in arrived})
                if self.used + est > self.budget and (inflight or planning or self.resident):
                    continue
                self.used += est
                reserved[k] = est
                planning[k] = self.pool.submit(self._make_plan, r)
                progressed = True
            for k in [k for k, f in planning.items() if f.done()]:
                try:
                    plan, stream, nbytes, secs = planning.pop(k).result()
                except HvoxError as e:
                    # The requests of this geometry fail; the server carries on.
                    self.used -= reserved.pop(k)
                    for r in [x for x in arrived if x._key == k]:
                        rep.errors[r.rid] = str(e)
                        arrived.remove(r)
                    progressed = True
                    continue
                self.used += nbytes - reserved.pop(k)
                self.resident[k] = _Resident(plan, stream, nbytes)
                rep.plan_s[k] = secs
                ready[k] = time.perf_counter() - t0
                progressed = True
            # admission
            admitted = []
            i = 0
            while i < len(arrived) and len(inflight) + len(admitted) < self.max_inflight:
                r = arrived[i]
                res = self.resident.get(r._key)
                if res is None or res.busy:
                    i += 1
                    if self.plain:
                        break
                    continue
                io = 16.0 * (len(r.pix) + len(r.uvw)) * 2
                if self.used + io > self.budget and (inflight or admitted):
                    break
                arrived.pop(i)
                res.busy = True
                self.used += io
                rep.peak_bytes = max(rep.peak_bytes, self.used)
                admitted.append((r, res, io))
            # launch: requests of one direction admitted together go through one batched
            # call (their direct sums share launches); a lone request uses its plan alone
            groups = {}
            for a in admitted:
                groups.setdefault(a[0].direction, []).append(a)
            for direction, grp in groups.items():
                t_start = time.perf_counter() - t0
                if len(grp) >= 2 and not self.plain:
                    for ent in self._launch_batch(direction, grp):
                        inflight.append(_Inflight(ent[0], ent[0]._key, ent[3], ent[4], ent[2], t_start))
                    rep.batches.append(len(grp))
                else:
                    for r, res, io in grp:
                        ev, out = self._launch_one(r, res)
                        inflight.append(_Inflight(r, r._key, ev, out, io, t_start))
                progressed = True
            # completions
            for f in [f for f in inflight if f.event.query()]:
                inflight.remove(f)
                done = time.perf_counter() - t0
                r = f.req
                arrival = (r.arrival * time_scale) if realtime else 0.0
                rep.latency_s[r.rid] = done - arrival
                plan_ready = max(arrival, ready.get(f.key, arrival))
                rep.phases[r.rid] = (plan_ready - arrival, f.start - plan_ready, done - f.start)
                rep.results[r.rid] = f.out.numpy().copy()
                res = self.resident[f.key]
                res.busy = False
                res.last_used = done
                self.used -= f.io_bytes
                if not self.keep_plans and not any(x._key == f.key for x in arrived):
                    res.plan.close()
                    self.used -= res.bytes
                    del self.resident[f.key]
                progressed = True
            if not progressed:
                time.sleep(0.0002)
        rep.makespan_s = (time.perf_counter() - t0) - (first_arrival or 0.0)
        return rep

    @staticmethod
    def _input(r, res):
        import torch
        dt = res.plan.real_dtype if r.direction == "s2v" else res.plan.complex_dtype
        return torch.as_tensor(r.data, dtype=dt).pin_memory().to("cuda", non_blocking=True)

    def _launch_one(self, r, res):
        import torch
        with torch.cuda.stream(res.stream):
            x = self._input(r, res)
            y = res.plan.synthesize(x) if r.direction == "s2v" else res.plan.analyze(x)
            out = torch.empty(y.shape, dtype=y.dtype, pin_memory=True)
            out.copy_(y, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(res.stream)
        return ev, out

    def _launch_batch(self, direction, grp):
        """One batched call over the plans of grp (on the first plan's stream): one event
        marks the whole group's completion."""
        import torch
        from . import analyze_batch, synthesize_batch
        s = grp[0][1].stream
        with torch.cuda.stream(s):
            xs = [self._input(r, res) for r, res, _ in grp]
            plans = [res.plan for _, res, _ in grp]
            ys = synthesize_batch(plans, xs) if direction == "s2v" else analyze_batch(plans, xs)
            outs = []
            for y in ys:
                o = torch.empty(y.shape, dtype=y.dtype, pin_memory=True)
                o.copy_(y, non_blocking=True)
                outs.append(o)
            ev = torch.cuda.Event()
            ev.record(s)
        return [(r, res, io, ev, o) for (r, res, io), o in zip(grp, outs)]

    def close(self):
        for r in self.resident.values():
            r.plan.close()
        self.resident.clear()
        self.used = 0.0
        self.pool.shutdown(wait=True)
