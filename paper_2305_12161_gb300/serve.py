"""Continuous-batching quench server over the C ABI.

Requests (L, t_max, replicas, seed) arrive over time.  A request is admitted as soon as
a slot and enough of the HBM budget are free; it then gets its own context (lattices
kept in HBM until it finishes) on its own CUDA stream, so the work of all admitted
requests overlaps on the device.  The scheduler issues each request's sweeps in
bounded quanta (never more than `max_inflight` quanta queued per request, so a long
request cannot monopolise the launch queue), measures at the request's log-spaced times
into device buffers, and on completion returns the l(t) series (e, m, l_E, l_C per
measured time and replica) and the integer records.  Time to result is completion time
minus arrival time.

This module only schedules: every sweep and measurement runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import inputs, ising


@dataclasses.dataclass
class Request:
    id: int
    L: int
    t_max: int
    replicas: int
    seed: int
    arrival_s: float = 0.0
    K: int = 12


@dataclasses.dataclass
class Result:
    request: Request
    times: list
    records: np.ndarray   # [K, replicas, record_len] int64 (t, M, B, D_a(r))
    derived: np.ndarray   # [K, replicas, 4] float64 (e, m, l_E, l_C)
    admitted_s: float
    finished_s: float

    @property
    def time_to_result_s(self) -> float:
        return self.finished_s - self.request.arrival_s


def footprint_bytes(L: int, replicas: int, K: int, **opts) -> int:
    """Device memory a request holds while it runs: its context as the library accounts it
    (ising_footprint_bytes: packed lattices, twice for the fused whole-sweep kernel, records
    and, for L >= 512, the tensor-core correlation scratch of 2 L^3 bytes) plus the server's
    own result buffers for K measured times (records and derived values of every replica).
    `opts`: the context options the request runs with (sweep kernel and tiling)."""
    ctx = ising.ising_footprint_bytes(L, replicas, **opts)
    if ctx < 0:
        raise ValueError(f"no context for L={L}, replicas={replicas}")
    return ctx + K * replicas * (ising.ising_record_len(L) * 8 + 4 * 8)


def admit(pending: list, n_active: int, used: float, budget: float, max_slots: int, footprint) -> tuple:
    """Admission by HBM footprint: walk the pending requests in arrival order and admit
    each one for which a slot is free and whose footprint fits in what is left of the
    budget (a smaller request may pass a larger one that does not fit yet).  Returns
    (admitted, still pending, bytes in use afterwards)."""
    admitted, keep = [], []
    for req in pending:
        fp = footprint(req)
        if n_active + len(admitted) < max_slots and used + fp <= budget:
            admitted.append(req)
            used += fp
        else:
            keep.append(req)
    return admitted, keep, used


def schedule_for(req: Request) -> list[int]:
    K = max(1, min(req.K, req.t_max))
    return inputs.log_schedule(req.t_max, K)


class _Active:
    def __init__(self, req: Request, now: float, torch, opts=None):
        self.req = req
        self.times = schedule_for(req)
        self.stream = torch.cuda.Stream()
        self.opts = dict(opts or {})
        self.ctx = ising.Ising(req.L, replicas=req.replicas, seed=req.seed, stream=self.stream, **self.opts)
        K = len(self.times)
        self.rec = torch.empty((K, req.replicas, self.ctx.record_len), dtype=torch.int64, device="cuda")
        self.der = torch.empty((K, req.replicas, 4), dtype=torch.float64, device="cuda")
        self.next_k = 0          # next measurement slot to reach
        self.inflight = []       # events of queued quanta
        self.admitted_s = now
        self.updates = 0

    def done_issuing(self) -> bool:
        return self.next_k >= len(self.times)


class QuenchServer:
    """`tune`: pick the sweep kernel and tiling of each request shape (lattice size and
    replica count) with the library's autotuner the first time a request of that shape is
    submitted (every choice gives the same results; the best kernel depends on the replica
    count as well as the size, since replicas share a launch; the fused whole-sweep kernel,
    which the tuner picks for the larger sizes, holds a second packed store, which the
    admission footprint counts)."""

    def __init__(self, budget_bytes: float = 150e9, max_slots: int = 16, quantum_mcs: int = 64,
                 max_inflight: int = 2, c: float = 0.5, tune: bool = True, pdl: int = 1):
        import torch
        self.torch = torch
        self.tune = tune
        self.pdl = pdl  # programmatic dependent launch of the sweep kernels (ising_opts.pdl)
        self.opts: dict[tuple, dict] = {}  # (L, replicas) -> context options
        self.budget = float(budget_bytes)
        self.max_slots = max_slots
        self.quantum = quantum_mcs
        self.max_inflight = max_inflight
        self.c = c
        self.pending: list[Request] = []
        self.active: list[_Active] = []
        self.results: list[Result] = []
        self.used = 0.0
        self.t0 = None
        self.updates = 0

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def options_for(self, L: int, replicas: int = 1) -> dict:
        """Context options of requests of size L with `replicas` lattices (autotuned once per
        shape when `tune`)."""
        key = (L, replicas)
        if key not in self.opts:
            o = {}
            if self.tune:
                t = ising.ising_tune_sweep(L, replicas, probe_mcs=4)
                o = {k: t[k] for k in ("variant", "tile_y", "tile_z", "depth")}
            o["pdl"] = self.pdl
            self.opts[key] = o
        return self.opts[key]

    def footprint(self, req: Request) -> int:
        return footprint_bytes(req.L, req.replicas, req.K, **self.options_for(req.L, req.replicas))

    def submit(self, req: Request) -> None:
        if self.footprint(req) > self.budget:
            raise ValueError(f"request {req.id} needs more than the whole HBM budget")
        self.pending.append(req)

    def _admit(self) -> None:
        admitted, self.pending, self.used = admit(self.pending, len(self.active), self.used, self.budget,
                                                  self.max_slots, self.footprint)
        for req in admitted:
            self.active.append(_Active(req, self.now(), self.torch, self.options_for(req.L, req.replicas)))

    def _issue(self, a: _Active) -> None:
        # one quantum: sweep towards the next measured time, measure when it is reached
        a.inflight = [e for e in a.inflight if not e.query()]
        while len(a.inflight) < self.max_inflight and not a.done_issuing():
            target = a.times[a.next_k]
            n = min(self.quantum, target - a.ctx.t)
            if n > 0:
                a.ctx.sweep(n)
                a.updates += n * a.req.replicas * a.req.L ** 3
            if a.ctx.t == target:
                a.ctx.measure_device(a.rec[a.next_k], a.der[a.next_k], c=self.c)
                a.next_k += 1
            ev = self.torch.cuda.Event()
            ev.record(a.stream)
            a.inflight.append(ev)

    def _retire(self) -> None:
        still = []
        for a in self.active:
            if a.done_issuing() and all(e.query() for e in a.inflight):
                rec = a.rec.cpu().numpy()
                der = a.der.cpu().numpy()
                self.results.append(Result(a.req, a.times, rec, der, a.admitted_s, self.now()))
                self.updates += a.updates
                self.used -= self.footprint(a.req)
                a.ctx.destroy()
            else:
                still.append(a)
        self.active = still

    def run(self, trace: list[Request], idle_sleep_s: float = 0.0005) -> list[Result]:
        """Serve `trace` (arrival_s relative to the start) until every request is done.  The
        request shapes in the trace are tuned before the clock starts."""
        for r in trace:
            self.options_for(r.L, r.replicas)
        self.t0 = time.perf_counter()
        queue = sorted(trace, key=lambda r: r.arrival_s)
        i = 0
        while i < len(queue) or self.pending or self.active:
            now = self.now()
            while i < len(queue) and queue[i].arrival_s <= now:
                self.submit(queue[i])
                i += 1
            self._admit()
            for a in self.active:
                self._issue(a)
            self._retire()
            if not self.active and not self.pending and i < len(queue):
                time.sleep(max(0.0, min(idle_sleep_s, queue[i].arrival_s - self.now())))
        return self.results

    def summary(self) -> dict:
        ttr = np.array([r.time_to_result_s for r in self.results])
        span = max(r.finished_s for r in self.results) if self.results else 0.0
        return {"requests": len(self.results), "p50_s": float(np.percentile(ttr, 50)) if len(ttr) else None,
                "p99_s": float(np.percentile(ttr, 99)) if len(ttr) else None, "makespan_s": span,
                "updates": self.updates, "updates_per_ns": self.updates / span / 1e9 if span > 0 else None}


def trace_requests(n: int, seed: int = 0, rate_hz: float = 20.0, K: int = 12, **kw) -> list[Request]:
    """The seeded Poisson request stream of inputs.serving_trace as Request objects."""
    return [Request(id=d["id"], L=d["L"], t_max=d["t_max"], replicas=d["replicas"], seed=d["seed"],
                    arrival_s=d["arrival_s"], K=K)
            for d in inputs.serving_trace(n, seed=seed, rate_hz=rate_hz, **kw)]


def run_alone(req: Request, c: float = 0.5, opts=None) -> Result:
    """The same request served by itself (reference for the mix), with the default sweep
    kernel unless `opts` names one."""
    import torch
    t0 = time.perf_counter()
    a = _Active(req, 0.0, torch, opts)
    for k, tk in enumerate(a.times):
        a.ctx.sweep(tk - a.ctx.t)
        a.ctx.measure_device(a.rec[k], a.der[k], c=c)
    a.ctx.sync()
    res = Result(req, a.times, a.rec.cpu().numpy(), a.der.cpu().numpy(), 0.0, time.perf_counter() - t0)
    a.ctx.destroy()
    return res
