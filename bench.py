#!/usr/bin/env python
"""Throughput benchmark of the zero-temperature checkerboard quench on GB300.

Workload (one step = one pass of the whole hot path over a 2048^3 lattice):
  leg (i):  T = infinity Philox start (seed 1), 1000 MCS of the checkerboard T -> 0
            Glauber dynamics, observables (M, B, D_a(r) for r = 0..1024, and e, m, l_E,
            l_C) at K log-spaced times;
  leg (ii): the configuration evolved to t = 10^4 MCS (sparse interfaces; prepared once,
            untimed, kept in HBM), 1000 further MCS, observables at K log-spaced times.
Metric: spin updates per ns over the whole step (2 x 1000 x 2048^3 updates).

`value` runs with every input already in HBM (checkpoint copied device-to-device,
records written to device buffers).  `e2e` runs the same step through the C ABI with
host buffers: the checkpoint is copied from pinned host memory and every record is
read back to the host, inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own independent lattice (replicas only; no exchange).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin updates/ns & % HBM roofline at L=2048; batched vs plain form on one GB300"
UNIT = "spin updates/ns"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", 1700.0))}
    except Exception:
        return {"hbm_gbs": 6800.0, "src": "fallback", "sm_max_mhz": 2070.0, "bf16_tflops_sustained": 1700.0}


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(sample_L: int = 1024, mcs: int = 2, single_L: int = 256, single_mcs: int = 2) -> dict:
    """The oracle as it stands, on this host's cores, on a bounded sample; and on one core,
    on a smaller sample."""
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    s = oracle.init(sample_L, 1)
    t0 = time.perf_counter()
    oracle.sweeps(s, 0, mcs, 1, oracle.TIE_GLAUBER)
    dt = time.perf_counter() - t0
    del s
    oracle.set_threads(1)
    s1 = oracle.init(single_L, 1)
    t1 = time.perf_counter()
    oracle.sweeps(s1, 0, single_mcs, 1, oracle.TIE_GLAUBER)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    return {"value": mcs * sample_L**3 / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{mcs} MCS of one {sample_L}^3 lattice from the T=inf start (sweeps only, "
                      f"no correlation pass), {dt:.1f} s",
            "single_thread": {"value": single_mcs * single_L**3 / dt1 / 1e9, "unit": UNIT, "cores": 1,
                              "sample": f"{single_mcs} MCS of one {single_L}^3 lattice from the T=inf start, "
                                        f"{dt1:.1f} s"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    L, mcs = args.ref_L, 1
    s = oracle.init(L, 1)
    for _ in range(args.warmup):
        oracle.sweeps(s, 0, mcs, 1, oracle.TIE_GLAUBER)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.sweeps(s, k * mcs, mcs, 1, oracle.TIE_GLAUBER)
    dt = time.perf_counter() - t0
    v = args.steps * mcs * L**3 / dt / 1e9
    sample = f"each step: {mcs} MCS of one {L}^3 lattice (oracle sweeps only)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": "L=2048 quench legs (oracle sample)", "L": L, "parallelism": "host threads"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_quench_case(args):
    """A short plain run of the hot path for ncu: T = infinity start, --mcs sweeps, one
    full measurement, every kernel launched on the context's stream."""
    import __graft_entry__
    from paper_2305_12161_gb300 import ising
    __graft_entry__.build()
    kw = {}
    if args.sweep_config:
        v, ty, tz, dp = (int(x) for x in args.sweep_config.split(","))
        kw = dict(variant=v, tile_y=ty, tile_z=tz, depth=dp)
    form = ising.FORM_PLAIN if args.form == "plain" else ising.FORM_PACKED
    with ising.Ising(args.L, replicas=1, seed=1, corr=args.corr, form=form, **kw) as q:
        q.sweep(args.mcs)
        rec, der = q.measure_ex(c=0.5)
        print(json.dumps({"case": "quench", "L": args.L, "mcs": args.mcs, "B": int(rec[0, 2]),
                          "l_E": float(der[0, 2]), "l_C": float(der[0, 3]), "launches": q.launch_count()}))


BATCH_CLASSES = [(64, 512, 1), (128, 64, 513), (256, 16, 577), (512, 4, 593)]  # seeds 1..596

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch from one ncu capture of
# the kernel as built (the file under profiles/ gives the command), by (kernel, L, tile_z,
# depth); kernels changed since their capture and configurations never captured report null
TRAFFIC_NCU = {("k_mcs_fused", 2048, 64, 26): (2.162e9, "ncu, profiles/k_mcs_fused_L2048.md (balanced tiling, "
                                                        "z-blocks fitted near 64 planes, five slots)")}


def run_batched(torch, ising, inputs, K: int = 20, window: int = 20) -> dict:
    """Mixed batch 512x64^3 + 64x128^3 + 16x256^3 + 4x512^3 (each lattice its own seed):
    the batched form runs 10^4 MCS with K log-spaced measurements as one CUDA graph
    (per segment a persistent launch for the 64^3 and 128^3 classes and the 256^3 and 512^3
    classes streamed beside it on side streams; work list, streamed kernels and stream order
    tuned by the autotuner); the plain form (one byte per spin, one launch per lattice) and
    the packed form launched per class (on the kernels the batch chose) are compared with it
    on the same window of `window` MCS from the T = inf start."""
    stream = torch.cuda.Stream()
    times = inputs.log_schedule(10_000, K)
    spins = sum(R * L**3 for L, R, _ in BATCH_CLASSES)

    def timed(fn):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    out = {"workload": "512x64^3 + 64x128^3 + 16x256^3 + 4x512^3, seeds 1..596, 10^4 MCS, "
                       f"{K} log-spaced measurements (M, B, D_a(r), e, m, l_E, l_C) in one CUDA graph",
           "spins": spins}
    with ising.Batch(BATCH_CLASSES, stream=stream) as bt:
        w = bt.tune(probe_mcs=4)
        out["autotuner_w_local"] = w
        out["plan"] = bt.plan()
        kernels = [bt.class_config(ci) for ci in range(len(BATCH_CLASSES))]
        out["streamed_beside_persistent"] = bt.overlap
        out["class_kernels"] = {f"{L}^3": ("persistent" if k["variant"] < 0 else
                                           f"variant {k['variant']}, tile_z {k['tile_z']}, depth {k['depth']}")
                                for (L, _, _), k in zip(BATCH_CLASSES, kernels)}
        rec = torch.empty((K, bt.record_words), dtype=torch.int64, device="cuda")
        der = torch.empty((K, bt.lattices, 4), dtype=torch.float64, device="cuda")
        bt.reinit()
        l0 = bt.launch_count()
        bt.run(times, rec=rec, derived=der, device=True)  # capture + warm
        bt.sync()
        out["graph_kernel_launches"] = bt.launch_count() - l0  # kernels captured into the schedule graph
        bt.reinit()
        ms = timed(lambda: bt.run(times, rec=rec, derived=der, device=True))
        bt.sync()
        out["batched_updates_per_ns"] = 10_000 * spins / (ms * 1e-3) / 1e9
        out["batched_ms"] = ms
        bt.reinit()
        bt.sweep(2)
        bt.reinit()
        ms_w = timed(lambda: bt.sweep(window))
        bt.sync()
        out["window_mcs"] = window
        out["batched_window_updates_per_ns"] = window * spins / (ms_w * 1e-3) / 1e9
    # the packed form per class runs every class on the kernel the batch gave it (the tuned
    # single-lattice kernel of a streamed class; the default kernel of the others)
    packed_kw = [dict(variant=k["variant"], tile_y=k["tile_y"], tile_z=k["tile_z"], depth=k["depth"])
                 if k["variant"] > 0 else {} for k in kernels]
    for form, key in ((ising.FORM_PLAIN, "plain_window_updates_per_ns"),
                      (ising.FORM_PACKED, "packed_per_class_window_updates_per_ns")):
        ctxs = [ising.Ising(L, replicas=R, seed=sd, form=form, stream=stream,
                            **(packed_kw[i] if form == ising.FORM_PACKED else {}))
                for i, (L, R, sd) in enumerate(BATCH_CLASSES)]
        for c in ctxs:
            c.sweep(1)
        ms_p = timed(lambda: [c.sweep(window) for c in ctxs])
        out[key] = window * spins / (ms_p * 1e-3) / 1e9
        for c in ctxs:
            c.destroy()
    out["batched_vs_plain"] = out["batched_window_updates_per_ns"] / out["plain_window_updates_per_ns"]
    out["batched_vs_packed_per_class"] = (out["batched_window_updates_per_ns"]
                                          / out["packed_per_class_window_updates_per_ns"])
    return out


def run_plain(torch, ising, pk, sizes=(1024, 2048), mcs: int = 10, warm: int = 2) -> dict:
    """The plain form at one lattice: one byte per spin, one kernel launch per half-sweep
    (k_sweep_plain), T = infinity start, `warm` untimed MCS then `mcs` timed MCS (CUDA
    events on the context's stream).  Algorithmic bytes: a half-sweep reads the whole
    L^3-byte lattice (the sites of both sublattices share every 32-byte sector) and writes
    back every sector that holds a site of the updated sublattice (L^3 bytes): 2 L^3 bytes
    per L^3/2 updates = 4 B/update.  Both lattices are larger than L2."""
    out = {}
    for L in sizes:
        stream = torch.cuda.Stream()
        with ising.Ising(L, replicas=1, seed=1, form=ising.FORM_PLAIN, stream=stream) as q:
            q.sweep(warm)
            q.sync()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            q.sweep(mcs)
            b.record(stream)
            q.sync()
            ms = a.elapsed_time(b)
        N = L**3
        half_s = ms * 1e-3 / (2 * mcs)
        gbs = 2 * N / half_s / 1e9
        out[str(L)] = {"updates_per_ns": N * mcs / (ms * 1e-3) / 1e9, "ms_per_mcs": ms / mcs,
                       "avg_launch_ms": half_s * 1e3, "bytes_per_launch": 2 * N, "achieved_gbs": gbs,
                       "peak_gbs": pk["hbm_gbs"], "frac": gbs / pk["hbm_gbs"], "mcs_timed": mcs,
                       "t_window": [warm, warm + mcs]}
        torch.cuda.empty_cache()
    return out


def run_serving(serve, requests: int = 16) -> dict:
    """Continuous-batching serving on the first `requests` arrivals of the seeded trace
    (Poisson 20/s, L log-uniform on {64..1024}, t_max = 10^U[3,5], 1-16 replicas, 12
    measured times each), 150 GB budget by library footprint, 16 slots."""
    trace = serve.trace_requests(requests, seed=0, K=12)
    offered = sum(r.L**3 * r.replicas * r.t_max for r in trace)
    srv = serve.QuenchServer(budget_bytes=150e9, max_slots=16, quantum_mcs=64)
    srv.run(trace)
    summ = srv.summary()
    arrivals = trace[-1].arrival_s
    return {"requests": summ["requests"], "p50_s": summ["p50_s"], "p99_s": summ["p99_s"],
            "makespan_s": summ["makespan_s"], "aggregate_updates_per_ns": summ["updates_per_ns"],
            "updates": summ["updates"],
            "offered_updates_per_s": offered / arrivals if arrivals > 0 else None,
            "trace": f"first {requests} arrivals: seeded Poisson 20/s, L log-uniform {{64,...,1024}}, "
                     "t_max=10^U[3,5], replicas U{1..16}, K=12; overloaded (offered >> capacity)",
            "slots": 16, "budget_gb": 150, "quantum_mcs": 64}


def aggregate_ranks(ms: float, updates: float, dist=None, device=None) -> tuple[float, float]:
    """Whole-job numbers over ranks: the slowest rank's time (MAX) and the units all
    ranks processed (SUM).  Without a process group, the local numbers."""
    if dist is None:
        return ms, updates
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([updates], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_batch_case(args):
    """A short plain run of the batched form for ncu: the mixed batch, --mcs sweeps as one
    segment (the persistent launch and the streamed classes' launches beside it), then one
    measurement of every lattice."""
    import __graft_entry__
    from paper_2305_12161_gb300 import ising
    __graft_entry__.build()
    with ising.Batch(BATCH_CLASSES) as b:
        b.sweep(args.mcs)
        rec, der = b.measure_ex()
        print(json.dumps({"case": "batch", "mcs": args.mcs, "plan": b.plan(), "launches": b.launch_count()}))


def run_dcb_case(args):
    """The double-checkerboard sweep (Supp. Methods I A) on one L^3 lattice from the T = inf
    start: 3 warm-up MCS, then --mcs MCS timed with CUDA events on the context stream, the
    checkerboard sweep timed the same way beside it.  The roofline counts, per colour
    launch, the algorithmic bytes of the blocks of one colour: both sublattices of every
    block row and halo row read once, both sublattices of every block row written once."""
    import torch

    import __graft_entry__
    from paper_2305_12161_gb300 import ising
    __graft_entry__.build()
    L, mcs = args.L, args.mcs
    by, bz = args.block_y, args.block_z
    N = L**3
    stream = torch.cuda.Stream()
    pk = _peaks()

    def timed(q, n):
        q.sweep(3)
        q.sync()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        l0 = q.launch_count()
        a.record(stream)
        q.sweep(n)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), q.launch_count() - l0

    clocks = ClockSampler(0)
    clocks.start()
    with ising.Ising(L, seed=1, scheme=ising.SCHEME_DOUBLE, block=(0, by, bz), stream=stream) as q:
        ms, launches = timed(q, mcs)
    with ising.Ising(L, seed=1, stream=stream, variant=3 if L % 256 == 0 and L <= 2048 else 0) as q:
        ms_cb, _ = timed(q, mcs)
    clk = clocks.stop()
    W = max(1, L // 64)
    rows_own = L * L  # every row of the lattice belongs to exactly one block
    nblk = (L // by) * (L // bz)
    halo_rows = nblk * ((2 * bz if by < L else 0) + (2 * by if bz < L else 0))
    bytes_mcs = 2 * 4 * W * (rows_own + halo_rows) + 2 * 4 * W * rows_own
    per_launch_s = ms * 1e-3 / launches
    bytes_launch = bytes_mcs / 2
    achieved = bytes_launch / per_launch_s / 1e9
    print(json.dumps({
        "case": "dcb", "metric": "spin updates/ns, double-checkerboard sweep (Supp. Methods I A), one GB300",
        "value": mcs * N / (ms * 1e-3) / 1e9, "unit": UNIT, "higher_is_better": True,
        "config": {"workload": f"L={L} single lattice, T=inf start + 3 MCS, then {mcs} MCS timed",
                   "block": [L, by, bz], "cycle": "01", "l2": "lattice larger than L2" if N // 8 > 129e6 else "in L2"},
        "ms_per_mcs": ms / mcs, "launches": launches,
        "roofline": {"kernel": "k_sweep_dcb_rows (one colour)", "bound": "hbm", "achieved": achieved,
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                     # DRAM bytes of one launch in one ncu capture (L=2048, 16 x 8 blocks, sweep t=1)
                     "traffic": 1.2026e9 if (L, by, bz) == (2048, 16, 8) else None,
                     "avg_launch_ms": per_launch_s * 1e3, "bytes_per_launch": bytes_launch},
        "checkerboard_updates_per_ns": mcs * N / (ms_cb * 1e-3) / 1e9, "checkerboard_ms_per_mcs": ms_cb / mcs,
        "clocks": clk}))


def run_radial_case(args):
    """The radially averaged 3-d correlation and structure factor (two cuFFT transforms and
    the library's unpack / power / binning kernels) of one L^3 lattice after --mcs sweeps
    from the T = inf start: one untimed call per precision, then --steps calls timed with
    CUDA events around each (the call synchronises its stream)."""
    import torch

    import __graft_entry__
    from paper_2305_12161_gb300 import ising
    __graft_entry__.build()
    L = args.L
    stream = torch.cuda.Stream()
    out = {"case": "radial", "metric": "ms per radial C(r) + S(k) measurement (Eq. 3, radial average), one GB300",
           "unit": "ms", "higher_is_better": False,
           "config": {"workload": f"L={L} single lattice after {args.mcs} MCS from the T=inf start",
                      "L": L, "steps": args.steps}}
    clocks = ClockSampler(0)
    clocks.start()
    with ising.Ising(L, seed=1, stream=stream) as q:
        q.sweep(args.mcs)
        for prec, name in ((ising.FFT_SINGLE, "fp32"), (ising.FFT_DOUBLE, "fp64")):
            r = q.measure_radial(precision=prec)
            ms = []
            for _ in range(args.steps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r = q.measure_radial(precision=prec)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            out[name] = {"ms": statistics.median(ms), "ell": r["ell"], "inexact": r["inexact"],
                         "C_1_to_4": [float(v) for v in r["C"][1:5]]}
    out["clocks"] = clocks.stop()
    out["value"] = out["fp32"]["ms"]
    print(json.dumps(out))


def run_hist_case(args):
    """Statistical cross-check against the paper's domain-size histogram (Supplementary
    Discussion II): --runs independent L=256 lattices (seeds 1..runs) quenched with the 01-cycle
    checkerboard to rescaled time 4000 MCS (2286 checkerboard MCS at the factor 1.75), then
    l from the radially averaged C (fp32 FFTs) and from the axis C of every lattice."""
    import torch

    import __graft_entry__
    from paper_2305_12161_gb300 import ising
    __graft_entry__.build()
    L, runs = 256, args.runs
    mcs = round(4000 / 1.75)
    stream = torch.cuda.Stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with ising.Ising(L, replicas=runs, seed=1, stream=stream) as q:
        a.record(stream)
        q.sweep(mcs)
        b.record(stream)
        _, der = q.measure_ex(c=0.5)
        ms_sweep = a.elapsed_time(b)
        t0 = time.perf_counter()
        ell_rad = [q.measure_radial(replica=r, precision=ising.FFT_SINGLE)["ell"] for r in range(runs)]
        s_rad = time.perf_counter() - t0
    import numpy as np
    er, ea = np.array(ell_rad), der[:, 3]
    print(json.dumps({
        "case": "hist", "metric": "mean domain size l at rescaled t=4000 MCS, L=256 (paper: 19.9 checkerboard)",
        "runs": runs, "mcs": mcs, "mean_ell_radial": float(er.mean()), "std_ell_radial": float(er.std(ddof=1)),
        "sem_ell_radial": float(er.std(ddof=1) / np.sqrt(runs)), "mean_ell_axis": float(ea.mean()),
        "sem_ell_axis": float(ea.std(ddof=1) / np.sqrt(runs)),
        "quantiles_radial": [float(v) for v in np.quantile(er, [0.05, 0.25, 0.5, 0.75, 0.95])],
        "sweep_updates_per_ns": runs * L**3 * mcs / (ms_sweep * 1e-3) / 1e9, "radial_s_total": s_rad}))


def run_serve_case(args):
    """Continuous-batching serving on a finite seeded trace: Poisson arrivals at 20/s,
    L log-uniform on {64..1024}, t_max = 10^U[3,5] MCS, 1-16 replicas, 12 log-spaced
    measurements per request, 150 GB HBM budget, 16 slots."""
    import torch

    import __graft_entry__
    from paper_2305_12161_gb300 import serve
    __graft_entry__.build()
    torch.cuda.init()
    trace = serve.trace_requests(args.requests, seed=0, K=12)
    offered = sum(r.L**3 * r.replicas * r.t_max for r in trace)
    srv = serve.QuenchServer(budget_bytes=150e9, max_slots=16, quantum_mcs=64)
    clocks = ClockSampler(0)
    clocks.start()
    res = srv.run(trace)
    clk = clocks.stop()
    summ = srv.summary()
    arrivals = trace[-1].arrival_s
    print(json.dumps({
        "case": "serve", "metric": "time to result and aggregate spin updates/ns (serving)",
        "requests": len(res), "p50_s": summ["p50_s"], "p99_s": summ["p99_s"], "makespan_s": summ["makespan_s"],
        "aggregate_updates_per_ns": summ["updates_per_ns"], "updates": summ["updates"],
        "offered_updates_per_s": offered / arrivals if arrivals > 0 else None,
        "trace": "seeded Poisson 20/s, L log-uniform {64,...,1024}, t_max=10^U[3,5], replicas U{1..16}, K=12",
        "slots": 16, "budget_gb": 150, "quantum_mcs": 64, "clocks": clk}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=2048)
    ap.add_argument("--mcs", type=int, default=1000)
    ap.add_argument("--corr", type=int, default=0, help="correlation method: 0 auto, 1 popcount, 2 tensor cores")
    ap.add_argument("--t-checkpoint", type=int, default=10_000)
    ap.add_argument("--K", type=int, default=4, help="measured times per leg (4: one per decade)")
    ap.add_argument("--ref-L", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--block-y", type=int, default=16, help="dcb case: block rows along y")
    ap.add_argument("--block-z", type=int, default=8, help="dcb case: block planes along z")
    ap.add_argument("--runs", type=int, default=1000, help="hist case: independent L=256 runs")
    ap.add_argument("--sweep-config", default="", help="variant,tile_y,tile_z,depth instead of the autotuner "
                                                        "(for launch lists: no tuning launches)")
    ap.add_argument("--case", default="bench", choices=["bench", "quench", "serve", "batch", "dcb", "radial", "hist"],
                    help="quench: init + --mcs sweeps + one measurement, untimed (for profilers); "
                         "serve: the serving loop on the first --requests arrivals of the seeded trace")
    ap.add_argument("--requests", type=int, default=24)
    ap.add_argument("--serve-requests", type=int, default=16, help="serving leg of the default run: first arrivals")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--form", default="packed", choices=["packed", "plain"], help="quench case: lattice form")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.case == "quench":
        run_quench_case(args)
        return
    if args.case == "serve":
        run_serve_case(args)
        return
    if args.case == "batch":
        run_batch_case(args)
        return
    if args.case == "dcb":
        run_dcb_case(args)
        return
    if args.case == "radial":
        run_radial_case(args)
        return
    if args.case == "hist":
        run_hist_case(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()  # before any GPU work

    import numpy as np
    import torch

    import __graft_entry__
    from paper_2305_12161_gb300 import inputs, ising

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()

    L, MCS, TCK, K = args.L, args.mcs, args.t_checkpoint, args.K
    N = L**3
    seed = 1 + 1000 * rank
    stream = torch.cuda.Stream()
    if args.sweep_config:  # fixed kernel configuration (variant,tile_y,tile_z,depth), no tuning launches
        v, ty, tz, dp = (int(x) for x in args.sweep_config.split(","))
        tuned = {"variant": v, "tile_y": ty, "tile_z": tz, "depth": dp, "ms_per_mcs": None}
    else:
        tuned = ising.ising_tune_sweep(L, 1, probe_mcs=8)  # the project's autotuner picks the kernel
    q = ising.Ising(L, replicas=1, seed=seed, stream=stream, variant=tuned["variant"], tile_y=tuned["tile_y"],
                    tile_z=tuned["tile_z"], depth=tuned["depth"], corr=args.corr)
    RL = q.record_len
    per_mcs = 1 if tuned["variant"] == 5 else 2  # sweep kernel launches per MCS
    offsets = inputs.log_schedule(MCS, K)
    nwords = ising.ising_packed_words(L)

    # leg (ii) input: the state at t = 10^4, prepared once (untimed)
    q.sweep(TCK)
    ck_dev = torch.empty(nwords, dtype=torch.int32, device="cuda")
    q.get_packed(0, out=ck_dev, device=True)
    ck_host = torch.empty(nwords, dtype=torch.int32, pin_memory=True)
    q.sync()
    ck_host.copy_(ck_dev.cpu())
    rec_dev = torch.empty((2, K, RL), dtype=torch.int64, device="cuda")
    der_dev = torch.empty((2, K, 4), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    # which correlation method the context runs (the tensor-core path launches 9 kernels per
    # measurement, the bit-count path 4); this first call also allocates its scratch
    l0 = q.launch_count()
    q.measure_device(rec_dev[0, 0], der_dev[0, 0], c=0.5)
    q.sync()
    tensor_corr = q.launch_count() - l0 > 4

    sweep_events, meas_events = [], []

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    # end-to-end leg: the step's results land in pinned host buffers (one read-back per step)
    rec_host = torch.empty((2, K, RL), dtype=torch.int64, pin_memory=True)
    der_host = torch.empty((2, K, 4), dtype=torch.float64, pin_memory=True)

    def step(e2e: bool, timing: bool):
        outs = []
        for leg in (0, 1):
            if leg == 0:
                q.reinit(seed)
                t0 = 0
            else:
                if e2e:  # from pinned host memory; the transfer overlaps leg (i) on the device
                    q.set_packed(ck_host, 0, asynchronous=True)
                else:
                    q.set_packed(ck_dev, 0, device=True)
                q.t = TCK
                t0 = TCK
            t = t0
            for k, off in enumerate(offsets):
                a = ev() if timing else None
                q.sweep(t0 + off - t)
                b = ev() if timing else None
                t = t0 + off
                q.measure_device(rec_dev[leg, k], der_dev[leg, k], c=0.5)
                c = ev() if timing else None
                if timing:
                    sweep_events.append((a, b, per_mcs * (off - (offsets[k - 1] if k else 0)), leg))
                    meas_events.append((b, c))
        if e2e:  # the device-to-host read of the step's records and derived quantities
            with torch.cuda.stream(stream):
                rec_host.copy_(rec_dev, non_blocking=True)
                der_host.copy_(der_dev, non_blocking=True)
            q.sync()
            outs.append((rec_host, der_host))
        return outs

    def timed(e2e: bool, n: int):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = q.launch_count()
        start = ev()
        for _ in range(n):
            step(e2e, timing=not e2e)
        end = ev()
        torch.cuda.synchronize()
        ms = start.elapsed_time(end)
        ms, _ = aggregate_ranks(ms, 0.0, dist, "cuda")
        return ms, q.launch_count() - l0

    for _ in range(args.warmup):
        step(False, timing=False)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches = timed(False, args.steps)
    clk = clocks.stop()
    e2e_ms = None
    if not args.no_e2e:
        step(True, timing=False)  # warm the host path
        e2e_ms, _ = timed(True, args.steps)

    batched = None
    if not args.no_batched and rank == 0:
        batched = run_batched(torch, ising, inputs)
    pk = _peaks()
    plain = None
    if not args.no_plain and rank == 0:
        plain = run_plain(torch, ising, pk)
    serving = None
    if not args.no_serve and rank == 0:
        from paper_2305_12161_gb300 import serve
        serving = run_serving(serve, args.serve_requests)

    updates_per_step = 2 * MCS * N
    _, job_updates = aggregate_ranks(ms, float(updates_per_step * args.steps), dist, "cuda")
    value = job_updates / (ms * 1e-3) / 1e9

    # per-kernel live timings (CUDA events on the launching stream, inside the timed region)
    sweep_ms = sum(a.elapsed_time(b) for a, b, _, _ in sweep_events)
    sweep_launches = sum(n for _, _, n, _ in sweep_events)
    leg_ms = [sum(a.elapsed_time(b) for a, b, _, lg in sweep_events if lg == g) for g in (0, 1)]
    leg_launches = [sum(n for _, _, n, lg in sweep_events if lg == g) for g in (0, 1)]
    meas_ms = sum(a.elapsed_time(b) for a, b in meas_events)
    fused = tuned["variant"] == 5
    # a half-sweep reads q and q-bar and writes q (1 bit per site each: 3 N/16 bytes); the fused
    # sweep reads both sublattices and writes both (N/4 bytes) and updates all N sites
    bytes_per_launch = N / 4 if fused else 3 * (N // 2) / 8
    sites_per_launch = N if fused else N // 2
    sweep_avg_s = sweep_ms * 1e-3 / sweep_launches
    sweep_gbs = bytes_per_launch / sweep_avg_s / 1e9
    # correlation pass: XOR+popc word operations, 3 axes x L/2 lags x N/32 words
    corr_ops = 3 * (L // 2) * (N // 32)
    n_meas = len(meas_events)
    meas_avg_s = meas_ms * 1e-3 / n_meas
    # Bound of the correlation kernel, which sums XOR words on two pipes at once.  Counted from
    # the source: a POPC-path word is 1 bit count (16 lanes per SM per clock) + 1 XOR on the
    # integer ALU (64 lanes per SM per clock), its add issuing as a multiply-add on the
    # otherwise idle FMA pipe; a carry-save word is 1/8 bit count + 22/8 ALU ops (8 XORs and
    # 7 adders of two 3-input ops per 8 words).  The best split f of words on the POPC path
    # balances the two pipes: f = 0.43, 32 words per SM per clock.
    p_pop, a_pop, p_csa, a_csa = 1.0, 1.0, 1.0 / 8, 22.0 / 8
    f_pop = (a_csa / 64 - p_csa / 16) / ((p_pop - p_csa) / 16 + (a_csa - a_pop) / 64)
    words_per_clk = 16 / (f_pop * p_pop + (1 - f_pop) * p_csa)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    popc_peak = sms * words_per_clk * pk["sm_max_mhz"] * 1e6 / 1e12  # T word pairs/s
    corr_tops = corr_ops / meas_avg_s / 1e12
    kname = {1: "k_sweep_word", 2: "k_sweep_zmarch", 3: "k_sweep_zfast", 4: "k_sweep_zdeep",
             5: "k_mcs_fused"}[tuned["variant"]]
    # DRAM bytes per launch are not measured here (that needs a profiler): they are quoted
    # from the ncu capture of the same kernel at L=2048 named in traffic_src, and only for
    # the kernel that capture measured
    traffic, traffic_src = TRAFFIC_NCU.get((kname, L, tuned["tile_z"], tuned["depth"]), (None, None))
    roof_sweep = {"kernel": kname + (" (whole sweep)" if fused else " (half-sweep)"), "bound": "hbm",
                  "achieved": sweep_gbs,
                  "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": sweep_gbs / pk["hbm_gbs"], "traffic": traffic,
                  "traffic_src": traffic_src,
                  "peak_src": pk["src"], "avg_launch_ms": sweep_avg_s * 1e3, "bytes_per_launch": bytes_per_launch,
                  "updates_per_ns": sites_per_launch / sweep_avg_s / 1e9}
    if tensor_corr:
        # tensor-core path: the upper block triangle of the three axes' Gram matrices,
        # npairs tiles of 128 x 128 over K = L^2 lines, 2 flops per multiply-add; against the
        # fp8 peak = measured sustained bf16 x 2 (the nominal fp8 : bf16 ratio), the kernel
        # running inside a long step
        nbt = L // 128
        gram_flops = 3 * (nbt * (nbt + 1) // 2) * 2 * 128 * 128 * L * L
        fp8_peak = 2 * pk["bf16_tflops_sustained"]
        gram_tflops = gram_flops / meas_avg_s / 1e12
        roof_corr = {"kernel": "measurement: k_expand_x_e4m3 + 3 x k_gram_tma (helper warps expand y, z) + k_mb4", "bound": "tensor",
                     "achieved": gram_tflops, "peak": fp8_peak, "unit": "TFLOP/s (fp8)",
                     "frac": gram_tflops / fp8_peak, "traffic": None, "peak_src": pk["src"] + " bf16 sustained x 2",
                     "avg_launch_ms": meas_avg_s * 1e3, "flops_per_launch": gram_flops}
    else:
        roof_corr = {"kernel": "k_corr + k_mb (one measurement)", "bound": "alu", "achieved": corr_tops,
                     "peak": popc_peak, "unit": "T XOR-word-pairs/s", "frac": corr_tops / popc_peak, "traffic": None,
                     "avg_launch_ms": meas_avg_s * 1e3, "ops_per_launch": corr_ops}
    roof = roof_sweep if sweep_ms >= meas_ms else roof_corr
    e2e = None
    if e2e_ms is not None:
        d2h = 2 * K * (RL * 8 + 4 * 8)
        e2e = {"value": world * updates_per_step * args.steps / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": nwords * 4, "d2h_bytes_per_step": d2h}
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32 (1-bit spins, integer logic)", "data": "synthetic",
            "config": {"workload": f"L={L} single lattice: T=inf start + {MCS} MCS, and t={TCK} state + {MCS} MCS; "
                                   f"M, B, D_a(r<=L/2), e, m, l_E, l_C at {K} log-spaced times per leg",
                       "L": L, "mcs_per_leg": MCS, "legs": 2, "measurements_per_leg": K, "form": "packed",
                       "l2": "inputs larger than L2 (1 GiB packed lattice > 129 MB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof, "roofline_sweep": roof_sweep, "roofline_measure": roof_corr,
            "breakdown_ms_per_step": {"sweeps": sweep_ms / args.steps, "measurements": meas_ms / args.steps,
                                      "sweeps_leg_i_t0": leg_ms[0] / args.steps,
                                      "sweeps_leg_ii_t1e4": leg_ms[1] / args.steps},
            "sweep_updates_per_ns_by_leg": [sites_per_launch * n / (ms_ * 1e-3) / 1e9 if ms_ > 0 else None
                                            for n, ms_ in zip(leg_launches, leg_ms)],
            "sweep_only_updates_per_ns": world * sites_per_launch / sweep_avg_s / 1e9,
            "sweep_config": tuned,
            "corr_method": "tensor cores (tcgen05 Gram)" if tensor_corr else "bit counts",
            "clocks": clk, "e2e": e2e, "gpu_launches": launches, "batched": batched,
            "plain": plain, "serving": serving,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out))
    q.destroy()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
