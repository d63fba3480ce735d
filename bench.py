#!/usr/bin/env python3
"""Benchmark of the DDPMA mesh-generation hot path on GB300.

One bench step = one pass of the whole hot path over one batch of seeded
synthetic requests: admission tables in device memory, every forward-Euler
step of every subdomain until each request meets its stop rule or its step
cap, and the owner-takes combination of every request into its global mesh.

  value      node-updates/s with the inputs resident in device memory,
             device time from CUDA events on the library's stream;
  e2e        the same through the public C API from host structs to host
             meshes (host<->device copies inside the timed region);
  roofline   the sweep kernel's algorithmic bytes (one read and one write of
             v per node-update) over its event-timed windows, against the
             measured HBM copy bandwidth;
  cpu_baseline  the FP64 oracle on a bounded sample, on the host cores.

Multi-GPU: the path does not exchange data between requests, so N GPUs run N
independent replicas (weak scaling); value = all ranks' node-updates over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

from paper_2006_14602_gb300 import workloads as W

METRIC = "PMA node-updates/s"
UNIT = "node-updates/s"

WORKLOADS = {
    "c4": "uneven batch: 512 independent 2D problems, sides log-uniform in [17,513], "
          "1-16 subdomains (overlap 4-8), 1-4 Gaussian bumps/rings, FP32, tol 1e-6 "
          "or 2000 steps",
    "c2": "2D 257x257 in 4x4 subdomains (overlap 8), ring and sine-wave monitors, FP32, "
          "2000 steps, all 32 subdomains in one launch",
    "c3": "3D 129^3 in 2x2x2 subdomains (overlap 6), spherical shell monitor, FP32 sweep, "
          "FP64 residual/stop test, 2000 steps",
    "c3x16": "3D: 16 requests of 129^3 in 2x2x2 subdomains (overlap 6), spherical shell "
             "monitor, FP32 sweep, FP64 residual/stop test, 2000 steps; 315 MB of state "
             "(larger than L2)",
    "c3big": "3D 257^3 in 4x4x4 subdomains (overlap 6), spherical shell monitor, FP32 sweep, "
             "FP64 residual/stop test, 2000 steps; 166 MB of state (larger than L2)",
    "c4x2": "uneven batch twice over: 1024 independent 2D problems (seeds 14602 and 14603), "
            "sides log-uniform in [17,513], 1-16 subdomains (overlap 4-8), 1-4 Gaussian "
            "bumps/rings, FP32, tol 1e-6 or 2000 steps; 213 MB of state (larger than L2)",
}


# ------------------------------------------------------------------ serving
def serving(args):
    """Serving stream: Poisson arrivals of mixed 2D / 3D requests submitted
    from a host thread to a context whose server thread batches them
    continuously.  First the whole stream at once (saturation throughput),
    then Poisson rates of 0.25x..1.5x that throughput (latency under load),
    a run with a small memory budget (admission back-pressure), and the
    first requests on the plain FP64 path (one launch per subdomain and
    step, no graphs) for comparison."""
    import torch
    from paper_2006_14602_gb300 import build, pma

    build.build()
    pma.load()
    torch.cuda.init()

    def run(stream, precision, plain, budget=120 << 30):
        reqs = [(t, p.replace(precision=precision)) for t, p in stream]
        opts = {"window_steps": args.window, "resident": args.resident,
                "resident_steps": args.resident_steps}
        if plain:
            opts.update(launch_mode=pma.PMA_LAUNCH_PER_SUBDOMAIN, use_graphs=0)
        with pma.Context(0, budget, **opts) as ctx:
            if pma.pma_serve_start(ctx.h) != pma.PMA_OK:
                raise RuntimeError("server did not start")
            ids = []
            t0 = time.perf_counter()
            for t_arr, p in reqs:
                d = t0 + t_arr - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                ids.append(ctx.submit(p))
            lat, nu = [], 0
            for (_, p), i in zip(reqs, ids):
                st = pma.pma_wait(ctx.h, i, 600_000_000)
                if st not in (pma.PMA_OK, pma.PMA_NOT_CONVERGED, pma.PMA_ERR_TANGLED):
                    raise RuntimeError("request failed: %s" % pma.STATUS_NAMES.get(st, st))
                _, info = pma.pma_get_info(ctx.h, i)
                lat.append(info.latency_us / 1e3)
                nu += info.steps * _sub_nodes(p)
                pma.pma_release(ctx.h, i)
            wall = time.perf_counter() - t0
            pma.pma_serve_stop(ctx.h)
        return {"meshes_per_s": len(reqs) / wall, "node_updates_per_s": nu / wall,
                "p10_ms": percentile(lat, 0.1), "p25_ms": percentile(lat, 0.25),
                "p50_ms": percentile(lat, 0.5), "p90_ms": percentile(lat, 0.9),
                "p99_ms": percentile(lat, 0.99), "wall_s": wall, "requests": len(reqs)}

    def stream_at(rate):
        return W.config5_stream(count=args.requests, rate_hz=rate,
                                max_steps=args.max_steps or 2000,
                                size2d=(33, args.max2d), size3d=(17, args.max3d))

    warm = W.config5_stream(seed=1, count=4, rate_hz=1e6, max_steps=50, size2d=(33, 65),
                            size3d=(17, 21))
    run(warm, "fp32", False)
    sat = run(stream_at(1e9), "fp32", False)
    rates = [args.rate] if args.rate else [f * sat["meshes_per_s"] for f in (0.25, 0.5, 1.0, 1.5)]
    sweep = []
    for r in rates:
        q = run(stream_at(r), "fp32", False)
        q["rate_per_s"] = r
        sweep.append(q)
    small = run(stream_at(rates[-1] if args.rate else sat["meshes_per_s"]), "fp32", False,
                budget=args.budget_mb << 20)
    small["budget_mb"] = args.budget_mb
    full = stream_at(1e9)
    plain_n = len(full) if args.plain_requests < 0 else args.plain_requests
    plain = run(full[:plain_n], "fp64", True) if plain_n else None
    same = run(full[:plain_n], "fp32", False) if plain_n and plain_n != len(full) else sat
    line = {
        "metric": "meshes/s (serving stream)", "value": sat["meshes_per_s"], "unit": "meshes/s",
        "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded Poisson stream, master seed %d)" % W.MASTER_SEED,
        "config": {"workload": "serving stream: %d mixed 2D (33^2-%d^2) and 3D (17^3-%d^3) "
                               "requests, 1-27 subdomains, random bump monitors, tol 1e-6 or "
                               "%d steps; value = all submitted at once"
                               % (args.requests, args.max2d, args.max3d, args.max_steps or 2000),
                   "requests": args.requests},
        "latency_ms": {"p10": sat["p10_ms"], "p25": sat["p25_ms"], "p50": sat["p50_ms"],
                       "p90": sat["p90_ms"], "p99": sat["p99_ms"]},
        "node_updates_per_s": sat["node_updates_per_s"],
        "poisson_sweep": sweep,
        "small_budget": small,
        "plain_fp64_per_subdomain": plain,
        "batched_fp32_same_requests": same,
        "budget_gb": 120,
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ per-config table
def config_table(args):
    """Configurations 1-4 on three device paths (FP32 batched, FP64 batched,
    the plain FP64 path: one launch per subdomain and step, no graphs) and
    the FP64 oracle on one host core (a bounded sample of each
    configuration, step caps scaled to ~1.5e8 node-updates).  Device time
    from CUDA events around pma_run on the context's stream; L2 flushed
    before each timed run.  One JSON line."""
    import torch
    from paper_2006_14602_gb300 import build, pma

    cap = args.max_steps or 400
    cfgs = {"c1": [W.config1("fp64")],
            "c2": [W.config2("ring", "fp64"), W.config2("sine", "fp64")],
            "c3": [W.config3("fp64")],
            "c4": W.config4(precision="fp64")}
    # the same step cap on every path (rates are per node-update)
    cfgs = {k: [p.replace(max_steps=min(p.max_steps, cap)) for p in v] for k, v in cfgs.items()}
    # oracle first, in spawned workers of one process each, before any GPU call
    oracle_rates = {}
    for name, probs in cfgs.items():
        work = sum(_sub_nodes(p) * p.max_steps for p in probs)
        scale = min(1.0, 1.5e8 / work)
        rng = np.random.default_rng(3)
        pick = probs if len(probs) <= 2 else [probs[i] for i in rng.permutation(len(probs))[:8]]
        sample = [p.replace(max_steps=max(1, int(p.max_steps * scale)), tol=0.0) for p in pick]
        v, wall, nu = run_oracle(sample, 1)
        oracle_rates[name] = {"node_updates_per_s": v, "sample_node_updates": nu, "wall_s": wall,
                              "cores": 1}
        print("oracle %s: %.3g node-updates/s" % (name, v), file=sys.stderr, flush=True)
    build.build()
    pma.load()
    torch.cuda.init()
    stream = torch.cuda.Stream(0)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=0)

    def timed(probs, precision, plain):
        opts = {"window_steps": 128}
        if plain:
            opts.update(launch_mode=pma.PMA_LAUNCH_PER_SUBDOMAIN, use_graphs=0)
        ps = [p.replace(precision=precision) for p in probs]
        with pma.Context(0, 0, stream.cuda_stream, **opts) as ctx:
            for _ in range(2):  # the first pass warms up
                ids = [ctx.submit(p) for p in ps]
                if pma.pma_admit(ctx.h) != pma.PMA_OK:
                    raise RuntimeError("admission failed")
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                pma.pma_get_stats(ctx.h, 1)
                e0.record(stream)
                ctx.run()
                e1.record(stream)
                e1.synchronize()
                _, st = pma.pma_get_stats(ctx.h, 1)
                steps = []
                for i in ids:
                    steps.append(pma.pma_get_info(ctx.h, i)[1].steps)
                    pma.pma_release(ctx.h, i)
            ms = e0.elapsed_time(e1)
        return {"node_updates_per_s": st.node_updates / (ms / 1e3), "meshes_per_s":
                len(ps) / (ms / 1e3), "ms": ms, "mean_steps": float(np.mean(steps))}

    table = {}
    for name, probs in cfgs.items():
        table[name] = {"oracle_1_core": oracle_rates[name]}
        for key, prec, plain in (("gpu_fp32_batched", "fp32", False),
                                 ("gpu_fp64_batched", "fp64", False),
                                 ("gpu_fp64_plain", "fp64", True)):
            table[name][key] = timed(probs, prec, plain)
            print("%s %s: %.3g node-updates/s" % (name, key, table[name][key]["node_updates_per_s"]),
                  file=sys.stderr, flush=True)
    line = {"metric": "per-configuration node-updates/s (configs 1-4, every request capped "
                      "at %d steps)" % cap, "unit": "node-updates/s",
            "n_gpus": 1, "data": "synthetic (seeded requests, master seed %d)" % W.MASTER_SEED,
            "configs": table}
    print(json.dumps(line))
    return 0


def make_workload(name: str, precision: str, max_steps=None):
    if name == "c4":
        probs = W.config4(precision=precision)
    elif name == "c2":
        probs = [W.config2("ring", precision), W.config2("sine", precision)]
    elif name == "c3":
        probs = [W.config3(precision)]
    elif name == "c3x16":
        probs = [W.config3(precision) for _ in range(16)]
    elif name == "c3big":
        n = (257, 257, 257)
        probs = [W.config3(precision).replace(n=n, parts=(4, 4, 4),
                                              dt=W.dt_for(n, 3, cfl=0.05))]
    elif name == "c4x2":
        probs = (W.config4(precision=precision) +
                 W.config4(seed=W.MASTER_SEED + 1, precision=precision))
    else:
        raise SystemExit("unknown workload %s" % name)
    if max_steps is not None:
        probs = [p.replace(max_steps=max_steps) for p in probs]
    return probs


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        med = statistics.median(sm) if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax or None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle leg
def _oracle_job(args):
    prob, = args
    import oracle
    t = time.perf_counter()
    r = oracle.solve(prob)
    dt = time.perf_counter() - t
    nodes = _sub_nodes(prob)
    return r.steps * nodes, dt


def _sub_nodes(prob) -> int:
    """Subdomain nodes of a problem (overlap duplicates counted), from the
    decomposition rule of the input description."""
    total = 1
    for a in range(prob.dim):
        n, p, o = prob.n[a], prob.parts[a], prob.overlap
        if p == 1:
            total *= n
            continue
        ol, oh = o // 2, o - o // 2
        b = [(2 * k * n + p) // (2 * p) for k in range(p + 1)]
        s = 0
        for k in range(p):
            lo = 0 if k == 0 else b[k] - ol
            hi = n - 1 if k == p - 1 else b[k + 1] - 1 + oh
            s += hi - lo + 1
        total *= s
    return total


def oracle_sample(probs, budget_node_updates: float = 1.2e9, seed: int = 7):
    """A bounded sample of the workload for the CPU oracle: a seeded subset
    of requests with their step caps scaled so that the whole sample is about
    budget_node_updates of work."""
    import oracle  # noqa: F401  (build before forking workers)
    oracle.build()
    rng = np.random.default_rng(seed)
    idx = list(rng.permutation(len(probs)))
    cores = max(1, min(os.cpu_count() or 1, 16))
    pick = [probs[i] for i in idx[: max(cores, 1)]]
    work = sum(_sub_nodes(p) * p.max_steps for p in pick)
    scale = min(1.0, budget_node_updates / max(work, 1))
    sample = [p.replace(max_steps=max(1, int(p.max_steps * scale)), tol=0.0,
                        precision="fp64") for p in pick]
    return sample, cores


def run_oracle(sample, cores):
    import multiprocessing as mp
    t = time.perf_counter()
    if cores > 1:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_job, [(p,) for p in sample])
    else:
        res = [_oracle_job((p,)) for p in sample]
    wall = time.perf_counter() - t
    nu = sum(r[0] for r in res)
    return nu / wall, wall, nu


# ------------------------------------------------------------------ helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha1()
    for f in ("pma_kernels.cu", "pma_device.cuh", "pma_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2006_14602_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def recorded_traffic(kernel: str, workload: str, precision: str):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(path):
        return None, None
    src = None
    val = None
    for line in open(path):
        if line.startswith("kernel_source_sha1:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            try:
                val = float(line.split(":", 1)[1].split()[0])
            except ValueError:
                val = None
        if line.startswith("node_updates_per_launch:"):
            pass
    if src != kernel_source_hash():
        return None, path
    return val, path


def percentile(xs, q):
    if not xs:
        return None
    xs = sorted(xs)
    k = (len(xs) - 1) * q
    f, c = math.floor(k), math.ceil(k)
    return xs[f] if f == c else xs[f] + (xs[c] - xs[f]) * (k - f)


# ------------------------------------------------------------------ native arm
def native(args, rank, world, device):
    import torch
    from paper_2006_14602_gb300 import build, pma

    build.build()
    pma.load()
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device)
    probs = make_workload(args.workload, args.precision, args.max_steps)
    # one step in 16 of every window has its sweep launch timed with events
    opts = {"window_steps": args.window, "resident": args.resident, "time_sweeps": 16,
            "groups": args.groups}
    tuned = None
    if args.autotune and args.tile2d is None and args.tile3d is None and not args.resident:
        # untimed: work shapes and window length measured on this batch
        from paper_2006_14602_gb300.autotune import autotune
        tuned = autotune(probs, device, groups=args.groups)
        opts.update(tile_2d=tuned["tile_2d"], tile_3d=tuned["tile_3d"],
                    window_steps=tuned["window_steps"])
    if args.tile2d is not None:
        opts["tile_2d"] = args.tile2d
    if args.tile3d is not None:
        opts["tile_3d"] = args.tile3d
    ctx = pma.Context(device, 0, stream.cuda_stream, **opts)
    nodes_out = [p.dim * p.nodes for p in probs]
    out = torch.empty(sum(nodes_out), dtype=torch.float64, device=device)
    offs = np.concatenate([[0], np.cumsum(nodes_out)])[:-1]
    ptrs = [out.data_ptr() + 8 * int(o) for o in offs]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    # end-to-end leg: the requests as the C structs a caller hands to
    # pma_submit, and one page-locked host buffer that receives every mesh
    host_out = torch.empty(sum(nodes_out), dtype=torch.float64, pin_memory=True)
    structs = [pma.to_structs(p) for p in probs]

    def one_step(timed_events: bool):
        ids = [ctx.submit(p) for p in probs]
        st = pma.pma_admit(ctx.h)
        if st != pma.PMA_OK:
            raise pma.PmaError("pma_admit", st)
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        pma.pma_get_stats(ctx.h, 1)
        e0.record(stream)
        ctx.run()
        st = pma.pma_get_mesh_device_batch(ctx.h, ids, ptrs, 1)
        if st != pma.PMA_OK:
            raise pma.PmaError("pma_get_mesh_device_batch", st)
        e1.record(stream)
        e1.synchronize()
        _, stats = pma.pma_get_stats(ctx.h, 1)
        infos = []
        for i in ids:
            infos.append(_info(pma, ctx, i))
            pma.pma_release(ctx.h, i)
        return e0.elapsed_time(e1), stats, infos

    def e2e_step():
        # the C ABI from host structs to host meshes: pma_submit (inputs
        # copied), pma_run (admission uploads the tables, then every step),
        # pma_get_mesh_batch (one combination and one device-to-host copy of
        # every mesh into the page-locked host buffer); wall clock around it
        torch.cuda.synchronize(device)
        pma.pma_get_stats(ctx.h, 1)
        t0 = time.perf_counter()
        ids = []
        for g, m, d, p in structs:
            st, rid = pma.pma_submit(ctx.h, g, m, d, p, None)
            if st != pma.PMA_OK:
                raise pma.PmaError("pma_submit", st)
            ids.append(rid)
        ctx.run()
        st = pma.pma_get_mesh_batch(ctx.h, ids, host_out.data_ptr())
        if st != pma.PMA_OK:
            raise pma.PmaError("pma_get_mesh_batch", st)
        t1 = time.perf_counter()
        _, stats = pma.pma_get_stats(ctx.h, 1)
        return (t1 - t0) * 1e3, stats

    for _ in range(args.warmup):
        one_step(False)
    sampler = ClockSampler(device) if rank == 0 else None
    _barrier(world, device)
    if sampler:
        sampler.start()
    times, all_stats, lat = [], [], []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        _barrier(world, device)
        torch.cuda.synchronize(device)
        ms, stats, infos = one_step(True)
        torch.cuda.synchronize(device)
        times.append(ms)
        all_stats.append(stats)
        lat.extend(i["latency_ms"] for i in infos)
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop() if sampler else None
    e2e_step()  # untimed: sizes the library's staging buffer for the batch's meshes
    e2e_times, e2e_stats = [], []
    for _ in range(max(1, min(args.steps, 3))):
        ms, stats = e2e_step()
        e2e_times.append(ms)
        e2e_stats.append(stats)

    node_updates = sum(s.node_updates for s in all_stats)
    total_ms = sum(times)
    sweep_ms = sum(s.window_ms for s in all_stats)
    sweep_bytes = sum(s.sweep_bytes for s in all_stats)
    kernel_ms = sum(s.sweep_kernel_ms for s in all_stats)
    kernel_launches = sum(s.sweep_kernel_launches for s in all_stats)
    launches = sum(s.sweep_launches for s in all_stats)
    sweep_steps = sum(s.sweep_steps for s in all_stats)
    other = sum(s.other_launches for s in all_stats)
    local = {
        "node_updates": node_updates, "ms": total_ms, "sweep_ms": sweep_ms,
        "sweep_bytes": sweep_bytes, "launches": launches + other, "sweep_launches": launches,
        "sweep_steps": sweep_steps,
        "kernel_ms": kernel_ms, "kernel_launches": kernel_launches,
        "e2e_ms": sum(e2e_times), "e2e_nu": sum(s.node_updates for s in e2e_stats),
        "h2d": sum(s.h2d_bytes for s in e2e_stats) / len(e2e_stats),
        "d2h": sum(s.d2h_bytes for s in e2e_stats) / len(e2e_stats),
        "e2e_host_ms": {k: sum(getattr(s, k) for s in e2e_stats) / len(e2e_stats)
                        for k in ("admit_ms", "rebuild_ms", "combine_ms")},
        "meshes": len(probs) * args.steps, "lat": lat, "wall_s": t_wall,
        # global-node updates (each node of a request's global grid once per
        # step it took, overlap copies not counted)
        "global_nu": sum(p.nodes * st for p, st in zip(probs, [i["steps"] for i in infos]))
                     * args.steps,
        "infos_steps": [i["steps"] for i in infos],
        "tuned": tuned, "window": opts["window_steps"],
    }
    agg = _gather(world, local, device)
    ctx.close()
    return agg, clocks, probs


def _info(pma, ctx, rid):
    st, info = pma.pma_get_info(ctx.h, rid)
    if st != pma.PMA_OK:
        raise pma.PmaError("pma_get_info", st)
    return {"status": info.status, "steps": info.steps, "latency_ms": info.latency_us / 1e3}


def _barrier(world, device):
    if world > 1:
        import torch.distributed as dist
        if dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def _gather(world, local, device):
    if world == 1:
        return [local]
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, local)
    return out


def aggregate(agg):
    """Whole-job throughput over replicas: every rank's node-updates over the
    slowest rank's time (device-resident and end to end)."""
    nu = sum(a["node_updates"] for a in agg)
    ms = max(a["ms"] for a in agg)
    e2e = sum(a["e2e_nu"] for a in agg) / (max(a["e2e_ms"] for a in agg) / 1e3)
    return nu / (ms / 1e3), ms, e2e


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="c4", choices=sorted(WORKLOADS) + ["c5", "table"])
    ap.add_argument("--resident", type=int, default=0,
                    help="k > 0: cluster-resident path for 2D requests that fit the "
                         "first k shared-memory classes (0: band kernels only)")
    ap.add_argument("--rate", type=float, default=None,
                    help="c5: one Poisson rate (default: 0.25x..1.5x the saturation throughput)")
    ap.add_argument("--resident-steps", type=int, default=0,
                    help="steps a resident launch takes per window (0: the window's)")
    ap.add_argument("--budget-mb", type=int, default=256,
                    help="c5: memory budget of the back-pressure run")
    ap.add_argument("--requests", type=int, default=64, help="c5: requests in the stream")
    ap.add_argument("--plain-requests", type=int, default=-1,
                    help="c5: requests of the stream replayed on the plain FP64 path "
                         "(-1: the whole stream)")
    ap.add_argument("--max2d", type=int, default=1025, help="c5: largest 2D side")
    ap.add_argument("--max3d", type=int, default=193, help="c5: largest 3D side")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--max-steps", type=int, default=None,
                    help="override the per-request step cap (testing only)")
    ap.add_argument("--window", type=int, default=64)
    ap.add_argument("--groups", type=int, default=1,
                    help="request groups per kernel class (1 or 2), each on its own stream")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the untimed autotuning of work shapes and window length")
    ap.add_argument("--tile2d", type=int, default=None, help="2D work shape id (default: auto)")
    ap.add_argument("--tile3d", type=int, default=None, help="3D work shape id (default: auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        return reference_arm(args, world)
    if args.workload == "c5":
        return serving(args) if rank == 0 else 0
    if args.workload == "table":
        return config_table(args) if rank == 0 else 0

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    # CPU baseline first (spawned workers, before the first GPU call)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        probs0 = make_workload(args.workload, args.precision, args.max_steps)
        sample, cores = oracle_sample(probs0)
        v, wall, nu = run_oracle(sample, cores)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d of the workload's requests (seeded), FP64 C oracle, step caps "
                         "scaled to %d node-updates in total, one spawned process per core; "
                         "%.1f s wall" % (len(sample), nu, wall)}

    agg, clocks, probs = native(args, rank, world, local_rank)
    if rank != 0:
        return 0
    value, ms, e2e_v = aggregate(agg)
    a0 = agg[0]
    peak, peak_kind = measured_peaks()
    # the sweep kernel's own device time: CUDA events around every sweep launch
    # on the library's stream (recorded inside the windows' graphs)
    if a0["kernel_ms"] > 0 and not args.resident:
        timing = ("CUDA events around the sweep launches of one step in 16 of the timed "
                  "region, on the launching streams: %d steps timed, mean %.1f us from the "
                  "first group's sweep start to the last one's end (request groups: %d, "
                  "their sweeps overlap)" % (
                      a0["kernel_launches"], 1e3 * a0["kernel_ms"] / max(a0["kernel_launches"], 1),
                      args.groups))
        # algorithmic bytes of one step's sweep launches over their timed span
        per_launch = a0["sweep_bytes"] / max(a0["sweep_steps"], 1)
        achieved = per_launch / (a0["kernel_ms"] / max(a0["kernel_launches"], 1) / 1e3) / 1e9
    else:
        achieved = a0["sweep_bytes"] / (a0["sweep_ms"] / 1e3) / 1e9
        timing = "CUDA events around the stepping windows"
        per_launch = None
    kname = "k_band2d" if probs[0].dim == 2 else "k_band3d"
    traffic, tpath = recorded_traffic(kname, args.workload, args.precision)
    lat = [x for x in a0["lat"] if x is not None]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic (seeded requests, master seed %d)" % W.MASTER_SEED,
        "config": {"workload": WORKLOADS[args.workload], "requests": len(probs),
                   "precision": args.precision, "window_steps": a0["window"],
                   "autotuned": ({k: v for k, v in a0["tuned"].items() if k != "rates"}
                                 if a0["tuned"] else None),
                   "resident": args.resident, "request_groups": args.groups,
                   "l2": "flushed (512 MB write) before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "meshes_per_s": a0["meshes"] / (a0["ms"] / 1e3),
        "global_node_updates_per_s": sum(a["global_nu"] for a in agg) / (ms / 1e3),
        "latency_ms": {"p50": percentile(lat, 0.5), "p99": percentile(lat, 0.99),
                       "what": "per request, submit to completion, all requests of a "
                               "step submitted together"},
        "mean_steps_per_request": float(np.mean(a0["infos_steps"])),
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": a0["h2d"],
                "d2h_bytes_per_step": a0["d2h"],
                "path": "C ABI: pma_submit per request from host structs, pma_run, "
                        "pma_get_mesh_batch into one page-locked host buffer",
                "host_ms_per_step": a0["e2e_host_ms"]},
        "gpu_launches": a0["launches"] // max(args.steps, 1),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None, "traffic": traffic,
                     "kernel": kname, "timing": timing,
                     "algorithmic_bytes_per_launch": per_launch,
                     "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind,
                     "algorithmic_bytes_per_node_update": 2 * (4 if args.precision == "fp32" else 8)},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "autotune_rates": a0["tuned"]["rates"] if a0["tuned"] else None,
    }
    print(json.dumps(line))
    return 0


def reference_arm(args, world):
    probs = make_workload(args.workload, args.precision, args.max_steps)
    sample, cores = oracle_sample(probs, budget_node_updates=1.0e8)
    for _ in range(args.warmup):
        run_oracle(sample[: max(1, len(sample) // 4)], cores)
    vals, walls, nus = [], [], []
    for _ in range(args.steps):
        v, wall, nu = run_oracle(sample, cores)
        vals.append(v)
        walls.append(wall)
        nus.append(nu)
    value = sum(nus) / sum(walls)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(walls) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded requests, master seed %d)" % W.MASTER_SEED,
        "config": {"workload": WORKLOADS[args.workload], "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d requests of the workload, step caps scaled to %d "
                                   "node-updates per step" % (len(sample), nus[0])},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
