#!/usr/bin/env python
"""Benchmark of the GB300 Pbit list sort.

One step = one pbit_sort_list call on a 2^27-node SoA list (int32 next[],
uint32 key[], seeded random list order, uniform keys, M = 32, K = 4): list
ranking, MSD passes, shared-memory finish and relink.  Inputs are resident in
HBM; before every step next[] is restored from a device copy outside the
timed events (inputs are 1 GiB, larger than the 129 MB L2, so no flush).

Prints ONE JSON line (rank 0).  --impl reference times the oracle (the
literal single-threaded CPU Pbit) on bounded samples of the same workload.
Multi-GPU (torchrun): every rank sorts its own replica list (the single-list
sort does not shard), value = all ranks' nodes / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "sorted list nodes/s (one 2^27-node SoA uint32 list, random order, M=32, K=4)"
UNIT = "nodes/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2n", type=int, default=27, help="list size (27 = the benchmark workload)")
    ap.add_argument("--key-bits", type=int, default=32,
                    help="keys uniform over this many low bits and M = this (32 = the benchmark workload)")
    ap.add_argument("--digit-bits", type=int, default=8,
                    help="GPU digit width of the timed sort (tune; 0 = the call's K, 4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-log2n", type=int, default=24)
    ap.add_argument("--no-batched", action="store_true", help="skip the 4096-list batched leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the request-serving leg")
    ap.add_argument("--batched-lists", type=int, default=4096)
    ap.add_argument("--cpu-batched-lists", type=int, default=512,
                    help="lists of the batched workload in the all-cores oracle sample")
    ap.add_argument("--serve-requests", type=int, default=20000, help="timed requests of each serving trace")
    ap.add_argument("--serve-warmup", type=int, default=1000)
    ap.add_argument("--serve-pools", type=int, default=1000, help="device pools the request stream cycles through")
    return ap.parse_args()


def workload(log2n, key_bits=32, digit_bits=0):
    return {"workload": f"pbit_sort_list: one 2^{log2n}-node list, SoA int32 next + uint32 key, "
                        f"seeded random list order, uniform keys, M={key_bits}, K=4"
                        + ("" if key_bits == 32 else f" (keys below 2^{key_bits})"),
            "n": 1 << log2n, "key": "uint32", "layout": "SoA", "M": key_bits, "K": 4,
            "gpu_digit_bits": digit_bits or 4,
            "digit_bits_note": "the GPU's MSD passes split on this many bits (tune); the result is the same for "
                               "any width, K=4 fixes only the paper's digit",
            "l2": "inputs (1 GiB at 2^27) larger than L2; no flush"}


def bench_keys(I, n, seed, key_bits):
    key = I.uniform_keys(n, 4, seed)
    if key_bits < 32:
        key &= np.uint32((1 << key_bits) - 1)
    return key


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"pbit_clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def whole_job_rate(units_per_rank, seconds, world, device):
    """Whole-job throughput: all ranks' units over the slowest rank's time
    (max over ranks; every rank does the same amount of work).  Returns
    (rate, max seconds).  Collective only when world > 1."""
    t = float(seconds)
    if world > 1:
        import torch
        import torch.distributed as tdist
        x = torch.tensor([t], dtype=torch.float64, device=device)
        tdist.all_reduce(x, op=tdist.ReduceOp.MAX)
        t = float(x.item())
    return world * units_per_rank / t, t


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(log2n, seed, key_bits=32):
    from oracle import oracle as O
    from paper_cs_0511020_gb300 import inputs as I
    n = 1 << log2n
    nxt, root = I.random_list(n, seed)
    key = bench_keys(I, n, seed + 1, key_bits)
    t0 = time.perf_counter()
    O.pbit_sort(nxt, key, root, key_bits, 4)
    dt = time.perf_counter() - t0
    return n, dt


def run_reference(a):
    ws, rank, _ = dist()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    log2n = min(21, a.log2n)
    times = []
    for i in range(a.warmup + a.steps):
        n, dt = oracle_sample(log2n, 0x0511020 + 2 + i, a.key_bits)
        if i >= a.warmup:
            times.append(dt)
    tot = sum(times)
    value = a.steps * (1 << log2n) / tot
    sample = f"{a.steps} timed steps, each the oracle on one 2^{log2n}-node list of the same recipe"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload(a.log2n, a.key_bits, a.digit_bits),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_ours(a):
    import torch
    import torch.distributed as tdist

    from paper_cs_0511020_gb300 import inputs as I
    from paper_cs_0511020_gb300 import pbit

    world, rank, local = dist()
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = 1 << a.log2n
    M = a.key_bits
    if not 4 <= M <= 32 or M % 4:
        raise SystemExit("--key-bits must be a multiple of 4 in [4, 32]")
    seed = I.SEED_BASE + 2 + 7919 * rank
    nxt, root = I.random_list(n, seed)
    key = bench_keys(I, n, seed + 1, M)
    d_next0 = torch.from_numpy(nxt).cuda()
    d_next = d_next0.clone()
    d_key = torch.from_numpy(key.view(np.int32)).cuda()
    pool = pbit.make_pool(d_next, d_key)
    tune = {"digit_bits": a.digit_bits} if a.digit_bits else None
    ws = pbit.alloc_workspace(pbit.workspace_size(n, 1, 4, tune))
    stream = torch.cuda.current_stream()

    def step():
        d_next.copy_(d_next0)
        st, r = pbit.sort_pool_list(pool, root, n, M, 4, ws=ws, stream=stream, check=False, tune=tune)
        if st != pbit.OK:
            raise pbit.PbitError(st, "bench step")
        return r

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    # Device time of a step = two CUDA events on the launching stream around
    # the call (its memsets, kernels and status read-back); next[] is restored
    # before the first event.  Per-kernel events are off here: they would
    # serialize the kernels' programmatic launches.
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    wall0 = time.perf_counter()
    for i in range(a.steps):
        d_next.copy_(d_next0)
        ev0[i].record(stream)
        st, _ = pbit.sort_pool_list(pool, root, n, M, 4, ws=ws, stream=stream, check=False, tune=tune)
        ev1[i].record(stream)
        if st != pbit.OK:
            raise pbit.PbitError(st, "bench step")
    torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    step_ms = [ev0[i].elapsed_time(ev1[i]) for i in range(a.steps)]
    launches_per_step = pbit.last_launch_count()
    # Per-kernel split (roofline objects): the same steps again with the
    # library's per-kernel events on.
    kernel_stats = {}
    pbit.profile_enable(True)
    for _ in range(a.steps):
        step()
        for k in pbit.profile_read():
            s = kernel_stats.setdefault(k["name"], {"launches": 0, "ms": 0.0, "bytes": 0.0})
            s["launches"] += k["launches"]
            s["ms"] += k["ms"]
            s["bytes"] += k["bytes"]
    pbit.profile_enable(False)
    value, tot_s = whole_job_rate(a.steps * n, sum(step_ms) / 1e3, world, "cuda")
    tot_ms = tot_s * 1e3

    # ---- end to end through the host-buffer C ABI call (pinned host memory)
    h_next0 = torch.from_numpy(nxt).pin_memory()
    h_next = h_next0.clone().pin_memory()
    h_key = torch.from_numpy(key.view(np.int32)).pin_memory()
    hpool = pbit.host_pool(h_next, h_key)
    ws_h = pbit.alloc_workspace(pbit.workspace_size_host(hpool, tune))
    del ws
    torch.cuda.empty_cache()
    e2e_times = []
    for i in range(a.warmup + a.steps):
        h_next.copy_(h_next0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, r = pbit.sort_pool_list_host(hpool, root, n, M, 4, ws=ws_h, stream=stream, check=False, tune=tune)
        dt = time.perf_counter() - t0
        if st != pbit.OK:
            raise pbit.PbitError(st, "bench e2e step")
        if i >= a.warmup:
            e2e_times.append(dt)
    e2e_value, _ = whole_job_rate(a.steps * n, sum(e2e_times), world, "cuda")

    if rank != 0:
        if world > 1:
            tdist.destroy_process_group()
        return
    # ---- roofline of the dominant kernel (largest share of device time), and
    # of the MSD pass kernel (the non-gather sort pass)
    peak, peak_kind = peaks()

    def roofline(name):
        s = kernel_stats.get(name)
        if not s or not s["ms"]:
            return None
        per_launch_ms = s["ms"] / max(1, s["launches"])
        achieved = s["bytes"] / (s["ms"] / 1e3) / 1e9
        traffic = traffic_for(name, s["launches"] / a.steps, a.log2n) if a.key_bits == 32 else None
        alg = s["bytes"] / max(1, s["launches"])
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind}", "traffic": traffic,
                "dram_frac": (traffic / (per_launch_ms / 1e3) / 1e9 / peak) if traffic else None,
                # algorithmic bytes / DRAM bytes: below 1 for random gathers (a
                # DRAM access moves far more than the 8-byte record it serves)
                "sector_efficiency": (alg / traffic) if traffic else None,
                "alg_bytes_per_launch": alg,
                "launches": s["launches"], "ms_total": s["ms"]}

    def roofline_msd():
        """The non-gather stages together: every MSD pass with its per-segment
        statistics and planning, and both finishes, against the algorithmic
        bytes of the passes and the finishes (the statistics' extra key reads
        and the planning count as overhead, not as work)."""
        parts = ("pass", "finish", "seg_stats", "plan", "scan")
        ms = sum(kernel_stats[k]["ms"] for k in parts if k in kernel_stats)
        alg = sum(kernel_stats[k]["bytes"] for k in ("pass", "finish") if k in kernel_stats)
        if not ms:
            return None
        achieved = alg / (ms / 1e3) / 1e9
        return {"kernels": list(parts), "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                "alg_bytes_per_step": alg / a.steps, "ms_per_step": ms / a.steps}

    dom = max(kernel_stats.items(), key=lambda kv: kv[1]["ms"])[0] if kernel_stats else None
    roof = roofline(dom) if dom else None
    roof_pass = roofline("pass")
    per_kernel = {k: {"ms_per_step": v["ms"] / a.steps, "GB/s": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] else None,
                      "share": v["ms"] / sum(x["ms"] for x in kernel_stats.values())}
                  for k, v in kernel_stats.items()}
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        m, dt = oracle_sample(a.cpu_sample_log2n, 0x0511020 + 2, a.key_bits)
        cpu = {"value": m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the oracle (single-threaded literal Pbit) on one 2^{a.cpu_sample_log2n}-node list "
                         f"of the same recipe ({dt:.1f} s); it stands in for the 2^{a.log2n}-node list, whose "
                         f"literal sort (one pointer-chasing pass per level over every node) would add "
                         f"~{dt * (1 << (a.log2n - a.cpu_sample_log2n)) * 1.1:.0f} s to the default run",
               "k_sweep_ms": oracle_k_sweep()}
    del d_next0, d_next, d_key, ws_h, h_next0, h_next, h_key
    torch.cuda.empty_cache()
    batched = None if (a.no_batched or world > 1) else run_batched(a, torch, pbit, I, local)
    torch.cuda.empty_cache()
    serve = None if (a.no_serve or world > 1) else run_serve(a, torch, pbit, I, local)
    torch.cuda.empty_cache()
    k_sweep = None if world > 1 else run_k_sweep(a, torch, pbit, I)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": tot_ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": dict(workload(a.log2n, a.key_bits, a.digit_bits), parallelism=("replicas" if world > 1 else "single GPU"),
                       timing="device time per step from two CUDA events on the launching stream around the "
                              "sort call; next[] restored from a device copy before each step, outside the "
                              "events; per-kernel figures from a second, profiled run of the same steps"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 4 * n + 8,
                "api": "pbit_sort_list_host (pinned host next/key, copies inside the call)"},
        "gpu_launches": launches_per_step * a.steps,
        "roofline": roof,
        "roofline_sort_pass": roof_pass,
        "roofline_msd_finish": roofline_msd(),
        "kernels": per_kernel,
        "cpu_baseline": cpu,
        "batched": batched,
        "serve": serve,
        "k_sweep": k_sweep,
        "clocks": clocks,
        "wall_s": wall,
    }
    print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()


def run_batched(a, torch, pbit, I, local=0):
    """Batched workload: 4096 lists in one pool, lengths log-uniform in
    [16, 2^20], uint32 keys, random order per list, M=32, K=4.  The batch is
    autotuned (digit width x shared-memory cutoff x ruler stride), captured
    once as a CUDA graph and replayed; the same lists are then sorted one
    pbit_sort_list call at a time (the plain per-list path, with the same
    tune).  Both paths are timed on both clocks: CUDA events on the stream
    around the whole step, and the host wall clock around launch + result."""
    gen = torch.Generator(device="cuda").manual_seed(I.SEED_BASE + 4)
    lens = I.config4_lengths(I.SEED_BASE + 4, a.batched_lists)
    d_next0, d_key, d_roots, d_off = I.device_batched_pool(lens, 4, gen)
    total = int(lens.sum())
    d_next = d_next0.clone()
    pool = pbit.make_pool(d_next, d_key)
    best, tune_ms = pbit.autotune_batched(pool, d_roots, d_off, 32, 4, reps=2)
    g = pbit.Graph.batched(pool, d_roots, d_off, 32, 4)  # tune = NULL: the autotuned choice
    stream = torch.cuda.current_stream()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    for _ in range(a.warmup):
        d_next.copy_(d_next0)
        g.launch(stream)
        g.result(stream)
    clk = Clocks(local)
    graph_wall = []
    for i in range(a.steps):
        d_next.copy_(d_next0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0[i].record(stream)
        g.launch(stream)
        e1[i].record(stream)
        g.result(stream)  # status of this replay (synchronizes; raises on an error)
        graph_wall.append(time.perf_counter() - t0)
    clocks = clk.stop()
    graph_ms = [e0[i].elapsed_time(e1[i]) for i in range(a.steps)]
    gm = statistics.median(graph_ms)
    gw = 1e3 * statistics.median(graph_wall)

    # the plain per-list path: one synchronous pbit_sort_list per list, in
    # order, each on its own slice of the pool with list-local indices
    off = d_off.cpu().numpy()
    lid = torch.repeat_interleave(torch.arange(lens.size, device="cuda"), torch.as_tensor(lens, device="cuda"))
    base = d_off[:-1][lid].to(torch.int32)
    loc0 = torch.where(d_next0 >= 0, d_next0 - base, d_next0)
    loc = loc0.clone()
    roots_loc = (d_roots - d_off[:-1].to(torch.int32)).cpu().numpy()
    tune = {k: best[k] for k in ("digit_bits", "smem_cutoff", "ruler_stride")}
    ws = pbit.alloc_workspace(pbit.workspace_size(int(lens.max()), 1, 4, tune))
    pools = [pbit.Pool(loc.data_ptr() + 4 * int(off[i]), 4, d_key.data_ptr() + 4 * int(off[i]), 4, 4, 0,
                       int(lens[i]), 0, 0) for i in range(lens.size)]
    fifo_wall, fifo_ev = [], []
    for rep in range(2):
        loc.copy_(loc0)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        f0.record(stream)
        for i in range(lens.size):
            st, _ = pbit.sort_pool_list(pools[i], int(roots_loc[i]), int(lens[i]), 32, 4, ws=ws, tune=tune,
                                        stream=stream, check=False)
            if st != pbit.OK:
                raise pbit.PbitError(st, "per-list sort")
        f1.record(stream)
        torch.cuda.synchronize()
        fifo_wall.append(1e3 * (time.perf_counter() - t0))
        fifo_ev.append(f0.elapsed_time(f1))
    # both paths give the same next[] (list-local vs pool indices)
    same = bool(torch.equal(torch.where(loc >= 0, loc + base, loc), d_next))
    fw, fe = min(fifo_wall), min(fifo_ev)
    out = {"workload": f"{lens.size} lists in one SoA pool, lengths log-uniform in [16, 2^20] (seeded), "
                       "uint32 keys uniform, random order per list, M=32, K=4",
           "nodes": total, "lists": int(lens.size),
           "graph": {"value": total / (gm / 1e3), "unit": UNIT, "ms_per_step": gm, "wall_ms_per_step": gw,
                     "steps": a.steps, "graph_nodes": g.node_count(),
                     "timing": "median over the steps; ms_per_step: CUDA events around each graph replay; "
                               "wall_ms_per_step: host clock around launch + status read-back; next[] restored "
                               "before, outside both",
                     "structure": "one graph launch per step; its nodes are the memsets and kernels of one "
                                  "batched sort, each stage a persistent, segmented kernel over all lists"},
           "per_list": {"value": total / (fe / 1e3), "unit": UNIT, "ms": fe, "wall_ms": fw,
                        "timing": "best of 2 loops over all lists; ms: CUDA events before the first and after the "
                                  "last call; wall_ms: host clock over the loop of synchronous calls"},
           "speedup_vs_per_list": {"events": fe / gm, "wall": fw / gw},
           "same_result": same, "clocks": clocks,
           "autotuned": {**best, "median_ms": tune_ms,
                         "searched": {"digit_bits": [4, 8], "smem_cutoff": [128, 256, 512],
                                      "ruler_stride": [16, 32, 64, 128]}}}
    g.close()
    if not a.no_cpu_baseline:
        out["cpu_baseline_all_cores"] = oracle_batched_sample(lens, a.cpu_batched_lists)
    return out


def oracle_batched_sample(lens, count):
    """The oracle on every host core at once: `count` lists of the batched
    workload (evenly spaced through the 4096, so their lengths span the
    range), one list per thread at a time (the C oracle runs outside the
    Python lock), nodes / wall time."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    from paper_cs_0511020_gb300 import inputs as I
    cores = len(os.sched_getaffinity(0))
    pick = np.linspace(0, lens.size - 1, count).astype(np.int64)
    lists = []
    for j in pick:
        n = int(lens[j])
        nxt, root = I.random_list(n, I.SEED_BASE + 40000 + int(j))
        lists.append((nxt, I.uniform_keys(n, 4, I.SEED_BASE + 50000 + int(j)), root))
    O.lib()
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(lambda x: O.pbit_sort(x[0], x[1], x[2], 32, 4), lists))
    dt = time.perf_counter() - t0
    nodes = int(sum(int(lens[j]) for j in pick))
    return {"value": nodes / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{count} of the {lens.size} lists (evenly spaced, {nodes} nodes), the oracle on "
                      f"{cores} threads ({dt:.1f} s)"}


def run_serve(a, torch, pbit, I, local=0):
    """Serving workload: open-loop Poisson arrivals, lengths log-uniform in
    [2^4, 2^24], key widths 2/4/8 bytes in 1:2:1 (M = 8 x width), uniform keys,
    random order, pools resident on the device, 16 GB admission budget.  Two
    traces: the request rate of the workload (mean gap 0.5 ms) and a
    saturating one (mean gap 0.1 ms, above what either arm can serve).  Each
    runs `--serve-requests` timed requests after `--serve-warmup` through a
    ring of `--serve-pools` device pools: request i sorts pool i mod P, and a
    pool is restored from its saved next[] on a side stream as soon as its
    request completes (before its next use; the copies share the GPU with the
    sorts in both arms).  Served arm: pbit_serve_*; FIFO arm: one synchronous
    pbit_sort_list call per request, in arrival order.  Latency = completion
    (seen by the scheduler, or the synchronous call's return) minus the
    scheduled arrival, host monotonic clock; throughput = nodes of the timed
    requests / (last completion - first timed arrival)."""
    W, N = a.serve_warmup, a.serve_requests
    R = W + N
    P = min(a.serve_pools, R)
    _, lens, kbs = I.config5_requests(P, I.SEED_BASE + 5)
    gen = torch.Generator(device="cuda").manual_seed(I.SEED_BASE + 5)
    pools = []
    for p in range(P):
        n, kb = int(lens[p]), int(kbs[p])
        nxt, root = I.device_random_list(n, gen)
        key = I.device_keys(n, kb, gen)
        pools.append({"next": nxt, "next0": nxt.clone(), "key": key, "root": root, "n": n, "kb": kb,
                      "pool": pbit.make_pool(nxt, key), "ready": None})
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    tune = {"digit_bits": 8}
    ws = pbit.alloc_workspace(max(pbit.workspace_size(1 << 24, 1, kb, tune) for kb in (2, 4, 8)))
    stream = torch.cuda.current_stream()

    def restore(p):
        pl = pools[p]
        ev = torch.cuda.Event()
        with torch.cuda.stream(side):
            pl["next"].copy_(pl["next0"])
            ev.record(side)
        pl["ready"] = ev

    def summarize(lat_ns, t_first, t_last, req_lens):
        lat = np.array(lat_ns, dtype=np.float64) / 1e6
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "value": float(sum(req_lens)) / ((t_last - t_first) / 1e9),
                "unit": UNIT}

    def served_arm(sched):
        srv = pbit.Server(mem_budget_bytes=16 << 30, streams=4, max_batch=64, tune=tune)
        tickets, done = [None] * R, [0] * R
        oldest = 0  # first request whose completion has not been seen
        next_poll = 0
        for i in range(R):
            p = i % P
            if i >= P and done[i - P] == 0:  # the ring came round before the pool's request finished
                st, _ = srv.wait(tickets[i - P], 600000)
                if st != pbit.OK:
                    raise pbit.PbitError(st, "served request")
                done[i - P] = srv.times(tickets[i - P])[1]
                restore(p)
            while True:  # until the arrival time: note completions and restore their pools
                while oldest < i and done[oldest]:
                    oldest += 1
                now = time.monotonic_ns()
                if oldest < i and now >= next_poll:  # (polls spaced out: the server's lock is shared)
                    next_poll = now + 20_000
                    st, _ = srv.poll(tickets[oldest])
                    if st != pbit.EPENDING:
                        if st != pbit.OK:
                            raise pbit.PbitError(st, "served request")
                        done[oldest] = srv.times(tickets[oldest])[1]
                        restore(oldest % P)
                        next_poll = 0
                        continue
                if now >= sched[i]:
                    break
            pl = pools[p]
            if pl["ready"] is not None:
                pl["ready"].synchronize()
                pl["ready"] = None
            tickets[i] = srv.submit(pl["pool"], pl["root"], pl["n"], 8 * pl["kb"], 4)
        for i in range(R):
            if done[i] == 0:
                st, _ = srv.wait(tickets[i], 600000)
                if st != pbit.OK:
                    raise pbit.PbitError(st, "served request")
                done[i] = srv.times(tickets[i])[1]
        stats = srv.stats()
        srv.close()
        return done, stats

    def fifo_arm(sched):
        done = [0] * R
        for i in range(R):
            p = i % P
            pl = pools[p]
            if pl["ready"] is not None:
                pl["ready"].synchronize()
                pl["ready"] = None
            while time.monotonic_ns() < sched[i]:
                pass
            st, _ = pbit.sort_pool_list(pl["pool"], pl["root"], pl["n"], 8 * pl["kb"], 4, ws=ws, tune=tune,
                                        stream=stream, check=False)
            if st != pbit.OK:
                raise pbit.PbitError(st, "FIFO request")
            done[i] = time.monotonic_ns()
            restore(p)
        return done

    out = {"workload": "open-loop Poisson arrivals; lengths log-uniform in [2^4, 2^24]; uint16/uint32/uint64 "
                       "keys 1:2:1, M = 8 x width, K = 4 (GPU digit width 8 by tune in both arms); random order; "
                       "uniform keys; 16 GB admission budget, 4 streams, batches of up to 64",
           "requests": N, "warmup_requests": W, "pools": P,
           "latency": "completion seen by the scheduler (served) or after the synchronous call returns (FIFO) "
                      "minus the scheduled arrival, host monotonic clock",
           "throughput": "nodes of the timed requests / (last completion - first timed arrival)"}
    for name, gap in (("rate_2000_per_s", 0.5e-3), ("saturating_10000_per_s", 0.1e-3)):
        arr = np.cumsum(I.rng(I.SEED_BASE + 50 + int(gap * 1e5)).exponential(gap, R))
        req_lens = [int(lens[i % P]) for i in range(W, R)]
        for pl in pools:
            pl["next"].copy_(pl["next0"])
            pl["ready"] = None
        torch.cuda.synchronize()
        clk = Clocks(local)
        t0 = time.monotonic_ns() + 20_000_000
        sched = [t0 + int(x * 1e9) for x in arr]
        done, stats = served_arm(sched)
        clocks = clk.stop()
        served = summarize([done[i] - sched[i] for i in range(W, R)], sched[W], max(done[W:]), req_lens)
        for pl in pools:
            pl["next"].copy_(pl["next0"])
            pl["ready"] = None
        torch.cuda.synchronize()
        t0 = time.monotonic_ns() + 20_000_000
        sched = [t0 + int(x * 1e9) for x in arr]
        fdone = fifo_arm(sched)
        fifo = summarize([fdone[i] - sched[i] for i in range(W, R)], sched[W], max(fdone[W:]), req_lens)
        out[name] = {"mean_gap_ms": gap * 1e3,
                     "offered_nodes_per_s": float(sum(req_lens) / (arr[-1] - arr[W])),
                     "served": {**served, "batches": stats["batches"], "max_batch": stats["max_batch"],
                                "peak_workspace_bytes": stats["peak_bytes"], "clocks": clocks},
                     "fifo_per_list": fifo,
                     "served_over_fifo_throughput": served["value"] / fifo["value"]}
    return out


K_SWEEP = (1, 2, 4, 8, 16)


def run_k_sweep(a, torch, pbit, I):
    """The paper's digit width K (its Sec. on the length of the bit pattern)
    swept on the GPU: one 2^24-node uint32 list, M=32, median of 5 sorts per
    K.  The result is K-independent and so is the GPU's work (its own digit
    width is fixed); the literal oracle's time per K is in cpu_baseline."""
    n = 1 << 24
    gen = torch.Generator(device="cuda").manual_seed(I.SEED_BASE + 24)
    d_next0, root = I.device_random_list(n, gen)
    d_key = I.device_keys(n, 4, gen)
    d_next = d_next0.clone()
    pool = pbit.make_pool(d_next, d_key)
    ws = pbit.alloc_workspace(pbit.workspace_size(n, 1, 4))
    stream = torch.cuda.current_stream()
    out = {}
    for K in K_SWEEP:
        t = []
        for rep in range(6):
            d_next.copy_(d_next0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pbit.sort_pool_list(pool, root, n, 32, K, ws=ws, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep:
                t.append(e0.elapsed_time(e1))
        out[str(K)] = statistics.median(t)
    return {"workload": "one 2^24-node SoA uint32 list, random order, uniform keys, M=32", "gpu_ms": out}


def oracle_k_sweep():
    """The literal oracle's time per K on one 2^18-node list (it visits every
    node M/K times: the paper's K experiment)."""
    from oracle import oracle as O
    from paper_cs_0511020_gb300 import inputs as I
    n = 1 << 18
    nxt, root = I.random_list(n, 0x0511020 + 24)
    key = I.uniform_keys(n, 4, 0x0511020 + 25)
    res = {}
    for K in K_SWEEP:
        t0 = time.perf_counter()
        O.pbit_sort(nxt, key, root, 32, K)
        res[str(K)] = 1e3 * (time.perf_counter() - t0)
    return {"n": n, "M": 32, "ms": res}


def traffic_for(name, launches_per_step, log2n):
    """DRAM bytes per launch from the committed ncu capture (profiles/traffic.json:
    the kernel kind's DRAM bytes in one sort), if it was taken on the current
    source of that kernel and on this list size; else None."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
    except Exception:
        return None
    e = t.get(name)
    if not e or e.get("log2n") != log2n:
        return None
    src = os.path.join(ROOT, "paper_cs_0511020_gb300", "csrc", e["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if h != e.get("source_sha") or not launches_per_step:
        return None
    return e["dram_bytes_total"] / launches_per_step


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
