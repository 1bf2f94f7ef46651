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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2n", type=int, default=27, help="list size (27 = the benchmark workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-log2n", type=int, default=24)
    return ap.parse_args()


def workload(log2n):
    return {"workload": f"pbit_sort_list: one 2^{log2n}-node list, SoA int32 next + uint32 key, "
                        "seeded random list order, uniform keys, M=32, K=4",
            "n": 1 << log2n, "key": "uint32", "layout": "SoA", "M": 32, "K": 4,
            "l2": "inputs (1 GiB at 2^27) larger than L2; no flush"}


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
        self.path = os.path.join(ROOT, "gpurun_out", f".clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
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


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(log2n, seed):
    from oracle import oracle as O
    from paper_cs_0511020_gb300 import inputs as I
    n = 1 << log2n
    nxt, root = I.random_list(n, seed)
    key = I.uniform_keys(n, 4, seed + 1)
    t0 = time.perf_counter()
    O.pbit_sort(nxt, key, root, 32, 4)
    dt = time.perf_counter() - t0
    return n, dt


def run_reference(a):
    ws, rank, _ = dist()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    log2n = min(22, a.log2n)
    times = []
    for i in range(a.warmup + a.steps):
        n, dt = oracle_sample(log2n, 0x0511020 + 2 + i)
        if i >= a.warmup:
            times.append(dt)
    tot = sum(times)
    value = a.steps * (1 << log2n) / tot
    sample = f"{a.steps} timed steps, each the oracle on one 2^{log2n}-node list of the same recipe"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload(a.log2n),
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
    seed = I.SEED_BASE + 2 + 7919 * rank
    nxt, root = I.random_list(n, seed)
    key = I.uniform_keys(n, 4, seed + 1)
    d_next0 = torch.from_numpy(nxt).cuda()
    d_next = d_next0.clone()
    d_key = torch.from_numpy(key.view(np.int32)).cuda()
    pool = pbit.make_pool(d_next, d_key)
    ws = pbit.alloc_workspace(pbit.workspace_size(n, 1, 4))
    stream = torch.cuda.current_stream()

    def step():
        d_next.copy_(d_next0)
        st, r = pbit.sort_pool_list(pool, root, n, 32, 4, ws=ws, stream=stream, check=False)
        if st != pbit.OK:
            raise pbit.PbitError(st, "bench step")
        return r

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    # Device time of a step = CUDA events the library records on the launching
    # stream: from before its first memset/kernel to after its last kernel.
    kernel_stats = {}
    step_ms = []
    pbit.profile_enable(True)
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    wall0 = time.perf_counter()
    for _ in range(a.steps):
        step()
        ks = pbit.profile_read()
        step_ms.append(sum(k["ms"] for k in ks))
        for k in ks:
            s = kernel_stats.setdefault(k["name"], {"launches": 0, "ms": 0.0, "bytes": 0.0})
            s["launches"] += k["launches"]
            s["ms"] += k["ms"]
            s["bytes"] += k["bytes"]
    torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    wall = time.perf_counter() - wall0
    clocks = clk.stop()
    pbit.profile_enable(False)
    launches_per_step = pbit.last_launch_count()
    tot_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([tot_ms], device="cuda")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = world * a.steps * n / (tot_ms / 1e3)

    # ---- end to end through the host-buffer C ABI call (pinned host memory)
    h_next0 = torch.from_numpy(nxt).pin_memory()
    h_next = h_next0.clone().pin_memory()
    h_key = torch.from_numpy(key.view(np.int32)).pin_memory()
    hpool = pbit.host_pool(h_next, h_key)
    ws_h = pbit.alloc_workspace(pbit.workspace_size_host(hpool))
    del ws
    torch.cuda.empty_cache()
    e2e_times = []
    for i in range(a.warmup + a.steps):
        h_next.copy_(h_next0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, r = pbit.sort_pool_list_host(hpool, root, n, 32, 4, ws=ws_h, stream=stream, check=False)
        dt = time.perf_counter() - t0
        if st != pbit.OK:
            raise pbit.PbitError(st, "bench e2e step")
        if i >= a.warmup:
            e2e_times.append(dt)
    e2e_tot = sum(e2e_times)
    if world > 1:
        t = torch.tensor([e2e_tot], device="cuda")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        e2e_tot = float(t.item())
    e2e_value = world * a.steps * n / e2e_tot

    if rank != 0:
        if world > 1:
            tdist.destroy_process_group()
        return
    # ---- roofline of the dominant kernel (largest share of device time)
    peak, peak_kind = peaks()
    dom = max(kernel_stats.items(), key=lambda kv: kv[1]["ms"]) if kernel_stats else None
    roof = None
    if dom:
        name, s = dom
        achieved = s["bytes"] / (s["ms"] / 1e3) / 1e9
        roof = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                "traffic": traffic_for(name, s["bytes"] / max(1, s["launches"]), a.log2n),
                "alg_bytes_per_launch": s["bytes"] / max(1, s["launches"]),
                "launches": s["launches"], "ms_total": s["ms"]}
    per_kernel = {k: {"ms_per_step": v["ms"] / a.steps, "GB/s": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] else None,
                      "share": v["ms"] / sum(x["ms"] for x in kernel_stats.values())}
                  for k, v in kernel_stats.items()}
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        m, dt = oracle_sample(a.cpu_sample_log2n, 0x0511020 + 2)
        cpu = {"value": m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the oracle (single-threaded literal Pbit) on one 2^{a.cpu_sample_log2n}-node list "
                         f"of the same recipe ({dt:.1f} s)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": tot_ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic",
        "config": dict(workload(a.log2n), parallelism=("replicas" if world > 1 else "single GPU"),
                       timing="device time per step from CUDA events recorded on the launching stream "
                              "around every kernel of the call; next[] restored from a device copy before "
                              "each step, outside the timed events"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 4 * n + 8,
                "api": "pbit_sort_list_host (pinned host next/key, copies inside the call)"},
        "gpu_launches": launches_per_step * a.steps,
        "roofline": roof,
        "kernels": per_kernel,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "wall_s": wall,
    }
    print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()


def traffic_for(name, alg_bytes, log2n):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of that kernel; else None."""
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
    return e["dram_bytes_per_launch"] if h == e.get("source_sha") else None


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
