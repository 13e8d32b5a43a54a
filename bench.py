#!/usr/bin/env python
"""Benchmark of the GB300 Multiway Powersort (arXiv 2209.06909).

Workload (one step = one complete sort through the C ABI): a single array of
n = 2^28 uint32 keys, a uniform random permutation of 0..n-1, fan-in k = 4;
keys resident in HBM before the timed region (1 GiB of input, larger than the
129 MB L2, so no flush is needed between steps).  Also reported on the same
line: the geometric random-runs input (mean run length 2^14) and k = 2 for
both inputs (fewer steps each), the end-to-end time from pinned host memory
through mps_sort_keys_host, the roofline of the dominant kernel, and the CPU
oracle timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mps|reference]

With N > 1 (launched by torchrun) every rank sorts its own independent array
(weak scaling, no collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 1 << 28
GEOM_MEAN = float(1 << 14)
NOMINAL_HBM_GBS = 8000.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mps", "reference"], default="mps")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--no-variants", action="store_true", help="skip the secondary inputs and fan-ins")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.1)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ helpers

def gen_input(kind, n, seed):
    from paper_2209_06909_gb300 import inputs
    if kind == "perm":
        return inputs.random_permutation(n, seed)
    return inputs.random_runs_geometric(n, seed, mean=GEOM_MEAN)


def time_sorts(mps, torch, d_in, d_out, ws, k, steps, warmup, stream, barrier=None):
    for _ in range(warmup):
        mps.sort_keys(d_in, k=k, out=d_out, ws=ws, stream=stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(steps):
        mps.sort_keys(d_in, k=k, out=d_out, ws=ws, stream=stream)
    end.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return start.elapsed_time(end) / steps


def cpu_baseline(n_sample, seed):
    """The oracle as it stands (single thread), timed on a bounded sample of the
    same workload (a random permutation of n_sample keys, k = 4)."""
    import oracle
    a = gen_input("perm", n_sample, seed)
    oracle.sort(a[:4096], k=4, want_tree=False)
    t0 = time.perf_counter()
    res = oracle.sort(a, k=4, want_tree=False)
    dt = time.perf_counter() - t0
    assert np.array_equal(res["keys"], np.arange(n_sample, dtype=np.uint32))
    return {"value": n_sample / dt / 1e9, "unit": "GKeys/s", "cores": 1, "kind": "oracle",
            "sample": f"one sort of a random permutation of 2^{int(math.log2(n_sample))} uint32 keys, k=4, "
                      f"{dt:.1f} s on one host core (nproc={os.cpu_count()})"}


# ------------------------------------------------------------------ arms

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n_sample = 1 << 21
    a = gen_input("perm", n_sample, 1234)
    for _ in range(args.warmup):
        oracle.sort(a, k=args.k, want_tree=False)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sort(a, k=args.k, want_tree=False)
        times.append(time.perf_counter() - t0)
    sec = float(np.mean(times))
    value = n_sample / sec / 1e9
    line = {"impl": "reference", "metric": "sorted_keys_per_second", "value": value, "unit": "GKeys/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "single-array sort, uint32 keys, uniform random permutation, k=%d "
                                   "(oracle steps sort a 2^21-key sample)" % args.k,
                       "n": n_sample, "k": args.k, "input": "random permutation"},
            "cpu_baseline": {"value": value, "unit": "GKeys/s", "cores": 1, "kind": "oracle",
                             "sample": "random permutation of 2^21 uint32 keys per step, one host core"},
            "e2e": {"value": value, "unit": "GKeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_mps(args):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
        barrier = lambda: dist.barrier(device_ids=[local])
    else:
        barrier = None

    from paper_2209_06909_gb300 import build, mps
    build.build()
    mps.lib()
    peaks, peak_src = measured_peaks()
    n, k = args.n, args.k
    stream = torch.cuda.current_stream(dev)

    a = gen_input("perm", n, 1000 + rank)
    d_in = mps.to_device(a, dev)
    d_out = torch.empty_like(d_in)
    ws = mps.workspace(n, 4, False, max(k, 2), dev)
    ws2 = mps.workspace(n, 4, False, 2, dev) if (not args.no_variants and k != 2) else ws

    # correctness spot check of this exact configuration (outside the timed region)
    mps.sort_keys(d_in, k=k, out=d_out, ws=ws, stream=stream)
    torch.cuda.synchronize()
    assert torch.equal(d_out, torch.arange(n, dtype=torch.int32, device=dev)), "sorted output is not 0..n-1"
    stats = mps.last_stats()

    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    clocks = None
    for attempt in range(2):
        sampler = ClockSampler(bus)
        mps.profile_enable(False)
        for _ in range(args.warmup):
            mps.sort_keys(d_in, k=k, out=d_out, ws=ws, stream=stream)
        torch.cuda.synchronize()
        sampler.start()
        mps.profile_enable(True)
        ms = time_sorts(mps, torch, d_in, d_out, ws, k, args.steps, 0, stream, barrier)
        prof = mps.profile_read()
        mps.profile_enable(False)
        clocks = sampler.stop()
        bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"} & set(clocks["reasons"])
        if not bad:
            break
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    value = world * n / (ms * 1e-3) / 1e9
    b = 4.0
    b_alg = b * (n + 2.0 * stats["merge_cost"])
    # dominant kernel: largest share of the timed region
    prof.sort(key=lambda e: -e["total_ms"])
    dom = prof[0]
    per_launch_ms = dom["total_ms"] / dom["launches"]
    achieved = dom["bytes"] / dom["launches"] / (per_launch_ms * 1e-3) / 1e9
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tf):
        with open(tf) as f:
            tj = json.load(f)
        src_sha = subprocess.run(["git", "-C", ROOT, "hash-object", os.path.join(ROOT, "paper_2209_06909_gb300", "csrc",
                                                                             "merge.cu")],
                                 capture_output=True, text=True).stdout.strip()
        ent = tj.get(dom["name"])
        if ent and ent.get("merge_cu_sha") == src_sha and ent.get("n") == n and ent.get("k") == k:
            traffic = ent["bytes_per_launch"]
    roofline = {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "peak_source": peak_src,
                "algorithmic_bytes_per_launch": dom["bytes"] / dom["launches"],
                "avg_launch_ms": per_launch_ms}
    kernels = [{"name": e["name"], "launches_per_step": e["launches"] / args.steps,
                "ms_per_step": e["total_ms"] / args.steps,
                "share": e["total_ms"] / sum(x["total_ms"] for x in prof)} for e in prof]

    line = {"metric": "sorted_keys_per_second", "value": value, "unit": "GKeys/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "single-array sort, n=2^28 uint32 keys, uniform random permutation, k=%d" % k,
                       "n": n, "k": k, "input": "random permutation", "per_gpu_arrays": 1,
                       "l2": "input 1 GiB > 129 MB L2 (no flush needed)"},
            "clocks": clocks, "gpu_launches": int(stats["launches"]) * args.steps,
            "roofline": roofline,
            "sort_roofline": {"b_alg_bytes": b_alg, "merge_cost_per_n": stats["merge_cost"] / n,
                              "frac_of_measured": b_alg / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                              "frac_of_8tbs": b_alg / (ms * 1e-3) / 1e9 / NOMINAL_HBM_GBS,
                              "levels_x2nb_bytes": 2.0 * n * b * stats["num_levels"]},
            "kernels": kernels,
            "tree": {"runs": stats["r"], "levels": stats["num_levels"], "level_merge_levels": stats["hbm_levels"],
                     "fused_subtrees": stats["frontier_nodes"], "level_nodes": stats["hbm_nodes"]}}

    if rank == 0:
        # end to end through the C ABI from pinned host memory
        h_in = torch.from_numpy(a.view(np.int32)).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        d_tmp = torch.empty_like(d_in)
        mps.sort_keys_host(h_in, h_out, d_tmp, d_out, ws, k=k, stream=stream)
        e2e_steps = 4
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            mps.sort_keys_host(h_in, h_out, d_tmp, d_out, ws, k=k, stream=stream)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        assert np.array_equal(h_out.numpy()[:1024].view(np.uint32), np.arange(1024, dtype=np.uint32))
        line["e2e"] = {"value": n / e2e_s / 1e9, "unit": "GKeys/s", "h2d_bytes_per_step": n * 4,
                       "d2h_bytes_per_step": n * 4, "ms_per_step": e2e_s * 1e3}
        del h_in, h_out, d_tmp

        if not args.no_variants:
            variants = []
            b_runs = gen_input("runs", n, 2000)
            d_runs = mps.to_device(b_runs, dev)
            for kind, dsrc in (("perm", d_in), ("runs", d_runs)):
                for kk in sorted({k, 2}):
                    if kind == "perm" and kk == k:
                        continue
                    w = ws if kk == k else ws2
                    vms = time_sorts(mps, torch, dsrc, d_out, w, kk, 8, 3, stream)
                    st = mps.last_stats()
                    ba = b * (n + 2.0 * st["merge_cost"])
                    variants.append({"input": "random permutation" if kind == "perm" else
                                     "geometric runs, mean 2^14", "k": kk, "ms": vms,
                                     "gkeys_s": n / (vms * 1e-3) / 1e9, "merge_cost_per_n": st["merge_cost"] / n,
                                     "levels": st["num_levels"],
                                     "sort_frac_of_measured": ba / (vms * 1e-3) / 1e9 / peaks["hbm_gbs"]})
            line["variants"] = variants
            del d_runs
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(1 << 24, 1234)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier(device_ids=[local])
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_mps(args)


if __name__ == "__main__":
    sys.exit(main())
