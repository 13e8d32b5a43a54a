"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Weak scaling with no collective on the data path: every rank sorts its own
independent array; the job's time is the maximum of the ranks' timed regions
(one all_reduce MAX) and its throughput counts the keys of all ranks.  The
reference arm under torchrun runs on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        ms = bench.job_time_ms(local_ms, dist)
        n = 1 << 20
        seed = bench.rank_seed(rank)
        a = bench.gen_input("perm", 4096, seed)
        res = {"rank": rank, "ms": ms, "value": bench.job_value(n, world, ms), "seed": seed,
               "head": a[:16].tolist()}
        dist.barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)


def test_job_time_is_max_over_ranks_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rs = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    assert [r["ms"] for r in rs] == [15.0, 15.0]
    want = world * (1 << 20) / 15e-3 / 1e9
    assert all(abs(r["value"] - want) < 1e-9 for r in rs)
    assert rs[0]["seed"] != rs[1]["seed"]
    assert rs[0]["head"] != rs[1]["head"]  # independent arrays


def test_single_rank_needs_no_process_group():
    assert bench.job_time_ms(12.5) == 12.5
    assert bench.job_value(1 << 28, 1, 1000.0) == pytest.approx((1 << 28) / 1e9)


def test_inputs_differ_per_rank_and_are_permutations():
    a0 = bench.gen_input("perm", 1 << 12, bench.rank_seed(0))
    a1 = bench.gen_input("perm", 1 << 12, bench.rank_seed(1))
    assert np.array_equal(np.sort(a0), np.arange(1 << 12)) and np.array_equal(np.sort(a1), np.arange(1 << 12))
    assert not np.array_equal(a0, a1)


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0", "--ref-sample-log2", "12"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [json.loads(x) for x in res.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
