"""Request queue with continuous batching (GPU).

Requests of both kinds (uint32 keys; uint64 keys with uint32 payloads) are
submitted together; every result must be bit for bit the sort the request
gets alone through mps_sort_keys / mps_sort_pairs, with the same merge cost.  Failures are made on the
host: an over-budget request, a malformed request, a wait that runs out while
admission is paused, and destroy with requests still pending.
"""
import threading

import numpy as np
import pytest
import torch

from paper_2209_06909_gb300 import inputs
from paper_2209_06909_gb300 import mps

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2209_06909_gb300 import build
    build.build()


def make_requests(seed, count):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(2 ** rng.uniform(4, 17)) if i % 7 else int(rng.integers(0, 3))
        kind = "keys" if i % 2 == 0 else "pairs"
        if kind == "keys":
            a = inputs.random_runs_loguniform(n, int(rng.integers(1 << 40)), log2_hi=10.0, distinct=1000,
                                              dtype=np.uint32) if n else np.zeros(0, np.uint32)
            reqs.append(("keys", a, None))
        else:
            a = inputs.random_runs_loguniform(n, int(rng.integers(1 << 40)), log2_hi=10.0, distinct=1000,
                                              dtype=np.uint64) if n else np.zeros(0, np.uint64)
            reqs.append(("pairs", a, np.arange(n, dtype=np.uint32)))
    return reqs


def alone(kind, a, v, k=4):
    """The request's sort and merge cost through the single-array calls."""
    if a.size == 0:
        return a, v, 0
    if kind == "keys":
        ok = mps.to_numpy(mps.sort_keys(mps.to_device(a, DEV), k=k), a.dtype)
        return ok, None, mps.last_stats()["merge_cost"]
    ok, ov = mps.sort_pairs(mps.to_device(a, DEV), mps.to_device(v, DEV), k=k)
    return mps.to_numpy(ok, a.dtype), mps.to_numpy(ov, np.uint32), mps.last_stats()["merge_cost"]


@pytest.mark.parametrize("k", [4, 2, 16])
def test_mixed_requests_match_alone(k):
    reqs = make_requests(1 + k, 80 if k == 4 else 40)
    pool = torch.empty(256 << 20, dtype=torch.uint8, device=DEV)
    q = mps.Queue(pool, max_inflight=3, max_batch=16, k=k)
    bufs, tickets = [], []
    lock = threading.Lock()

    def client(part):
        for i in part:
            kind, a, v = reqs[i]
            d_in = mps.to_device(a, DEV)
            d_out = torch.empty_like(d_in)
            if kind == "keys":
                t = q.submit(d_in, d_out, tag=i)
                with lock:
                    bufs.append((i, d_out, None))
                    tickets.append(t)
            else:
                dv = mps.to_device(v, DEV)
                dvo = torch.empty_like(dv)
                t = q.submit(d_in, d_out, dv, dvo, tag=i)
                with lock:
                    bufs.append((i, d_out, dvo))
                    tickets.append(t)

    torch.cuda.synchronize()
    threads = [threading.Thread(target=client, args=(range(j, len(reqs), 4),)) for j in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    results = {}
    for t in tickets:
        r = q.wait(t, timeout_ms=60000)
        assert r["status"] == 0, r
        assert r["t_submit_ms"] <= r["t_admit_ms"] <= r["t_done_ms"]
        results[r["tag"]] = r
    q.close()
    assert len(results) == len(reqs)
    for i, d_out, dvo in bufs:
        kind, a, v = reqs[i]
        wk, wv, wcost = alone(kind, a, v, k)
        assert np.array_equal(mps.to_numpy(d_out, a.dtype), wk), i
        assert results[i]["merge_cost"] == wcost, i
        if kind == "pairs":
            assert np.array_equal(mps.to_numpy(dvo, np.uint32), wv), i


def test_batch_of_empty_requests():
    """A batch with nothing to sort completes with status 0 (reused pool memory
    holds stale data)."""
    pool = torch.full((32 << 20,), 255, dtype=torch.uint8, device=DEV)
    q = mps.Queue(pool, max_batch=8)
    e = torch.empty(0, dtype=torch.int32, device=DEV)
    ts = [q.submit(e, torch.empty_like(e)) for _ in range(5)]
    for t in ts:
        assert q.wait(t)["status"] == 0
    q.close()


def test_budget_and_malformed_requests():
    pool = torch.empty(1 << 20, dtype=torch.uint8, device=DEV)
    q = mps.Queue(pool)
    big = torch.zeros(1 << 20, dtype=torch.int32, device=DEV)
    with pytest.raises(mps.MpsError) as e:
        q.submit(big, torch.empty_like(big))
    assert e.value.code == 6  # MPS_ERR_BUDGET
    req = mps.Request(0, 0, 10, None, None, None, None, 0)
    t = mps.ctypes.c_uint64(0)
    assert mps.lib().mps_queue_submit(q.handle, mps.ctypes.byref(req), mps.ctypes.byref(t)) == 1
    q.close()


def test_wait_times_out_while_paused_then_completes():
    pool = torch.empty(64 << 20, dtype=torch.uint8, device=DEV)
    q = mps.Queue(pool)
    q.pause(True)
    a = inputs.random_permutation(5000, 3)
    d_in = mps.to_device(a, DEV)
    d_out = torch.empty_like(d_in)
    t = q.submit(d_in, d_out)
    with pytest.raises(mps.MpsError) as e:
        q.wait(t, timeout_ms=200)
    assert e.value.code == 5  # MPS_ERR_TIMEOUT
    q.pause(False)
    r = q.wait(t, timeout_ms=60000)
    assert r["status"] == 0
    assert np.array_equal(mps.to_numpy(d_out, np.uint32), np.arange(5000, dtype=np.uint32))
    q.close()


def test_destroy_cancels_pending():
    pool = torch.empty(64 << 20, dtype=torch.uint8, device=DEV)
    q = mps.Queue(pool)
    q.pause(True)
    d_in = mps.to_device(inputs.random_permutation(1000, 4), DEV)
    d_out = torch.full_like(d_in, -1)
    q.submit(d_in, d_out)
    q.close()  # returns without running the paused request
    torch.cuda.synchronize()
    assert int(d_out[0].item()) == -1
