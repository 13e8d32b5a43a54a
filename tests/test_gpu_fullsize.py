"""Parity at the full workload sizes, in the launch configuration bench.py
times (GPU): default workspace, k as timed, inputs from the same generators.

The oracle's sort is O(n log r) C, so it runs whole at these sizes except for
the 4096-array batch, where it sorts a sample of arrays and every array's
tree is still checked through its merge cost:
  * random permutation of 0..n-1 (n = 2^28, k = 4, 2, 8 and 16): the output is
    exactly 0..n-1; runs, powers, node table, leaf depths and merge cost equal
    the oracle's run scan and tree from run lengths;
  * geometric random runs (n = 2^28, mean 2^14, k = 4 and 2): keys and tree
    equal the oracle's; and at n = 2^31 + 4099 (k = 4) the tree, with the
    output checked for order, sum and xor;
  * pairs (n = 2^27, uint64 keys with 2^16 distinct values, payload = index):
    keys and payload order equal the oracle's;
  * records (n = 2^26, uint64 keys and uint64 payloads, runs of geometric
    mean sqrt(n)): keys equal the oracle's, payloads follow its order;
  * 4096-array batch: every 61st array equals the oracle's sort, every array is
    non-decreasing with the same sum and xor as its input, and the batch's
    merge cost is the sum of the oracle's per-array merge costs;
  * served stream (sizes log-uniform in [2^10, 2^24], both request kinds,
    64 GiB pool): every result through the queue equals the oracle's sort.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_06909_gb300 import inputs
from paper_2209_06909_gb300 import mps

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
N = 1 << 28


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2209_06909_gb300 import build
    build.build()
    oracle.build()


def check_tree(t, a, k):
    """Runs, powers, canonical node table, leaf depths and merge cost against
    the oracle's linear-time run scan and tree from run lengths."""
    rs, rd = oracle.find_runs(a)
    want = oracle.tree_from_lengths(np.diff(rs.astype(np.int64)), k)
    assert t["r"] == rs.size - 1
    assert np.array_equal(t["run_starts"], rs) and np.array_equal(t["run_desc"], rd)
    assert np.array_equal(t["powers"], want["powers"])
    assert t["num_nodes"] == want["num_nodes"] and np.array_equal(t["nodes"], want["nodes"])
    assert np.array_equal(t["node_first"], want["node_first"])
    assert np.array_equal(t["leaf_depth"], want["leaf_depth"])
    assert t["num_levels"] == want["num_levels"] and t["merge_cost"] == want["merge_cost"]


@pytest.mark.parametrize("k", [4, 2, 8, 16])
def test_permutation_2e28(k):
    a = inputs.random_permutation(N, 1000 + k)
    tb = mps.TreeBuffers.alloc(N, DEV)
    out = mps.sort_keys(mps.to_device(a, DEV), k=k, tree=tb)
    torch.cuda.synchronize()
    assert torch.equal(out, torch.arange(N, dtype=torch.int32, device=DEV))
    del out
    check_tree(tb.to_numpy(), a, k)


@pytest.mark.parametrize("k", [4, 2])
def test_geometric_runs_2e28(k):
    a = inputs.random_runs_geometric(N, 2000 + k, mean=float(1 << 14))
    tb = mps.TreeBuffers.alloc(N, DEV)
    out = mps.sort_keys(mps.to_device(a, DEV), k=k, tree=tb)
    torch.cuda.synchronize()
    got = mps.to_numpy(out, np.uint32)
    del out
    check_tree(tb.to_numpy(), a, k)
    want = oracle.sort(a, k=k, want_tree=False)
    assert np.array_equal(got, want["keys"])


def test_geometric_runs_above_2e31():
    """n = 2^31 + 4099 uint32 keys, past the size where 2n needs 33 bits (the
    power kernel's quotient), geometric runs of mean 2^14, k = 4: the output is
    non-decreasing with the input's sum and xor, and runs, powers, node table,
    leaf depths and merge cost equal the oracle's run scan and tree from run
    lengths."""
    n = (1 << 31) + 4099
    a = inputs.random_runs_geometric(n, 3100, mean=float(1 << 14))
    tb = mps.TreeBuffers.alloc(n, DEV)
    d = mps.to_device(a, DEV)
    out = mps.sort_keys(d, k=4, tree=tb)
    torch.cuda.synchronize()
    del d
    got = mps.to_numpy(out, np.uint32)
    del out
    assert np.all(got[1:] >= got[:-1])
    assert int(got.sum(dtype=np.uint64)) == int(a.sum(dtype=np.uint64))
    assert np.bitwise_xor.reduce(got) == np.bitwise_xor.reduce(a)
    del got
    check_tree(tb.to_numpy(), a, 4)


def test_pairs_2e27():
    n = 1 << 27
    a = inputs.random_runs_loguniform(n, 31)
    v = inputs.payload_index(n)
    ok, ov = mps.sort_pairs(mps.to_device(a, DEV), mps.to_device(v, DEV), k=4)
    torch.cuda.synchronize()
    got_k = mps.to_numpy(ok, np.uint64)
    got_v = mps.to_numpy(ov, np.uint32)
    del ok, ov
    want = oracle.sort(a, v, k=4, want_tree=False)
    assert np.array_equal(got_k, want["keys"])
    assert np.array_equal(got_v, want["vals"])


def test_records_2e26():
    n = 1 << 26
    a = inputs.random_runs_geometric(n, 41, mean=float(np.sqrt(n)), dtype=np.uint64)
    v = inputs.record_payload(n, 41)
    ok, ov = mps.sort_records(mps.to_device(a, DEV), mps.to_device(v, DEV), k=4)
    torch.cuda.synchronize()
    got_k = mps.to_numpy(ok, np.uint64)
    got_v = mps.to_numpy(ov, np.uint64)
    del ok, ov
    want = oracle.sort(a, inputs.payload_index(n), k=4, want_tree=False)
    assert np.array_equal(got_k, want["keys"])
    assert np.array_equal(got_v, v[want["vals"]])


def test_batch_4096_arrays():
    keys, offsets = inputs.batch_arrays(4096, 77)
    n, m = keys.size, offsets.size - 1
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    out = mps.sort_batch(mps.to_device(keys, DEV), d_off, k=4)
    torch.cuda.synchronize()
    cost = mps.last_stats()["merge_cost"]
    got = mps.to_numpy(out, np.uint32)
    del out
    starts = offsets[:-1].astype(np.int64)
    sizes = np.diff(offsets.astype(np.int64))
    assert np.all(sizes > 0)
    inner = np.ones(n - 1, bool)
    inner[starts[1:] - 1] = False  # pairs that straddle two arrays
    assert np.all(got[1:][inner] >= got[:-1][inner])
    assert np.array_equal(np.add.reduceat(keys.astype(np.uint64), starts),
                          np.add.reduceat(got.astype(np.uint64), starts))
    assert np.array_equal(np.bitwise_xor.reduceat(keys, starts), np.bitwise_xor.reduceat(got, starts))
    want_cost = 0
    for i in range(m):
        lo, hi = int(offsets[i]), int(offsets[i + 1])
        if i % 61 == 0:
            w = oracle.sort(keys[lo:hi], k=4, want_tree=False)
            assert np.array_equal(got[lo:hi], w["keys"]), f"array {i}"
            want_cost += w["merge_cost"]
        else:
            rs, _ = oracle.find_runs(keys[lo:hi])
            want_cost += oracle.tree_from_lengths(np.diff(rs.astype(np.int64)), 4)["merge_cost"]
    assert cost == want_cost


def test_served_stream_full_sizes():
    reqs = inputs.request_stream(40, 505, rate_per_s=1000.0)
    pool = torch.empty(64 << 30, dtype=torch.uint8, device=DEV)
    q = mps.Queue(pool, max_inflight=4, max_batch=64, k=4)
    held = []
    for i, r in enumerate(reqs):
        a, v = inputs.request_keys(r)
        d_in = mps.to_device(a, DEV)
        d_out = torch.empty_like(d_in)
        if v is None:
            t = q.submit(d_in, d_out, tag=i)
            held.append((t, r, d_out, None))
        else:
            dv = mps.to_device(v, DEV)
            t = q.submit(d_in, d_out, dv, torch.empty_like(dv), tag=i)
            held.append((t, r, d_out, q.keep[t][3]))
    for t, r, d_out, dvo in held:
        res = q.wait(t, timeout_ms=120000)
        assert res["status"] == 0 and res["device_status"] == 0
        a, v = inputs.request_keys(r)
        want = oracle.sort(a, v, k=4, want_tree=False)
        assert np.array_equal(mps.to_numpy(d_out, a.dtype), want["keys"]), f"request {res['tag']}"
        if v is not None:
            assert np.array_equal(mps.to_numpy(dvo, np.uint32), want["vals"]), f"request {res['tag']}"
    q.close()
