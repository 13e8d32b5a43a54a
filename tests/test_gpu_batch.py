"""Batched sorts (mps_sort_batch*) against the oracle, array by array (GPU).

Each array of a batch is its own Multiway Powersort problem: its own runs,
powers (Def. 3.1 with the array's length) and merge tree.  The batch output
must equal the concatenation of the per-array sorts, and the reported merge
cost must equal the sum of the oracle's per-array merge costs.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_06909_gb300 import inputs
from paper_2209_06909_gb300 import mps

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2209_06909_gb300 import build
    build.build()
    oracle.build()


def make_batch(seed, count, dtype=np.uint32, max_log2=15):
    rng = np.random.default_rng(seed)
    arrays = []
    special = [0, 1, 2, 3, 0, 5]
    for i in range(count):
        if i < len(special):
            m = special[i]
        else:
            m = int(2 ** rng.uniform(2, max_log2))
        kind = i % 6
        s = int(rng.integers(1 << 40))
        if kind == 0:
            a = inputs.random_permutation(m, s, dtype=dtype)
        elif kind == 1:
            a = inputs.random_runs_geometric(m, s, mean=max(1.0, m ** 0.5), dtype=dtype) if m else np.zeros(0, dtype)
        elif kind == 2:
            a = np.sort(rng.integers(0, 1 << 31, m).astype(dtype))[::-1].copy()  # one or few descending runs
        elif kind == 3:
            a = np.full(m, 7, dtype)
        elif kind == 4:
            a = (np.arange(m, dtype=np.uint64) ^ 1).astype(dtype)  # zigzag: runs of two
        else:
            a = inputs.random_runs_uniform_len(m, s, hi=max(2, m // 4)).astype(dtype) if m else np.zeros(0, dtype)
        arrays.append(np.ascontiguousarray(a, dtype=dtype))
    offsets = np.zeros(count + 1, np.uint64)
    offsets[1:] = np.cumsum([a.size for a in arrays])
    return arrays, offsets


def oracle_cost(arrays, k):
    return sum(oracle.sort(a, k=k, want_tree=False)["merge_cost"] for a in arrays if a.size)


@pytest.mark.parametrize("k", [2, 4, 8])
def test_batch_keys(k):
    arrays, offsets = make_batch(10 + k, 120)
    keys = np.concatenate(arrays)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    out = mps.sort_batch(mps.to_device(keys, DEV), d_off, k=k, max_len=int(max(a.size for a in arrays)))
    torch.cuda.synchronize()
    got = mps.to_numpy(out, np.uint32)
    want = np.concatenate([np.sort(a) for a in arrays])
    assert np.array_equal(got, want)
    assert mps.last_stats()["merge_cost"] == oracle_cost(arrays, k)


def test_batch_large_arrays_level_merges():
    """Arrays larger than a fused tile exercise the level merges of a batch."""
    arrays, offsets = make_batch(77, 16, max_log2=19)
    keys = np.concatenate(arrays)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    out = mps.sort_batch(mps.to_device(keys, DEV), d_off, k=4)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(out, np.uint32), np.concatenate([np.sort(a) for a in arrays]))
    assert mps.last_stats()["merge_cost"] == oracle_cost(arrays, 4)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_batch_pairs_stable(dtype):
    arrays, offsets = make_batch(5, 60, dtype=dtype)
    arrays = [np.ascontiguousarray(a % np.array(97, dtype)) for a in arrays]  # many equal keys
    keys = np.concatenate(arrays)
    vals = np.arange(keys.size, dtype=np.uint32)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    ok, ov = mps.sort_batch_pairs(mps.to_device(keys, DEV), mps.to_device(vals, DEV), d_off, k=4)
    torch.cuda.synchronize()
    want_k, want_v = [], []
    for i, a in enumerate(arrays):
        idx = np.arange(offsets[i], offsets[i + 1], dtype=np.uint32)
        order = np.lexsort((idx, a))
        want_k.append(a[order])
        want_v.append(idx[order])
    assert np.array_equal(mps.to_numpy(ok, dtype), np.concatenate(want_k))
    assert np.array_equal(mps.to_numpy(ov, np.uint32), np.concatenate(want_v))


def test_batch_graph_and_autotune():
    arrays, offsets = make_batch(3, 200)
    keys = np.concatenate(arrays)
    d_in = mps.to_device(keys, DEV)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    out = torch.empty_like(d_in)
    ws = mps.batch_workspace(keys.size, len(arrays), 4, False, 0, DEV)
    best = mps.batch_autotune(d_in, d_off, out, ws)
    assert best in (2, 4, 8)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = mps.BatchGraph(d_in, d_off, out, ws, k=0, stream=stream)
        for _ in range(2):
            out.fill_(-1)
            g.launch(stream=stream, check=True)
            assert np.array_equal(mps.to_numpy(out, np.uint32), np.concatenate([np.sort(a) for a in arrays]))
        g.close()
