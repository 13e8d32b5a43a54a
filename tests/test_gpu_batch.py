"""Batched sorts (mps_sort_batch*) against the oracle, array by array (GPU).

Each array of a batch is its own Multiway Powersort problem: its own runs,
powers (Def. 3.1 with the array's length) and merge tree.  The batch output
must equal the concatenation of the per-array sorts, each array's merge cost
(Sec. 2.2) must equal the oracle's for that array sorted alone, and the
reported total must equal their sum.
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


def oracle_costs(arrays, k):
    """Merge cost of every array sorted alone (0 for an empty array)."""
    return np.array([oracle.sort(a, k=k, want_tree=False)["merge_cost"] if a.size else 0 for a in arrays],
                    dtype=np.int64)


def cost_buffer(m):
    # filled with garbage: the call must overwrite every entry
    return torch.full((m,), -1, dtype=torch.int64, device=DEV)


@pytest.mark.parametrize("k", [2, 4, 8])
def test_batch_keys(k):
    arrays, offsets = make_batch(10 + k, 120)
    keys = np.concatenate(arrays)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    costs = cost_buffer(len(arrays))
    out = mps.sort_batch(mps.to_device(keys, DEV), d_off, k=k, max_len=int(max(a.size for a in arrays)),
                         merge_costs=costs)
    torch.cuda.synchronize()
    got = mps.to_numpy(out, np.uint32)
    want = np.concatenate([np.sort(a) for a in arrays])
    assert np.array_equal(got, want)
    want_costs = oracle_costs(arrays, k)
    assert np.array_equal(costs.cpu().numpy(), want_costs)
    assert mps.last_stats()["merge_cost"] == int(want_costs.sum())


@pytest.mark.parametrize("tile", [0, 1, 2])
@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_batch_tile_choices(k, tile):
    """Every (fan-in, tile) configuration that k = 0 can select gives the
    per-array sorts and merge costs, keys and pairs; arrays up to 2^17 cross
    every tile size, so both fused subtrees and level merges run."""
    arrays, offsets = make_batch(40 + tile + 3 * k, 150, max_log2=17)
    keys = np.concatenate(arrays)
    n, m = keys.size, len(arrays)
    mps.batch_set_config(4, False, n, m, k, tile)
    mps.batch_set_config(4, True, n, m, k, tile)
    cfg = mps.batch_tuned_config(4, False, n, m)
    assert cfg["k"] == k and cfg["c_fused"] * cfg["items_per_thread"] > 0
    d_in = mps.to_device(keys, DEV)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    costs = cost_buffer(m)
    ws = mps.batch_workspace(n, m, 4, True, 0, DEV)
    out = mps.sort_batch(d_in, d_off, k=0, ws=ws, merge_costs=costs)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(out, np.uint32), np.concatenate([np.sort(a) for a in arrays]))
    assert np.array_equal(costs.cpu().numpy(), oracle_costs(arrays, k))
    v = inputs.payload_index(n)
    ok, ov = mps.sort_batch_pairs(d_in, mps.to_device(v, DEV), d_off, k=0, ws=ws)
    torch.cuda.synchronize()
    want_v = []
    for i, a in enumerate(arrays):
        idx = np.arange(offsets[i], offsets[i + 1], dtype=np.uint32)
        want_v.append(idx[np.lexsort((idx, a))])
    assert np.array_equal(mps.to_numpy(ov, np.uint32), np.concatenate(want_v))


def test_batch_large_arrays_level_merges():
    """Arrays larger than a fused tile exercise the level merges of a batch."""
    arrays, offsets = make_batch(77, 16, max_log2=19)
    keys = np.concatenate(arrays)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    costs = cost_buffer(len(arrays))
    out = mps.sort_batch(mps.to_device(keys, DEV), d_off, k=4, merge_costs=costs)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(out, np.uint32), np.concatenate([np.sort(a) for a in arrays]))
    want_costs = oracle_costs(arrays, 4)
    assert np.array_equal(costs.cpu().numpy(), want_costs)
    assert mps.last_stats()["merge_cost"] == int(want_costs.sum())


def test_batch_costs_many_small_and_empty_arrays():
    """Per-array costs where many arrays share one mask tile, with empty arrays
    between them (the cost of an array depends on its runs only)."""
    rng = np.random.default_rng(2024)
    arrays = []
    for i in range(3000):
        m = 0 if i % 7 == 3 else int(rng.integers(1, 200))
        arrays.append(inputs.random_runs_uniform_len(m, int(rng.integers(1 << 40)), hi=max(2, m // 3)).astype(np.uint32)
                      if m else np.zeros(0, np.uint32))
    offsets = np.zeros(len(arrays) + 1, np.uint64)
    offsets[1:] = np.cumsum([a.size for a in arrays])
    keys = np.concatenate(arrays)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    costs = cost_buffer(len(arrays))
    out = mps.sort_batch(mps.to_device(keys, DEV), d_off, k=4, merge_costs=costs)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(out, np.uint32), np.concatenate([np.sort(a) for a in arrays]))
    assert np.array_equal(costs.cpu().numpy(), oracle_costs(arrays, 4))


def test_batch_of_many_tiny_arrays():
    """Every array of two or more runs that fits a tile is its own fused root,
    so a batch of many tiny arrays has far more fused subtrees than nodes
    above T_max: the fused list is sized by the number of arrays."""
    rng = np.random.default_rng(31)
    m = 120_000
    sizes = rng.integers(3, 9, m)
    keys = rng.integers(0, 1 << 32, int(sizes.sum()), dtype=np.uint64).astype(np.uint32)
    offsets = np.zeros(m + 1, np.uint64)
    offsets[1:] = np.cumsum(sizes)
    arrays = [keys[int(offsets[i]):int(offsets[i + 1])] for i in range(m)]
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    costs = cost_buffer(m)
    out = mps.sort_batch(mps.to_device(keys, DEV), d_off, k=4, max_len=8, merge_costs=costs)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(out, np.uint32), np.concatenate([np.sort(a) for a in arrays]))
    assert mps.last_stats()["frontier_nodes"] > 50_000
    assert np.array_equal(costs.cpu().numpy(), oracle_costs(arrays, 4))


def test_batch_longer_than_max_len_is_reported():
    """An array longer than the caller's max_len is a device-side check
    failure (status 16), not a silently short level loop."""
    arrays, offsets = make_batch(9, 40, max_log2=14)
    keys = np.concatenate(arrays)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    longest = int(max(a.size for a in arrays))
    with pytest.raises(mps.MpsError) as ei:
        mps.sort_batch(mps.to_device(keys, DEV), d_off, k=4, max_len=longest - 1)
    assert mps.STATUS[ei.value.code] == "device-side check failed"
    assert mps.last_stats()["device_status"] == 16
    # the same batch with a sufficient bound sorts
    out = mps.sort_batch(mps.to_device(keys, DEV), d_off, k=4, max_len=longest)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(out, np.uint32), np.concatenate([np.sort(a) for a in arrays]))


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_batch_pairs_stable(dtype):
    arrays, offsets = make_batch(5, 60, dtype=dtype)
    arrays = [np.ascontiguousarray(a % np.array(97, dtype)) for a in arrays]  # many equal keys
    keys = np.concatenate(arrays)
    vals = np.arange(keys.size, dtype=np.uint32)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(DEV)
    costs = cost_buffer(len(arrays))
    ok, ov = mps.sort_batch_pairs(mps.to_device(keys, DEV), mps.to_device(vals, DEV), d_off, k=4, merge_costs=costs)
    torch.cuda.synchronize()
    assert np.array_equal(costs.cpu().numpy(), oracle_costs(arrays, 4))
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
    cfg = mps.batch_tuned_config(4, False, keys.size, len(arrays))
    assert cfg["k"] == best and cfg["c_fused"] in (4096, 6144, 2048)
    stream = torch.cuda.Stream()
    costs = cost_buffer(len(arrays))
    want_costs = oracle_costs(arrays, best)
    with torch.cuda.stream(stream):
        g = mps.BatchGraph(d_in, d_off, out, ws, k=0, stream=stream, merge_costs=costs)
        for _ in range(2):
            out.fill_(-1)
            costs.fill_(-1)
            g.launch(stream=stream, check=True)
            assert np.array_equal(mps.to_numpy(out, np.uint32), np.concatenate([np.sort(a) for a in arrays]))
            assert np.array_equal(costs.cpu().numpy(), want_costs)  # rewritten by every replay
        g.close()
