"""Minimum run length on the GPU (Sec. 5, "Minimal run length": runs shorter
than m are extended to m elements and sorted) against the oracle's
min_run_len sort, element by element: keys, payload order, run starts, the
direction of each run's natural part, powers, node_first, node table, leaf
depths, levels and merge cost (GPU)."""
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
    assert torch.cuda.is_available()


def check_minrun(a: np.ndarray, k: int, m: int):
    want = oracle.sort(a, k=k, min_run_len=m)
    tb = mps.TreeBuffers.alloc(a.size, DEV)
    out = mps.sort_keys_minrun(mps.to_device(a, DEV), min_run_len=m, k=k, tree=tb)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(out, a.dtype), want["keys"]), f"keys (n={a.size}, k={k}, m={m})"
    t = tb.to_numpy()
    assert t["r"] == want["r"], (t["r"], want["r"])
    for key in ("run_starts", "run_desc", "powers", "node_first", "leaf_depth"):
        assert np.array_equal(t[key], want[key]), f"{key} differs (n={a.size}, k={k}, m={m})"
    assert t["num_nodes"] == want["num_nodes"] and np.array_equal(t["nodes"], want["nodes"])
    assert t["num_levels"] == want["num_levels"] and t["merge_cost"] == want["merge_cost"]


def edge_arrays(m):
    yield np.zeros(1, np.uint32)
    yield np.array([5, 3], np.uint32)
    for n in (m - 1, m, m + 1, 2 * m - 1, 2 * m, 2 * m + 1, 3 * m + 2):
        yield inputs.random_permutation(max(n, 1), seed=n)
    yield np.full(1000, 7, np.uint32)
    yield np.arange(5000, dtype=np.uint32)
    yield np.arange(5000, dtype=np.uint32)[::-1].copy()
    yield np.tile(np.array([1, 0], np.uint32), 3000)           # alternating pairs
    yield np.concatenate([np.arange(m - 1), np.arange(m + 5), np.arange(3)[::-1], np.arange(4 * m)]).astype(np.uint32)
    yield np.array([0xFFFFFFFF, 0, 0xFFFFFFFF, 0] * 100, np.uint32)


@pytest.mark.parametrize("m", [2, 5, 24, 32])
@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_minrun_edges(k, m):
    for a in edge_arrays(m):
        check_minrun(a, k, m)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
@pytest.mark.parametrize("m", [7, 24])
def test_minrun_permutation(k, m):
    check_minrun(inputs.random_permutation(300007, seed=m + k), k, m)


@pytest.mark.parametrize("k", [4, 2])
def test_minrun_config1_shape(k):
    """n = 2^20, run lengths U[1, 2000], half strictly descending, m = 24."""
    check_minrun(inputs.random_runs_uniform_len(1 << 20, seed=12), k, 24)


@pytest.mark.parametrize("mean", [3.0, 20.0, 64.0, 4096.0])
def test_minrun_geometric(mean):
    check_minrun(inputs.random_runs_geometric(250001, seed=int(mean), mean=mean), 4, 24)


def test_minrun_u64_and_pairs():
    b = inputs.random_runs_loguniform(200003, seed=3, log2_hi=8.0, distinct=512, dtype=np.uint64)
    check_minrun(b, 4, 24)
    v = inputs.payload_index(b.size)
    want = oracle.sort(b, v, k=4, want_tree=False, min_run_len=24)
    ok, ov = mps.sort_pairs_minrun(mps.to_device(b, DEV), mps.to_device(v, DEV), min_run_len=24, k=4)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(ok, np.uint64), want["keys"])
    assert np.array_equal(mps.to_numpy(ov, np.uint32), want["vals"])


def test_minrun_one_is_the_plain_sort():
    a = inputs.random_runs_uniform_len(100003, seed=4, hi=50)
    check_minrun(a, 4, 1)


def test_minrun_rejects_unsupported_lengths():
    a = mps.to_device(np.arange(100, dtype=np.uint32), DEV)
    with pytest.raises(mps.MpsError) as e:
        mps.sort_keys_minrun(a, min_run_len=33, k=4, ws=torch.empty(1 << 20, dtype=torch.uint8, device=DEV))
    assert e.value.code == 2


def test_minrun_permutation_2e28():
    """The bench's min-run variant at full size (n = 2^28 permutation, m = 24,
    k = 4): the output is 0..n-1; runs, directions, powers, node table, leaf
    depths and merge cost equal the oracle's run scan and tree from run lengths."""
    n = 1 << 28
    a = inputs.random_permutation(n, 1004)
    tb = mps.TreeBuffers.alloc(n, DEV)
    out = mps.sort_keys_minrun(mps.to_device(a, DEV), min_run_len=24, k=4, tree=tb)
    torch.cuda.synchronize()
    assert torch.equal(out, torch.arange(n, dtype=torch.int32, device=DEV))
    del out
    t = tb.to_numpy()
    rs, rd = oracle.find_runs(a, min_run_len=24)
    want = oracle.tree_from_lengths(np.diff(rs.astype(np.int64)), 4)
    assert t["r"] == rs.size - 1
    assert np.array_equal(t["run_starts"], rs) and np.array_equal(t["run_desc"], rd)
    assert np.array_equal(t["powers"], want["powers"])
    assert t["num_nodes"] == want["num_nodes"] and np.array_equal(t["nodes"], want["nodes"])
    assert np.array_equal(t["node_first"], want["node_first"])
    assert np.array_equal(t["leaf_depth"], want["leaf_depth"])
    assert t["merge_cost"] == want["merge_cost"]
