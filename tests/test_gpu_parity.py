"""CUDA path vs the CPU oracle, element by element (GPU).

Everything is integer work, so the bar is bit-exact: sorted keys, payload
order, run starts and directions, powers, node_first, the canonical node
table, leaf depths, number of levels and the merge cost.  Sizes span several
detection tiles, fused tiles and level-merge units, with ragged tails.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_06909_gb300 import inputs
from paper_2209_06909_gb300 import mps

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
U32_MAX = (1 << 32) - 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2209_06909_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available()


def check_keys_and_tree(a: np.ndarray, k: int):
    want = oracle.sort(a, k=k)
    dt = a.dtype
    tb = mps.TreeBuffers.alloc(a.size, DEV)
    out = mps.sort_keys(mps.to_device(a, DEV), k=k, tree=tb)
    torch.cuda.synchronize()
    got = mps.to_numpy(out, dt)
    assert np.array_equal(got, want["keys"]), f"keys differ (n={a.size}, k={k})"
    t = tb.to_numpy()
    assert t["r"] == want["r"]
    for key in ("run_starts", "run_desc", "powers", "node_first", "leaf_depth"):
        assert np.array_equal(t[key], want[key]), f"{key} differs (n={a.size}, k={k})"
    assert t["num_nodes"] == want["num_nodes"]
    assert np.array_equal(t["nodes"], want["nodes"]), f"node table differs (n={a.size}, k={k})"
    assert t["num_levels"] == want["num_levels"]
    assert t["merge_cost"] == want["merge_cost"]
    st = mps.last_stats()
    assert st["merge_cost"] == want["merge_cost"] and st["r"] == want["r"]


def check_pairs(a: np.ndarray, k: int):
    v = inputs.payload_index(a.size)
    want = oracle.sort(a, v, k=k, want_tree=False)
    ok, ov = mps.sort_pairs(mps.to_device(a, DEV), mps.to_device(v, DEV), k=k)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(ok, a.dtype), want["keys"])
    assert np.array_equal(mps.to_numpy(ov, np.uint32), want["vals"])


@pytest.mark.parametrize("k", [2, 4, 8, 16])
@pytest.mark.parametrize("n", [2, 3, 17, 1000, 4097, 65536 + 123, 300001])
def test_random_runs_uniform(n, k):
    check_keys_and_tree(inputs.random_runs_uniform_len(n, seed=n + k, hi=min(2000, max(2, n // 8))), k)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_config1_shape_full(k):
    """n = 2^20 uint32, run lengths U[1, 2000], half strictly descending."""
    check_keys_and_tree(inputs.random_runs_uniform_len(1 << 20, seed=11), k)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
@pytest.mark.parametrize("n", [5000, 100003, 1 << 20])
def test_permutation(n, k):
    check_keys_and_tree(inputs.random_permutation(n, seed=n % 97 + k), k)


@pytest.mark.parametrize("k", [2, 4, 16])
@pytest.mark.parametrize("mean", [3.0, 64.0, 4096.0])
def test_geometric_runs(mean, k):
    check_keys_and_tree(inputs.random_runs_geometric(400000, seed=int(mean) + k, mean=mean), k)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_u64_keys_duplicates(k):
    check_keys_and_tree(inputs.random_runs_loguniform(200000, seed=3 + k, log2_hi=12.0, distinct=1 << 10), k)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_pairs_stable(k, dtype):
    a = inputs.random_runs_loguniform(150001, seed=5 + k, log2_hi=11.0, distinct=300, dtype=dtype)
    check_pairs(a, k)
    check_pairs(a[::-1].copy(), k)


def edge_arrays():
    m = U32_MAX
    rng = np.random.default_rng(0)
    yield "one", np.array([7], np.uint32)
    yield "two_desc", np.array([2, 1], np.uint32)
    yield "equal", np.full(100000, 5, np.uint32)
    yield "ascending", np.arange(200000, dtype=np.uint32)
    yield "strict_desc", np.arange(200000, 0, -1).astype(np.uint32)
    yield "zigzag", np.arange(100000, dtype=np.uint32) ^ 1
    yield "extremes", rng.choice(np.array([0, 1, m - 1, m], np.uint32), 77777)
    yield "max_runs", np.tile(np.array([m, 0], np.uint32), 40000)
    big = np.concatenate([np.sort(rng.integers(0, 1 << 32, 300000)).astype(np.uint32),
                          rng.integers(0, 1 << 32, 50).astype(np.uint32),
                          np.sort(rng.integers(0, 1 << 32, 200000)).astype(np.uint32)[::-1]])
    yield "skewed", big
    yield "two_runs", np.concatenate([np.arange(70000), np.arange(70000)]).astype(np.uint32)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_edge_cases(k):
    for name, a in edge_arrays():
        check_keys_and_tree(a, k)
        check_pairs(a, k)


def test_empty():
    a = np.zeros(0, np.uint32)
    tb = mps.TreeBuffers.alloc(0, DEV)
    out = mps.sort_keys(mps.to_device(a, DEV), k=4, tree=tb)
    torch.cuda.synchronize()
    assert out.numel() == 0 and tb.to_numpy()["r"] == 0


def test_merge_tree_leaves_keys_untouched():
    a = inputs.random_runs_uniform_len(123457, seed=9, hi=300)
    d = mps.to_device(a, DEV)
    tb = mps.merge_tree(d, k=4)
    torch.cuda.synchronize()
    want = oracle.sort(a, k=4)
    t = tb.to_numpy()
    assert np.array_equal(mps.to_numpy(d, np.uint32), a)
    for key in ("run_starts", "run_desc", "powers", "node_first", "leaf_depth"):
        assert np.array_equal(t[key], want[key])
    assert np.array_equal(t["nodes"], want["nodes"]) and t["merge_cost"] == want["merge_cost"]


def test_repeat_calls_same_workspace():
    a = inputs.random_permutation(300000, seed=4)
    ws = mps.workspace(a.size, 4, False, 4, DEV)
    d = mps.to_device(a, DEV)
    o1 = mps.sort_keys(d, k=4, ws=ws).clone()
    o2 = mps.sort_keys(d, k=4, ws=ws)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)
    assert np.array_equal(mps.to_numpy(o2, np.uint32), np.arange(a.size, dtype=np.uint32))


def test_host_entry_point():
    a = inputs.random_runs_geometric(200000, seed=8, mean=100.0)
    h_in = torch.from_numpy(a.view(np.int32)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_in = torch.empty(a.size, dtype=torch.int32, device=DEV)
    d_out = torch.empty_like(d_in)
    ws = mps.workspace(a.size, 4, False, 4, DEV)
    mps.sort_keys_host(h_in, h_out, d_in, d_out, ws, k=4)
    assert np.array_equal(h_out.numpy().view(np.uint32), np.sort(a))


def test_host_async_pipeline():
    """Six arrays through mps_sort_keys_host_async on two streams, each stream
    with its own device buffers and workspace, queued without waiting: every
    host result must be that array's sort."""
    n = 300000
    arrays = [inputs.random_runs_geometric(n, seed=40 + i, mean=50.0) if i % 2 else inputs.random_permutation(n, seed=40 + i)
              for i in range(6)]
    h_in = [torch.from_numpy(a.view(np.int32)).pin_memory() for a in arrays]
    h_out = [torch.empty_like(h).pin_memory() for h in h_in]
    streams = [torch.cuda.Stream(device=DEV) for _ in range(2)]
    d_in = [torch.empty(n, dtype=torch.int32, device=DEV) for _ in range(2)]
    d_out = [torch.empty_like(d) for d in d_in]
    ws = [mps.workspace(n, 4, False, 4, DEV) for _ in range(2)]
    torch.cuda.synchronize()
    for i in range(6):
        s = i % 2
        mps.sort_keys_host_async(h_in[i], h_out[i], d_in[s], d_out[s], ws[s], k=4, stream=streams[s])
    torch.cuda.synchronize()
    for i, a in enumerate(arrays):
        assert np.array_equal(h_out[i].numpy().view(np.uint32), np.sort(a)), i


def test_argument_errors():
    a = mps.to_device(np.arange(1000, dtype=np.uint32), DEV)
    with pytest.raises(mps.MpsError) as e:
        mps.sort_keys(a, k=3)
    assert e.value.code == 2
    ws = torch.empty(16, dtype=torch.uint8, device=DEV)
    with pytest.raises(mps.MpsError) as e:
        mps.sort_keys(a, k=4, ws=ws)
    assert e.value.code == 3
    v = torch.empty(1000, dtype=torch.int32, device=DEV)
    with pytest.raises(mps.MpsError) as e:
        mps.sort_pairs(a, v, k=4, out_keys=a, out_vals=a)  # keys and payloads in the same memory
    assert e.value.code == 1


def test_host_async_rejects_before_copying():
    """A rejected mps_sort_keys_host_async call queues nothing: the device
    input buffer keeps its contents."""
    n = 5000
    h_in = torch.from_numpy(np.arange(n, dtype=np.int32)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_in = torch.full((n,), 7, dtype=torch.int32, device=DEV)
    d_out = torch.empty_like(d_in)
    small = torch.empty(16, dtype=torch.uint8, device=DEV)
    for k, ws, code in ((4, small, 3), (3, mps.workspace(n, 4, False, 4, DEV), 2)):
        with pytest.raises(mps.MpsError) as e:
            mps.sort_keys_host_async(h_in, h_out, d_in, d_out, ws, k=k)
        assert e.value.code == code
    torch.cuda.synchronize()
    assert bool((d_in == 7).all())


@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_sort_in_place(k):
    """d_keys_out == d_keys_in (and payloads in place): the same result as the oracle."""
    a = inputs.random_runs_uniform_len(300001, seed=21 + k, hi=2000)
    d = mps.to_device(a, DEV)
    mps.sort_keys(d, k=k, out=d)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(d, np.uint32), oracle.sort(a, k=k)["keys"])
    b = inputs.random_runs_loguniform(200003, seed=5, log2_hi=12.0, distinct=1024, dtype=np.uint64)
    v = inputs.payload_index(b.size)
    want = oracle.sort(b, v, k=k, want_tree=False)
    dk, dv = mps.to_device(b, DEV), mps.to_device(v, DEV)
    mps.sort_pairs(dk, dv, k=k, out_keys=dk, out_vals=dv)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(dk, np.uint64), want["keys"])
    assert np.array_equal(mps.to_numpy(dv, np.uint32), want["vals"])


def test_calls_queue_without_waiting():
    """Several sorts queued back to back on one stream and one workspace, then
    one synchronisation: each output is right, and the status word is clear."""
    ws = mps.workspace(400000, 4, False, 4, DEV)
    arrays = [inputs.random_permutation(400000, seed=s) for s in (1, 2)] + \
             [inputs.random_runs_geometric(399999, seed=3, mean=50.0)]
    outs = []
    for a in arrays:
        outs.append(mps.sort_keys(mps.to_device(a, DEV), k=4, ws=ws))
    mps.sync_status(ws)
    for a, o in zip(arrays, outs):
        assert np.array_equal(mps.to_numpy(o, np.uint32), np.sort(a))
    st = mps.last_stats()
    assert st["device_status"] == 0 and st["r"] == oracle.find_runs(arrays[-1])[0].size - 1
