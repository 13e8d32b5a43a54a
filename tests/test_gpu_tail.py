"""Final-collapse variants on the GPU (mps_sort_keys_tail) against the oracle.

Alg. 2's run stack, once the last run is pushed, is emptied either by the
power rule (Alg. 1's tree), by the last loop as printed (pop up to k-1
entries per merge) or by the appendix's merge_down.  The oracle builds each
policy's tree on the run lengths (``oracle.tree_tail``, pinned by hand-written
trees and by a separate cost-only loop).  Bit-exact: sorted keys, run starts
and directions, the powers of Def. 3.1, node_first, leaf depths, the merge
cost and the set of nodes (first run, end run, degree); the node table's
power field holds relabelled powers and is compared through node shapes.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_06909_gb300 import inputs
from paper_2209_06909_gb300 import mps

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
POLICIES = ["alg2_pop_k_minus_1", "merge_down"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2209_06909_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available()


def _shape(nodes):
    return sorted((int(x["first_run"]), int(x["end_run"]), int(x["degree"])) for x in nodes)


def check_tail(a: np.ndarray, k: int, policy: str):
    base = oracle.sort(a, k=k)
    lengths = np.diff(base["run_starts"].astype(np.int64))
    want = oracle.tree_tail(lengths, k, policy) if lengths.size else None
    tb = mps.TreeBuffers.alloc(a.size, DEV)
    out = mps.sort_keys_tail(mps.to_device(a, DEV), policy, k=k, tree=tb)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(out, a.dtype), base["keys"]), f"keys differ (n={a.size}, k={k}, {policy})"
    t = tb.to_numpy()
    assert t["r"] == base["r"]
    for key in ("run_starts", "run_desc", "powers"):
        assert np.array_equal(t[key], base[key]), f"{key} differs (n={a.size}, k={k}, {policy})"
    if want is None:
        return
    assert t["num_nodes"] == want["num_nodes"]
    assert _shape(t["nodes"]) == _shape(want["nodes"]), f"nodes differ (n={a.size}, k={k}, {policy})"
    assert np.array_equal(t["node_first"], want["node_first"])
    assert np.array_equal(t["leaf_depth"], want["leaf_depth"])
    assert t["merge_cost"] == want["merge_cost"]
    assert mps.last_stats()["merge_cost"] == want["merge_cost"]


@pytest.mark.parametrize("policy", POLICIES)
@pytest.mark.parametrize("k", [2, 4, 8, 16])
@pytest.mark.parametrize("n", [2, 17, 4097, 65536 + 123, 300001])
def test_random_runs(n, k, policy):
    check_tail(inputs.random_runs_uniform_len(n, seed=n + 3 * k, hi=min(2000, max(2, n // 8))), k, policy)


@pytest.mark.parametrize("policy", POLICIES)
@pytest.mark.parametrize("k", [4, 8, 16])
def test_permutation_and_geometric(k, policy):
    check_tail(inputs.random_permutation(1 << 20, seed=40 + k), k, policy)
    check_tail(inputs.random_runs_geometric(400000, seed=50 + k, mean=64.0), k, policy)


@pytest.mark.parametrize("policy", POLICIES)
def test_edge_cases(policy):
    m = (1 << 32) - 1
    cases = [np.array([7], np.uint32), np.array([2, 1], np.uint32), np.arange(100000, dtype=np.uint32),
             np.arange(100000, 0, -1).astype(np.uint32), np.tile(np.array([m, 0], np.uint32), 30000),
             np.concatenate([np.arange(70000), np.arange(70000)]).astype(np.uint32)]
    for a in cases:
        for k in (4, 16):
            check_tail(a, k, policy)


@pytest.mark.parametrize("k", [4, 8])
def test_power_rule_policy_is_sort_keys(k):
    """Policy 0 is the power rule: every tree output equals mps_sort_keys'."""
    a = inputs.random_runs_uniform_len(200003, seed=60 + k, hi=500)
    d = mps.to_device(a, DEV)
    t0, t1 = mps.TreeBuffers.alloc(a.size, DEV), mps.TreeBuffers.alloc(a.size, DEV)
    o0 = mps.sort_keys(d, k=k, tree=t0)
    o1 = mps.sort_keys_tail(d, "kway_tree", k=k, tree=t1)
    torch.cuda.synchronize()
    assert torch.equal(o0, o1)
    x, y = t0.to_numpy(), t1.to_numpy()
    for key in ("run_starts", "run_desc", "powers", "node_first", "leaf_depth", "nodes"):
        assert np.array_equal(x[key], y[key]), key
    assert x["merge_cost"] == y["merge_cost"]


@pytest.mark.parametrize("policy", POLICIES)
def test_permutation_2e26_merge_cost(policy):
    """The bench's input shape at 2^26, k = 4: output 0..n-1 and the merge
    cost of the oracle's cost-only loop for the policy."""
    n = 1 << 26
    a = inputs.random_permutation(n, 77)
    rs, _ = oracle.find_runs(a)
    out = mps.sort_keys_tail(mps.to_device(a, DEV), policy, k=4)
    torch.cuda.synchronize()
    assert torch.equal(out, torch.arange(n, dtype=torch.int32, device=DEV))
    assert mps.last_stats()["merge_cost"] == oracle.merge_cost_tail(np.diff(rs.astype(np.int64)), 4, policy)


def test_bad_policy():
    a = mps.to_device(np.arange(100, dtype=np.uint32), DEV)
    ws = mps.workspace(100, 4, False, 4, DEV)
    code = mps.lib().mps_sort_keys_tail(a.data_ptr(), a.data_ptr(), 100, 0, 4, 3, ws.data_ptr(), ws.numel(), None, None)
    assert code == 1  # MPS_ERR_INVALID_ARG, returned before anything is queued
