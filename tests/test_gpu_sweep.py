"""Seeded random sweep of the CUDA path against the oracle (GPU).

Each case draws a size (log-uniform up to about 2^20, or one of the tile and
unit boundaries), a key type, a fan-in, an input shape and a call: keys with
the full tree, pairs, records, a minimum run length, or a final-collapse
variant.  The comparison is the same bit-exact one as the other parity tests:
keys, payload order, runs, powers, node_first, node table, leaf depths, levels
and merge cost.  A failure names its case, so it can be rerun alone.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_06909_gb300 import inputs
from paper_2209_06909_gb300 import mps

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
CASES = 256
POLICIES = ["alg2_pop_k_minus_1", "merge_down"]
# tile and unit sizes of the kernels and their neighbours
EDGE_SIZES = [0, 1, 2, 3, 31, 32, 33, 2047, 2048, 4095, 4096, 4097, 6144, 8191, 8192, 8193, 9215, 9216, 9217,
              16384, 65537]
SHAPES = ["uniform_runs", "perm", "geom", "loguniform", "few", "equal", "asc", "desc_strict", "desc_pairs",
          "saw", "organ", "extreme"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2209_06909_gb300 import build
    build.build()
    oracle.build()
    assert torch.cuda.is_available()


def draw_case(i: int) -> dict:
    rng = np.random.default_rng(90_000 + i)
    dtype = np.uint32 if rng.random() < 0.6 else np.uint64
    n = int(rng.choice(EDGE_SIZES)) if rng.random() < 0.2 else int(2 ** rng.uniform(2.0, 20.3))
    shape = SHAPES[int(rng.integers(len(SHAPES)))]
    seed = int(rng.integers(1 << 30))
    top = np.iinfo(dtype).max
    if shape == "uniform_runs":
        lo = int(rng.integers(1, 9))
        hi = lo + int(2 ** rng.uniform(2.0, 11.0))
        if hi < 64:
            n = min(n, 1 << 16)  # the generator loops over runs in Python
        a = inputs.random_runs_uniform_len(n, seed, lo=lo, hi=hi, p_desc=float(rng.random())).astype(dtype)
    elif shape == "perm":
        a = inputs.random_permutation(n, seed, dtype)
    elif shape == "geom":
        a = inputs.random_runs_geometric(n, seed, mean=float(2 ** rng.uniform(0.0, 14.0)), dtype=dtype)
    elif shape == "loguniform":
        a = inputs.random_runs_loguniform(n, seed, log2_hi=float(rng.uniform(1.0, 16.0)),
                                          distinct=int(2 ** rng.uniform(1.0, 16.0)), dtype=dtype)
    elif shape == "few":
        a = rng.integers(0, 3, n).astype(dtype)
    elif shape == "equal":
        a = np.full(n, rng.integers(0, 1000), dtype)
    elif shape == "asc":
        a = np.arange(n, dtype=dtype)
    elif shape == "desc_strict":
        a = np.arange(n, dtype=dtype)[::-1].copy()
    elif shape == "desc_pairs":  # non-strictly descending: equal neighbours split it into short runs
        a = (np.arange(n, dtype=np.int64) // 2)[::-1].astype(dtype)
    elif shape == "saw":
        a = (np.arange(n, dtype=np.int64) % int(rng.integers(2, 5000))).astype(dtype)
    elif shape == "organ":
        h = n // 2
        a = np.concatenate([np.arange(h, dtype=np.int64), np.arange(n - h, dtype=np.int64)[::-1]]).astype(dtype)
    else:  # extreme values of the key type, with ties
        a = rng.choice(np.array([0, 1, top - 1, top], dtype=dtype), n)
    a = np.ascontiguousarray(a[:n], dtype=dtype)
    mode = str(rng.choice(["keys", "pairs", "records", "minrun", "minrun_pairs", "tail"],
                          p=[0.3, 0.15, 0.1, 0.2, 0.1, 0.15]))
    return {"a": a, "k": int(rng.choice([2, 4, 8, 16])), "mode": mode, "m": int(rng.integers(2, 33)),
            "policy": POLICIES[int(rng.integers(2))], "shape": shape, "seed": seed}


def check_tree(t: dict, want: dict, what: str):
    assert t["r"] == want["r"], what
    for key in ("run_starts", "run_desc", "powers", "node_first", "leaf_depth"):
        assert np.array_equal(t[key], want[key]), f"{key}: {what}"
    assert t["num_nodes"] == want["num_nodes"], what
    assert np.array_equal(t["nodes"], want["nodes"]), f"node table: {what}"
    assert t["num_levels"] == want["num_levels"], what
    assert t["merge_cost"] == want["merge_cost"], what


def node_shape(nodes):
    return sorted((int(x["first_run"]), int(x["end_run"]), int(x["degree"])) for x in nodes)


@pytest.mark.parametrize("case", range(CASES), ids=lambda c: f"case{c}")
def test_sweep(case):
    c = draw_case(case)
    a, k, mode = c["a"], c["k"], c["mode"]
    n = a.size
    what = f"case {case}: n={n} {a.dtype} k={k} {c['shape']} {mode}"
    if mode == "keys":
        want = oracle.sort(a, k=k)
        tb = mps.TreeBuffers.alloc(n, DEV)
        out = mps.sort_keys(mps.to_device(a, DEV), k=k, tree=tb)
        torch.cuda.synchronize()
        assert np.array_equal(mps.to_numpy(out, a.dtype), want["keys"]), what
        check_tree(tb.to_numpy(), want, what)
    elif mode in ("pairs", "minrun_pairs"):
        m = c["m"] if mode == "minrun_pairs" else 1
        v = inputs.payload_index(n)
        want = oracle.sort(a, v, k=k, want_tree=False, min_run_len=m)
        if m > 1:
            ok, ov = mps.sort_pairs_minrun(mps.to_device(a, DEV), mps.to_device(v, DEV), min_run_len=m, k=k)
        else:
            ok, ov = mps.sort_pairs(mps.to_device(a, DEV), mps.to_device(v, DEV), k=k)
        torch.cuda.synchronize()
        assert np.array_equal(mps.to_numpy(ok, a.dtype), want["keys"]), what
        assert np.array_equal(mps.to_numpy(ov, np.uint32), want["vals"]), what
    elif mode == "records":
        vals = inputs.record_payload(n, c["seed"])
        want = oracle.sort(a, inputs.payload_index(n), k=k, want_tree=False)
        ok, ov = mps.sort_records(mps.to_device(a, DEV), mps.to_device(vals, DEV), k=k)
        torch.cuda.synchronize()
        assert np.array_equal(mps.to_numpy(ok, a.dtype), want["keys"]), what
        assert np.array_equal(mps.to_numpy(ov, np.uint64), vals[want["vals"]]), what
    elif mode == "minrun":
        want = oracle.sort(a, k=k, min_run_len=c["m"])
        tb = mps.TreeBuffers.alloc(n, DEV)
        out = mps.sort_keys_minrun(mps.to_device(a, DEV), min_run_len=c["m"], k=k, tree=tb)
        torch.cuda.synchronize()
        assert np.array_equal(mps.to_numpy(out, a.dtype), want["keys"]), what
        check_tree(tb.to_numpy(), want, what + f" m={c['m']}")
    else:
        base = oracle.sort(a, k=k)
        lengths = np.diff(base["run_starts"].astype(np.int64))
        tb = mps.TreeBuffers.alloc(n, DEV)
        out = mps.sort_keys_tail(mps.to_device(a, DEV), c["policy"], k=k, tree=tb)
        torch.cuda.synchronize()
        assert np.array_equal(mps.to_numpy(out, a.dtype), base["keys"]), what
        t = tb.to_numpy()
        for key in ("run_starts", "run_desc", "powers"):
            assert np.array_equal(t[key], base[key]), f"{key}: {what}"
        if lengths.size:
            want = oracle.tree_tail(lengths, k, c["policy"])
            assert node_shape(t["nodes"]) == node_shape(want["nodes"]), what
            assert np.array_equal(t["node_first"], want["node_first"]), what
            assert np.array_equal(t["leaf_depth"], want["leaf_depth"]), what
            assert t["merge_cost"] == want["merge_cost"], what
