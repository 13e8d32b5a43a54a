"""The seeded input generators produce the shapes the input recipe states
(sizes, run lengths, value pools, mixes), deterministically per seed.  They
hold none of the method's arithmetic; the natural runs counted here use the
oracle's greedy scan, pinned in test_oracle_pins.py."""
import numpy as np

import oracle
from paper_2209_06909_gb300 import inputs


def test_generators_are_deterministic_per_seed():
    for gen in (lambda s: inputs.random_permutation(5000, s),
                lambda s: inputs.random_runs_uniform_len(5000, s, hi=300),
                lambda s: inputs.random_runs_geometric(5000, s, mean=50.0),
                lambda s: inputs.random_runs_loguniform(5000, s, log2_hi=10.0, distinct=256)):
        assert np.array_equal(gen(3), gen(3))
        assert not np.array_equal(gen(3), gen(4))


def test_permutation_is_a_permutation():
    a = inputs.random_permutation(1 << 16, 1000)
    assert a.dtype == np.uint32 and np.array_equal(np.sort(a), np.arange(1 << 16, dtype=np.uint32))


def test_uniform_length_runs_and_directions():
    """Config 1: run lengths U[1, 2000]; about half of the runs strictly
    descending.  Natural runs can fuse at a boundary, so the detected count is
    a little below the generated one."""
    n = 1 << 20
    a = inputs.random_runs_uniform_len(n, 7)
    assert a.size == n and a.dtype == np.uint32
    starts, desc = oracle.find_runs(a)
    r = starts.size - 1
    assert 0.85 * n / 1000.5 < r < 1.1 * n / 1000.5
    assert 0.4 < desc.mean() < 0.6


def test_geometric_runs_have_the_stated_mean():
    """Config 2b shape: ascending runs of geometric mean length; with long runs
    of uniform values, neighbours almost never fuse, so the detected mean
    length matches the generator's mean."""
    n, mean = 1 << 21, 1024.0
    a = inputs.random_runs_geometric(n, 11, mean=mean)
    starts, desc = oracle.find_runs(a)
    lengths = np.diff(starts.astype(np.int64))
    assert abs(lengths.mean() / mean - 1) < 0.1
    # descending "runs" appear only at fused boundaries, as pairs of elements
    assert np.all(lengths[desc == 1] <= 2)


def test_loguniform_runs_draw_from_the_pool():
    """Config 3 shape: keys from 2^16 distinct values (uint64), weakly
    ascending runs of lengths floor(2^U(1, 16))."""
    n = 1 << 20
    a = inputs.random_runs_loguniform(n, 31)
    assert a.size == n and a.dtype == np.uint64
    assert np.unique(a).size <= 1 << 16
    pool = inputs.distinct_pool(1 << 16, 31)
    assert np.all(np.isin(a[:4096], pool))
    starts, _ = oracle.find_runs(a)
    lengths = np.diff(starts.astype(np.int64))
    assert lengths.max() <= (1 << 16) + 2


def test_batch_arrays_recipe():
    """Config 4: sizes floor(2^U(4, 20)), half permutations, the rest ascending
    runs; offsets delimit the arrays."""
    keys, off = inputs.batch_arrays(400, 77)
    sizes = np.diff(off.astype(np.int64))
    assert off[0] == 0 and off[-1] == keys.size and sizes.size == 400
    assert sizes.min() >= 16 and sizes.max() < 1 << 20
    perms = sum(np.array_equal(np.sort(keys[off[i]:off[i + 1]]), np.arange(sizes[i], dtype=np.uint32))
                for i in range(400))
    assert 140 < perms < 260


def test_request_stream_recipe():
    """Config 5: Poisson arrivals at the given rate, sizes floor(2^U(10, 24)),
    the two kinds half and half."""
    rate = 1000.0
    reqs = inputs.request_stream(4000, 5, rate)
    t = np.array([q["t"] for q in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.diff(t).mean() * rate - 1) < 0.1
    sizes = np.array([q["n"] for q in reqs])
    assert sizes.min() >= 1 << 10 and sizes.max() < 1 << 24
    assert 0.45 < np.mean([q["kind"] == "keys" for q in reqs]) < 0.55
    small = dict(reqs[0], n=5000)
    k, v = inputs.request_keys(small)
    assert (k.dtype, v is None) in ((np.uint32, True), (np.uint64, False))
