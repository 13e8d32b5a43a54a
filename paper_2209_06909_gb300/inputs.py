"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers; it holds none of the sorting method's
arithmetic.  The same generated arrays feed the CUDA path, the CPU oracle and
the benchmark.  Every generator takes an explicit seed and uses numpy's PCG64.

Workloads (Sec. 5, "random runs" and "random permutations" inputs):
  * ``random_runs_uniform_len``: run lengths uniform in [lo, hi], run values
    uniform 32-bit and sorted, each run ascending with probability ``p_desc``
    complement, else strictly descending;
  * ``random_permutation``: a uniform permutation of 0..n-1;
  * ``random_runs_geometric``: ascending runs with geometric lengths of a given
    mean (support 1, 2, ...), values uniform over the key type;
  * ``random_runs_loguniform``: ascending runs with lengths floor(2^U(a, b)),
    keys drawn from a pool of distinct values (heavy duplicates);
  * ``record_payload``: 64-bit payloads of the records workload (a long key
    and a pointer, random runs of geometric mean sqrt(n));
  * ``batch_arrays`` and ``request_stream`` for the batched and served modes.
The last run is truncated at n.  Generated runs are not necessarily the
detected runs (adjacent runs may fuse); the sort detects runs itself.
"""
from __future__ import annotations

import numpy as np

U32_MAX = (1 << 32) - 1


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _fill_runs(lengths: np.ndarray, draw, sort_desc_mask=None) -> np.ndarray:
    """Concatenates runs; ``draw(m)`` returns m values, each run is sorted
    ascending, and runs flagged in ``sort_desc_mask`` are reversed."""
    parts = []
    for i, L in enumerate(lengths.tolist()):
        v = np.sort(draw(L))
        if sort_desc_mask is not None and sort_desc_mask[i]:
            v = v[::-1]
        parts.append(v)
    return np.concatenate(parts) if parts else np.zeros(0, np.uint32)


def _lengths_until(n: int, draw_len) -> np.ndarray:
    out, total = [], 0
    while total < n:
        chunk = draw_len(max(16, (n - total) // 64 + 1))
        chunk = chunk[chunk > 0]
        c = np.cumsum(chunk)
        take = int(np.searchsorted(c, n - total, side="left")) + 1
        take = min(take, chunk.size)
        out.append(chunk[:take])
        total += int(c[take - 1])
    L = np.concatenate(out).astype(np.int64)
    excess = int(L.sum()) - n
    if excess > 0:
        L[-1] -= excess
    return L[L > 0]


def random_runs_uniform_len(n: int, seed: int, lo: int = 1, hi: int = 2000, p_desc: float = 0.5) -> np.ndarray:
    """uint32 keys: run lengths U[lo, hi]; values U[0, 2^32) sorted per run;
    each run strictly descending with probability p_desc (values redrawn until
    distinct), else ascending."""
    rng = _rng(seed)
    L = _lengths_until(n, lambda m: rng.integers(lo, hi + 1, m))
    desc = rng.random(L.size) < p_desc
    parts = []
    for i, m in enumerate(L.tolist()):
        while True:
            v = np.sort(rng.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32))
            if not desc[i] or m < 2 or np.all(v[1:] != v[:-1]):
                break
        parts.append(v[::-1] if desc[i] else v)
    return np.concatenate(parts) if parts else np.zeros(0, np.uint32)


def random_permutation(n: int, seed: int, dtype=np.uint32) -> np.ndarray:
    """A uniform random permutation of 0..n-1."""
    return _rng(seed).permutation(n).astype(dtype)


def random_runs_geometric(n: int, seed: int, mean: float, dtype=np.uint32) -> np.ndarray:
    """Ascending runs with geometric lengths of the given mean (support >= 1),
    values uniform over the key type."""
    rng = _rng(seed)
    p = 1.0 / float(mean)
    L = _lengths_until(n, lambda m: rng.geometric(p, m))
    bits = 32 if dtype == np.uint32 else 64
    if bits == 32:
        draw = lambda m: rng.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    else:
        draw = lambda m: rng.integers(0, np.iinfo(np.uint64).max, m, dtype=np.uint64, endpoint=True)
    return _fill_runs(L, draw)


def distinct_pool(count: int, seed: int) -> np.ndarray:
    """``count`` distinct uint64 values, sorted."""
    rng = _rng(seed ^ 0x5EED)
    pool = np.unique(rng.integers(0, np.iinfo(np.uint64).max, count * 2, dtype=np.uint64, endpoint=True))
    while pool.size < count:
        pool = np.unique(np.concatenate([pool, rng.integers(0, np.iinfo(np.uint64).max, count, dtype=np.uint64)]))
    return np.sort(rng.choice(pool, count, replace=False))


def random_runs_loguniform(n: int, seed: int, log2_lo: float = 1.0, log2_hi: float = 16.0,
                           distinct: int = 1 << 16, dtype=np.uint64) -> np.ndarray:
    """Ascending (weakly) runs with lengths floor(2^U(log2_lo, log2_hi)); keys
    drawn uniformly from ``distinct`` distinct values (heavy duplicates)."""
    rng = _rng(seed)
    pool = distinct_pool(distinct, seed)
    if dtype == np.uint32:
        pool = np.unique((pool >> np.uint64(32)).astype(np.uint32))
    L = _lengths_until(n, lambda m: np.floor(np.exp2(rng.uniform(log2_lo, log2_hi, m))).astype(np.int64))
    return _fill_runs(L, lambda m: pool[rng.integers(0, pool.size, m)])


def record_payload(n: int, seed: int) -> np.ndarray:
    """uint64 payloads standing in for pointers: uniform 64-bit values."""
    return _rng(seed ^ 0xACE).integers(0, np.iinfo(np.uint64).max, n, dtype=np.uint64, endpoint=True)


def payload_index(n: int) -> np.ndarray:
    """uint32 payload = original index."""
    return np.arange(n, dtype=np.uint32)


def batch_arrays(count: int, seed: int, log2_lo: float = 4.0, log2_hi: float = 20.0):
    """Independent uint32 arrays with sizes floor(2^U(log2_lo, log2_hi)); each is
    a random permutation with probability 0.5, else ascending random runs of
    geometric mean length sqrt(size).  Returns (keys concatenated, offsets[m+1])."""
    rng = _rng(seed)
    sizes = np.floor(np.exp2(rng.uniform(log2_lo, log2_hi, count))).astype(np.int64)
    kinds = rng.random(count) < 0.5
    arrays = []
    for i, (m, perm) in enumerate(zip(sizes.tolist(), kinds.tolist())):
        s = int(rng.integers(0, 1 << 62))
        if perm:
            arrays.append(random_permutation(m, s))
        else:
            arrays.append(random_runs_geometric(m, s, mean=max(1.0, float(np.sqrt(m)))))
    offsets = np.zeros(count + 1, np.uint64)
    offsets[1:] = np.cumsum(sizes)
    return np.concatenate(arrays).astype(np.uint32), offsets


def request_stream(count: int, seed: int, rate_per_s: float, log2_lo: float = 10.0, log2_hi: float = 24.0):
    """Poisson arrivals of sort requests.  Each request: arrival time (s), kind
    ('keys' = uint32 keys, 'pairs' = uint64 keys + uint32 payload, 50/50), size
    floor(2^U(log2_lo, log2_hi)), and a seed for its random-runs content (runs
    log-uniform in [2, 2^16], keys from 2^16 distinct values)."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, count)
    t = np.cumsum(gaps)
    sizes = np.floor(np.exp2(rng.uniform(log2_lo, log2_hi, count))).astype(np.int64)
    kinds = np.where(rng.random(count) < 0.5, "keys", "pairs")
    seeds = rng.integers(0, 1 << 62, count)
    return [dict(t=float(t[i]), kind=str(kinds[i]), n=int(sizes[i]), seed=int(seeds[i])) for i in range(count)]


def request_keys(req: dict):
    """Materialises one request of ``request_stream``: (keys, vals or None)."""
    n, s = req["n"], req["seed"]
    if req["kind"] == "keys":
        return random_runs_loguniform(n, s, dtype=np.uint32), None
    return random_runs_loguniform(n, s, dtype=np.uint64), payload_index(n)
