"""Pins the CPU oracle to things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped term in
the power, an exclusive/inclusive interval end, a wrong tie-break, a wrong tail
rule, a wrong leaf depth) fails at least one of them:
  * values the paper prints for worked examples (Fig. 1, Fig. 3; tests/golden);
  * Def. 3.1 evaluated with exact rationals, written from its sums of run
    fractions rather than from the midpoint form the oracle uses;
  * Alg. 1 restated in Python and the oracle's own Alg. 1 and Alg. 2 builders;
  * closed forms: the sorted multiset, the stable order (key, original index);
  * the paper's invariants and bounds (Fact 3.2, Thm. 3.3, the power range);
  * the squish identity between 2-way and 4-way powers (Sec. 3.1);
  * Tab. 1's merge costs for its random-runs workload (statistical).
"""
import itertools
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2209_06909_gb300 import inputs


# ---------------------------------------------------------------- helpers ---

def power_def31(lengths, i, k):
    """Def. 3.1: a_i = sum_{j<i} l_j - l_{i-1}/2, b_i = sum_{j<i} l_j + l_i/2,
    P_i = min{p : floor(a_i k^p) < floor(b_i k^p)} with exact rationals."""
    n = sum(lengths)
    ell = [Fraction(L, n) for L in lengths]
    prefix = sum(ell[:i], Fraction(0))
    a = prefix - ell[i - 1] / 2
    b = prefix + ell[i] / 2
    p = 0
    while not (math.floor(a * k ** p) < math.floor(b * k ** p)):
        p += 1
    return p


def kway_tree_py(powers, r):
    """Alg. 1 restated: split [lo, hi) at every boundary of minimum power.
    Returns {(first_run, end_run): (power, degree, parent_key)}."""
    nodes = {}

    def rec(lo, hi, parent):
        if hi - lo < 2:
            return
        pmin = min(powers[lo + 1:hi])
        cuts = [i for i in range(lo + 1, hi) if powers[i] == pmin]
        nodes[(lo, hi)] = (pmin, len(cuts) + 1, parent)
        bounds = [lo] + cuts + [hi]
        for a, b in zip(bounds[:-1], bounds[1:]):
            rec(a, b, (lo, hi))

    rec(0, r, None)
    return nodes


def canon_from_oracle(nodes):
    out = {}
    for v in nodes:
        par = None
        if v["parent"] != 0xFFFFFFFF:
            p = nodes[v["parent"]]
            par = (int(p["first_run"]), int(p["end_run"]))
        out[(int(v["first_run"]), int(v["end_run"]))] = (int(v["power"]), int(v["degree"]), par)
    return out


def greedy_runs_bruteforce(a):
    """First run = the longest prefix that is weakly increasing or strictly
    decreasing (for length >= 2 the two kinds exclude each other)."""
    starts, desc, b = [], [], 0
    n = len(a)
    while b < n:
        for L in range(n - b, 0, -1):
            seg = a[b:b + L]
            inc = all(seg[t] <= seg[t + 1] for t in range(L - 1))
            dec = all(seg[t] > seg[t + 1] for t in range(L - 1))
            if inc or dec:
                starts.append(b)
                desc.append(1 if (dec and L >= 2) else 0)
                b += L
                break
    return starts + [n], desc


def lengths_from_starts(rs):
    return np.diff(rs.astype(np.int64))


# ------------------------------------------------------ worked examples ---

def test_fig1_powers_and_trees():
    g = read_golden("fig1_n16.txt")
    L = [int(x) for x in g["run_lengths"].split()]
    assert sum(L) == int(g["n"])
    for k in (2, 4):
        want_p = [int(x) for x in g[f"powers_k{k}"].split()]
        got = oracle.tree_from_lengths(L, k)
        assert list(got["powers"][1:len(L)]) == want_p
        assert [power_def31(L, i, k) for i in range(1, len(L))] == want_p
        want_nodes = set()
        for item in g[f"tree_k{k}"].split("|"):
            fr, er, pw, dg = (int(x) for x in item.split())
            want_nodes.add((fr, er, pw, dg))
        have = {(int(v["first_run"]), int(v["end_run"]), int(v["power"]), int(v["degree"]))
                for v in got["nodes"]}
        assert have == want_nodes
        assert got["merge_cost"] == int(g[f"merge_cost_k{k}"])
        # M = sum_i d_i L_i (Sec. 2.2)
        assert int(np.dot(got["leaf_depth"].astype(np.int64), L)) == got["merge_cost"]


def test_fig3_single_boundary():
    g = read_golden("fig3_power.txt")
    n, b1, e1, b2, e2 = (int(g[x]) for x in ("n", "b1", "e1", "b2", "e2"))
    assert oracle.power(n, b1, e1, b2, e2, 4) == int(g["power_k4"])
    assert oracle.power(n, b1, e1, b2, e2, 2) == int(g["power_k2"])
    # the same boundary through Def. 3.1 with the surrounding runs as fillers
    lengths = [b1, e1 - b1, e2 - b2, n - e2]
    assert power_def31(lengths, 2, 4) == int(g["power_k4"])
    assert power_def31(lengths, 2, 2) == int(g["power_k2"])


# ------------------------------------------------------------ powers ---

@pytest.mark.parametrize("k", [2, 3, 4, 8, 16])
def test_powers_exhaustive_small_against_def31(k):
    """Every composition of n <= 11 into runs: oracle powers == Def. 3.1."""
    for n in range(2, 12):
        for cuts in itertools.product([0, 1], repeat=n - 1):
            L, cur = [], 1
            for c in cuts:
                if c:
                    L.append(cur)
                    cur = 1
                else:
                    cur += 1
            L.append(cur)
            if len(L) < 2:
                continue
            got = oracle.tree_from_lengths(L, k)["powers"]
            for i in range(1, len(L)):
                assert got[i] == power_def31(L, i, k), (L, i, k)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_powers_random_against_def31(k):
    rng = random.Random(7 + k)
    for _ in range(40):
        r = rng.randint(2, 60)
        L = [rng.choice([1, 2, 3, rng.randint(1, 5000)]) for _ in range(r)]
        got = oracle.tree_from_lengths(L, k)["powers"]
        assert [int(x) for x in got[1:r]] == [power_def31(L, i, k) for i in range(1, r)]


def test_squish_identity():
    """Sec. 3.1: P4 = floor((P2 - 1)/2) + 1; likewise P8 = ceil(P2 / 3) and
    P16 = ceil(P2 / 4)."""
    rng = np.random.default_rng(3)
    for _ in range(30):
        L = rng.integers(1, 3000, rng.integers(2, 400))
        p2 = oracle.tree_from_lengths(L, 2)["powers"][1:L.size].astype(int)
        p4 = oracle.tree_from_lengths(L, 4)["powers"][1:L.size].astype(int)
        p8 = oracle.tree_from_lengths(L, 8)["powers"][1:L.size].astype(int)
        p16 = oracle.tree_from_lengths(L, 16)["powers"][1:L.size].astype(int)
        assert np.array_equal(p4, (p2 - 1) // 2 + 1)
        assert np.array_equal(p8, -(-p2 // 3))
        assert np.array_equal(p16, -(-p2 // 4))


def test_power_range_bound():
    """1 <= P_i <= ceil(log_k n + 1) (Sec. 3.3, proof of the stack bound)."""
    rng = np.random.default_rng(11)
    for k in (2, 4, 8, 16):
        for _ in range(20):
            L = rng.integers(1, 100000, rng.integers(2, 300))
            n = int(L.sum())
            P = oracle.tree_from_lengths(L, k)["powers"][1:L.size].astype(int)
            hi = 1
            while k ** (hi - 1) < n:  # smallest hi with hi >= log_k n + 1
                hi += 1
            assert P.min() >= 1 and P.max() <= hi


# -------------------------------------------------------------- runs ---

def test_run_detection_exhaustive_small():
    """All arrays over {0,1,2,3} with n <= 6 against the brute-force greedy."""
    for n in range(0, 7):
        for a in itertools.product(range(4), repeat=n):
            rs, rd = oracle.find_runs(np.array(a, np.uint64))
            want_s, want_d = greedy_runs_bruteforce(list(a))
            assert list(rs) == want_s and list(rd) == want_d, a


def test_run_detection_edge_cases():
    m = (1 << 32) - 1
    cases = {
        "empty": ([], [0], []),
        "one": ([5], [0, 1], [0]),
        "equal": ([7, 7, 7, 7], [0, 4], [0]),
        "strict_desc": ([4, 3, 2, 1], [0, 4], [1]),
        "desc_then_equal": ([4, 3, 3, 2], [0, 2, 4], [1, 1]),
        "extremes": ([m, 0, m, m, 0], [0, 2, 4, 5], [1, 0, 0]),
        "zigzag": ([1, 0, 3, 2, 5, 4], [0, 2, 4, 6], [1, 1, 1]),
    }
    for name, (a, s, d) in cases.items():
        rs, rd = oracle.find_runs(np.array(a, np.uint64))
        assert list(rs) == s and list(rd) == d, name


# -------------------------------------------------------------- trees ---

@pytest.mark.parametrize("k", [2, 3, 4, 8, 16])
def test_stack_tree_equals_kway_tree(k):
    """Alg. 2 (with the power-rule final collapse) builds Alg. 1's tree: the
    oracle's stack builder, its recursive builder and a Python Alg. 1 agree."""
    rng = np.random.default_rng(100 + k)
    for t in range(120):
        r = int(rng.integers(1, 90))
        L = rng.choice([1, 2, 3, 50, 700], r) if t % 2 else rng.integers(1, 2000, r)
        st = oracle.tree_from_lengths(L, k)
        rs = np.concatenate([[0], np.cumsum(L)]).astype(np.uint32)
        rec = oracle.tree_from_powers(st["powers"], rs)
        for key in ("node_first", "leaf_depth"):
            assert np.array_equal(st[key], rec[key])
        assert np.array_equal(st["nodes"], rec["nodes"])
        assert st["merge_cost"] == rec["merge_cost"]
        py = kway_tree_py([int(x) for x in st["powers"]], r)
        assert canon_from_oracle(st["nodes"]) == py


def test_tree_invariants():
    """Degree in [2, k], Fact 3.2 depth(m(B_j)) <= P_j - 1, node_first
    consistency, and M = sum d_i L_i."""
    rng = np.random.default_rng(5)
    for k in (2, 4, 8, 16):
        for _ in range(40):
            L = rng.integers(1, 500, int(rng.integers(2, 200)))
            t = oracle.tree_from_lengths(L, k)
            nodes = t["nodes"]
            assert np.all(nodes["degree"] >= 2) and np.all(nodes["degree"] <= k)
            depth = np.zeros(len(nodes), int)
            for i in range(len(nodes)):
                d, u = 0, int(nodes[i]["parent"])
                while u != 0xFFFFFFFF:
                    d += 1
                    u = int(nodes[u]["parent"])
                depth[i] = d
            lookup = {}
            for i, v in enumerate(nodes):
                lookup[(int(v["power"]), int(v["first_run"]))] = i
            P = t["powers"]
            for j in range(1, L.size):
                # the node owning boundary j has power P_j; its first boundary is node_first[j]
                nf = int(t["node_first"][j])
                assert P[nf] == P[j] and nf <= j
                owners = [i for i, v in enumerate(nodes)
                          if v["power"] == P[j] and v["first_run"] < j < v["end_run"]]
                assert len(owners) == 1
                assert depth[owners[0]] <= int(P[j]) - 1
            assert int(np.dot(t["leaf_depth"].astype(np.int64), L)) == t["merge_cost"]


def test_merge_cost_bounds():
    """Thm. 3.3: M/n <= sum l_i ceil(log_k(1/l_i) + 1) <= H/lg k + 2."""
    rng = np.random.default_rng(9)
    for k in (2, 4, 8):
        for _ in range(40):
            L = rng.integers(1, 10000, int(rng.integers(2, 500)))
            n = int(L.sum())
            M = oracle.tree_from_lengths(L, k)["merge_cost"]
            bound1 = 0
            for Li in L.tolist():
                c = 1  # smallest integer c >= log_k(n / Li) + 1
                while k ** (c - 1) * Li < n:
                    c += 1
                bound1 += Li * c
            H = float(sum((Li / n) * math.log2(n / Li) for Li in L.tolist()))
            assert M <= bound1 <= H * n / math.log2(k) + 2 * n + 1e-6 * n


def test_table1_merge_cost_statistical():
    """Tab. 1: n = 10^8, random runs with mean length 10^4; merge cost of 4P and
    2P within 1.5% of the printed values and the 4P/2P ratio near 0.52."""
    g = read_golden("table1_merge_cost.txt")
    n, mean = int(g["n"]), int(g["mean_run_length"])
    ratios, m4s, m2s = [], [], []
    for seed in range(3):
        rng = np.random.default_rng(1000 + seed)
        L = rng.geometric(1.0 / mean, 2 * n // mean)
        c = np.cumsum(L)
        L = L[: int(np.searchsorted(c, n)) + 1]
        L[-1] -= int(L.sum()) - n
        L = L[L > 0]
        m4 = oracle.tree_from_lengths(L, 4)["merge_cost"]
        m2 = oracle.tree_from_lengths(L, 2)["merge_cost"]
        m4s.append(m4)
        m2s.append(m2)
        ratios.append(m4 / m2)
    assert abs(np.mean(m4s) / int(g["merge_cost_k4"]) - 1) < 0.015
    assert abs(np.mean(m2s) / int(g["merge_cost_k2"]) - 1) < 0.015
    assert abs(np.mean(ratios) - float(g["ratio_k4_over_k2"])) < 0.01


# ------------------------------------------------------------ sorting ---

@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_sort_keys_closed_form(k):
    gens = [
        lambda s: inputs.random_runs_uniform_len(5000, s, hi=200),
        lambda s: inputs.random_permutation(3000, s),
        lambda s: inputs.random_runs_geometric(4000, s, mean=64.0),
        lambda s: inputs.random_runs_loguniform(4000, s, log2_hi=8.0, distinct=64),
    ]
    for gi, gen in enumerate(gens):
        a = gen(gi + 10 * k)
        res = oracle.sort(a, k=k)
        assert np.array_equal(res["keys"], np.sort(a))
        rs, rd = oracle.find_runs(a.astype(np.uint64))
        assert np.array_equal(res["run_starts"], rs) and np.array_equal(res["run_desc"], rd)
        # the tree of the full sort is the tree of its run lengths
        t = oracle.tree_from_lengths(lengths_from_starts(rs), k)
        assert np.array_equal(t["nodes"], res["nodes"]) and t["merge_cost"] == res["merge_cost"]


@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_sort_pairs_is_stable(k):
    """Payload = original index: output must equal the lexicographic order of
    (key, index), the unique stable sort."""
    for s in range(4):
        a = inputs.random_runs_loguniform(6000, s, log2_hi=9.0, distinct=32, dtype=np.uint64)
        if s % 2:
            a = a[::-1].copy()  # strictly descending stretches appear only with distinct neighbours
        idx = inputs.payload_index(a.size)
        res = oracle.sort(a, idx, k=k)
        order = np.lexsort((idx, a))
        assert np.array_equal(res["keys"], a[order])
        assert np.array_equal(res["vals"], idx[order])


def test_sort_edge_cases():
    m = np.uint32((1 << 32) - 1)
    for a in ([], [3], [2, 1], [1, 1], [m, 0, m, 0], [m] * 5, list(range(10, 0, -1))):
        arr = np.array(a, np.uint32)
        for k in (2, 4, 8):
            res = oracle.sort(arr, np.arange(arr.size, dtype=np.uint32), k=k)
            assert np.array_equal(res["keys"], np.sort(arr))
            order = np.lexsort((np.arange(arr.size), arr))
            assert np.array_equal(res["vals"], order.astype(np.uint32))
            if arr.size <= 1:
                assert res["merge_cost"] == 0 and res["num_nodes"] == 0


# ---------------------------------------------------------------- final collapse variants

def _random_lengths(rng, r, hi):
    return rng.integers(1, hi + 1, r).astype(np.uint64)


@pytest.mark.parametrize("k", [2, 3, 4, 8])
def test_tail_kway_tree_policy_is_the_oracle_tree(k):
    """Policy "kway_tree" is the oracle's own final collapse (power rule against
    a final power 0), i.e. the merge cost of Alg. 1's tree."""
    rng = np.random.default_rng(70 + k)
    for _ in range(300):
        L = _random_lengths(rng, int(rng.integers(1, 60)), int(rng.choice([3, 50, 2000])))
        assert oracle.merge_cost_tail(L, k, "kway_tree") == oracle.tree_from_lengths(L, k)["merge_cost"]


def test_tail_policies_agree_for_binary_merges():
    """For k = 2 every node has one boundary, so the power rule, "pop k-1" and
    merge_down all merge the top run with the current one: the same cost."""
    rng = np.random.default_rng(72)
    for _ in range(300):
        L = _random_lengths(rng, int(rng.integers(1, 80)), 1000)
        c = [oracle.merge_cost_tail(L, 2, p) for p in oracle.TAIL_POLICIES]
        assert c[0] == c[1] == c[2]


def test_merge_down_never_costs_more_than_kway_tree():
    """Appendix (merge_down for k = 4): the changed final collapse "can only
    reduce the resulting merge cost" relative to the tree of KwayTree_k."""
    rng = np.random.default_rng(74)
    lower = 0
    for _ in range(2000):
        L = _random_lengths(rng, int(rng.integers(1, 40)), int(rng.choice([4, 100, 5000])))
        md = oracle.merge_cost_tail(L, 4, "merge_down")
        kt = oracle.merge_cost_tail(L, 4, "kway_tree")
        assert md <= kt
        lower += md < kt
    assert lower > 0  # the variants do differ


def test_alg2_printed_tail_can_cost_more():
    """Alg. 2's last loop (pop up to k-1 runs per merge) builds a different tree
    from Alg. 1's at the end and can have a higher merge cost (k = 4)."""
    rng = np.random.default_rng(76)
    higher = 0
    for _ in range(2000):
        L = _random_lengths(rng, int(rng.integers(1, 40)), int(rng.choice([4, 100, 5000])))
        higher += oracle.merge_cost_tail(L, 4, "alg2_pop_k_minus_1") > oracle.merge_cost_tail(L, 4, "kway_tree")
    assert higher > 0


# ---- minimum run length (Sec. 5 "Minimal run length"; the appendix's
# 4-way Powersort extends a natural run shorter than minRunLen to minRunLen
# elements and insertion-sorts it; minRunLen = 1 keeps the natural runs)

def _mixed_inputs(rng, count):
    for i in range(count):
        n = int(rng.integers(0, 300))
        kind = i % 4
        if kind == 0:
            yield rng.integers(0, 5, n).astype(np.uint32)           # many ties
        elif kind == 1:
            yield rng.permutation(n).astype(np.uint32)               # short runs
        elif kind == 2:
            yield inputs.random_runs_uniform_len(n, int(rng.integers(1 << 30)), hi=30) if n else np.zeros(0, np.uint32)
        else:
            yield np.repeat(rng.integers(0, 1 << 31, max(1, n // 7)), 7)[:n].astype(np.uint32)


def test_min_run_len_one_is_the_natural_run_sort():
    rng = np.random.default_rng(80)
    for a in _mixed_inputs(rng, 60):
        for k in (2, 4):
            x, y = oracle.sort(a, k=k), oracle.sort(a, k=k, min_run_len=1)
            for key in ("keys", "run_starts", "run_desc", "powers", "node_first", "leaf_depth", "merge_cost"):
                assert np.array_equal(x[key], y[key]), key


@pytest.mark.parametrize("m0", [2, 3, 7, 24])
def test_min_run_len_run_rule(m0):
    """Every run is the longer of the natural run at its start (the greedy
    scan, pinned above against brute force) and m0 elements, clipped at n;
    only the last run can be shorter than m0."""
    rng = np.random.default_rng(81 + m0)
    for a in _mixed_inputs(rng, 80):
        n = a.size
        rs, _ = oracle.find_runs(a, min_run_len=m0)
        assert rs[0] == 0 and rs[-1] == n and np.all(np.diff(rs.astype(np.int64)) > 0) if n else rs.tolist() == [0]
        for j in range(rs.size - 1):
            s, e = int(rs[j]), int(rs[j + 1])
            natural = int(oracle.find_runs(a[s:])[0][1])  # end of the first natural run of the suffix
            assert e - s == max(natural, min(m0, n - s)), (m0, j, s, e, natural)
            if j + 1 < rs.size - 1:
                assert e - s >= m0


@pytest.mark.parametrize("m0", [2, 5, 24])
def test_min_run_len_sort_is_stable(m0):
    """The output is the sorted multiset and equal keys keep their input
    order: reversal touches only strictly decreasing parts, and insertion
    sort moves an element only past strictly larger keys."""
    rng = np.random.default_rng(90 + m0)
    for a in _mixed_inputs(rng, 60):
        idx = np.arange(a.size, dtype=np.uint32)
        res = oracle.sort(a, vals=idx, k=4, min_run_len=m0)
        order = np.lexsort((idx, a))
        assert np.array_equal(res["keys"], a[order])
        assert np.array_equal(res["vals"], idx[order])


@pytest.mark.parametrize("k,h", [(2, 8), (4, 5), (8, 3)])
def test_min_run_len_equal_runs_give_the_complete_tree(k, h):
    """A zigzag (natural runs of two) with minRunLen 24 and n = 24 k^h has
    r = k^h runs of exactly 24 elements.  For equal runs, boundary i has power
    h - v_k(i) (Def. 3.1: the only multiple of k^-p in the midpoint interval
    can be i / r), so Alg. 1 builds the complete k-ary tree of height h and
    every element sits at depth h: M = h n."""
    n = 24 * k ** h
    a = (np.arange(n, dtype=np.uint32) ^ 1).astype(np.uint32)  # 1, 0, 3, 2, ...
    res = oracle.sort(a, k=k, min_run_len=24)
    r = k ** h
    assert np.array_equal(res["keys"], np.arange(n, dtype=np.uint32))
    assert np.array_equal(res["run_starts"], np.arange(r + 1, dtype=np.uint32) * 24)
    assert res["merge_cost"] == h * n
    assert np.all(res["leaf_depth"] == h)
    assert res["num_levels"] == h

    def vk(i):
        t = 0
        while i % k == 0:
            i //= k
            t += 1
        return t
    assert [int(p) for p in res["powers"][1:r]] == [h - vk(i) for i in range(1, r)]


def _powers_exact(lengths, k):
    """Def. 3.1 with exact rationals: the power of the boundary between
    consecutive runs, from the runs' normalised midpoints."""
    n = sum(lengths)
    s = [0]
    for x in lengths:
        s.append(s[-1] + x)
    out = []
    for i in range(1, len(lengths)):
        a = Fraction(s[i - 1] + s[i], 2 * n)
        b = Fraction(s[i] + s[i + 1], 2 * n)
        p = 0
        while math.floor(a * k ** p) == math.floor(b * k ** p):
            p += 1
        out.append(p)
    return out


# Final-collapse pins written out by hand (k = 4).  Every input has weakly
# increasing powers, so Alg. 2's main loop merges nothing and the whole run
# stack is left to the final collapse; the merge sequences are spelled out in
# the comments (M = sum of merge result sizes, Sec. 2.2).
TAIL_CASES = [
    # L = 1 2 2 2 | 1, powers 1 1 1 2: stack [1 2 2 2], current 1.
    #  kway_tree: {2}+1 = 3, then {1 2 2}+3 = 8             -> 11
    #  pop k-1:   {2 2 2}+1 = 7, then {1}+7 = 8             -> 15
    #  merge_down: x = 4 mod 3 = 1: {2}+1 = 3, {2 2 1}+3 = 8 -> 11
    ((1, 2, 2, 2, 1), [1, 1, 1, 2], {"kway_tree": 11, "alg2_pop_k_minus_1": 15, "merge_down": 11}),
    # L = 1 3 3 1 1 | 1, powers 1 1 1 2 2: stack [1 3 3 1 1], current 1.
    #  kway_tree: {1 1}+1 = 3, then {1 3 3}+3 = 10            -> 13
    #  pop k-1:   {1 1 3}+1 = 6, then {3 1}+6 = 10            -> 16
    #  merge_down: x = 5 mod 3 = 2: {1 1}+1 = 3, {3 3 1}+3 = 10 -> 13
    ((1, 3, 3, 1, 1, 1), [1, 1, 1, 2, 2], {"kway_tree": 13, "alg2_pop_k_minus_1": 16, "merge_down": 13}),
    # L = 10 1 1 1 | 1, powers 1 2 2 2: stack [10 1 1 1], current 1.
    #  kway_tree: {1 1 1}+1 = 4, then {10}+4 = 14             -> 18
    #  pop k-1:   {1 1 1}+1 = 4, then {10}+4 = 14             -> 18
    #  merge_down: x = 4 mod 3 = 1: {1}+1 = 2, {1 1 10}+2 = 14 -> 16
    ((10, 1, 1, 1, 1), [1, 2, 2, 2], {"kway_tree": 18, "alg2_pop_k_minus_1": 18, "merge_down": 16}),
]


@pytest.mark.parametrize("lengths,pw,want", TAIL_CASES)
def test_tail_policies_hand_derived(lengths, pw, want):
    assert _powers_exact(list(lengths), 4) == pw
    for policy, m in want.items():
        assert oracle.merge_cost_tail(list(lengths), 4, policy) == m, policy
    # the KwayTree tail is Alg. 1's tree: its merge cost from the canonical tree
    assert oracle.tree_from_lengths(np.array(lengths), 4)["merge_cost"] == want["kway_tree"]


# The trees of the same three inputs, node by node (first run, end run,
# degree), from the merge sequences written out above.
TAIL_SHAPES = [
    {"kway_tree": {(3, 5, 2), (0, 5, 4)}, "alg2_pop_k_minus_1": {(1, 5, 4), (0, 5, 2)},
     "merge_down": {(3, 5, 2), (0, 5, 4)}},
    {"kway_tree": {(3, 6, 3), (0, 6, 4)}, "alg2_pop_k_minus_1": {(2, 6, 4), (0, 6, 3)},
     "merge_down": {(3, 6, 3), (0, 6, 4)}},
    {"kway_tree": {(1, 5, 4), (0, 5, 2)}, "alg2_pop_k_minus_1": {(1, 5, 4), (0, 5, 2)},
     "merge_down": {(3, 5, 2), (0, 5, 4)}},
]


def _shape(nodes):
    return {(int(x["first_run"]), int(x["end_run"]), int(x["degree"])) for x in nodes}


@pytest.mark.parametrize("case", range(len(TAIL_CASES)))
def test_tail_trees_hand_derived(case):
    lengths, _, want = TAIL_CASES[case]
    for policy, shape in TAIL_SHAPES[case].items():
        t = oracle.tree_tail(np.array(lengths), 4, policy)
        assert _shape(t["nodes"]) == shape, policy
        assert t["merge_cost"] == want[policy], policy


@pytest.mark.parametrize("k", [2, 3, 4, 8, 16])
def test_tail_trees_against_cost_loop(k):
    """The tree builder's merge cost (sum of node sizes, cross-checked inside
    against sum_i depth_i L_i) equals the separate cost-only loop for every
    policy; policy "kway_tree" is Alg. 1's tree node for node; the nodes made
    before the last run (end run < r) are the same under every policy, and a
    final-collapse node has at most k children."""
    rng = np.random.default_rng(90 + k)
    for _ in range(150):
        L = _random_lengths(rng, int(rng.integers(1, 120)), int(rng.choice([3, 50, 2000])))
        r = L.size
        base = oracle.tree_from_lengths(L, k)
        main = {x for x in _shape(base["nodes"]) if x[1] < r}
        for policy in oracle.TAIL_POLICIES:
            t = oracle.tree_tail(L, k, policy)
            assert t["merge_cost"] == oracle.merge_cost_tail(L, k, policy), policy
            sh = _shape(t["nodes"])
            assert {x for x in sh if x[1] < r} == main
            assert all(2 <= x[2] <= k for x in sh)
            if policy == "kway_tree":
                assert np.array_equal(t["nodes"], base["nodes"])
                assert np.array_equal(t["leaf_depth"], base["leaf_depth"])
                assert np.array_equal(t["node_first"], base["node_first"])
