"""Sequential CPU oracle for Multiway Powersort (arXiv 2209.06909).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2209_06909_gb300``) never imports, loads or calls it, and the two share
no code: the oracle is plain C in ``mps_oracle.c`` (see its header for the
paper passages each function follows), compiled with gcc, and loaded here with
ctypes.

Outputs use the canonical tree encoding:
  * ``run_starts[r+1]`` (uint32), ``run_desc[r]`` (uint8);
  * ``powers[r+1]`` (uint8) with ``powers[i]`` the power of boundary i between
    run i-1 and run i, and ``powers[0] = powers[r] = 0``;
  * ``nodes`` (structured array, see ``NODE_DTYPE``) sorted by
    (power, first_run), ``parent`` indexing that table (0xFFFFFFFF at the root);
  * ``node_first[r]``: smallest boundary of the node owning boundary i;
  * ``leaf_depth[r]``; ``counts = (r, num_nodes, num_levels, merge_cost)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_BUILD = _HERE / "_build"
_SO = _BUILD / "libmps_oracle.so"
_SRC = _HERE / "mps_oracle.c"

NODE_DTYPE = np.dtype([("first_run", "<u4"), ("end_run", "<u4"), ("power", "u1"),
                       ("degree", "u1"), ("pad", "<u2"), ("parent", "<u4")])
assert NODE_DTYPE.itemsize == 16


_REF_SO = _BUILD / "libstd_stable_sort.so"
_REF_SRC = _HERE / "std_stable_sort.cpp"


def build(force: bool = False) -> Path:
    """Compiles the oracle with gcc (portable flags: runs on x86 and Arm), and
    the std::stable_sort reference used by the CPU baseline with g++."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _SO.exists() or _SO.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _SO.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-shared", "-fPIC", "-Wall",
                               "-o", str(tmp), str(_SRC)])
        os.replace(tmp, _SO)
    if force or not _REF_SO.exists() or _REF_SO.stat().st_mtime < _REF_SRC.stat().st_mtime:
        tmp = _REF_SO.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-shared", "-fPIC", "-Wall",
                               "-o", str(tmp), str(_REF_SRC)])
        os.replace(tmp, _REF_SO)
    return _SO


_ref_lib = None


def std_stable_sort(keys):
    """std::stable_sort of a copy of ``keys`` (uint32 or uint64) on one host
    thread: the second CPU reference of the baseline (not part of the oracle's
    method; sorted keys are unique, so it also cross-checks the oracle)."""
    global _ref_lib
    if _ref_lib is None:
        build()
        _ref_lib = ctypes.CDLL(str(_REF_SO))
    a = np.array(keys, copy=True)
    if a.dtype == np.uint32:
        _ref_lib.ref_stable_sort_u32(ctypes.c_void_p(a.ctypes.data), ctypes.c_uint64(a.size))
    elif a.dtype == np.uint64:
        _ref_lib.ref_stable_sort_u64(ctypes.c_void_p(a.ctypes.data), ctypes.c_uint64(a.size))
    else:
        raise TypeError("keys must be uint32 or uint64")
    return a


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        P = ctypes.c_void_p
        U64 = ctypes.c_uint64
        lib.mpso_sort.argtypes = [P, P, P, P, U64, ctypes.c_int, ctypes.c_uint32, P, P, P, P, P, P, P]
        lib.mpso_sort.restype = ctypes.c_int
        lib.mpso_sort_min_run.argtypes = [P, P, P, P, U64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                          P, P, P, P, P, P, P]
        lib.mpso_sort_min_run.restype = ctypes.c_int
        lib.mpso_find_runs_min.argtypes = [P, U64, ctypes.c_uint32, P, P, P]
        lib.mpso_find_runs_min.restype = U64
        lib.mpso_power.argtypes = [U64, U64, U64, U64, U64, ctypes.c_uint32]
        lib.mpso_power.restype = ctypes.c_uint32
        lib.mpso_find_runs.argtypes = [P, U64, P, P]
        lib.mpso_find_runs.restype = U64
        lib.mpso_tree_from_powers.argtypes = [P, P, U64, P, P, P, P]
        lib.mpso_tree_from_powers.restype = ctypes.c_int
        lib.mpso_tree_from_lengths.argtypes = [P, U64, ctypes.c_uint32, P, P, P, P, P]
        lib.mpso_tree_from_lengths.restype = ctypes.c_int
        lib.mpso_merge_cost_tail.argtypes = [P, U64, ctypes.c_uint32, ctypes.c_int, P]
        lib.mpso_merge_cost_tail.restype = ctypes.c_int
        lib.mpso_tree_tail.argtypes = [P, U64, ctypes.c_uint32, ctypes.c_int, P, P, P, P]
        lib.mpso_tree_tail.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError(f"oracle returned error code {rc}")


def power(n, b1, e1, b2, e2, k):
    """Power_k(n, b1, e1, b2, e2) of Alg. 2 (exact integer arithmetic)."""
    return int(_load().mpso_power(n, b1, e1, b2, e2, k))


def find_runs(keys, min_run_len=1):
    """Greedy run detection (Sec. 2); returns (run_starts[r+1], run_desc[r]).
    With min_run_len > 1 a shorter natural run is extended to min_run_len
    elements (Sec. 5 "Minimal run length"); run_desc then flags a strictly
    decreasing natural part."""
    a = np.ascontiguousarray(keys, dtype=np.uint64)
    n = a.size
    starts = np.zeros(n + 2, np.uint32)
    desc = np.zeros(n + 1, np.uint8)
    r = int(_load().mpso_find_runs_min(_ptr(a), n, int(min_run_len), _ptr(starts), _ptr(desc), None))
    return starts[: r + 1].copy(), desc[:r].copy()


def sort(keys, vals=None, k=4, want_tree=True, min_run_len=1):
    """Multiway Powersort of ``keys`` (uint32 or uint64), optional uint32 payload.

    Returns a dict with ``keys`` (and ``vals``) plus, if ``want_tree``, the run
    structure and canonical tree (see the module docstring).  ``min_run_len``
    > 1 extends shorter natural runs to that length and insertion-sorts them
    (Sec. 5 "Minimal run length"); 1 sorts the natural runs."""
    keys = np.ascontiguousarray(keys)
    if keys.dtype not in (np.uint32, np.uint64):
        raise TypeError("keys must be uint32 or uint64")
    n = keys.size
    kb = keys.dtype.itemsize
    out = np.empty_like(keys)
    vin = vout = None
    if vals is not None:
        vin = np.ascontiguousarray(vals, dtype=np.uint32)
        vout = np.empty_like(vin)
    m = max(n, 1)
    rs = np.zeros(m + 2, np.uint32) if want_tree else None
    rd = np.zeros(m + 1, np.uint8) if want_tree else None
    pw = np.zeros(m + 2, np.uint8) if want_tree else None
    nodes = np.zeros(m, NODE_DTYPE) if want_tree else None
    nf = np.zeros(m + 1, np.uint32) if want_tree else None
    ld = np.zeros(m + 1, np.uint8) if want_tree else None
    counts = np.zeros(4, np.uint64)
    rc = _load().mpso_sort_min_run(_ptr(keys), _ptr(vin), _ptr(out), _ptr(vout), n, kb, k, int(min_run_len),
                                   _ptr(rs), _ptr(rd), _ptr(pw), _ptr(nodes), _ptr(nf), _ptr(ld), _ptr(counts))
    _check(rc)
    r, nn, lv, mc = (int(x) for x in counts)
    res = {"keys": out, "r": r, "num_nodes": nn, "num_levels": lv, "merge_cost": mc}
    if vals is not None:
        res["vals"] = vout
    if want_tree:
        res.update(run_starts=rs[: r + 1].copy(), run_desc=rd[:r].copy(), powers=pw[: r + 1].copy(),
                   nodes=nodes[:nn].copy(), node_first=nf[:r].copy(), leaf_depth=ld[:r].copy())
    return res


def tree_from_powers(powers, run_starts):
    """Alg. 1 (KwayTree_k) from powers[0..r] and run_starts[0..r]."""
    pw = np.ascontiguousarray(powers, dtype=np.uint8)
    rs = np.ascontiguousarray(run_starts, dtype=np.uint32)
    r = rs.size - 1
    m = max(r, 1)
    nodes = np.zeros(m, NODE_DTYPE)
    nf = np.zeros(m + 1, np.uint32)
    ld = np.zeros(m + 1, np.uint8)
    counts = np.zeros(4, np.uint64)
    _check(_load().mpso_tree_from_powers(_ptr(pw), _ptr(rs), r, _ptr(nodes), _ptr(nf), _ptr(ld), _ptr(counts)))
    nn = int(counts[1])
    return {"nodes": nodes[:nn].copy(), "node_first": nf[:r].copy(), "leaf_depth": ld[:r].copy(),
            "r": int(counts[0]), "num_nodes": nn, "num_levels": int(counts[2]), "merge_cost": int(counts[3])}


def tree_from_lengths(lengths, k):
    """Powers (Alg. 2's Power_k) and the stack policy of Alg. 2 on run lengths
    alone, without data; returns powers and the canonical tree."""
    ln = np.ascontiguousarray(lengths, dtype=np.uint64)
    r = ln.size
    m = max(r, 1)
    nodes = np.zeros(m, NODE_DTYPE)
    nf = np.zeros(m + 1, np.uint32)
    ld = np.zeros(m + 1, np.uint8)
    pw = np.zeros(m + 2, np.uint8)
    counts = np.zeros(4, np.uint64)
    _check(_load().mpso_tree_from_lengths(_ptr(ln), r, k, _ptr(nodes), _ptr(nf), _ptr(ld), _ptr(counts), _ptr(pw)))
    nn = int(counts[1])
    return {"powers": pw[: r + 1].copy(), "nodes": nodes[:nn].copy(), "node_first": nf[:r].copy(),
            "leaf_depth": ld[:r].copy(), "r": r, "num_nodes": nn, "num_levels": int(counts[2]),
            "merge_cost": int(counts[3])}


TAIL_POLICIES = {"kway_tree": 0, "alg2_pop_k_minus_1": 1, "merge_down": 2}


def merge_cost_tail(lengths, k, policy):
    """Merge cost of Alg. 2's run stack on run lengths alone, with the final
    collapse done by ``policy``: "kway_tree" (power rule against a final power
    0, the tree of Alg. 1), "alg2_pop_k_minus_1" (Alg. 2's last loop as
    printed) or "merge_down" (the appendix's merge_down taken to any k)."""
    ln = np.ascontiguousarray(lengths, dtype=np.uint64)
    out = np.zeros(1, np.uint64)
    _check(_load().mpso_merge_cost_tail(_ptr(ln), ln.size, k, TAIL_POLICIES[policy], _ptr(out)))
    return int(out[0])


def tree_tail(lengths, k, policy):
    """The full tree of Alg. 2's run stack on run lengths alone, with the stack
    left after the last run emptied by ``policy`` (as in ``merge_cost_tail``).
    Same outputs as ``tree_from_lengths`` minus the powers; a node made by the
    final collapse of "alg2_pop_k_minus_1" or "merge_down" carries the smallest
    power among its boundaries."""
    ln = np.ascontiguousarray(lengths, dtype=np.uint64)
    r = ln.size
    m = max(r, 1)
    nodes = np.zeros(m, NODE_DTYPE)
    nf = np.zeros(m + 1, np.uint32)
    ld = np.zeros(m + 1, np.uint8)
    counts = np.zeros(4, np.uint64)
    _check(_load().mpso_tree_tail(_ptr(ln), r, k, TAIL_POLICIES[policy], _ptr(nodes), _ptr(nf), _ptr(ld), _ptr(counts)))
    nn = int(counts[1])
    return {"nodes": nodes[:nn].copy(), "node_first": nf[:r].copy(), "leaf_depth": ld[:r].copy(), "r": r,
            "num_nodes": nn, "merge_cost": int(counts[3])}
