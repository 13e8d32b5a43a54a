"""Thin ctypes binding of libmps.so (include/mps.h).

Argument marshalling only: every step of the sort runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  Keys are
passed as tensors whose element size selects the key type (4 bytes: uint32,
8 bytes: uint64); signed dtypes are accepted and their bits read as unsigned.
If libmps.so is missing the binding raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from .build import LIB

STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "workspace too small", 4: "CUDA runtime error",
          5: "timed out", 6: "budget exceeded", 7: "device-side check failed", 8: "not ready", 9: "cancelled"}

NODE_DTYPE = np.dtype([("first_run", "<u4"), ("end_run", "<u4"), ("power", "u1"), ("degree", "u1"),
                       ("pad", "<u2"), ("parent", "<u4")])


class MpsError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn}: {STATUS.get(code, code)} ({code})")
        self.code = code


class Tree(ctypes.Structure):
    _fields_ = [("run_starts", ctypes.c_void_p), ("run_desc", ctypes.c_void_p), ("powers", ctypes.c_void_p),
                ("node_first", ctypes.c_void_p), ("nodes", ctypes.c_void_p), ("leaf_depth", ctypes.c_void_p),
                ("counts", ctypes.c_void_p)]


class QueueConfig(ctypes.Structure):
    _fields_ = [("d_pool", ctypes.c_void_p), ("pool_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("timeout_ms", ctypes.c_uint32), ("k", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("kt", ctypes.c_int), ("has_payload", ctypes.c_int), ("n", ctypes.c_uint64),
                ("d_keys_in", ctypes.c_void_p), ("d_vals_in", ctypes.c_void_p), ("d_keys_out", ctypes.c_void_p),
                ("d_vals_out", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("device_status", ctypes.c_uint32), ("tag", ctypes.c_uint64),
                ("merge_cost", ctypes.c_uint64), ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double)]


def _result_dict(res: "Result") -> dict:
    return {name: getattr(res, name) for name, _ in Result._fields_}


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("r", ctypes.c_uint64), ("merge_cost", ctypes.c_uint64),
                ("frontier_nodes", ctypes.c_uint64), ("hbm_nodes", ctypes.c_uint64),
                ("num_levels", ctypes.c_uint32), ("hbm_levels", ctypes.c_uint32),
                ("bytes_fused", ctypes.c_uint64), ("bytes_levels", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("device_status", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


EXPORTS = ["mps_workspace_size", "mps_sort_keys", "mps_sort_pairs", "mps_merge_tree", "mps_sort_keys_host",
           "mps_profile_enable", "mps_profile_read", "mps_last_stats", "mps_status_string", "mps_sort_keys_noalloc",
           "mps_batch_workspace_size", "mps_sort_batch", "mps_sort_batch_pairs", "mps_batch_autotune",
           "mps_batch_graph_create", "mps_batch_graph_launch", "mps_batch_graph_destroy",
           "mps_queue_create", "mps_queue_submit", "mps_queue_poll", "mps_queue_wait", "mps_queue_pause",
           "mps_queue_destroy", "mps_records_workspace_size", "mps_sort_records", "mps_sync_status",
           "mps_workspace_size_minrun", "mps_sort_keys_minrun", "mps_sort_pairs_minrun", "mps_sort_keys_tail",
           "mps_batch_tuned_config", "mps_batch_set_config", "mps_sort_keys_host_async"]

# Largest n accepted by mps_sort_keys_noalloc (its scratch is compiled into the library).
NOALLOC_MAX_N = 1 << 20

_lib = None


def lib():
    """Loads libmps.so (built by paper_2209_06909_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB.exists():
        raise RuntimeError(f"{LIB} is missing: build it with paper_2209_06909_gb300.build.build() (no CPU fallback)")
    L = ctypes.CDLL(str(LIB))
    P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    L.mps_workspace_size.argtypes = [U64, I, I, I, ctypes.POINTER(ctypes.c_size_t)]
    L.mps_sort_keys.argtypes = [P, P, U64, I, I, P, ctypes.c_size_t, P, P]
    L.mps_sort_pairs.argtypes = [P, P, P, P, U64, I, I, P, ctypes.c_size_t, P, P]
    L.mps_merge_tree.argtypes = [P, U64, I, I, P, P, ctypes.c_size_t, P]
    L.mps_sort_keys_host.argtypes = [P, P, U64, I, I, P, P, P, ctypes.c_size_t, P]
    L.mps_sort_keys_host_async.argtypes = [P, P, U64, I, I, P, P, P, ctypes.c_size_t, P]
    L.mps_profile_enable.argtypes = [I]
    L.mps_profile_enable.restype = None
    L.mps_profile_read.argtypes = [P, I]
    L.mps_profile_read.restype = I
    L.mps_last_stats.argtypes = [P]
    L.mps_sync_status.argtypes = [P, P]
    L.mps_sync_status.restype = I
    L.mps_workspace_size_minrun.argtypes = [U64, I, I, I, ctypes.c_uint32, ctypes.POINTER(ctypes.c_size_t)]
    L.mps_sort_keys_minrun.argtypes = [P, P, U64, I, I, ctypes.c_uint32, P, ctypes.c_size_t, P, P]
    L.mps_sort_pairs_minrun.argtypes = [P, P, P, P, U64, I, I, ctypes.c_uint32, P, ctypes.c_size_t, P, P]
    L.mps_sort_keys_tail.argtypes = [P, P, U64, I, I, I, P, ctypes.c_size_t, P, P]
    L.mps_sort_keys_tail.restype = I
    L.mps_batch_tuned_config.argtypes = [I, I, U64, ctypes.c_uint32, P, P, P]
    L.mps_batch_tuned_config.restype = I
    L.mps_batch_set_config.argtypes = [I, I, U64, ctypes.c_uint32, I, I]
    L.mps_batch_set_config.restype = I
    for fn in ("mps_workspace_size_minrun", "mps_sort_keys_minrun", "mps_sort_pairs_minrun"):
        getattr(L, fn).restype = I
    L.mps_sort_keys_noalloc.argtypes = [P, P, U64, I, I, P]
    L.mps_sort_keys_noalloc.restype = I
    U32 = ctypes.c_uint32
    L.mps_batch_workspace_size.argtypes = [U64, U32, I, I, I, ctypes.POINTER(ctypes.c_size_t)]
    L.mps_sort_batch.argtypes = [P, P, P, U32, U64, U64, I, I, P, ctypes.c_size_t, P, P]
    L.mps_sort_batch_pairs.argtypes = [P, P, P, P, P, U32, U64, U64, I, I, P, ctypes.c_size_t, P, P]
    L.mps_batch_autotune.argtypes = [P, P, P, U32, U64, U64, I, P, ctypes.c_size_t, P, ctypes.POINTER(I)]
    L.mps_batch_graph_create.argtypes = [P, P, P, U32, U64, U64, I, I, P, ctypes.c_size_t, P, P, ctypes.POINTER(P)]
    L.mps_batch_graph_launch.argtypes = [P, P, I]
    L.mps_batch_graph_destroy.argtypes = [P]
    for fn in ("mps_batch_workspace_size", "mps_sort_batch", "mps_sort_batch_pairs", "mps_batch_autotune",
               "mps_batch_graph_create", "mps_batch_graph_launch", "mps_batch_graph_destroy"):
        getattr(L, fn).restype = I
    L.mps_queue_create.argtypes = [P, ctypes.POINTER(P)]
    L.mps_queue_submit.argtypes = [P, P, ctypes.POINTER(U64)]
    L.mps_queue_poll.argtypes = [P, U64, P]
    L.mps_queue_wait.argtypes = [P, U64, U32, P]
    L.mps_queue_pause.argtypes = [P, I]
    L.mps_queue_destroy.argtypes = [P]
    for fn in ("mps_queue_create", "mps_queue_submit", "mps_queue_poll", "mps_queue_wait", "mps_queue_pause",
               "mps_queue_destroy"):
        getattr(L, fn).restype = I
    L.mps_records_workspace_size.argtypes = [U64, I, I, ctypes.POINTER(ctypes.c_size_t)]
    L.mps_sort_records.argtypes = [P, P, P, P, U64, I, I, P, ctypes.c_size_t, P]
    for fn in ("mps_records_workspace_size", "mps_sort_records"):
        getattr(L, fn).restype = I
    L.mps_status_string.argtypes = [I]
    L.mps_status_string.restype = ctypes.c_char_p
    for fn in ("mps_workspace_size", "mps_sort_keys", "mps_sort_pairs", "mps_merge_tree", "mps_sort_keys_host",
               "mps_sort_keys_host_async", "mps_last_stats"):
        getattr(L, fn).restype = I
    _lib = L
    return L


def _check(fn, code):
    if code in (5, 7):  # device-side check or bounded device wait: report which one
        s = Stats()
        lib().mps_last_stats(ctypes.byref(s))
        err = MpsError(fn, code)
        err.args = (f"{err.args[0]} [device status {s.device_status}]",)
        raise err
    if code != 0:
        raise MpsError(fn, code)


def _key_type(t: torch.Tensor) -> int:
    if t.element_size() == 4:
        return 0
    if t.element_size() == 8:
        return 1
    raise TypeError("keys must have 4-byte or 8-byte elements")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def workspace_size(n: int, key_bytes: int, has_payload: bool = False, k: int = 4) -> int:
    out = ctypes.c_size_t(0)
    _check("mps_workspace_size", lib().mps_workspace_size(n, 0 if key_bytes == 4 else 1, int(has_payload), k,
                                                          ctypes.byref(out)))
    return out.value


def workspace(n: int, key_bytes: int, has_payload: bool = False, k: int = 4, device="cuda") -> torch.Tensor:
    return torch.empty(max(workspace_size(n, key_bytes, has_payload, k), 16), dtype=torch.uint8, device=device)


@dataclass
class TreeBuffers:
    """Device buffers for the tree outputs (sized for n runs)."""
    run_starts: torch.Tensor
    run_desc: torch.Tensor
    powers: torch.Tensor
    node_first: torch.Tensor
    nodes: torch.Tensor
    leaf_depth: torch.Tensor
    counts: torch.Tensor

    @staticmethod
    def alloc(n: int, device) -> "TreeBuffers":
        m = max(n, 1)
        return TreeBuffers(
            run_starts=torch.zeros(m + 2, dtype=torch.int32, device=device),
            run_desc=torch.zeros(m + 1, dtype=torch.uint8, device=device),
            powers=torch.zeros(m + 2, dtype=torch.uint8, device=device),
            node_first=torch.zeros(m + 1, dtype=torch.int32, device=device),
            nodes=torch.zeros((m + 1) * 4, dtype=torch.int32, device=device),
            leaf_depth=torch.zeros(m + 1, dtype=torch.uint8, device=device),
            counts=torch.zeros(4, dtype=torch.int64, device=device))

    def struct(self) -> Tree:
        return Tree(self.run_starts.data_ptr(), self.run_desc.data_ptr(), self.powers.data_ptr(),
                    self.node_first.data_ptr(), self.nodes.data_ptr(), self.leaf_depth.data_ptr(),
                    self.counts.data_ptr())

    def to_numpy(self) -> dict:
        """Host copy trimmed to the actual sizes (canonical encoding)."""
        counts = self.counts.cpu().numpy().astype(np.uint64)
        r, nn, lv, mc = (int(x) for x in counts)
        nodes = self.nodes.cpu().numpy().view(np.uint32)[: 4 * nn].view(NODE_DTYPE)
        return {"r": r, "num_nodes": nn, "num_levels": lv, "merge_cost": mc,
                "run_starts": self.run_starts.cpu().numpy().view(np.uint32)[: r + 1].copy(),
                "run_desc": self.run_desc.cpu().numpy()[:r].copy(),
                "powers": self.powers.cpu().numpy()[: r + 1].copy(),
                "node_first": self.node_first.cpu().numpy().view(np.uint32)[:r].copy(),
                "nodes": nodes.copy(),
                "leaf_depth": self.leaf_depth.cpu().numpy()[:r].copy()}


def sort_keys(keys: torch.Tensor, k: int = 4, out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
              tree: TreeBuffers | None = None, stream=None) -> torch.Tensor:
    """Sorts a device tensor of uint32/uint64 keys (mps_sort_keys)."""
    n = keys.numel()
    kt = _key_type(keys)
    if out is None:
        out = torch.empty_like(keys)
    if ws is None:
        ws = workspace(n, keys.element_size(), False, k, keys.device)
    ts = ctypes.byref(tree.struct()) if tree is not None else None
    _check("mps_sort_keys", lib().mps_sort_keys(keys.data_ptr(), out.data_ptr(), n, kt, k, ws.data_ptr(),
                                                ws.numel(), ts, _stream(stream)))
    _hold(ws)
    return out


def sort_pairs(keys: torch.Tensor, vals: torch.Tensor, k: int = 4, out_keys=None, out_vals=None, ws=None,
               tree: TreeBuffers | None = None, stream=None):
    """Stable key/value sort (mps_sort_pairs); vals are 4-byte payloads."""
    n = keys.numel()
    kt = _key_type(keys)
    if vals.element_size() != 4 or vals.numel() != n:
        raise TypeError("vals must be n 4-byte values")
    out_keys = torch.empty_like(keys) if out_keys is None else out_keys
    out_vals = torch.empty_like(vals) if out_vals is None else out_vals
    if ws is None:
        ws = workspace(n, keys.element_size(), True, k, keys.device)
    ts = ctypes.byref(tree.struct()) if tree is not None else None
    _check("mps_sort_pairs", lib().mps_sort_pairs(keys.data_ptr(), vals.data_ptr(), out_keys.data_ptr(),
                                                  out_vals.data_ptr(), n, kt, k, ws.data_ptr(), ws.numel(), ts,
                                                  _stream(stream)))
    _hold(ws)
    return out_keys, out_vals


def records_workspace(n: int, key_bytes: int, k: int = 4, device="cuda") -> torch.Tensor:
    b = ctypes.c_size_t(0)
    _check("mps_records_workspace_size",
           lib().mps_records_workspace_size(n, 0 if key_bytes == 4 else 1, k, ctypes.byref(b)))
    return torch.empty(max(b.value, 16), dtype=torch.uint8, device=device)


def sort_records(keys: torch.Tensor, vals: torch.Tensor, k: int = 4, out_keys=None, out_vals=None, ws=None,
                 stream=None):
    """Stable sort of records with 8-byte payloads (mps_sort_records)."""
    n = keys.numel()
    kt = _key_type(keys)
    if vals.element_size() != 8 or vals.numel() != n:
        raise TypeError("vals must be n 8-byte values")
    out_keys = torch.empty_like(keys) if out_keys is None else out_keys
    out_vals = torch.empty_like(vals) if out_vals is None else out_vals
    if ws is None:
        ws = records_workspace(n, keys.element_size(), k, keys.device)
    _check("mps_sort_records", lib().mps_sort_records(keys.data_ptr(), vals.data_ptr(), out_keys.data_ptr(),
                                                      out_vals.data_ptr(), n, kt, k, ws.data_ptr(), ws.numel(),
                                                      _stream(stream)))
    _hold(ws)
    return out_keys, out_vals


def merge_tree(keys: torch.Tensor, k: int = 4, ws=None, stream=None) -> TreeBuffers:
    """Run structure, powers and canonical merge tree (mps_merge_tree)."""
    n = keys.numel()
    tb = TreeBuffers.alloc(n, keys.device)
    if ws is None:
        ws = workspace(n, keys.element_size(), False, k, keys.device)
    t = tb.struct()
    _check("mps_merge_tree", lib().mps_merge_tree(keys.data_ptr(), n, _key_type(keys), k, ctypes.byref(t),
                                                  ws.data_ptr(), ws.numel(), _stream(stream)))
    _hold(ws)
    return tb


def sort_keys_host(h_in: torch.Tensor, h_out: torch.Tensor, d_in: torch.Tensor, d_out: torch.Tensor,
                   ws: torch.Tensor, k: int = 4, stream=None) -> None:
    """End-to-end sort from (pinned) host memory through mps_sort_keys_host."""
    n = h_in.numel()
    _check("mps_sort_keys_host", lib().mps_sort_keys_host(h_in.data_ptr(), h_out.data_ptr(), n, _key_type(h_in), k,
                                                          d_in.data_ptr(), d_out.data_ptr(), ws.data_ptr(),
                                                          ws.numel(), _stream(stream)))


def sort_keys_host_async(h_in: torch.Tensor, h_out: torch.Tensor, d_in: torch.Tensor, d_out: torch.Tensor,
                         ws: torch.Tensor, k: int = 4, stream=None) -> None:
    """The same, queued on `stream` without waiting (mps_sort_keys_host_async):
    h_out holds the result once the stream has passed the call.  The caller
    keeps every buffer alive and untouched until then."""
    n = h_in.numel()
    _check("mps_sort_keys_host_async", lib().mps_sort_keys_host_async(h_in.data_ptr(), h_out.data_ptr(), n,
                                                                      _key_type(h_in), k, d_in.data_ptr(),
                                                                      d_out.data_ptr(), ws.data_ptr(), ws.numel(),
                                                                      _stream(stream)))


def sort_keys_noalloc(keys: torch.Tensor, out: torch.Tensor, k: int = 4, stream=None) -> torch.Tensor:
    """Sorts up to NOALLOC_MAX_N keys with the library's built-in scratch
    (mps_sort_keys_noalloc): for callers that cannot allocate device memory.
    Calls that overlap on the GPU share that scratch and must be serialised."""
    _check("mps_sort_keys_noalloc", lib().mps_sort_keys_noalloc(keys.data_ptr(), out.data_ptr(), keys.numel(),
                                                                _key_type(keys), k, _stream(stream)))
    return out


def batch_workspace(n: int, m: int, key_bytes: int, has_payload: bool = False, k: int = 0, device="cuda") -> torch.Tensor:
    out = ctypes.c_size_t(0)
    _check("mps_batch_workspace_size", lib().mps_batch_workspace_size(n, m, 0 if key_bytes == 4 else 1,
                                                                      int(has_payload), k, ctypes.byref(out)))
    return torch.empty(max(out.value, 16), dtype=torch.uint8, device=device)


# The calls return once their kernels are queued, and the statistics of a
# single-array sort stay in its workspace until mps_last_stats reads them: the
# workspace of the most recent call is kept alive here until the next call, so
# that one allocated inside a call is not reused before its sort has finished.
_held = None


def _hold(ws):
    global _held
    _held = ws


def _ptr(t: torch.Tensor | None):
    return t.data_ptr() if t is not None else None


def sort_batch(keys: torch.Tensor, offsets: torch.Tensor, k: int = 0, out: torch.Tensor | None = None,
               ws: torch.Tensor | None = None, max_len: int = 0, stream=None,
               merge_costs: torch.Tensor | None = None) -> torch.Tensor:
    """Sorts every array of a batch (mps_sort_batch); offsets: int64 device
    tensor of m+1 array starts.  merge_costs: optional int64 device tensor of
    m entries that receives each array's merge cost."""
    n, m = keys.numel(), offsets.numel() - 1
    out = torch.empty_like(keys) if out is None else out
    ws = batch_workspace(n, m, keys.element_size(), False, k, keys.device) if ws is None else ws
    _check("mps_sort_batch", lib().mps_sort_batch(keys.data_ptr(), out.data_ptr(), offsets.data_ptr(), m, n, max_len,
                                                  _key_type(keys), k, ws.data_ptr(), ws.numel(), _ptr(merge_costs),
                                                  _stream(stream)))
    _hold(ws)
    return out


def sort_batch_pairs(keys: torch.Tensor, vals: torch.Tensor, offsets: torch.Tensor, k: int = 0, out_keys=None,
                     out_vals=None, ws=None, max_len: int = 0, stream=None, merge_costs: torch.Tensor | None = None):
    n, m = keys.numel(), offsets.numel() - 1
    out_keys = torch.empty_like(keys) if out_keys is None else out_keys
    out_vals = torch.empty_like(vals) if out_vals is None else out_vals
    ws = batch_workspace(n, m, keys.element_size(), True, k, keys.device) if ws is None else ws
    _check("mps_sort_batch_pairs", lib().mps_sort_batch_pairs(keys.data_ptr(), vals.data_ptr(), out_keys.data_ptr(),
                                                              out_vals.data_ptr(), offsets.data_ptr(), m, n, max_len,
                                                              _key_type(keys), k, ws.data_ptr(), ws.numel(),
                                                              _ptr(merge_costs), _stream(stream)))
    _hold(ws)
    return out_keys, out_vals


def batch_autotune(keys: torch.Tensor, offsets: torch.Tensor, out: torch.Tensor, ws: torch.Tensor, max_len: int = 0,
                   stream=None) -> int:
    best = ctypes.c_int(0)
    n, m = keys.numel(), offsets.numel() - 1
    _check("mps_batch_autotune", lib().mps_batch_autotune(keys.data_ptr(), out.data_ptr(), offsets.data_ptr(), m, n,
                                                          max_len, _key_type(keys), ws.data_ptr(), ws.numel(),
                                                          _stream(stream), ctypes.byref(best)))
    return best.value


class BatchGraph:
    """A batch sort captured once in a CUDA graph (mps_batch_graph_*)."""

    def __init__(self, keys, offsets, out, ws, k=0, max_len=0, stream=None, merge_costs=None):
        self.handle = ctypes.c_void_p()
        self.keep = (keys, offsets, out, ws, merge_costs)
        n, m = keys.numel(), offsets.numel() - 1
        _check("mps_batch_graph_create", lib().mps_batch_graph_create(
            keys.data_ptr(), out.data_ptr(), offsets.data_ptr(), m, n, max_len, _key_type(keys), k, ws.data_ptr(),
            ws.numel(), _ptr(merge_costs), _stream(stream), ctypes.byref(self.handle)))

    def launch(self, stream=None, check=False):
        _check("mps_batch_graph_launch", lib().mps_batch_graph_launch(self.handle, _stream(stream), int(check)))

    def close(self):
        if self.handle:
            lib().mps_batch_graph_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Queue:
    """Request queue with continuous batching (mps_queue_*).  The pool tensor is
    the device memory budget; request buffers must stay alive until done."""

    def __init__(self, pool: torch.Tensor, max_inflight: int = 2, max_batch: int = 256, k: int = 4):
        self.pool = pool
        cfg = QueueConfig(pool.data_ptr(), pool.numel() * pool.element_size(), max_inflight, max_batch, 0, k)
        self.handle = ctypes.c_void_p()
        _check("mps_queue_create", lib().mps_queue_create(ctypes.byref(cfg), ctypes.byref(self.handle)))
        self.keep = {}

    def submit(self, keys_in, keys_out, vals_in=None, vals_out=None, tag=0) -> int:
        req = Request(_key_type(keys_in), int(vals_in is not None), keys_in.numel(), keys_in.data_ptr(),
                      vals_in.data_ptr() if vals_in is not None else None, keys_out.data_ptr(),
                      vals_out.data_ptr() if vals_out is not None else None, tag)
        t = ctypes.c_uint64(0)
        _check("mps_queue_submit", lib().mps_queue_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self.keep[t.value] = (keys_in, keys_out, vals_in, vals_out)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000) -> dict:
        res = Result()
        code = lib().mps_queue_wait(self.handle, ticket, timeout_ms, ctypes.byref(res))
        _check("mps_queue_wait", code)
        self.keep.pop(ticket, None)
        return _result_dict(res)

    def poll(self, ticket: int):
        res = Result()
        code = lib().mps_queue_poll(self.handle, ticket, ctypes.byref(res))
        if code == 8:
            return None
        _check("mps_queue_poll", code)
        self.keep.pop(ticket, None)
        return _result_dict(res)

    def pause(self, paused: bool = True):
        _check("mps_queue_pause", lib().mps_queue_pause(self.handle, int(paused)))

    def close(self):
        if self.handle:
            lib().mps_queue_destroy(self.handle)
            self.handle = ctypes.c_void_p()
            self.keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



def batch_tuned_config(key_bytes: int, has_payload: bool, n: int, m: int) -> dict:
    """Configuration chosen by k = 0 for such batches (mps_batch_tuned_config)."""
    k, cf, cl = ctypes.c_int(0), ctypes.c_uint32(0), ctypes.c_uint32(0)
    _check("mps_batch_tuned_config", lib().mps_batch_tuned_config(0 if key_bytes == 4 else 1, int(has_payload), n, m,
                                                                  ctypes.byref(k), ctypes.byref(cf), ctypes.byref(cl)))
    return {"k": k.value, "c_fused": cf.value, "c_level": cl.value, "items_per_thread": cf.value // 256}


def batch_set_config(key_bytes: int, has_payload: bool, n: int, m: int, k: int, tile: int) -> None:
    """Sets the configuration k = 0 selects (mps_batch_set_config)."""
    _check("mps_batch_set_config", lib().mps_batch_set_config(0 if key_bytes == 4 else 1, int(has_payload), n, m, k, tile))

def profile_enable(on: bool = True) -> None:
    lib().mps_profile_enable(int(on))


def profile_read() -> list[dict]:
    cap = 64
    arr = (ProfileEntry * cap)()
    m = lib().mps_profile_read(ctypes.cast(arr, ctypes.c_void_p), cap)
    return [{"name": arr[i].name.decode(), "launches": int(arr[i].launches), "total_ms": float(arr[i].total_ms),
             "bytes": float(arr[i].bytes)} for i in range(min(m, cap))]


def last_stats() -> dict:
    s = Stats()
    _check("mps_last_stats", lib().mps_last_stats(ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in Stats._fields_}


def to_device(a: np.ndarray, device="cuda") -> torch.Tensor:
    """uint32/uint64 numpy array -> device tensor with the same bits."""
    signed = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}[a.dtype]
    return torch.from_numpy(np.ascontiguousarray(a).view(signed)).to(device)


def to_numpy(t: torch.Tensor, dtype) -> np.ndarray:
    """Device tensor -> numpy array of the given unsigned dtype (same bits)."""
    return t.cpu().numpy().view(dtype)


def sync_status(ws: torch.Tensor, stream=None) -> None:
    """Waits for the stream and raises if the last sort on this workspace
    reported a device-side failure (mps_sync_status)."""
    _check("mps_sync_status", lib().mps_sync_status(ws.data_ptr(), _stream(stream)))


def workspace_minrun(n: int, key_bytes: int, has_payload: bool = False, k: int = 4, min_run_len: int = 24,
                     device="cuda") -> torch.Tensor:
    """Workspace for the minimum-run-length sorts (mps_workspace_size_minrun)."""
    b = ctypes.c_size_t(0)
    kt = 0 if key_bytes == 4 else 1
    _check("mps_workspace_size_minrun", lib().mps_workspace_size_minrun(n, kt, int(has_payload), k, min_run_len,
                                                                        ctypes.byref(b)))
    return torch.empty(max(b.value, 16), dtype=torch.uint8, device=device)


def sort_keys_minrun(keys: torch.Tensor, min_run_len: int = 24, k: int = 4, out: torch.Tensor | None = None,
                     ws: torch.Tensor | None = None, tree: TreeBuffers | None = None, stream=None) -> torch.Tensor:
    """Sort with runs extended to min_run_len (mps_sort_keys_minrun)."""
    n = keys.numel()
    out = torch.empty_like(keys) if out is None else out
    if ws is None:
        ws = workspace_minrun(n, keys.element_size(), False, k, min_run_len, keys.device)
    ts = ctypes.byref(tree.struct()) if tree is not None else None
    _check("mps_sort_keys_minrun", lib().mps_sort_keys_minrun(keys.data_ptr(), out.data_ptr(), n, _key_type(keys), k,
                                                              min_run_len, ws.data_ptr(), ws.numel(), ts,
                                                              _stream(stream)))
    _hold(ws)
    return out


TAIL_POLICIES = {"kway_tree": 0, "alg2_pop_k_minus_1": 1, "merge_down": 2}


def sort_keys_tail(keys: torch.Tensor, policy: str, k: int = 4, out: torch.Tensor | None = None,
                   ws: torch.Tensor | None = None, tree: TreeBuffers | None = None, stream=None) -> torch.Tensor:
    """Sort whose run stack is emptied by a final-collapse policy (mps_sort_keys_tail)."""
    n = keys.numel()
    out = torch.empty_like(keys) if out is None else out
    if ws is None:
        ws = workspace(n, keys.element_size(), False, k, keys.device)
    ts = ctypes.byref(tree.struct()) if tree is not None else None
    _check("mps_sort_keys_tail", lib().mps_sort_keys_tail(keys.data_ptr(), out.data_ptr(), n, _key_type(keys), k,
                                                          TAIL_POLICIES[policy], ws.data_ptr(), ws.numel(), ts,
                                                          _stream(stream)))
    _hold(ws)
    return out


def sort_pairs_minrun(keys: torch.Tensor, vals: torch.Tensor, min_run_len: int = 24, k: int = 4, out_keys=None,
                      out_vals=None, ws=None, tree: TreeBuffers | None = None, stream=None):
    """Stable key/value sort with runs extended to min_run_len (mps_sort_pairs_minrun)."""
    n = keys.numel()
    out_keys = torch.empty_like(keys) if out_keys is None else out_keys
    out_vals = torch.empty_like(vals) if out_vals is None else out_vals
    if ws is None:
        ws = workspace_minrun(n, keys.element_size(), True, k, min_run_len, keys.device)
    ts = ctypes.byref(tree.struct()) if tree is not None else None
    _check("mps_sort_pairs_minrun", lib().mps_sort_pairs_minrun(keys.data_ptr(), vals.data_ptr(), out_keys.data_ptr(),
                                                                out_vals.data_ptr(), n, _key_type(keys), k, min_run_len,
                                                                ws.data_ptr(), ws.numel(), ts, _stream(stream)))
    _hold(ws)
    return out_keys, out_vals
