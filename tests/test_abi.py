"""The C ABI library builds, loads and exports every entry point declared in
include/mps.h; host-side argument checks (no GPU needed)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2209_06909_gb300 import build
    path = build.build()
    return ctypes.CDLL(str(path))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "mps.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mps_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2209_06909_gb300 import mps
    assert sorted(mps.EXPORTS) == sorted(n for n in declared_functions())


def test_workspace_size_host_checks(lib):
    from paper_2209_06909_gb300 import mps
    small = mps.workspace_size(1000, 4, False, 4)
    big = mps.workspace_size(1 << 20, 4, False, 4)
    pairs = mps.workspace_size(1 << 20, 8, True, 4)
    assert 0 < small < big < pairs
    with pytest.raises(mps.MpsError) as e:
        mps.workspace_size(1000, 4, False, 3)
    assert e.value.code == 2
    with pytest.raises(mps.MpsError):
        mps.workspace_size(1 << 32, 4, False, 4)


def test_sort_rejects_bad_fan_in_before_any_device_work(lib):
    P = ctypes.c_void_p
    lib.mps_sort_keys.argtypes = [P, P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P, P]
    assert lib.mps_sort_keys(None, None, 10, 0, 3, None, 0, None, None) == 2
    assert lib.mps_sort_keys(None, None, 1 << 32, 0, 4, None, 0, None, None) == 2
    # n >= 2^31 with a minimum run length
    assert mps_minrun_code(lib, 1 << 31) == 2 and mps_minrun_code(lib, (1 << 31) - 1) == 1
    lib.mps_status_string.restype = ctypes.c_char_p
    assert lib.mps_status_string(3) == b"workspace too small"


def mps_minrun_code(lib, n):
    P = ctypes.c_void_p
    lib.mps_sort_keys_minrun.argtypes = [P, P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, P,
                                         ctypes.c_size_t, P, P]
    return lib.mps_sort_keys_minrun(None, None, n, 0, 4, 24, None, 0, None, None)


# C structs shared with the binding: (C type, ctypes class or numpy dtype name)
_STRUCTS = [("mps_tree", "Tree"), ("mps_queue_config", "QueueConfig"), ("mps_request", "Request"),
            ("mps_result", "Result"), ("mps_profile_entry", "ProfileEntry"), ("mps_stats", "Stats")]


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors in the binding have the header's size and field
    offsets (compiles a probe against include/mps.h with the host compiler)."""
    import json
    import shutil
    import subprocess

    import numpy as np

    from paper_2209_06909_gb300 import mps
    gcc = shutil.which("gcc")
    cuda_inc = "/usr/local/cuda/include"
    if gcc is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime_api.h")):
        pytest.skip("needs gcc and the CUDA headers")
    lines = ['#include <stdio.h>', '#include "mps.h"', "int main(void) {", '  printf("{");']
    first = True
    for cname, pyname in _STRUCTS + [("mps_node", None)]:
        fields = ([f for f, _ in getattr(mps, pyname)._fields_] if pyname else list(mps.NODE_DTYPE.names))
        sep = "" if first else ","
        first = False
        lines.append(f'  printf("{sep}\\"{cname}\\": [%zu", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf(", %zu", offsetof({cname}, {f}));')
        lines.append('  printf("]");')
    lines += ['  printf("}\\n");', "  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)])
    got = json.loads(subprocess.check_output([str(exe)]).decode())
    for cname, pyname in _STRUCTS:
        cls = getattr(mps, pyname)
        want = [ctypes.sizeof(cls)] + [getattr(cls, f).offset for f, _ in cls._fields_]
        assert got[cname] == want, (cname, got[cname], want)
    dt = mps.NODE_DTYPE
    assert got["mps_node"] == [dt.itemsize] + [dt.fields[f][1] for f in dt.names]


def _header_prototypes():
    txt = open(os.path.join(ROOT, "include", "mps.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(mps_[a-z_]+)\s*\(([^;{]*?)\)\s*;", txt):
        params = " ".join(m.group(2).split())
        protos[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return protos


def test_binding_argument_counts_match_the_header():
    from paper_2209_06909_gb300 import build, mps
    build.build()
    L = mps.lib()
    protos = _header_prototypes()
    assert set(mps.EXPORTS) <= set(protos)
    checked = 0
    for name in mps.EXPORTS:
        argtypes = getattr(L, name).argtypes
        if argtypes is None:
            continue
        assert len(argtypes) == protos[name], (name, len(argtypes), protos[name])
        checked += 1
    assert checked >= 20


def test_fan_in_sixteen_and_tail_policy_checks(lib):
    """k = 16 is accepted (and sizes a larger workspace than k = 8); the
    final-collapse entry point rejects a policy outside 0..2 and a bad fan-in
    before any device work."""
    from paper_2209_06909_gb300 import mps
    w8 = mps.workspace_size(1 << 20, 4, False, 8)
    w16 = mps.workspace_size(1 << 20, 4, False, 16)
    assert w16 > w8 > 0
    with pytest.raises(mps.MpsError) as e:
        mps.workspace_size(1 << 20, 4, False, 32)
    assert e.value.code == 2
    L = mps.lib()
    assert L.mps_sort_keys_tail(None, None, 10, 0, 4, 3, None, 0, None, None) == 1
    assert L.mps_sort_keys_tail(None, None, 10, 0, 4, -1, None, 0, None, None) == 1
    assert L.mps_sort_keys_tail(None, None, 10, 0, 5, 1, None, 0, None, None) == 2


def test_batch_configuration_host_logic(lib):
    """The configuration that k = 0 selects: default (k = 4, the default
    tiles) until set; per key type, payload flag and mean-size bucket; bad
    fan-in or tile rejected; the workspace for k = 0 covers every tile."""
    from paper_2209_06909_gb300 import mps
    n, m = 3_000_000, 700  # a mean size no other test of this process tunes
    cfg = mps.batch_tuned_config(4, False, n, m)
    assert cfg == {"k": 4, "c_fused": 4096, "c_level": 9216, "items_per_thread": 16}
    mps.batch_set_config(4, False, n, m, 8, 2)
    assert mps.batch_tuned_config(4, False, n, m) == {"k": 8, "c_fused": 2048, "c_level": 4096, "items_per_thread": 8}
    assert mps.batch_tuned_config(4, True, n, m)["k"] == 4      # the payload flag has its own entry
    assert mps.batch_tuned_config(4, False, n, m * 64)["k"] == 4  # so does another mean size
    mps.batch_set_config(8, True, n, m, 16, 1)
    assert mps.batch_tuned_config(8, True, n, m) == {"k": 16, "c_fused": 2048, "c_level": 3072, "items_per_thread": 8}
    for bad_k, bad_tile, code in ((3, 0, 2), (4, 3, 1), (4, -1, 1)):
        with pytest.raises(mps.MpsError) as e:
            mps.batch_set_config(4, False, n, m, bad_k, bad_tile)
        assert e.value.code == code
    # k = 0 sizes the workspace for every configuration it may select
    w0 = mps.batch_workspace(n, m, 4, False, 0, "meta").numel()
    for k in (2, 4, 8, 16):
        assert mps.batch_workspace(n, m, 4, False, k, "meta").numel() <= w0
