"""The allocation-free sort entry point (GPU).

mps_sort_keys_noalloc serves callers that cannot allocate device memory when
they need a sort (a memory pool they do not own, a host that forbids device
allocations after start-up, a latency-critical path): it uses a scratch array
compiled into the library instead of a caller-provided workspace.  These tests
call it through the C ABI and compare its output with mps_sort_keys, bit for
bit, on two calls in a row -- the second call finds the scratch holding the
first call's leftovers.  This file is collected last on purpose, so that a
run that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2209_06909_gb300 import inputs
from paper_2209_06909_gb300 import mps

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def L():
    from paper_2209_06909_gb300 import build
    build.build()
    return mps.lib()


def _noalloc(L, d_in, d_out, k):
    kt = 0 if d_in.element_size() == 4 else 1
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.mps_sort_keys_noalloc(d_in.data_ptr(), d_out.data_ptr(), d_in.numel(), kt, k, stream)


@pytest.mark.parametrize("k", [2, 4, 8, 16])
def test_noalloc_matches_sort_keys_two_calls(L, k):
    arrays = [inputs.random_permutation(mps.NOALLOC_MAX_N, seed=21 + k),
              inputs.random_runs_uniform_len(300001, seed=22 + k, hi=700),
              inputs.random_runs_loguniform(mps.NOALLOC_MAX_N, seed=23 + k, log2_hi=12.0, distinct=4096)]
    for a in arrays:
        d_in = mps.to_device(a, DEV)
        want = mps.sort_keys(d_in, k=k)
        for _ in range(2):
            got = torch.full_like(d_in, -1)
            assert _noalloc(L, d_in, got, k) == 0
            torch.cuda.synchronize()
            assert torch.equal(got, want)
        assert np.array_equal(mps.to_numpy(got, a.dtype), np.sort(a))


def test_noalloc_rejects_too_large(L):
    n = mps.NOALLOC_MAX_N + 1
    d_in = torch.zeros(n, dtype=torch.int32, device=DEV)
    d_out = torch.empty_like(d_in)
    assert _noalloc(L, d_in, d_out, 4) == 3  # MPS_ERR_WORKSPACE
