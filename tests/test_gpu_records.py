"""Records (Sec. 5: a long key and a pointer, 16 bytes) through
mps_sort_records, against the oracle (GPU).

The oracle sorts (key, input index) pairs stably; the expected payloads are
the input payloads taken in that order.  Keys and payloads must match bit
for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_06909_gb300 import inputs
from paper_2209_06909_gb300 import mps

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2209_06909_gb300 import build
    build.build()
    oracle.build()


def check_records(a: np.ndarray, k: int, seed: int = 1):
    n = a.size
    vals = inputs.record_payload(n, seed)
    want = oracle.sort(a, inputs.payload_index(n), k=k, want_tree=False)
    ok, ov = mps.sort_records(mps.to_device(a, DEV), mps.to_device(vals, DEV), k=k)
    torch.cuda.synchronize()
    assert np.array_equal(mps.to_numpy(ok, a.dtype), want["keys"])
    assert np.array_equal(mps.to_numpy(ov, np.uint64), vals[want["vals"]])


@pytest.mark.parametrize("k", [2, 4, 8, 16])
@pytest.mark.parametrize("n", [1, 2, 17, 1000, 100003, 1 << 20])
def test_records_geometric_sqrt_n(n, k):
    mean = max(1.0, float(np.sqrt(n)))
    check_records(inputs.random_runs_geometric(n, n + k, mean=mean, dtype=np.uint64), k)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_records_heavy_duplicates_stable(dtype):
    check_records(inputs.random_runs_loguniform(300001, 9, log2_hi=10.0, distinct=50, dtype=dtype), 4)


def test_records_edge_cases():
    check_records(np.full(5000, 7, np.uint64), 4)                      # all equal: input order kept
    check_records(np.arange(4096, dtype=np.uint64)[::-1].copy(), 4)    # one strictly descending run
    empty = torch.empty(0, dtype=torch.int64, device=DEV)
    ok, ov = mps.sort_records(empty, empty, k=4)
    assert ok.numel() == 0 and ov.numel() == 0


def test_records_argument_errors():
    a = mps.to_device(np.arange(1000, dtype=np.uint64), DEV)
    v = mps.to_device(np.arange(1000, dtype=np.uint64), DEV)
    with pytest.raises(mps.MpsError):  # payload output overlapping its input
        mps.sort_records(a, v, k=4, out_vals=v)
    small = torch.empty(64, dtype=torch.uint8, device=DEV)
    with pytest.raises(mps.MpsError):
        mps.sort_records(a, v, k=4, ws=small)
