"""Host logic of the serving queue's admission: the first-fit pool allocator
(csrc/pool_alloc.h), compiled with the host compiler and driven against a
plain interval model (no GPU)."""
import os
import random
import shutil
import subprocess

import pytest

from conftest import ROOT

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include "pool_alloc.h"
// stdin: "size" then ops "a bytes" / "r off bytes"; prints "ok off" / "fail" per alloc,
// and after every op "u used blocks"
int main() {
    size_t size;
    if (scanf("%zu", &size) != 1) return 1;
    mps::PoolAllocator pool(size);
    char op;
    while (scanf(" %c", &op) == 1) {
        if (op == 'a') {
            size_t b, off = 0;
            scanf("%zu", &b);
            if (pool.alloc(b, &off)) printf("ok %zu\n", off); else printf("fail\n");
        } else {
            size_t off, b;
            scanf("%zu %zu", &off, &b);
            pool.release(off, b);
        }
        printf("u %zu %zu\n", pool.used(), pool.free_blocks());
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    d = tmp_path_factory.mktemp("pool")
    (d / "h.cpp").write_text(HARNESS)
    exe = d / "h"
    subprocess.check_call([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2209_06909_gb300", "csrc"),
                           str(d / "h.cpp"), "-o", str(exe)])
    return exe


def run(exe, size, ops):
    lines = [str(size)] + [f"a {b}" if o == "a" else f"r {b[0]} {b[1]}" for o, b in ops]
    out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return out.stdout.split("\n")


def up(x):
    return (max(x, 1) + 255) // 256 * 256


class Model:
    """Free list as sorted (offset, length) intervals; first fit; merge on release."""

    def __init__(self, size):
        self.free = [(0, size)]

    def alloc(self, b):
        b = up(b)
        for i, (o, ln) in enumerate(self.free):
            if ln >= b:
                self.free[i:i + 1] = [(o + b, ln - b)] if ln > b else []
                return o
        return None

    def release(self, off, b):
        self.free.append((off, up(b)))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged


def test_first_fit_and_coalescing(harness):
    ops = [("a", 1000), ("a", 256), ("a", 5000), ("r", (1024, 256)), ("a", 100), ("r", (0, 1000)),
           ("r", (1024, 100)), ("r", (1280, 5000))]
    out = run(harness, 1 << 20, ops)
    allocs = [l for l in out if l.startswith(("ok", "fail"))]
    assert allocs == ["ok 0", "ok 1024", "ok 1280", "ok 1024"]  # the freed hole is reused first
    last = [l for l in out if l.startswith("u")][-1]
    assert last == "u 0 1"  # everything released: one free block again


def test_budget_exhaustion_and_reuse(harness):
    out = run(harness, 4096, [("a", 4096), ("a", 1), ("r", (0, 4096)), ("a", 4000)])
    assert [l for l in out if l.startswith(("ok", "fail"))] == ["ok 0", "fail", "ok 0"]


def test_random_sequences_match_the_model(harness):
    rnd = random.Random(5)
    for trial in range(20):
        size = rnd.choice([1 << 16, 1 << 20, 3 * 1000 * 1000])
        model, live, ops, want = Model(size), [], [], []
        for _ in range(400):
            if live and rnd.random() < 0.45:
                off, b = live.pop(rnd.randrange(len(live)))
                ops.append(("r", (off, b)))
                model.release(off, b)
            else:
                b = rnd.choice([1, 200, 256, 3000, 70000, rnd.randrange(1, size // 4)])
                ops.append(("a", b))
                off = model.alloc(b)
                want.append("fail" if off is None else f"ok {off}")
                if off is not None:
                    live.append((off, b))
        got = run(harness, size, ops)
        assert [l for l in got if l.startswith(("ok", "fail"))] == want
        # used bytes equal the live blocks; live blocks never overlap
        used = sum(up(b) for _, b in live)
        assert [l for l in got if l.startswith("u")][-1].split()[1] == str(used)
        spans = sorted((o, o + up(b)) for o, b in live)
        assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
