"""Host logic of the serving loop's budget allocator (csrc/arena.h), compiled
with the system C++ compiler and driven through random alloc / release
sequences: ranges never overlap, stay inside the capacity, free ranges are
fully merged, used bytes are accounted exactly, the peak never exceeds the
budget, and once everything is released the whole capacity is one range
again.  No GPU needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2309_08235_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <utility>
#include "arena.h"

static unsigned long long rs = 88172645463325252ull;
static unsigned long long nxt() { rs ^= rs << 13; rs ^= rs >> 7; rs ^= rs << 17; return rs; }

int main() {
    const size_t cap = size_t(1) << 24;
    priest::Arena a(cap + 100, 256);  // capacity rounds down to the alignment
    if (a.capacity() != cap || !a.check()) { std::puts("bad init"); return 1; }
    std::vector<std::pair<size_t, size_t>> live;  // (offset, requested bytes)
    size_t fails = 0;
    for (int step = 0; step < 200000; ++step) {
        const bool do_alloc = live.empty() || (nxt() % 100) < 55;
        if (do_alloc) {
            const size_t bytes = 1 + nxt() % (size_t(1) << (8 + nxt() % 12));
            size_t off = 0;
            const size_t before = a.used();
            if (a.alloc(bytes, &off)) {
                if (off % 256 || off + a.round(bytes) > cap) { std::puts("out of range"); return 1; }
                for (auto &r : live) {
                    const size_t lo = r.first, hi = r.first + a.round(r.second);
                    if (off < hi && lo < off + a.round(bytes)) { std::puts("overlap"); return 1; }
                }
                if (a.used() != before + a.round(bytes)) { std::puts("used"); return 1; }
                live.push_back({off, bytes});
            } else {
                ++fails;
                if (a.largest_free() >= a.round(bytes)) { std::puts("false failure"); return 1; }
                if (a.used() != before) { std::puts("failed alloc changed state"); return 1; }
            }
        } else {
            const size_t k = nxt() % live.size();
            a.release(live[k].first, live[k].second);
            live[k] = live.back();
            live.pop_back();
        }
        if (a.peak() > cap || a.used() > a.peak()) { std::puts("peak"); return 1; }
        if ((step & 1023) == 0 && !a.check()) { std::puts("invariant"); return 1; }
    }
    for (auto &r : live) a.release(r.first, r.second);
    if (a.used() != 0 || a.free_ranges() != 1 || a.largest_free() != cap || !a.check()) {
        std::puts("not merged back");
        return 1;
    }
    std::printf("ok %zu\n", fails);
    return fails > 0 ? 0 : 2;  // the sequence must have hit a full arena at least once
}
"""


def test_arena_invariants(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    src = tmp_path / "arena_check.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "arena_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
