"""Host arithmetic of the static-obstacle grid's table region
(csrc/priest_internal.cuh: grid_side, grid_layout, table_layout), compiled
with the system C++ compiler: for every static-obstacle count up to the
library's limit, the cell-start array holds nx * ny + 1 entries for any grid
the set-up kernel may choose (nx, ny <= grid_side), the entry array holds the
at most 4 cells per obstacle, the set-up's range scratch holds one word per
obstacle, every block is 32-byte aligned (the kernel stages the region with
16-byte loads), and the FP32 table allocation, sized by the obstacle count,
holds the region of every static count up to it.  No GPU needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2309_08235_gb300", "csrc")
INC = os.path.join(ROOT, "include")

DRIVER = r"""
#include <cstdio>
#include "priest_internal.cuh"

using namespace priest;

int main() {
    if (kGridMinStatic != 16 || kGridCellMax != 64) { std::puts("constants changed"); return 1; }
    size_t prev = 0;
    for (int ns = 0; ns <= PRIEST_MAX_OBS; ++ns) {
        const GridLayout g = grid_layout(ns);
        if (g.start != 8 || g.start % 8 || g.ent % 8 || g.rng % 8 || g.total % 8) { std::printf("align %d\n", ns); return 1; }
        if (ns < kGridMinStatic) {
            if (g.ent != 8 || g.rng != 8 || g.smem != 8 || g.total != 8) { std::printf("header only %d\n", ns); return 1; }
        } else {
            const int gs = grid_side(ns);
            if (gs < 4 || gs > 32 || (gs * gs < 2 * ns && gs != 32)) { std::printf("side %d %d\n", ns, gs); return 1; }
            if (2 * (g.ent - g.start) < size_t(gs * gs + 1)) { std::printf("starts %d\n", ns); return 1; }
            if (2 * (g.rng - g.ent) < size_t(4 * ns)) { std::printf("entries %d\n", ns); return 1; }
            if (g.total - g.rng < size_t(ns)) { std::printf("ranges %d\n", ns); return 1; }
            if (g.smem != g.rng) { std::printf("smem %d\n", ns); return 1; }
            if (4 * ns > 65535) { std::printf("uint16 entries %d\n", ns); return 1; }
        }
        if (g.total < prev) { std::printf("not monotone %d\n", ns); return 1; }
        prev = g.total;
    }
    const int dims[2] = {2, 3}, nps[3] = {20, 100, 512};
    for (int d : dims)
        for (int np : nps)
            for (int n_obs = 0; n_obs <= PRIEST_MAX_OBS; n_obs += 7) {
                const TableLayout t = table_layout(d, 11, 5, np, n_obs);
                if (t.grid != t.total || t.grid % 8) { std::printf("grid offset %d\n", n_obs); return 1; }
                for (int ns = 0; ns <= n_obs; ns += 5)
                    if (t.total32 - t.grid < grid_layout(ns).total) { std::printf("alloc %d %d\n", n_obs, ns); return 1; }
            }
    std::puts("ok");
    return 0;
}
"""


def cuda_include():
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


def test_grid_layout_capacities(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = cuda_include()
    if not cxx or not inc:
        pytest.skip("no C++ compiler or CUDA headers")
    src = tmp_path / "grid_layout_check.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "grid_layout_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", INC, "-I", inc, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
