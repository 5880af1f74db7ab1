"""Host check of the FP32 BS-record layout (rec_brick_index in common.cuh, compiled for the host
with nvcc): every site of a box gets its own slot below rec_brick_count, and the two sites a
two-site sweep thread handles (x even, x + 1) get adjacent slots starting on an even slot, i.e.
one aligned 32-byte sector of 16-byte records. Odd and even sizes, 2D and 3D."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1105_2904_gb300", "csrc")

PROGRAM = r'''
#include <cstdio>
#include <vector>
#include "common.cuh"
using namespace lbmp;
int check(int nx, int ny, int nz)
{
    Geom g{};
    g.nx = nx; g.ny = ny; g.nz = nz;
    const size_t n = rec_brick_count(g);
    std::vector<char> used(n, 0);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const unsigned r = rec_brick_index(g, x, y, z);
                if (r >= n || used[r]) return 1;
                used[r] = 1;
                if (x % 2 == 0 && x + 1 < nx) {
                    const unsigned r1 = rec_brick_index(g, x + 1, y, z);
                    if (r % 2 != 0 || r1 != r + 1) return 2;
                }
            }
    if (n > 8 * (size_t)((nx + 1) / 2) * ((ny + 1) / 2) * ((nz + 1) / 2)) return 3;
    return 0;
}
int main()
{
    const int dims[][3] = {{1, 1, 1}, {2, 2, 2}, {7, 5, 3}, {8, 6, 4}, {33, 17, 9}, {64, 48, 1}, {65, 31, 1}, {10, 1, 1}};
    for (auto& d : dims) {
        const int e = check(d[0], d[1], d[2]);
        if (e) { std::printf("fail %d %d %d: %d\n", d[0], d[1], d[2], e); return 1; }
    }
    std::printf("ok\n");
    return 0;
}
'''


def test_brick_index_is_a_bijection_with_pairs_in_one_sector(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "layout.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "layout"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
