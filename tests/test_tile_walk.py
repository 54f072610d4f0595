"""The image-tile walk of the query kernels (encoding.cuh: niv_tile_count, niv_record_of,
NivTileWalk), compiled for the host: every record of an image or record list is visited by
exactly one (tile, thread slot) pair, whatever the grid of persistent warpgroups, and the
incremental walk agrees with the direct record formula.  A walk that skipped or repeated a
tile would leave pixels unwritten or written twice without any numerical test noticing."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "paper_2602_12949_gb300", "csrc", "encoding.cuh")

DRIVER = r"""
#include <cstdio>
#include <vector>
int main() {
    int bad = 0;
    struct C { int64_t n; int32_t w; };
    const C cs[] = {{1920LL * 1080, 1920}, {3840LL * 2160, 3840}, {37 * 29, 37}, {37 * 29 - 5, 37},
                    {960 * 540, 960}, {1000, 0}, {130, 33}, {1, 1}, {127, 0}, {129, 0}, {65, 200}};
    const int grids[] = {1, 3, 152, 1000};
    const int wgs[] = {8, 4, 1};
    for (const C& c : cs)
        for (int B : grids)
            for (int kWG : wgs) {
                const int64_t nt = niv_tile_count(c.n, c.w);
                std::vector<int> seen(c.n, 0);
                for (int b = 0; b < B; ++b)
                    for (int wg = 0; wg < kWG; ++wg)
                        for (int k = 0; k < 128; ++k) {
                            NivTileWalk walk;
                            walk.init((int64_t)b * kWG + wg, (int64_t)B * kWG, k, c.w);
                            for (; walk.tile < nt; walk.next()) {
                                const int64_t r = walk.record(k, c.n, c.w), r2 = niv_record_of(walk.tile, k, c.n, c.w);
                                if (r != r2 && !(r >= c.n && r2 >= c.n)) ++bad;
                                if (r < c.n) ++seen[r];
                            }
                        }
                for (int64_t i = 0; i < c.n; ++i)
                    if (seen[i] != 1) ++bad;
            }
    printf("bad=%d\n", bad);
    return bad != 0;
}
"""


def _tile_section():
    text = open(HEADER).read()
    a, b = text.index("// Image tiles:"), text.index("__host__ __forceinline__ int64_t niv_tile_count_host")
    body = text[a:b].replace("__device__ __forceinline__", "__host__ __device__ __forceinline__")
    return body.replace("__host__ __host__", "__host__")


def test_tile_walk_visits_every_record_once(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "walk.cu"
    src.write_text("#include <cstdint>\n#include <cuda_runtime.h>\n"
                   "struct IoArgs { int32_t sub; int32_t src_width; };\n" + _tile_section() + DRIVER)
    exe = tmp_path / "walk"
    r = subprocess.run([nvcc, "-O2", "-std=c++17", str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "bad=0" in r.stdout, r.stdout + r.stderr
