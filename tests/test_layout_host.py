"""The block-group layout of the 7-point warp-tile step kernel (lat_layout.cuh),
compiled for the host: for every tile count, group count and plane count
tried, each (y tile, z plane) unit of a step is marched by exactly one group,
and the groups' work (planes, plus 2.5 per extra run) is balanced where the
groups march the tiles in step."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0911_5692_gb300", "csrc")

PROGRAM = r'''
#include <algorithm>
#include <cstdio>
#include <vector>
#include "lat_layout.cuh"
using lat::Layout;
using lat::tile_layout;

static int check(int T, int G, int zn, double* spread)
{
    std::vector<int> cover((size_t)T * zn, 0);
    double hi = 0, lo = 1e30;
    for (int g = 0; g < G; g++) {
        const Layout L = tile_layout(T, G, g, zn);
        int runs = 0, load = 0;
        for (int u = L.ubeg; u < L.uend;) {
            const int yt = u / L.zspan, zrel = u % L.zspan, z0 = L.zoff + zrel;
            const int nz = std::min(L.zspan - zrel, L.uend - u);
            if (yt < 0 || yt >= T || z0 < 0 || nz < 1 || z0 + nz > zn) return 1;
            for (int z = z0; z < z0 + nz; z++) cover[(size_t)yt * zn + z]++;
            u += nz;
            runs++;
            load += nz;
        }
        const double cost = load + 2.5 * (runs > 0 ? runs - 1 : 0);
        hi = std::max(hi, cost);
        lo = std::min(lo, cost);
    }
    for (int c : cover)
        if (c != 1) return 1;
    *spread = hi / lo;
    return 0;
}

int main()
{
    double s;
    for (int T : {1, 2, 4, 8, 16, 32, 64})
        for (int G = 1; G <= 160; G++)
            for (int zn : {1, 2, 3, 5, 7, 16, 31, 64, 100, 128, 256})
                if (check(T, G, zn, &s)) { printf("bad T=%d G=%d zn=%d\n", T, G, zn); return 1; }
    // the benchmark geometries: 512^3 (32 tiles, 38 groups), 256^3 (16, 76), a
    // 512^3 slab of 128 planes
    const int cases[3][3] = {{32, 38, 512}, {16, 76, 256}, {32, 38, 128}};
    for (auto& c : cases) {
        if (check(c[0], c[1], c[2], &s)) return 1;
        printf("spread %d %d %d %.4f\n", c[0], c[1], c[2], s);
    }
    printf("ok\n");
    return 0;
}
'''


def test_layout_covers_every_unit_once(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "layout.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "layout"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    lines = out.stdout.splitlines()
    assert lines[-1] == "ok"
    spreads = [float(l.split()[-1]) for l in lines if l.startswith("spread")]
    assert len(spreads) == 3 and max(spreads[:2]) <= 1.05, spreads
