"""Host check of the tiled kernel's tile placement (tvspec_internal.h: tiles_edge_aligned,
tile_count, tile_span), compiled from the library's own header with nvcc.

For every tile shape of the kernel and every image extent up to a few tiles (plus the 512 and
2048 sides of the benchmarked images), along both axes:
  * the stored ranges [a, b) of the tiles partition [0, n) in order (every pixel is written by
    exactly one tile);
  * with edge-aligned placement every tile reads inside the image, starts on a V-column
    boundary (x), stores whole V-column groups, and every stored pixel lies at least the halo
    (TB rows, roundup(TB, V) columns) from each tile edge that is not an image border -- so
    it is exact after up to TB Chambolle iterations (the stencil of one iteration reaches one
    pixel in each direction); the first tile starts at 0 and the last ends at n;
  * otherwise each tile's read range is its stored range widened by the halo on both sides.
The checker is compiled by nvcc (the header also holds device code) but runs on the host
only: no GPU is needed. The test is skipped when nvcc is not found.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2006_10004_gb300", "csrc")

CHECKER = r"""
#include <cstdio>
#include <cstdlib>
#include "tvspec_internal.h"
#include "k_tiled_shapes.inc"
using namespace tvspec;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails++ < 20) { std::printf(__VA_ARGS__); std::printf("\n"); } } } while (0)

// one axis of n pixels: tile extent T, halo h, centre c, alignment unit u (V for x, 1 for y)
static void axis(const char *name, int shape, int n, int T, int h, int c, int u, bool aligned) {
    const int m = tile_count(n, T, c, aligned);
    CHECK(m >= 1, "%s shape %d n %d: %d tiles", name, shape, n, m);
    int next = 0;
    for (int t = 0; t < m; ++t) {
        const TileSpan sp = tile_span(t, m, n, T, h, c, aligned);
        CHECK(sp.a == next, "%s shape %d n %d tile %d: stores from %d, expected %d", name, shape, n, t, sp.a, next);
        CHECK(sp.b > sp.a, "%s shape %d n %d tile %d: empty [%d,%d)", name, shape, n, t, sp.a, sp.b);
        next = sp.b;
        if (aligned) {
            CHECK(sp.s >= 0 && sp.s + T <= n, "%s shape %d n %d tile %d: reads [%d,%d)", name, shape, n, t, sp.s, sp.s + T);
            CHECK(sp.s % u == 0 && sp.a % u == 0 && sp.b % u == 0, "%s shape %d n %d tile %d: unaligned", name, shape, n, t);
            CHECK(sp.first == (t == 0) && sp.last == (t == m - 1), "%s shape %d n %d tile %d: border flags", name, shape, n, t);
            CHECK(sp.a >= sp.s && sp.b <= sp.s + T, "%s shape %d n %d tile %d: stores outside its tile", name, shape, n, t);
            if (!sp.first) CHECK(sp.a - sp.s >= h, "%s shape %d n %d tile %d: left margin %d < %d", name, shape, n, t, sp.a - sp.s, h);
            else CHECK(sp.s == 0, "%s shape %d n %d: first tile reads from %d", name, shape, n, sp.s);
            if (!sp.last) CHECK(sp.s + T - sp.b >= h, "%s shape %d n %d tile %d: right margin %d < %d", name, shape, n, t, sp.s + T - sp.b, h);
            else CHECK(sp.s + T == n, "%s shape %d n %d: last tile ends at %d", name, shape, n, sp.s + T);
        } else {
            CHECK(sp.s == sp.a - h && !sp.first && !sp.last, "%s shape %d n %d tile %d: masked read range", name, shape, n, t);
            CHECK(sp.b <= sp.a + c, "%s shape %d n %d tile %d: stores more than the centre", name, shape, n, t);
        }
    }
    CHECK(next == n, "%s shape %d n %d: stores end at %d", name, shape, n, next);
}

int main() {
    const int shapes[][4] = {TVSPEC_TEST_SHAPES};
    const int n_shapes = sizeof(shapes) / sizeof(shapes[0]);
    int cases = 0;
    for (int i = 0; i < n_shapes; ++i) {
        const int V = shapes[i][0], R = shapes[i][1], RW = shapes[i][2], TB = shapes[i][3];
        const int TW = 32 * V, TH = RW * R, HX = (TB + V - 1) / V * V;
        const int OW = TW - 2 * HX, OH = TH - 2 * TB;
        int sizes[600];
        int ns = 0;
        for (int n = 1; n <= 4 * (TW > TH ? TW : TH) + 3 && ns < 590; ++n) sizes[ns++] = n;
        sizes[ns++] = 512; sizes[ns++] = 1000; sizes[ns++] = 1024; sizes[ns++] = 2048;
        for (int k = 0; k < ns; ++k) {
            const int n = sizes[k];
            // x: the other extent large enough, so alignment depends on W alone
            axis("x", i, n, TW, HX, OW, V, tiles_edge_aligned(TH, n, TH, TW, V));
            axis("y", i, n, TH, TB, OH, 1, tiles_edge_aligned(n, TW, TH, TW, V));
            // and an image too small along the other axis: no edge alignment anywhere
            axis("x", i, n, TW, HX, OW, V, tiles_edge_aligned(TH - 1, n, TH, TW, V));
            cases += 3;
        }
    }
    std::printf("%d axis cases, %d failures\n", cases, fails);
    return fails ? 1 : 0;
}
"""


def _shapes():
    """(V, R, RW, TB) of every tile shape, read from the kernel's shape list."""
    import re

    src = open(os.path.join(CSRC, "k_tiled.cuh")).read()
    block = src[src.index("#define TVSPEC_TILE_SHAPES(X)"):]
    block = block[:block.index("\n\n")]
    rows = re.findall(r"X\((\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\)", block)
    assert rows, "no tile shapes found"
    return [tuple(int(v) for v in r[1:5]) for r in rows]


def _nvcc():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        p = os.path.join(d, "bin", "nvcc") if d else ""
        if p and os.path.exists(p):
            return p
    return shutil.which("nvcc")


def test_tile_placement_partitions_and_keeps_the_halo(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("no nvcc")
    shapes = _shapes()
    (tmp_path / "k_tiled_shapes.inc").write_text(
        "#define TVSPEC_TEST_SHAPES " + ", ".join("{%d, %d, %d, %d}" % s for s in shapes) + "\n")
    (tmp_path / "check.cu").write_text(CHECKER)
    exe = tmp_path / "check"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", CSRC, "-I", str(tmp_path), str(tmp_path / "check.cu"), "-o", str(exe)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    print(out.stdout)
    assert out.returncode == 0, out.stdout[-3000:]
