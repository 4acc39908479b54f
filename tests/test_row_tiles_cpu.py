"""Binning's row resolution, run on the CPU from the CUDA source itself.

k_bin_count and k_bin_scatter do not evaluate the FP32 tile test once per
tile: `row_tiles` (csrc/mgs_binning.cu) finds the interval of a rectangle
row's tiles that pass it from a few evaluations, because the test is
monotone along the row up to its vertex.  This test lifts `tile_may_hit` and
`row_tiles` out of the .cu file verbatim, compiles them for the host with
the rounding intrinsics mapped to plain IEEE single-precision operations
(`-ffp-contract=off`, so no product is fused unless the source says fma),
and checks on seeded synthetic Gaussians -- ordinary ellipses, needles at
every angle, means far off-screen, rows 1000 tiles wide, near-degenerate
factors, interval ends placed exactly at a tile centre -- that every row's interval (or, where `row_tiles` declines, the
per-tile fallback) is exactly the set of tiles that pass `tile_may_hit`.
The GPU tests compare the lists with the oracle's; this one runs without a
GPU.
"""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2603_11531_gb300", "csrc", "mgs_binning.cu")

SHIM = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <stdint.h>
#include <algorithm>
using std::max;
using std::min;
#define __device__
#define __forceinline__ inline
#define __noinline__
static const int kTile = 16;
static inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
static inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
static inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
static inline float __fmaf_rn(float a, float b, float c) { return fmaf(a, b, c); }
"""

MAIN = r"""
int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    fseek(f, 0, SEEK_END);
    const long sz = ftell(f);
    fseek(f, 0, SEEK_SET);
    const long n = sz / 36;
    float *g = (float *)malloc(sz);
    if (fread(g, 4, n * 9, f) != (size_t)(n * 9)) return 2;
    fclose(f);
    long rows = 0, pairs = 0, mism = 0, declined = 0;
    for (long i = 0; i < n; ++i) {
        const float *q = g + 9 * i;
        const int x0 = (int)q[5], y0 = (int)q[6], x1 = (int)q[7], y1 = (int)q[8];
        for (int ty = y0; ty < y1; ++ty) {
            ++rows;
            int a, b;
            const bool one = row_tiles(q[0], q[1], q[2], q[3], q[4], x0, x1, ty, a, b);
            if (!one) ++declined;
            if (one && a <= b && (a < x0 || b >= x1)) ++mism;   // interval inside the rectangle
            for (int tx = x0; tx < x1; ++tx) {
                const bool ref = tile_may_hit(q[0], q[1], q[2], q[3], q[4], tx, ty);
                const bool got = one ? (tx >= a && tx <= b) : ref;
                pairs += ref;
                mism += ref != got;
            }
        }
    }
    printf("%ld %ld %ld %ld\n", rows, pairs, mism, declined);
    return 0;
}
"""


def _extract():
    src = open(SRC).read()
    a = src.index("__device__ __forceinline__ bool tile_may_hit(")
    b = src.index("// Plan cost of a rectangle row:")
    body = src[a:b]
    assert "bool row_tiles(" in body
    return body


@pytest.fixture(scope="module")
def row_tool(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("rowtiles")
    cpp = d / "rows.cpp"
    cpp.write_text(SHIM + _extract() + MAIN)
    exe = d / "rows"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-o", str(exe), str(cpp)], check=True,
                   capture_output=True, text=True)
    return exe, d


def _gaussians(rng, n, tiles_x, tiles_y, mode):
    """Rows of (m_x, m_y, l11, l21, l22, x_lo, y_lo, x_hi, y_hi) in pixels / tiles."""
    a = np.zeros((n, 9), np.float32)
    W, H = 16 * tiles_x, 16 * tiles_y
    if mode == "ellipses":           # ordinary 2D ellipses on and around the image
        a[:, 0] = rng.uniform(-0.2 * W, 1.2 * W, n)
        a[:, 1] = rng.uniform(-0.2 * H, 1.2 * H, n)
        sx = np.exp(rng.uniform(0.0, 4.5, n))
        sy = np.exp(rng.uniform(0.0, 4.5, n))
        th = rng.uniform(0, np.pi, n)
        c, s = np.cos(th), np.sin(th)
        # covariance R diag(sx^2, sy^2) R^T, inverse = L L^T with L lower triangular:
        # q = (l11 dx + l21 dy)^2 + (l22 dy)^2
        cxx = c * c * sx * sx + s * s * sy * sy
        cyy = s * s * sx * sx + c * c * sy * sy
        cxy = c * s * (sx * sx - sy * sy)
        det = cxx * cyy - cxy * cxy
        ia, ib, ic = cyy / det, -cxy / det, cxx / det          # inverse [[ia, ib], [ib, ic]]
        l11 = np.sqrt(ia)
        l21 = ib / l11
        l22 = np.sqrt(np.maximum(ic - l21 * l21, 1e-30))
        a[:, 2], a[:, 3], a[:, 4] = l11, l21, l22
        r = 3.0 * np.sqrt(np.maximum(cxx, cyy)) + 1.0
        lo_x = np.floor((a[:, 0] - r) / 16)
        hi_x = np.ceil((a[:, 0] + r) / 16)
        lo_y = np.floor((a[:, 1] - r) / 16)
        hi_y = np.ceil((a[:, 1] + r) / 16)
    elif mode == "boundaries":       # an interval end exactly at (or a hair from) a tile centre
        l11 = np.exp(rng.uniform(-4.0, 0.0, n))
        a[:, 2] = np.where(rng.random(n) < 0.5, -l11, l11)
        a[:, 3] = np.where(rng.random(n) < 0.5, 0.0, rng.normal(0, 1e-3, n))
        a[:, 4] = 10.0 ** rng.uniform(-3, 0, n)
        k = rng.integers(2, tiles_x - 2, n)
        # left end of |l11 (x - m_x)| - 7.5 |l11| <= K at the centre of tile k
        # (l21 = 0): K = 3 for half of them, and for the other half the
        # largest bound of the row (3 + the margin at the rectangle's far
        # end, about 2^-18 of |l11| |dxb|), so that rounding decides the tile
        f32 = np.float32
        far = f32(16.0 * tiles_x)
        kmax = f32(3.0) + f32(3.814697265625e-06) * (f32(np.abs(l11)) * (far + f32(7.5)) + f32(4.0))
        K = np.where(rng.random(n) < 0.5, 3.0, kmax.astype(np.float64))
        half = K / l11 + 7.5
        a[:, 0] = 16.0 * k + 8.0 + half + rng.choice([0.0, 1e-4, -1e-4, 0.01, -0.01], n)
        a[:, 1] = rng.uniform(0, H, n)
        lo_x = np.zeros(n)
        hi_x = np.full(n, tiles_x)
        lo_y = np.floor(a[:, 1] / 16) - 1
        hi_y = lo_y + 3
    else:                             # adversarial: needles, far means, extreme factors, wide rows
        a[:, 0] = rng.uniform(-1e5, 2e5, n)
        a[:, 1] = rng.uniform(0, H, n)
        l11 = 10.0 ** rng.uniform(-9, 1, n)
        a[:, 2] = np.where(rng.random(n) < 0.5, -l11, l11)
        a[:, 3] = rng.normal(0, 1, n) * 10.0 ** rng.uniform(-9, 1, n)
        a[:, 4] = 10.0 ** rng.uniform(-5, 1, n)
        lo_x = rng.integers(0, tiles_x, n).astype(np.float64)
        hi_x = lo_x + rng.integers(1, tiles_x, n)
        lo_y = np.floor(a[:, 1] / 16) - rng.integers(0, 3, n)
        hi_y = lo_y + rng.integers(1, 6, n)
    a[:, 5] = np.clip(lo_x, 0, tiles_x)
    a[:, 7] = np.clip(hi_x, 0, tiles_x)
    a[:, 6] = np.clip(lo_y, 0, tiles_y)
    a[:, 8] = np.clip(hi_y, 0, tiles_y)
    keep = (a[:, 7] > a[:, 5]) & (a[:, 8] > a[:, 6])
    return a[keep]


@pytest.mark.parametrize("mode,tiles", [("ellipses", (100, 67)), ("boundaries", (256, 40)),
                                        ("adversarial", (1024, 40))])
def test_row_intervals_equal_the_per_tile_test(row_tool, mode, tiles):
    exe, d = row_tool
    seed, n = {"ellipses": (2603, 20000), "boundaries": (71, 20000), "adversarial": (11531, 6000)}[mode]
    g = _gaussians(np.random.default_rng(seed), n, *tiles, mode)
    path = d / f"{mode}.bin"
    g.astype(np.float32).tofile(path)
    out = subprocess.run([str(exe), str(path)], check=True, capture_output=True, text=True).stdout
    rows, pairs, mism, declined = (int(x) for x in out.split())
    assert rows > 10000 and pairs > 10000, out
    assert mism == 0, out
    # the per-tile fallback is the exception, not the rule
    assert declined <= rows // 100, out


def test_source_markers_present():
    body = _extract()
    assert re.search(r"bool row_tiles\(", body)
    assert "tile_may_hit" in body
