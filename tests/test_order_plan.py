"""Tile geometry of the work order (csrc/order_plan.h), compiled with the host C++ compiler: tiles cover
every ray once, samples lie in the image, and placing the tiles in descending order of random keys
(stable within a key) through tile_entry gives a permutation of the rays in which each tile's rays are
contiguous and row-major.  Images with ragged edges and a partial last row, one-pixel-wide images, a
width beyond the batch, and runs of 32 rays."""
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1811_03510_gb300", "csrc")

HARNESS = r'''
#include <cstdio>
#include <vector>
#include "order_plan.h"
using namespace ccs;
template <class S> int run(unsigned n, unsigned w, unsigned seed) {
    const OrderGeom g = order_geom<S>(n, w);
    std::vector<unsigned> key(g.n_tiles), size(g.n_tiles);
    unsigned long long total = 0, h = seed * 2654435761u + 1;
    for (unsigned t = 0; t < g.n_tiles; ++t) {
        h = h * 6364136223846793005ull + 1442695040888963407ull;
        key[t] = (unsigned)(h >> 60);   // 0..15
        size[t] = tile_size<S>(g, (t % g.tiles_x) * S::TW, (t / g.tiles_x) * S::TH);
        total += size[t];
        for (unsigned s = 0; s < S::SPT; ++s) {
            unsigned j;
            if (tile_sample<S>(g, t, s, &j) && j >= n) { printf("BADSAMPLE\n"); return 0; }
        }
    }
    if (total != n) { printf("BADSIZE %llu\n", total); return 0; }
    std::vector<unsigned> pos(g.n_tiles);   // stable counting sort, keys descending
    unsigned p = 0;
    for (int k = kOrderKeys - 1; k >= 0; --k)
        for (unsigned t = 0; t < g.n_tiles; ++t)
            if ((int)key[t] == k) { pos[t] = p; p += size[t]; }
    std::vector<long long> perm(n, -1);
    for (unsigned t = 0; t < g.n_tiles; ++t) {
        const unsigned x0 = (t % g.tiles_x) * S::TW, y0 = (t / g.tiles_x) * S::TH;
        unsigned last = 0, count = 0;
        for (unsigned e = 0; e < S::TW * S::TH; ++e) {
            unsigned j, off;
            if (!tile_entry<S>(g, x0, y0, e, &j, &off)) continue;
            if (j >= n || off >= size[t] || perm[pos[t] + off] != -1) { printf("BADENTRY\n"); return 0; }
            if (count && j <= last) { printf("BADORDER\n"); return 0; }
            perm[pos[t] + off] = j;
            last = j;
            ++count;
        }
        if (count != size[t]) { printf("BADCOUNT\n"); return 0; }
    }
    std::vector<char> seen(n, 0);
    for (unsigned q = 0; q < n; ++q) {
        if (perm[q] < 0 || seen[perm[q]]) { printf("NOTPERM\n"); return 0; }
        seen[perm[q]] = 1;
    }
    printf("OK %u %u\n", g.n_tiles, order_blocks<S>(g));
    return 0;
}
int main() {
    unsigned n, w, seed;
    while (scanf("%u %u %u", &n, &w, &seed) == 3) {
        if (w) run<ImageShape>(n, w, seed); else run<RunShape>(n, n, seed);
    }
    return 0;
}
'''

CASES = [(1920 * 1080, 1920), (333 * 77 + 100, 333), (37 * 5, 37), (1000, 1), (5000, 4096), (63, 64),
         (1000, 1 << 30), (1, 1), (64 * 64, 64), (100003, 0), (31, 0), (1, 0), (4001, 0)]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("order")
    (d / "h.cpp").write_text(HARNESS)
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", CSRC, str(d / "h.cpp"), "-o", str(d / "h")], check=True)
    text = "\n".join(f"{n} {w} {k + 1}" for k, (n, w) in enumerate(CASES)) + "\n"
    out = subprocess.run([str(d / "h")], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    return dict(zip(CASES, out))


@pytest.mark.parametrize("case", CASES)
def test_tiles_place_every_ray_once(results, case):
    assert results[case].startswith("OK"), results[case]


def test_tile_counts(results):
    assert results[(1920 * 1080, 1920)] == "OK 32400 507"    # 240 x 135 tiles of 8 x 8, 64 per block
    assert results[(100003, 0)] == f"OK {(100003 + 31) // 32} {int(np.ceil((100003 + 31) // 32 / 32))}"
