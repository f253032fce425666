"""Host BVH builder (binned SAH, binary, and its collapse to 4-wide nodes), compiled with the host C++
compiler and checked on CPU: every patch is reached exactly once, every child box contains the boxes of
the patches below it, parent and slot links and leaf back-links agree, and the depth bound holds."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1811_03510_gb300", "csrc")

HARNESS = r'''
#include <cstdio>
#include <vector>
#include <string>
#include "bvh_build.h"
int main(int argc, char **argv) {
    unsigned n; int bins, width;
    if (scanf("%u %d %d", &n, &bins, &width) != 3) return 2;
    std::vector<float> lo(3 * (size_t)n), hi(3 * (size_t)n);
    for (unsigned i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) if (scanf("%f %f", &lo[3 * i + k], &hi[3 * i + k]) != 2) return 2;
    ccs::BvhHost bin, out;
    std::string err;
    if (!ccs::build_bvh(lo, hi, n, bins, bin, err)) { printf("ERR %s\n", err.c_str()); return 0; }
    const ccs::BvhHost *b = &bin;
    if (width == 4) {
        if (!ccs::collapse_bvh4(bin, n, out, err)) { printf("ERR %s\n", err.c_str()); return 0; }
        b = &out;
    }
    printf("OK %zu %d\n", b->nodes.size(), b->max_depth);
    FILE *f = fopen(argv[1], "wb");
    fwrite(b->nodes.data(), 4, b->nodes.size(), f);
    fwrite(b->leaf_parent.data(), 4, b->leaf_parent.size(), f);
    fclose(f);
    return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("bvh")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", CSRC, str(src), os.path.join(CSRC, "bvh_build.cpp"), "-o",
                    str(exe)], check=True)
    return exe, d


def build(harness, lo, hi, width, bins=16):
    exe, d = harness
    n = len(lo)
    text = f"{n} {bins} {width}\n" + "\n".join(" ".join(f"{float(lo[i, k]):.9g} {float(hi[i, k]):.9g}" for k in range(3))
                                               for i in range(n))
    out = d / "out.bin"
    r = subprocess.run([str(exe), str(out)], input=text, capture_output=True, text=True, check=True)
    head = r.stdout.split()
    if head[0] == "ERR":
        return None
    n_floats, depth = int(head[1]), int(head[2])
    raw = out.read_bytes()
    nodes = np.frombuffer(raw[:4 * n_floats], np.float32)
    links = np.frombuffer(raw[4 * n_floats:], np.int32)
    return nodes, links, depth


def check_tree(nodes, links, depth, lo, hi, width):
    per = 16 if width == 2 else 32
    nn = len(nodes) // per
    ints = nodes.view(np.int32).reshape(nn, per)
    f = nodes.reshape(nn, per)
    EMPTY = 0x7FFFFFFF
    seen = np.zeros(len(lo), int)

    def child_box(node, s):
        if width == 2:
            return (np.array([f[node, 4 * a + 2 * s] for a in range(3)]),
                    np.array([f[node, 4 * a + 2 * s + 1] for a in range(3)]))
        return (np.array([f[node, 8 * a + s] for a in range(3)]), np.array([f[node, 8 * a + 4 + s] for a in range(3)]))

    def child_word(node, s):
        return ints[node, 12 + s] if width == 2 else ints[node, 24 + s]

    def walk(node, d):
        assert d <= depth
        leaves = []
        for s in range(width):
            c = child_word(node, s)
            if c == EMPTY:
                continue
            blo, bhi = child_box(node, s)
            if c < 0:
                p = ~c
                seen[p] += 1
                assert np.array_equal(blo, lo[p]) and np.array_equal(bhi, hi[p])   # exact patch box
                shift = 1 if width == 2 else 2
                assert links[p] >> shift == node and links[p] & (width - 1) == s
                sub = [p]
            else:
                parent = ints[c, 14] if width == 2 else ints[c, 28]
                slot = ints[c, 15] if width == 2 else ints[c, 29]
                assert parent == node and slot == s
                sub = walk(c, d + 1)
            assert (blo <= lo[sub].min(0)).all() and (bhi >= hi[sub].max(0)).all()
            leaves += sub
        if width == 4:
            present = sum(child_word(node, s) != EMPTY for s in range(4))
            assert ints[node, 30] == present and (node == 0 or present >= 2 or len(lo) == 1)
        return leaves

    walk(0, 1)
    assert (seen == 1).all()
    return nn


@pytest.mark.parametrize("n", [1, 2, 3, 5, 96, 1000])
def test_binary_and_four_wide_trees_are_valid(harness, n):
    rng = np.random.default_rng(n)
    c = rng.normal(size=(n, 3)).astype(np.float32)
    e = rng.uniform(0.01, 0.2, size=(n, 3)).astype(np.float32)
    lo, hi = c - e, c + e
    b = build(harness, lo, hi, 2)
    nb = check_tree(*b, lo, hi, 2)
    w = build(harness, lo, hi, 4)
    n4 = check_tree(*w, lo, hi, 4)
    if n > 4:
        assert n4 < nb and w[2] < b[2]   # fewer nodes and a shallower tree
        assert w[2] <= (b[2] + 1) // 2 + 1


def test_coincident_boxes_split_by_index(harness):
    lo = np.zeros((40, 3), np.float32)
    hi = np.ones((40, 3), np.float32)
    for width in (2, 4):
        check_tree(*build(harness, lo, hi, width), lo, hi, width)


def test_four_wide_tree_deeper_than_the_stack_is_refused(harness):
    """Boxes at exponentially shrinking offsets make the SAH peel about two patches per level: a binary
    tree of more than 42 levels is still traversable, its 4-wide collapse (more than 21 levels, three
    pushes per level) would overflow the 64-entry traversal stack and is refused."""
    n = 110
    c = np.array([[2.0 ** -k, 0.0, 0.0] for k in range(n)], np.float32)
    e = np.array([[2.0 ** -(k + 3)] * 3 for k in range(n)], np.float32)
    lo, hi = c - e, c + e
    b = build(harness, lo, hi, 2)
    assert b is not None and b[2] > 42
    check_tree(*b, lo, hi, 2)
    assert build(harness, lo, hi, 4) is None
