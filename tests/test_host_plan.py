"""The host-buffer path's chunk plan (csrc/host_plan.h), compiled with the host C++ compiler: at most 8
chunks that cover [0, n) in order, short end chunks around ~2^20-ray middle chunks by default, equal
chunks for a given size, and inner boundaries on multiples of the image alignment."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1811_03510_gb300", "csrc")

HARNESS = r'''
#include <cstdio>
#include "host_plan.h"
int main() {
    unsigned n, chunk; unsigned long long align;
    while (scanf("%u %u %llu", &n, &chunk, &align) == 3) {
        size_t cut[ccs::kHostMaxChunks + 1];
        const unsigned c = ccs::host_chunk_plan(n, chunk, (size_t)align, cut);
        printf("%u", c);
        for (unsigned k = 0; k <= c; ++k) printf(" %zu", cut[k]);
        printf("\n");
    }
    return 0;
}
'''

CASES = [(0, 0, 1), (1, 0, 1), (100000, 0, 1), (1 << 17, 0, 1), (333918, 0, 1), (2073600, 0, 1), (2073600, 0, 15360),
         (3 * (1 << 20) + 5, 0, 1), (8294400, 0, 30720), (2 ** 32 - 1, 0, 1), (700001, 100003, 1), (700001, 1, 1),
         (5000, 0, 1 << 33), (2000001, 0, 15360)]


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("plan")
    (d / "h.cpp").write_text(HARNESS)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, str(d / "h.cpp"), "-o", str(d / "h")], check=True)
    text = "\n".join(f"{n} {c} {a}" for n, c, a in CASES) + "\n"
    out = subprocess.run([str(d / "h")], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    return {case: [int(x) for x in line.split()] for case, line in zip(CASES, out)}


@pytest.mark.parametrize("case", CASES)
def test_plan_covers_the_batch_in_order(plans, case):
    n, chunk, align = case
    c, *cut = plans[case]
    assert 1 <= c <= 8 and len(cut) == c + 1
    assert cut[0] == 0 and cut[-1] == n
    assert all(a <= b for a, b in zip(cut, cut[1:]))
    assert all(x % align == 0 for x in cut[1:-1])


def test_default_plan_shapes(plans):
    c, *cut = plans[(2073600, 0, 1)]   # the 1080p primary batch: 1/8, two middle chunks, 1/8
    assert [b - a for a, b in zip(cut, cut[1:])] == [259200, 777600, 777600, 259200]
    c, *cut = plans[(333918, 0, 1)]    # its diffuse rays: one middle chunk between two short ones
    assert c == 3 and cut[1] == 333918 // 8
    assert plans[(100000, 0, 1)] == [1, 0, 100000]   # below 2^17 rays: one chunk
    c, *cut = plans[(2 ** 32 - 1, 0, 1)]             # the most rays: 262144 at each end, 6 middle chunks
    assert c == 8 and cut[1] == 1 << 18 and cut[-1] - cut[-2] == 1 << 18
    c, *cut = plans[(700001, 100003, 1)]             # a given chunk size: seven equal chunks
    assert c == 7 and max(b - a for a, b in zip(cut, cut[1:])) - min(b - a for a, b in zip(cut, cut[1:])) <= 1
    assert plans[(700001, 1, 1)][0] == 8             # never more than 8
    c, *cut = plans[(5000, 0, 1 << 33)]              # an alignment beyond the batch: one non-empty chunk
    assert cut[-1] == 5000 and all(x == 0 for x in cut[:-1])
