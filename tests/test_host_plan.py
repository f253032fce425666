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


BATCH_HARNESS = r'''
#include <cstdio>
#include <vector>
#include "host_plan.h"
int main() {
    unsigned nb;
    while (scanf("%u", &nb) == 1) {
        std::vector<unsigned> n(nb), c(nb);
        std::vector<size_t> a(nb);
        for (unsigned j = 0; j < nb; ++j) {
            unsigned long long al;
            if (scanf("%u %u %llu", &n[j], &c[j], &al) != 3) return 1;
            a[j] = (size_t)al;
        }
        const std::vector<ccs::HostChunk> ch = ccs::host_batch_chunks(nb, n.data(), c.data(), a.data());
        printf("%zu", ch.size());
        for (const ccs::HostChunk &k : ch) printf(" %u %zu %zu", k.j, k.a, k.m);
        printf("\n");
    }
    return 0;
}
'''

BATCH_CASES = [
    [(2073600, 0, 15360), (333918, 0, 1)],                 # the bench's end-to-end step
    [(2073600, 0, 15360), (0, 0, 1), (333918, 40000, 1), (17, 0, 1)],
    [(0, 0, 1)],
    [],
    [(5, 1, 1), (5, 1, 1)],                                # at most 8 chunks per batch
    [(8294400, 0, 30720), (1399374, 0, 1), (1, 0, 1)],
]


def test_batch_chunks_are_each_batch_plan_in_order(plans, tmp_path):
    """The chunk list of several batches is the concatenation of the batches' own plans, in batch order,
    with empty chunks and empty batches left out."""
    (tmp_path / "b.cpp").write_text(BATCH_HARNESS)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, str(tmp_path / "b.cpp"), "-o", str(tmp_path / "b")],
                   check=True)
    text = "\n".join(" ".join([str(len(bs))] + [f"{n} {c} {a}" for n, c, a in bs]) for bs in BATCH_CASES) + "\n"
    out = subprocess.run([str(tmp_path / "b")], input=text, capture_output=True, text=True, check=True).stdout
    for bs, line in zip(BATCH_CASES, out.split("\n")):
        count, *rest = [int(x) for x in line.split()]
        got = [tuple(rest[3 * i:3 * i + 3]) for i in range(count)]
        want = []
        for j, (n, c, a) in enumerate(bs):
            if n == 0:
                continue
            single = plans.get((n, c, a))
            if single is None:   # not among the single-batch cases: check coverage only
                mine = [x for x in got if x[0] == j]
                assert mine[0][1] == 0 and sum(m for _, _, m in mine) == n and len(mine) <= 8
                assert all(p[1] + p[2] == q[1] for p, q in zip(mine, mine[1:]))
                want += mine
                continue
            k, *cut = single
            want += [(j, x, y - x) for x, y in zip(cut, cut[1:]) if y > x]
        assert got == want, (bs, got)
        assert all(m > 0 for _, _, m in got)
        assert [j for j, _, _ in got] == sorted(j for j, _, _ in got)
