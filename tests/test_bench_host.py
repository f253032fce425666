"""Host logic of bench.py that runs without a GPU: the kernel-source hash and the figures it reads from the
committed ncu summaries (DRAM traffic per launch, thread-instruction issue over the FP32 lane peak, the
dominant kernel's share of the step)."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_kernel_source_hash_is_stable_and_short():
    h = bench.kernel_source_hash()
    assert re.fullmatch(r"[0-9a-f]{16}", h)
    assert bench.kernel_source_hash() == h


def test_profile_figures_parse_and_follow_the_hash():
    traffic, t_src = bench.measured_traffic()
    issue, i_src = bench.measured_issue()
    share, s_src = bench.measured_share()
    assert t_src and os.path.exists(t_src) and i_src and os.path.exists(i_src) and s_src and os.path.exists(s_src)
    for src, val in ((t_src, traffic), (i_src, issue), (s_src, share)):
        text = open(src).read()
        m = re.search(r"kernel sources sha256\[:16\]: ([0-9a-f]{16})", text)
        assert m, src
        # a figure is reported exactly when the capture was taken on the current kernel sources
        assert (val is not None) == (m.group(1) == bench.kernel_source_hash()), src
    if traffic is not None:   # the subdivision pass reads its tasks and candidates (about 20 B per primary ray)
        p, d = traffic
        assert p > 10 * 1920 * 1080 and 0 < d < p
    if share is not None:
        assert 0.3 < share < 1
    if issue is not None:
        a, f = issue
        assert 0 < f < a < 1
