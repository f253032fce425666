"""The allocation-free batched entry point (for callers that cannot call cudaMalloc while tracing,
e.g. hosts that own all device memory through their own pools) against the allocating one.

Collected last on purpose; it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest

from paper_1811_03510_gb300 import ccs, scenegen as sg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_03510_gb300 import build_ext
    build_ext.build()
    torch.cuda.set_device(0)


def _inputs(seed):
    scenes = [sg.make_scene(n, 0.03, 3, seed + n, gregory_ring=(n == 5)) for n in (2, 5, 3)]
    rays = [sg.random_rays(4000 + 1000 * k, seed=seed + k) for k in range(3)]
    return scenes, rays


def test_noalloc_matches_allocating_entry_on_two_calls_in_a_row():
    handles = None
    for call, seed in enumerate((11, 23)):
        scenes, rays = _inputs(seed)
        handles = [ccs.Scene(s.P, s.types) for s in scenes]
        rdev = [ccs.rays_to_device(r.soa()) for r in rays]
        ref = [ccs.alloc_hits(r.n) for r in rays]
        out = [ccs.alloc_hits(r.n) for r in rays]
        for h in out:   # stale contents must not leak into the answer
            for p in h:
                p.fill_(7)
        ccs.ccs_intersect_batched(handles, rdev, ref, ccs.make_opts())
        ccs.ccs_intersect_batched_noalloc(handles, rdev, out, ccs.make_opts())
        torch.cuda.synchronize()
        hit_total = 0
        for a, b in zip(ref, out):
            ga, gb = ccs.hits_to_numpy(a), ccs.hits_to_numpy(b)
            for k in ("t", "u", "v", "pid"):
                # the tolerance of the parity tests between two GPU runs of one answer: exact
                assert np.array_equal(ga[k], gb[k]), (call, k)
            hit_total += int((ga["pid"] != ccs.MISS).sum())
        assert hit_total > 1000
        for h in handles:
            h.close()


def test_noalloc_rejects_too_many_scenes():
    s = sg.config_scene(1)
    h = ccs.Scene(s.P, s.types)
    r = ccs.rays_to_device(sg.random_rays(32, seed=1).soa())
    hits = ccs.alloc_hits(32)
    n = ccs.CCS_NOALLOC_MAX_SCENES + 1
    with pytest.raises(ccs.CcsError) as e:
        ccs.ccs_intersect_batched_noalloc([h] * n, [r] * n, [hits] * n, ccs.make_opts())
    assert e.value.status == ccs.CCS_ERR_INVALID_ARG and "CCS_NOALLOC_MAX_SCENES" in str(e.value)
    h.close()
