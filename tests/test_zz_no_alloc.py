"""The allocation-free batched entry point (for callers that cannot call cudaMalloc while tracing,
e.g. hosts that own all device memory through their own pools) against the allocating one.

The file name sorts it after every other test file, so that a run that stops at its first failure has
run every other test before this entry point's; nothing in it depends on that order (the entry point
clears its queue head and status word at every call and looks up its array's address each time), and
it passes alone in a fresh process too."""
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


def _compare_batches(handles, rdev, counts, hit_total_min=0):
    ref = [ccs.alloc_hits(max(c, 1)) for c in counts]
    out = [ccs.alloc_hits(max(c, 1)) for c in counts]
    for h in out:
        for p in h:
            p.fill_(7)
    hits_ref = [h if c else ccs.ccs_hits() for h, c in zip(ref, counts)]
    hits_out = [h if c else ccs.ccs_hits() for h, c in zip(out, counts)]
    ccs.ccs_intersect_batched(handles, rdev, hits_ref, ccs.make_opts())
    ccs.ccs_intersect_batched_noalloc(handles, rdev, hits_out, ccs.make_opts())
    torch.cuda.synchronize()
    total = 0
    for a, b, c in zip(ref, out, counts):
        if not c:
            assert all(bool((p == 7).all()) for p in b)   # nothing written for an empty scene
            continue
        ga, gb = ccs.hits_to_numpy(a), ccs.hits_to_numpy(b)
        for k in ("t", "u", "v", "pid"):
            assert np.array_equal(ga[k][:c], gb[k][:c]), k
        total += int((ga["pid"][:c] != ccs.MISS).sum())
    assert total >= hit_total_min


def test_noalloc_many_small_scenes_with_empty_ones():
    """70 scenes (more than two 32-scene chunks of the table upload), some with no rays and NULL planes."""
    base = [sg.make_scene(n, 0.02 * n, 3, n) for n in (2, 3, 4)]
    shared = [ccs.Scene(s.P, s.types) for s in base]
    handles, rdev, counts = [], [], []
    for k in range(70):
        handles.append(shared[k % 3])
        n = 0 if k % 9 == 4 else 200 + 37 * (k % 11)
        counts.append(n)
        rdev.append(ccs.rays_to_device(sg.random_rays(n, seed=100 + k).soa()) if n else ccs.ccs_rays())
    _compare_batches(handles, rdev, counts, hit_total_min=1000)
    for h in shared:
        h.close()


def test_noalloc_at_the_scene_limit():
    s = sg.config_scene(1)
    h = ccs.Scene(s.P, s.types)
    n = ccs.CCS_NOALLOC_MAX_SCENES
    rdev = [ccs.rays_to_device(sg.random_rays(64, seed=300 + k).soa()) for k in range(n)]
    _compare_batches([h] * n, rdev, [64] * n, hit_total_min=500)
    h.close()


def test_noalloc_status_is_cleared_between_calls():
    """A call whose rays reach the iteration cap reports CCS_ERR_TRAVERSAL_LIMIT; the next call, with the
    default cap, reports CCS_OK and the allocating entry point's hits."""
    scenes, rays = _inputs(31)
    handles = [ccs.Scene(s.P, s.types) for s in scenes]
    rdev = [ccs.rays_to_device(r.soa()) for r in rays]
    out = [ccs.alloc_hits(r.n) for r in rays]
    with pytest.raises(ccs.CcsError) as e:
        ccs.ccs_intersect_batched_noalloc(handles, rdev, out, ccs.make_opts(iter_cap=3))
    assert e.value.status == ccs.CCS_ERR_TRAVERSAL_LIMIT
    _compare_batches(handles, rdev, [r.n for r in rays], hit_total_min=1000)
    for h in handles:
        h.close()
