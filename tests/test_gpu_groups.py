"""Thread groups of three lanes per ray (Sec. 3.5), lanes_per_ray = 3, through the C ABI: hits and
traversal counters bit-identical to the one-lane-per-ray kernel, parity with the FP64 oracle, ragged
ray counts against groups of three and warps of ten rays, the iteration cap and batched launches."""
import numpy as np
import pytest

import oracle
from paper_1811_03510_gb300 import ccs, scenegen as sg
from parity import MISS, compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_03510_gb300 import build_ext
    build_ext.build()
    oracle.build()
    torch.cuda.set_device(0)


def run(sc, rays, counters=False, **kw):
    cnt = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device="cuda") if counters else None
    hits = ccs.intersect(sc, ccs.rays_to_device(rays.soa()), ccs.make_opts(counters=cnt, **kw))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    out = ccs.hits_to_numpy(hits)
    return (out, cnt.cpu().numpy()) if counters else out


def same(a, b, what):
    for k in ("t", "u", "v", "pid"):
        assert np.array_equal(a[k], b[k]), (what, k)


@pytest.mark.parametrize("which", ["cfg1_primary", "cfg2_random", "gregory_ring", "cfg2_primary"])
def test_groups_bit_identical_to_one_lane_per_ray(which):
    if which == "cfg1_primary":
        s, r = sg.config_scene(1), sg.pinhole_rays(64, 64)
    elif which == "cfg2_random":
        s, r = sg.config_scene(2), sg.random_rays(40000, seed=5)
    elif which == "gregory_ring":
        s, r = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True), sg.random_rays(30000, seed=6, target=1.0)
    else:
        s, r = sg.config_scene(2), sg.pinhole_rays(480, 270)
    sc = ccs.Scene(s.P, s.types)
    for K in (0, 2):
        ref, cref = run(sc, r, counters=True, cache_slots=K)
        got, cgot = run(sc, r, counters=True, cache_slots=K, lanes_per_ray=3)
        same(ref, got, (which, K))
        # every ray does the same sequence of steps in both layouts, so the work counts agree exactly
        w = ccs.NUM_WORK_COUNTERS
        assert np.array_equal(cref[:w], cgot[:w]), (which, K, cref, cgot)
    sc.close()


@pytest.mark.parametrize("L", [1, 4, 11, 15])
def test_groups_leaf_depths(L):
    s = sg.config_scene(1)
    r = sg.random_rays(5000, seed=200 + L)
    sc = ccs.Scene(s.P, s.types)
    same(run(sc, r, leaf_depth=L), run(sc, r, leaf_depth=L, lanes_per_ray=3), L)
    sc.close()


def test_groups_launch_shapes_do_not_change_hits():
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(30000, seed=22)
    sc = ccs.Scene(s.P, s.types)
    ref = run(sc, r)
    for kw in [dict(block_threads=32), dict(block_threads=64, refill=1, chunk=32), dict(block_threads=96, chunk=1024),
               dict(blocks_per_sm=1, refill=10), dict(blocks_per_sm=6, bvh_burst=1), dict(vote=3),
               dict(vote=8, cache_slots=0), dict(refill=32, bvh_burst=16)]:
        same(ref, run(sc, r, lanes_per_ray=3, **kw), kw)
    sc.close()


def test_groups_match_oracle():
    s = sg.config_scene(1)
    r = sg.random_rays(20000, seed=31)
    sc = ccs.Scene(s.P, s.types)
    g = run(sc, r, lanes_per_ray=3)
    o = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True)
    rep = compare(g, o, 8)
    assert rep["hits"] > 5000
    sc.close()


def test_groups_full_size_primary_launch_sampled():
    """1920 x 1080 primary rays of the 1536-patch scene, grouped layout; the oracle checks 4000 rays."""
    s = sg.config_scene(2)
    r = sg.pinhole_rays(1920, 1080)
    sc = ccs.Scene(s.P, s.types)
    g = run(sc, r, lanes_per_ray=3)
    rng = np.random.default_rng(8)
    hit_idx = np.nonzero(g["pid"] != MISS)[0]
    assert 0.1 < len(hit_idx) / r.n < 0.3
    pick = np.unique(np.concatenate([rng.choice(r.n, 2000, replace=False), rng.choice(hit_idx, 2000, replace=False)]))
    o = oracle.intersect(s.P, s.types, r.subset(pick).soa(), L=8, flags=True)
    compare({k: v[pick] for k, v in g.items()}, o, 8)
    sc.close()


@pytest.mark.parametrize("n", [1, 2, 3, 9, 10, 11, 29, 31, 33, 41, 1001])
def test_groups_ragged_ray_counts(n):
    s = sg.config_scene(1)
    r = sg.random_rays(n, seed=300 + n, target=0.5)
    sc = ccs.Scene(s.P, s.types)
    for kw in (dict(), dict(block_threads=32, chunk=32, refill=1)):
        same(run(sc, r), run(sc, r, lanes_per_ray=3, **kw), (n, kw))
    sc.close()


def test_groups_invalid_rays_and_empty_scene():
    s = sg.config_scene(1)
    r = sg.pinhole_rays(32, 32)
    o, d, tmin, tmax = r.o.copy(), r.d.copy(), r.tmin.copy(), r.tmax.copy()
    o[0, 1] = np.nan
    d[1, 0] = np.nan
    tmin[2], tmax[2] = 5.0, 1.0
    tmax[3:100] = 0.5
    rr = sg.Rays(o, d, tmin, tmax)
    sc = ccs.Scene(s.P, s.types)
    g = run(sc, rr, lanes_per_ray=3)
    assert (g["pid"][:100] == MISS).all() and np.isinf(g["t"][:100]).all()
    same(run(sc, rr), g, "invalid")
    sc.close()
    empty = ccs.Scene(s.P[:0], s.types[:0])
    g = run(empty, r, lanes_per_ray=3)
    assert (g["pid"] == MISS).all()
    empty.close()


def test_groups_iteration_cap_reports_status():
    s = sg.config_scene(1)
    r = sg.pinhole_rays(64, 64)
    sc = ccs.Scene(s.P, s.types)
    hits = ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(iter_cap=5, lanes_per_ray=3))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_ERR_TRAVERSAL_LIMIT
    assert (ccs.hits_to_numpy(hits)["pid"] == MISS).all()
    g = run(sc, r, lanes_per_ray=3)
    assert (g["pid"] != MISS).sum() > 500
    sc.close()


def test_groups_batched_launch_equals_per_scene():
    scenes = [sg.make_scene(n, 0.02 * (k % 3), 3, k + 1, gregory_ring=(k == 1)) for k, n in enumerate([2, 5, 3])]
    rays = [sg.pinhole_rays(64, 48), sg.random_rays(4001, seed=3), sg.random_rays(17, seed=4)]
    handles = [ccs.Scene(s.P, s.types) for s in scenes]
    ref = [run(h, r) for h, r in zip(handles, rays)]
    rdev = [ccs.rays_to_device(r.soa()) for r in rays]
    hits = [ccs.alloc_hits(r.n) for r in rays]
    ccs.ccs_intersect_batched(handles, rdev, hits, ccs.make_opts(lanes_per_ray=3))
    torch.cuda.synchronize()
    for h, rf in zip(hits, ref):
        same(ccs.hits_to_numpy(h), rf, "batched")
    for h in handles:
        h.close()


def test_lanes_per_ray_is_validated():
    s = sg.config_scene(1)
    sc = ccs.Scene(s.P, s.types)
    r = sg.pinhole_rays(4, 4)
    with pytest.raises(ccs.CcsError):
        ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(lanes_per_ray=2))
    sc.close()
