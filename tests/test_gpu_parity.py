"""GPU parity of the plain closest-hit kernel against the FP64 oracle, through the C ABI."""
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


def gpu_run(P, types, rays, L=8, scene=None, **kw):
    own = scene is None
    sc = scene or ccs.Scene(P, types)
    hits = ccs.intersect(sc, ccs.rays_to_device(rays.soa()), ccs.make_opts(leaf_depth=L, **kw))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    out = ccs.hits_to_numpy(hits)
    if own:
        sc.close()
    return out


def surface_rays(s, n_primary_w, n_primary_h, seed, L=8):
    """Outgoing rays from the oracle's primary hits: origin on the hit leaf surface point, offset along
    the normal, random direction in the normal's hemisphere (incoherent secondary rays)."""
    cam = sg.pinhole_rays(n_primary_w, n_primary_h)
    o = oracle.intersect(s.P, s.types, cam.soa(), L=L)
    idx = np.nonzero(o["pid"] != MISS)[0]
    rng = np.random.default_rng(seed)
    org, dirs = [], []
    for i in idx:
        pid = int(o["pid"][i])
        f, fu, fv = oracle.patch_frame(s.P[pid].astype(float), bool(s.types[pid]), float(o["u"][i]), float(o["v"][i]))
        nrm = np.cross(fu, fv)
        nrm /= np.linalg.norm(nrm)
        if nrm @ cam.d[i] > 0:
            nrm = -nrm
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if d @ nrm < 0:
            d = -d
        org.append(f + 2e-3 * nrm)
        dirs.append(d)
    org, dirs = np.array(org), np.array(dirs)
    n = len(org)
    return sg.Rays(org.astype(np.float32), dirs.astype(np.float32), np.zeros(n, np.float32),
                   np.full(n, np.inf, np.float32))


def test_cfg1_primary_rays_all_match():
    s = sg.config_scene(1)
    r = sg.pinhole_rays(64, 64)
    g = gpu_run(s.P, s.types, r, 8)
    o = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True)
    rep = compare(g, o, 8)
    assert rep["hits"] > 500


def test_cfg1_random_incoherent_rays():
    s = sg.config_scene(1)
    r = sg.random_rays(20000, seed=11)
    g = gpu_run(s.P, s.types, r, 8)
    o = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True)
    rep = compare(g, o, 8)
    assert rep["hits"] > 5000


def test_gregory_heavy_scene():
    """8x8 noisy cube-sphere with the 2-ring of each extraordinary vertex as Gregory patches (6.25 %)."""
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(20000, seed=12, target=1.0)
    g = gpu_run(s.P, s.types, r, 8)
    o = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True)
    rep = compare(g, o, 8)
    greg_hits = np.isin(o["pid"], np.nonzero(s.types == 1)[0]).sum()
    assert greg_hits > 100, rep


def test_secondary_rays_from_surface():
    s = sg.config_scene(2)
    r = surface_rays(s, 160, 90, seed=3)
    g = gpu_run(s.P, s.types, r, 8)
    o = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True)
    compare(g, o, 8)


@pytest.mark.parametrize("L", [1, 2, 5, 11, 15])
def test_leaf_depths(L):
    s = sg.config_scene(1)
    r = sg.random_rays(3000, seed=100 + L)
    g = gpu_run(s.P, s.types, r, L)
    o = oracle.intersect(s.P, s.types, r.soa(), L=L, flags=True)
    # deep leaves are small against the FP32 box error, so more rays are ambiguous there
    compare(g, o, L, max_flagged_frac=0.05 if L <= 8 else 0.12)


def test_full_size_primary_launch_sampled():
    """1920 x 1080 primary rays of the 1536-patch scene in one launch (the benchmark's launch
    configuration); the oracle checks a sample of 4000 rays, half of them inside the sphere's outline."""
    s = sg.config_scene(2)
    r = sg.pinhole_rays(1920, 1080)
    g = gpu_run(s.P, s.types, r, 8)
    rng = np.random.default_rng(7)
    hit_idx = np.nonzero(g["pid"] != MISS)[0]
    assert 0.1 < len(hit_idx) / r.n < 0.3
    pick = np.unique(np.concatenate([rng.choice(r.n, 2000, replace=False), rng.choice(hit_idx, 2000, replace=False)]))
    sub = r.subset(pick)
    o = oracle.intersect(s.P, s.types, sub.soa(), L=8, flags=True)
    gs = {k: v[pick] for k, v in g.items()}
    compare(gs, o, 8)


def test_edge_cases_nan_inverted_interval_and_short_tmax():
    s = sg.config_scene(1)
    r = sg.pinhole_rays(32, 32)
    n = r.n
    o = r.o.copy()
    d = r.d.copy()
    tmin = r.tmin.copy()
    tmax = r.tmax.copy()
    o[0, 0] = np.nan
    d[1, 2] = np.nan
    tmin[2], tmax[2] = 5.0, 1.0          # inverted interval
    tmax[3:200] = 0.5                    # ends before the sphere
    tmin[200:300] = 100.0                # starts after it
    # exactly representable axis-aligned directions
    d[300] = [0, 0, -1]
    o[300] = [0, 0, 3]
    d[301] = [0, -1, 0]
    o[301] = [0.1, 3, 0.05]
    rr = sg.Rays(o, d, tmin, tmax)
    g = gpu_run(s.P, s.types, rr, 8)
    assert (g["pid"][:300] == MISS).all()
    assert np.isinf(g["t"][:300]).all()
    orc = oracle.intersect(s.P, s.types, rr.soa(), L=8, flags=True)
    compare(g, orc, 8)
    assert g["pid"][300] != MISS and g["pid"][301] != MISS


def test_tmax_bound_is_inclusive_and_tmin_clips():
    s = sg.config_scene(1)
    r = sg.pinhole_rays(48, 48)
    g0 = gpu_run(s.P, s.types, r, 8)
    hit = g0["pid"] != MISS
    # with tmax equal to the reported t the same leaf is still found
    r2 = sg.Rays(r.o, r.d, r.tmin, np.where(hit, g0["t"], np.inf).astype(np.float32))
    g1 = gpu_run(s.P, s.types, r2, 8)
    assert np.array_equal(g1["pid"], g0["pid"]) and np.array_equal(g1["t"][hit], g0["t"][hit])
    # a tmin past the front surface finds the back side
    r3 = sg.Rays(r.o, r.d, np.where(hit, g0["t"] + 0.2, 0).astype(np.float32), r.tmax)
    g3 = gpu_run(s.P, s.types, r3, 8)
    assert (g3["t"][hit] > g0["t"][hit]).all()
    o3 = oracle.intersect(s.P, s.types, r3.soa(), L=8, flags=True)
    compare(g3, o3, 8)


def test_empty_and_single_patch_scenes():
    s = sg.config_scene(1)
    r = sg.random_rays(2000, seed=4)
    g = gpu_run(s.P[:0], s.types[:0], r, 8)
    assert (g["pid"] == MISS).all()
    for p in (0, 5, 40):   # Bezier and Gregory singles
        P1, t1 = s.P[p:p + 1], s.types[p:p + 1]
        c = P1[0].mean(0)
        rr = sg.random_rays(3000, seed=p, radius=2.0)
        rr = sg.Rays(rr.o, (c[None] + 0.05 * np.random.default_rng(p).normal(size=(3000, 3)) - rr.o).astype(np.float32),
                     rr.tmin, rr.tmax)
        g = gpu_run(P1, t1, rr, 8)
        o = oracle.intersect(P1, t1, rr.soa(), L=8, flags=True)
        rep = compare(g, o, 8)
        assert rep["hits"] > 100


def test_zero_rays_is_a_no_op():
    s = sg.config_scene(1)
    sc = ccs.Scene(s.P, s.types)
    hits = ccs.alloc_hits(1)
    rays = ccs.rays_to_device(sg.pinhole_rays(1, 1).soa())
    ccs.ccs_intersect(sc.handle, rays, 0, hits, ccs.make_opts())
    torch.cuda.synchronize()
    sc.close()


@pytest.mark.parametrize("case", ["one_chunk", "two_ragged_chunks_local", "four_chunks", "seven_given_chunks",
                                  "screen_space"])
def test_host_buffer_path_matches_device_path(case):
    """The host-buffer entry (chunked copies overlapping the traversal) returns the device path's hits."""
    s = sg.config_scene(2)
    if case == "one_chunk":
        r, local, kw = sg.pinhole_rays(320, 180), False, {}
    elif case == "two_ragged_chunks_local":   # 2,000,001 rays: chunks of 1,000,000 and 1,000,001
        r, local, kw = sg.pinhole_rays(1920, 1080).subset(np.arange(2000001)), True, {}
    elif case == "four_chunks":               # 3 * 2^20 + 5 rays
        r, local, kw = sg.random_rays(3 * (1 << 20) + 5, seed=77), True, {}
    elif case == "seven_given_chunks":        # 700,001 rays in chunks of 100,003 (the last one short)
        r, local, kw = sg.random_rays(700001, seed=78), False, dict(host_chunk=100003)
    else:
        r, local, kw = sg.pinhole_rays(640, 480), False, dict(pixel_spread=2.0 * np.tan(np.radians(30.0)) / 480)
    sc = ccs.Scene(s.P, s.types, local=local)
    g = ccs.hits_to_numpy(ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(**kw)))
    torch.cuda.synchronize()
    planes = [np.ascontiguousarray(a) for a in r.soa()]
    block = np.stack(planes)                               # rays as rows of one block (pitched copies)
    for rep in range(2):   # the second call reuses the scene's staging buffer, streams and events
        ht = np.empty(r.n, np.float32)
        hu = np.empty(r.n, np.float32)
        hv = np.empty(r.n, np.float32)
        hp = np.empty(r.n, np.uint32)
        ccs.ccs_intersect_host(sc.handle, [a.ctypes.data for a in planes], r.n,
                               [ht.ctypes.data, hu.ctypes.data, hv.ctypes.data, hp.ctypes.data], ccs.make_opts(**kw))
        assert np.array_equal(hp, g["pid"]) and np.array_equal(ht, g["t"])
        assert np.array_equal(hu, g["u"]) and np.array_equal(hv, g["v"])
        out = np.full((4, r.n + 3), -7, np.float32)      # hits as rows of one block with a wider pitch
        ccs.ccs_intersect_host(sc.handle, [block[c].ctypes.data for c in range(8)], r.n,
                               [out[c].ctypes.data for c in range(4)], ccs.make_opts(**kw))
        assert np.array_equal(out[3, :r.n].view(np.uint32), g["pid"]) and np.array_equal(out[0, :r.n], g["t"])
        assert np.array_equal(out[1, :r.n], g["u"]) and np.array_equal(out[2, :r.n], g["v"])
        assert (out[:, r.n:] == -7).all()
    assert (g["pid"] != MISS).sum() > 1000
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    sc.close()


def test_launch_timeline_counters():
    """Counters 20..22 of a counting launch: first warp start <= queue found empty <= last warp exit."""
    s = sg.config_scene(2)
    r = sg.pinhole_rays(480, 270)
    sc = ccs.Scene(s.P, s.types)
    cnt = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(counters=cnt))
    ev[1].record()
    torch.cuda.synchronize()
    tl = ccs.timeline(dict(zip(ccs.COUNTER_NAMES, cnt.cpu().tolist())))
    assert 0.0 < tl["drain_us"] < tl["launch_us"] <= 1e3 * ev[0].elapsed_time(ev[1]) + 5.0, tl
    sc.close()


def test_bit_identical_across_launch_configurations():
    """The answer does not depend on scheduling: block size, warps per SM and queue chunk."""
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(30000, seed=21)
    sc = ccs.Scene(s.P, s.types)
    ref = gpu_run(s.P, s.types, r, 8, scene=sc)
    for kw in [dict(block_threads=32), dict(block_threads=64, refill=16, chunk=32), dict(blocks_per_sm=1, refill=32),
               dict(cache_slots=0, bvh_burst=1), dict(cache_slots=0, refill=8, block_threads=96, chunk=1024, bvh_burst=16),
               dict(min_blocks=4), dict(min_blocks=4, cache_slots=0), dict(vote=12), dict(vote=24, bvh_burst=1)]:
        g = gpu_run(s.P, s.types, r, 8, scene=sc, **kw)
        for k in ("t", "u", "v", "pid"):
            assert np.array_equal(g[k], ref[k]), (kw, k)
    sc.close()


def test_iteration_cap_reports_status_and_context_survives():
    s = sg.config_scene(1)
    r = sg.pinhole_rays(64, 64)
    sc = ccs.Scene(s.P, s.types)
    hits = ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(iter_cap=5))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_ERR_TRAVERSAL_LIMIT
    g = ccs.hits_to_numpy(hits)
    assert (g["pid"] == MISS).all()
    # status was cleared; a normal launch works
    g2 = gpu_run(s.P, s.types, r, 8, scene=sc)
    assert (g2["pid"] != MISS).sum() > 500
    sc.close()


def test_refit_after_update_equals_fresh_build():
    """Deformed control points through update + refit give the same hits as a scene built from them."""
    s = sg.config_scene(2)
    P1 = sg.deform(s.P, 2, 8, seed=5)
    r = sg.random_rays(20000, seed=9)
    sc = ccs.Scene(s.P, s.types)
    x = torch.from_numpy(np.ascontiguousarray(P1[..., 0]).reshape(-1)).cuda()
    y = torch.from_numpy(np.ascontiguousarray(P1[..., 1]).reshape(-1)).cuda()
    z = torch.from_numpy(np.ascontiguousarray(P1[..., 2]).reshape(-1)).cuda()
    ccs.ccs_scene_update_points(sc.handle, x, y, z)
    ccs.ccs_bvh_refit(sc.handle)
    g = gpu_run(P1, s.types, r, 8, scene=sc)
    fresh = gpu_run(P1, s.types, r, 8)
    for k in ("t", "u", "v", "pid"):
        assert np.array_equal(g[k], fresh[k]), k
    o = oracle.intersect(P1, s.types, r.soa(), L=8, flags=True)
    compare(g, o, 8)
    sc.close()


def test_counters_count_the_work():
    """On single-patch scenes (no BVH ordering differences) the kernel expands the same nodes as the
    oracle's stack traversal, up to FP32 box differences."""
    s = sg.config_scene(1)
    for p in (0, int(np.nonzero(s.types == 1)[0][0])):
        P1, t1 = s.P[p:p + 1], s.types[p:p + 1]
        c = P1[0].mean(0)
        rr = sg.random_rays(4000, seed=p, radius=2.0)
        rr = sg.Rays(rr.o, (c[None] + 0.05 * np.random.default_rng(p).normal(size=(4000, 3)) - rr.o).astype(np.float32),
                     rr.tmin, rr.tmax)
        sc = ccs.Scene(P1, t1)
        cnt = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device="cuda")
        rays = ccs.rays_to_device(rr.soa())
        hits = ccs.alloc_hits(rr.n)
        ccs.ccs_intersect(sc.handle, rays, rr.n, hits, ccs.make_opts(counters=cnt))
        torch.cuda.synchronize()
        c = dict(zip(ccs.COUNTER_NAMES, cnt.cpu().tolist()))
        o = oracle.intersect(P1, t1, rr.soa(), L=8, stats=True)
        key = "gregory_splits" if t1[0] else "bezier_splits"
        exp = int(o["stats"][:, 2 if t1[0] else 1].sum())
        assert c["pairs"] > 1000 and c["leaves"] > 500
        assert abs(c[key] - exp) <= 0.01 * exp, (p, c, exp)
        sc.close()


@pytest.mark.parametrize("layout", ["mapped", "page_locked_copies", "one_plane_pageable"])
def test_host_path_on_page_locked_memory(layout):
    """With CCS_TRACE_HOST_MAPPED, page-locked planes are read and written by the launch through their
    device mapping; without it, or with one pageable plane among them, the copy pipeline runs.  All give
    the device path's hits."""
    s = sg.config_scene(2)
    r = sg.pinhole_rays(1920, 1080).subset(np.arange(1920 * 900 + 11))
    sc = ccs.Scene(s.P, s.types, local=True)
    kw = dict(order=True, image_width=1920)
    g = ccs.hits_to_numpy(ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(**kw)))
    torch.cuda.synchronize()
    rays = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in r.soa()]
    out = [torch.full((r.n,), -7.0).pin_memory() for _ in range(4)]
    if layout == "one_plane_pageable":
        rays[3] = torch.from_numpy(np.ascontiguousarray(r.soa()[3]))
    opts = ccs.make_opts(host_mapped=layout != "page_locked_copies", **kw)
    for _ in range(2):
        ccs.ccs_intersect_host(sc.handle, rays, r.n, out, opts)
        got = dict(t=out[0].numpy(), u=out[1].numpy(), v=out[2].numpy(), pid=out[3].numpy().view(np.uint32))
        for k in ("t", "u", "v", "pid"):
            assert np.array_equal(got[k], g[k]), (layout, k)
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    sc.close()


@pytest.mark.parametrize("kw", [{}, dict(order=True, image_width=960), dict(pairs=True)])
def test_concurrent_launches_on_one_scene_use_separate_queues(kw):
    """Two launches on one scene at the same time on two streams (each takes its own work-queue head, and
    its own work-order or pair-engine scratch from the library's pool) give the hits each gives alone."""
    s = sg.config_scene(2)
    sc = ccs.Scene(s.P, s.types, local=True)
    ra, rb = sg.pinhole_rays(960, 540), sg.random_rays(200000, seed=91)
    da, db = ccs.rays_to_device(ra.soa()), ccs.rays_to_device(rb.soa())
    ref_a = ccs.hits_to_numpy(ccs.intersect(sc, da, ccs.make_opts()))
    ref_b = ccs.hits_to_numpy(ccs.intersect(sc, db, ccs.make_opts()))
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(3):
        ha, hb = ccs.alloc_hits(ra.n), ccs.alloc_hits(rb.n)
        torch.cuda.synchronize()
        ccs.ccs_intersect(sc.handle, da, ra.n, ha, ccs.make_opts(**kw), s1)
        ccs.ccs_intersect(sc.handle, db, rb.n, hb, ccs.make_opts(**kw), s2)
        torch.cuda.synchronize()
        for got, ref in ((ccs.hits_to_numpy(ha), ref_a), (ccs.hits_to_numpy(hb), ref_b)):
            for k in ("t", "u", "v", "pid"):
                assert np.array_equal(got[k], ref[k]), k
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    sc.close()


def test_host_batches_match_the_device_path_batch_by_batch():
    """ccs_intersect_host_batches: host batches with options of their own go through one copy/trace
    pipeline (a batch's copies and launches overlap the end of the one before) and each gets its device
    path's hits.  Page-locked and pageable planes, an empty batch, a batch of 17 rays, and more chunks
    than the scene has event pairs; an invalid batch is refused before anything runs."""
    s = sg.config_scene(2)
    sc = ccs.Scene(s.P, s.types, local=True, bvh_width="both")
    prim = sg.pinhole_rays(1920, 1080).subset(np.arange(1920 * 700 + 13))
    diff = sg.random_rays(333918, seed=93)
    tiny = sg.random_rays(17, seed=94)
    rays = [prim, tiny, diff, tiny]
    n_list = [prim.n, 0, diff.n, tiny.n]
    opts = [ccs.make_opts(order=True, image_width=1920), None,
            ccs.make_opts(bvh_width=4, host_chunk=40000), ccs.make_opts(lanes_per_ray=3)]
    refs = []
    for r, n, o in zip(rays, n_list, opts):
        refs.append(ccs.hits_to_numpy(ccs.intersect(sc, ccs.rays_to_device(r.soa()), o or ccs.make_opts()))
                    if n else None)
    torch.cuda.synchronize()
    # the first batch in page-locked memory, the others pageable
    planes = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in prim.soa()]]
    planes += [[np.ascontiguousarray(a) for a in r.soa()] for r in rays[1:]]
    ray_ptrs = [[a.data_ptr() if torch.is_tensor(a) else a.ctypes.data for a in p] for p in planes]
    for rep in range(2):    # the second call reuses the staging buffer, streams and events
        outs = [[torch.full((max(n, 1),), -7.0).pin_memory() for _ in range(4)] if j == 0 else
                [np.full(max(n, 1), -7, np.float32) for _ in range(4)] for j, n in enumerate(n_list)]
        hit_ptrs = [[h.data_ptr() if torch.is_tensor(h) else h.ctypes.data for h in o] for o in outs]
        ccs.ccs_intersect_host_batches(sc.handle, ray_ptrs, n_list, hit_ptrs, opts)
        for j, (o, ref) in enumerate(zip(outs, refs)):
            got = [h.numpy() if torch.is_tensor(h) else h for h in o]
            if ref is None:
                assert (got[0] == -7).all()
                continue
            assert np.array_equal(got[3].view(np.uint32), ref["pid"]), (rep, j)
            for k, c in (("t", 0), ("u", 1), ("v", 2)):
                assert np.array_equal(got[c], ref[k]), (rep, j, k)
    with pytest.raises(ccs.CcsError):      # an invalid BVH width in the third batch
        ccs.ccs_intersect_host_batches(sc.handle, ray_ptrs[:3], n_list[:3], hit_ptrs[:3],
                                       [None, None, ccs.make_opts(bvh_width=8)])
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    assert (refs[0]["pid"] != MISS).sum() > 1000 and (refs[2]["pid"] != MISS).sum() > 1000
    sc.close()
