"""The pair engine (CCS_TRACE_PAIRS): a BVH pass that keeps each ray's 8 nearest candidate patches (with
local frames, only those whose root box in the patch frame the ray comes near), then a subdivision pass
that runs Algorithm 3 on one (ray, patch) pair per lane; a ray whose dropped candidates could still hold
the answer has its lane walk the BVH again for the next ones.  The answer is the smallest leaf key over all
nested intervals (readings A14/A15), so every hit must be bit-identical to the ray-persistent kernel's,
which the FP64 oracle pins; scenes with more than 8 candidate boxes along a ray drive the second walks."""
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


def run(sc, r, counters=None, **kw):
    """Hits of rays r, the hit planes filled with a pattern first so that an unwritten record shows."""
    rays = ccs.rays_to_device(r.soa())
    hits = [torch.full((r.n,), -7.0, device="cuda") for _ in range(3)] + \
        [torch.full((r.n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")]
    ccs.ccs_intersect(sc.handle, rays, r.n, hits, ccs.make_opts(counters=counters, **kw))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    return ccs.hits_to_numpy(hits)


def same(a, b, what):
    for k in ("t", "u", "v", "pid"):
        assert np.array_equal(a[k], b[k]), (what, k, int((a[k] != b[k]).sum()))


def tunnel_scene(n_u=40, gregory_every=0):
    """n_u U-shaped patches along x (patch k over x in [k, k+1], y in [-1, 1], the surface below z = -0.2 at
    y = 0), a ray along +x at y = 0, z = 0.3 crossing every patch box without touching a surface, then a
    wall at x = n_u + 0.5 facing -x.  With gregory_every = m every m-th U is a Gregory patch (p^u = p^v)."""
    P = np.zeros((n_u + 1, 20, 3), np.float32)
    ys = np.array([-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0])
    zs = np.array([1.0, -0.6, -0.6, 1.0])
    for k in range(n_u):
        for j in range(4):
            for i in range(4):
                P[k, 4 * j + i] = (k + i / 3.0, ys[j], zs[j])
        P[k, 16:20] = P[k, [5, 6, 9, 10]]
    for j in range(4):
        for i in range(4):
            P[n_u, 4 * j + i] = (n_u + 0.5, -1.0 + 2.0 * i / 3.0, -1.0 + 2.0 * j / 3.0)
    P[n_u, 16:20] = P[n_u, [5, 6, 9, 10]]
    types = np.zeros(n_u + 1, np.uint8)
    if gregory_every:
        types[:n_u:gregory_every] = 1
    return P, types


def tunnel_rays(n_u=40):
    """Rays along the tunnel (they reach the wall after several walks for dropped candidates), rays sloping
    down onto a U within the first 16 patches (answered within one or two lists), rays straight down into
    single U patches, and rays that leave the tunnel sideways."""
    o, d = [], []
    for z in np.linspace(0.05, 0.6, 12):
        for y in np.linspace(-0.3, 0.3, 7):
            o.append((-1.0, y, z))
            d.append((1.0, 0.0, 0.0))
    for s in np.linspace(0.03, 0.09, 9):
        o.append((-1.0, 0.0, 0.3))
        d.append((1.0, 0.0, -s))
    for k in range(0, n_u, 3):
        o.append((k + 0.37, 0.11, 0.5))
        d.append((0.0, 0.0, -1.0))
    for a in np.linspace(0.2, 1.2, 8):
        o.append((-1.0, 0.0, 0.3))
        d.append((1.0, a, 0.05))
    o = np.array(o, np.float32)
    d = np.array(d, np.float64)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    n = len(o)
    return sg.Rays(o, d, np.zeros(n, np.float32), np.full(n, np.inf, np.float32))


@pytest.mark.parametrize("local", [False, True])
@pytest.mark.parametrize("width", [2, 4])
def test_pairs_hits_equal_ray_kernel_across_options(local, width):
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(30000, seed=71)
    sc = ccs.Scene(s.P, s.types, local=local, bvh_width=width)
    ref = run(sc, r)
    assert (ref["pid"] != MISS).sum() > 1000
    for kw in [{}, dict(cache_slots=0), dict(cache_slots=1), dict(cache_slots=2, refill=1), dict(refill=24),
               dict(refill=32, cache_slots=1)]:
        same(run(sc, r, pairs=True, **kw), ref, kw)
    sc.close()


def test_pairs_match_oracle_on_primary_image_with_local_frames():
    s = sg.config_scene(2)
    cam = sg.pinhole_rays(480, 270)
    sc = ccs.Scene(s.P, s.types, local=True)
    g = run(sc, cam, pairs=True, cache_slots=1)
    same(g, run(sc, cam), "primary")
    rep = compare(g, oracle.intersect(s.P, s.types, cam.soa(), L=8, flags=True, local=True), 8,
                  max_flagged_frac=0.05)
    assert rep["hits"] > 10000
    sc.close()


def test_pairs_candidate_pass_in_image_tiles():
    """With image_width a multiple of 8 the candidate pass gives each warp an 8 x 4 pixel tile: the threads
    cover whole bands of 4 rows, those past the last ray (a ragged band, a partial last row, a host chunk
    that starts mid-row) have none, and every ray is traced once with the same answer."""
    s = sg.config_scene(2)
    r = sg.pinhole_rays(336, 211)   # 211 rows: the last band holds 3
    sc = ccs.Scene(s.P, s.types, local=True)
    ref = run(sc, r)
    assert (ref["pid"] != MISS).sum() > 10000
    for w in (336, 8, 333, 0):   # 333 is not a multiple of 8: rays in their own order
        same(run(sc, r, pairs=True, cache_slots=1, image_width=w), ref, w)
    # a partial last row: the first n - 5 rays, the rest of the hit planes untouched
    m = r.n - 5
    rays = ccs.rays_to_device(r.soa())
    hits = [torch.full((r.n,), -7.0, device="cuda") for _ in range(3)] + \
        [torch.full((r.n,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")]
    ccs.ccs_intersect(sc.handle, rays, m, hits, ccs.make_opts(pairs=True, image_width=336))
    torch.cuda.synchronize()
    got = ccs.hits_to_numpy(hits)
    same({k: v[:m] for k, v in got.items()}, {k: v[:m] for k, v in ref.items()}, "partial row")
    assert (got["t"][m:] == -7.0).all() and (got["pid"][m:] == 0x5A5A5A5A).all()
    # the any-hit query takes the same tiles: occlusion equals the closest hit's answer
    occ = ccs.occluded(sc, rays, ccs.make_opts(pairs=True, image_width=336))
    torch.cuda.synchronize()
    assert np.array_equal(occ.cpu().numpy().astype(bool), ref["pid"] != MISS)
    # host chunks of 20,000 rays: each chunk is tiled from its own first ray
    planes = [np.ascontiguousarray(a) for a in r.soa()]
    out = [np.empty(r.n, np.float32) for _ in range(3)] + [np.empty(r.n, np.uint32)]
    ccs.ccs_intersect_host(sc.handle, [a.ctypes.data for a in planes], r.n, [a.ctypes.data for a in out],
                           ccs.make_opts(pairs=True, image_width=336, host_chunk=20000))
    same(dict(t=out[0], u=out[1], v=out[2], pid=out[3]), ref, "host chunks")
    sc.close()


@pytest.mark.parametrize("gregory_every", [0, 3])
@pytest.mark.parametrize("width", [2, 4])
def test_pairs_walk_again_when_candidates_are_dropped(gregory_every, width):
    P, types = tunnel_scene(40, gregory_every)
    r = tunnel_rays(40)
    sc = ccs.Scene(P, types, bvh_width=width)
    g = run(sc, r, pairs=True)
    same(g, run(sc, r), "tunnel")
    o = oracle.intersect(P, types, r.soa(), L=6, flags=True)
    compare(run(sc, r, pairs=True, leaf_depth=6), o, 6, max_flagged_frac=0.5)
    # the rays along the tunnel reach the wall; the sloping ones end on a U patch
    assert (g["pid"][:84] == 40).all()
    assert ((g["pid"][84:93] != MISS) & (g["pid"][84:93] < 40)).all()
    cnt = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device="cuda")
    run(sc, r, counters=cnt, pairs=True)
    assert int(cnt[7]) > 0 and int(cnt[1]) > 0
    assert int(cnt[10]) >= 84   # the rays along the tunnel walked again for their dropped candidates
    sc.close()


def test_pairs_any_hit_equals_closest_hit_and_ray_kernel():
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(20000, seed=72)
    r.tmax[:] = np.random.default_rng(3).uniform(0.5, 6.0, r.n).astype(np.float32)
    sc = ccs.Scene(s.P, s.types, local=True)
    rays = ccs.rays_to_device(r.soa())
    occ_p = ccs.occluded(sc, rays, ccs.make_opts(pairs=True))
    occ_r = ccs.occluded(sc, rays, ccs.make_opts())
    torch.cuda.synchronize()
    assert torch.equal(occ_p, occ_r)
    hit = run(sc, r, pairs=True)["pid"] != MISS
    assert np.array_equal(occ_p.cpu().numpy().astype(bool), hit)
    assert 1000 < hit.sum() < r.n - 1000
    P, types = tunnel_scene(40, 4)
    t = tunnel_rays(40)
    t.tmax[:] = 100.0
    tsc = ccs.Scene(P, types)
    trays = ccs.rays_to_device(t.soa())
    occ = ccs.occluded(tsc, trays, ccs.make_opts(pairs=True))
    torch.cuda.synchronize()
    assert torch.equal(occ, ccs.occluded(tsc, trays, ccs.make_opts()))
    assert bool(occ[:84].all())
    sc.close()
    tsc.close()


def test_pairs_host_path_ragged_empty_and_cap():
    s = sg.config_scene(2)
    r = sg.pinhole_rays(333, 211)
    sc = ccs.Scene(s.P, s.types, local=True)
    ref = run(sc, r)
    planes = [np.ascontiguousarray(a) for a in r.soa()]
    out = [np.empty(r.n, np.float32) for _ in range(3)] + [np.empty(r.n, np.uint32)]
    ccs.ccs_intersect_host(sc.handle, [a.ctypes.data for a in planes], r.n, [a.ctypes.data for a in out],
                           ccs.make_opts(pairs=True, host_chunk=20000))
    got = dict(t=out[0], u=out[1], v=out[2], pid=out[3])
    same(got, ref, "host path")
    # n = 0 is a no-op
    ccs.ccs_intersect(sc.handle, ccs.rays_to_device(r.soa()), 0, ccs.alloc_hits(1), ccs.make_opts(pairs=True))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    # the iteration cap latches the status; the next launch runs normally
    hits = ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(pairs=True, iter_cap=5))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_ERR_TRAVERSAL_LIMIT
    assert (ccs.hits_to_numpy(hits)["pid"][ref["pid"] != MISS] == MISS).all()
    same(run(sc, r, pairs=True), ref, "after the cap")
    sc.close()


def test_pairs_invalid_rays_and_one_patch():
    s = sg.config_scene(1)
    r = sg.random_rays(4000, seed=73, radius=2.0)
    r.o[::7, 0] = np.nan
    r.tmin[1::11] = 5.0
    r.tmax[1::11] = 1.0
    sc = ccs.Scene(s.P, s.types)
    g = run(sc, r, pairs=True)
    same(g, run(sc, r), "invalid rays")
    assert (g["pid"][::7] == MISS).all() and (g["pid"][1::11] == MISS).all()
    one = ccs.Scene(s.P[:1], s.types[:1])
    same(run(one, r, pairs=True), run(one, r), "one patch")
    sc.close()
    one.close()


def test_pairs_batched_and_graph_replay_equal_single_scenes():
    scenes = [sg.make_scene(n, 0.02 * k, 3, k + 1, gregory_ring=k == 1) for k, n in enumerate([2, 5, 3, 4])]
    rays = [sg.pinhole_rays(64, 48), sg.random_rays(4001, seed=3), sg.random_rays(517, seed=4),
            sg.random_rays(0, seed=5)]
    handles = [ccs.Scene(x.P, x.types, local=k % 2 == 0) for k, x in enumerate(scenes)]
    ref = [run(h, r) if r.n else None for h, r in zip(handles, rays)]
    dev_rays = [ccs.rays_to_device(r.soa()) for r in rays]
    hits = [ccs.alloc_hits(max(r.n, 1)) for r in rays]
    ccs.ccs_intersect_batched(handles, dev_rays, hits, ccs.make_opts(pairs=True))
    torch.cuda.synchronize()
    for h, rf, r in zip(hits, ref, rays):
        if r.n:
            same({k: v[:r.n] for k, v in ccs.hits_to_numpy(h).items()}, rf, "batched")
    # an image width over a batch tiles the concatenated rays, which are no image: the same answers
    ccs.ccs_intersect_batched(handles, dev_rays, hits, ccs.make_opts(pairs=True, image_width=64))
    torch.cuda.synchronize()
    for h, rf, r in zip(hits, ref, rays):
        if r.n:
            same({k: v[:r.n] for k, v in ccs.hits_to_numpy(h).items()}, rf, "batched, tiled")
    b = ccs.ccs_batch_create(handles, dev_rays, hits, n_rays=[r.n for r in rays])
    ccs.ccs_batch_capture(b, ccs.CCS_BATCH_INTERSECT, ccs.make_opts(pairs=True, cache_slots=1))
    for _ in range(2):
        for h in hits:
            for p in h:
                p.fill_(-3)
        ccs.ccs_batch_launch(b)
        assert ccs.ccs_batch_sync_status(b) == ccs.CCS_OK
        for h, rf, r in zip(hits, ref, rays):
            if r.n:
                same({k: v[:r.n] for k, v in ccs.hits_to_numpy(h).items()}, rf, "graph")
    ccs.ccs_batch_destroy(b)
    for h in handles:
        h.close()


@pytest.mark.parametrize("local", [False, True])
def test_pairs_subtrees_handed_to_idle_lanes(local):
    """A batch much smaller than the GPU: the queue empties at once and idle lanes search subtrees of the
    busy lanes' pairs (counter 11 counts the hand-overs); the hits stay bit-identical."""
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(3000, seed=75, target=1.05)
    sc = ccs.Scene(s.P, s.types, local=local)
    ref = run(sc, r)
    cnt = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device="cuda")
    for K in (0, 1, 2):
        same(run(sc, r, pairs=True, cache_slots=K), ref, K)
    got = run(sc, r, counters=cnt, pairs=True)
    same(got, ref, "counting")
    assert int(cnt[11]) > 100
    compare(got, oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True, local=local), 8, max_flagged_frac=0.05)
    sc.close()


@pytest.mark.parametrize("width", [2, 4])
def test_pairs_root_box_cull_keeps_every_hit(width):
    """With local frames the candidate pass drops Bezier patches whose root box (in the patch frame) the
    ray does not come near (counter 17).  Rays that graze the surface, just above it and nearly tangent,
    are the ones a too-tight test would lose: their hits stay bit-identical to the ray-persistent kernel's,
    which never culls.  Without local frames nothing is culled."""
    s = sg.config_scene(2)
    cam = sg.pinhole_rays(160, 90)
    sc = ccs.Scene(s.P, s.types, local=True, bvh_width=width)
    h = run(sc, cam)
    hit = h["pid"] != MISS
    p = cam.o[hit].astype(np.float64) + cam.d[hit].astype(np.float64) * h["t"][hit][:, None]
    rng = np.random.default_rng(17)
    nrm = p / np.linalg.norm(p, axis=1, keepdims=True)
    tan = np.cross(nrm, rng.normal(size=p.shape))
    tan /= np.linalg.norm(tan, axis=1, keepdims=True)
    oo, dd = [], []
    for lift in (1e-5, 1e-4, 1e-3, 1e-2):
        tilt = rng.uniform(-2.0, 2.0, (len(p), 1)) * lift
        dv = tan - tilt * nrm
        dv /= np.linalg.norm(dv, axis=1, keepdims=True)
        oo.append(p * (1.0 + lift) - 2.0 * dv)
        dd.append(dv)
    oo, dd = np.concatenate(oo).astype(np.float32), np.concatenate(dd).astype(np.float32)
    n = len(oo)
    r = sg.Rays(oo, dd, np.zeros(n, np.float32), np.full(n, np.inf, np.float32))
    ref = run(sc, r)
    assert 0.2 * n < (ref["pid"] != MISS).sum() < n
    cnt = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device="cuda")
    same(run(sc, r, counters=cnt, pairs=True), ref, "grazing")
    assert int(cnt[17]) > n // 4
    same(run(sc, cam, pairs=True), h, "primary")
    sc.close()
    sw = ccs.Scene(s.P, s.types, local=False, bvh_width=width)
    cnt.zero_()
    same(run(sw, r, counters=cnt, pairs=True), run(sw, r), "world axes")
    assert int(cnt[17]) == 0
    sw.close()
