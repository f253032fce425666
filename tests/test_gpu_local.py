"""Local frames (Sec. 3.4, CCS_SCENE_LOCAL_FRAMES) through the C ABI: parity with the FP64 oracle under the
same frames, hits independent of the launch options and layouts, watertight shared boundaries in FP32,
the secondary-ray generators, and the batched, any-hit, learned and screen-space paths on such scenes."""
import numpy as np
import pytest

import oracle
from oracle.raygen import diffuse_rays
from paper_1811_03510_gb300 import ccs, scenegen as sg
from parity import MISS, compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
RNG = np.random.default_rng(99)


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_03510_gb300 import build_ext
    build_ext.build()
    oracle.build()
    torch.cuda.set_device(0)


def run(sc, r, **kw):
    hits = ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(**kw))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    return ccs.hits_to_numpy(hits)


def same(a, b, what):
    for k in ("t", "u", "v", "pid"):
        assert np.array_equal(a[k], b[k]), (what, k)


@pytest.mark.parametrize("which", ["cfg1_primary", "cfg2_random", "gregory_ring"])
def test_local_frames_match_oracle(which):
    if which == "cfg1_primary":
        s, r = sg.config_scene(1), sg.pinhole_rays(64, 64)
    elif which == "cfg2_random":
        s, r = sg.config_scene(2), sg.random_rays(20000, seed=51)
    else:
        s, r = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True), sg.random_rays(20000, seed=52, target=1.0)
    sc = ccs.Scene(s.P, s.types, local=True)
    g = run(sc, r)
    o = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True, local=True)
    # the FP32 transform of the ray into the patch frame widens the error model with the distance of the
    # origin from the patch (random rays start 3 units away), so more rays are flagged than in world frames
    rep = compare(g, o, 8, max_flagged_frac=0.05)
    assert rep["hits"] > 500
    sc.close()


def test_local_frames_full_size_primary_launch_sampled():
    s = sg.config_scene(2)
    r = sg.pinhole_rays(1920, 1080)
    sc = ccs.Scene(s.P, s.types, local=True)
    g = run(sc, r)
    hit_idx = np.nonzero(g["pid"] != MISS)[0]
    assert 0.1 < len(hit_idx) / r.n < 0.3
    pick = np.unique(np.concatenate([RNG.choice(r.n, 2000, replace=False), RNG.choice(hit_idx, 2000, replace=False)]))
    o = oracle.intersect(s.P, s.types, r.subset(pick).soa(), L=8, flags=True, local=True)
    compare({k: v[pick] for k, v in g.items()}, o, 8, max_flagged_frac=0.03)
    sc.close()


def test_local_frame_hits_do_not_depend_on_launch_options():
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(30000, seed=53)
    sc = ccs.Scene(s.P, s.types, local=True)
    ref = run(sc, r)
    for kw in [dict(block_threads=32), dict(cache_slots=0, refill=1), dict(vote=16, bvh_burst=2), dict(min_blocks=4),
               dict(lanes_per_ray=3), dict(lanes_per_ray=3, cache_slots=0, blocks_per_sm=6)]:
        same(run(sc, r, **kw), ref, kw)
    sc.close()


def test_local_frames_are_watertight_in_fp32():
    """Rays through points on shared patch boundaries of the closed cube-sphere (edges at 0, 1/4, 1/2, 3/4,
    corners included) always hit in FP32 (Sec. 3.4: false positives only)."""
    s = sg.config_scene(1)
    P = s.P.astype(float)
    targets = []
    for f in range(s.n):
        for slots in [(0, 1, 2, 3), (3, 7, 11, 15), (15, 14, 13, 12), (12, 8, 4, 0)]:
            b = P[f, list(slots)]
            for t in (0.0, 0.25, 0.5, 0.75):
                w = np.array([(1 - t) ** 3, 3 * t * (1 - t) ** 2, 3 * t * t * (1 - t), t ** 3])
                targets.append(w @ b)
    targets = np.array(targets)
    o = RNG.normal(size=targets.shape)
    o *= 3.0 / np.linalg.norm(o, axis=1, keepdims=True)
    flip = np.einsum("ij,ij->i", o, targets) < 0
    o[flip] *= -1
    d = targets - o
    r = sg.Rays(o.astype(np.float32), d.astype(np.float32), np.zeros(len(o), np.float32),
                np.full(len(o), np.inf, np.float32))
    for local in (False, True):
        sc = ccs.Scene(s.P, s.types, local=local)
        g = run(sc, r)
        assert (g["pid"] != MISS).all(), (local, int((g["pid"] == MISS).sum()))
        sc.close()


def test_generators_on_local_frame_scenes_match_the_oracle_generator():
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    cam = sg.pinhole_rays(160, 90)
    o = oracle.intersect(s.P, s.types, cam.soa(), L=8)
    sc = ccs.Scene(s.P, s.types, local=True)
    rays = ccs.rays_to_device(cam.soa())
    hits = [torch.from_numpy(np.where(o["pid"] != MISS, o["t"], np.inf).astype(np.float32)).cuda(),
            torch.from_numpy(o["u"]).cuda(), torch.from_numpy(o["v"]).cuda(),
            torch.from_numpy(o["pid"].view(np.int32)).cuda()]
    got = [p.cpu().numpy() for p in ccs.gen_diffuse(sc, rays, hits, seed=7)]
    torch.cuda.synchronize()
    ref = diffuse_rays(s.P, s.types, cam.soa(), o, seed=7)
    act = ref[7] >= ref[6]
    assert act.sum() > 1000 and np.array_equal(got[7] >= got[6], act)
    for k in range(6):
        np.testing.assert_allclose(got[k][act], ref[k][act], atol=3e-5)
    sc.close()


def test_batched_any_hit_learned_and_screen_space_on_local_frame_scenes():
    scenes = [sg.make_scene(n, 0.02 * (k % 3), 3, k + 1, gregory_ring=(k == 1)) for k, n in enumerate([2, 5, 3])]
    rays = [sg.pinhole_rays(64, 48), sg.random_rays(4001, seed=3), sg.random_rays(517, seed=4)]
    handles = [ccs.Scene(x.P, x.types, local=True) for x in scenes]
    ref = [run(h, r) for h, r in zip(handles, rays)]
    hits = [ccs.alloc_hits(r.n) for r in rays]
    ccs.ccs_intersect_batched(handles, [ccs.rays_to_device(r.soa()) for r in rays], hits, ccs.make_opts())
    torch.cuda.synchronize()
    for h, rf in zip(hits, ref):
        same(ccs.hits_to_numpy(h), rf, "batched")
    # any hit equals the closest hit's hit/miss
    for h, r, rf in zip(handles, rays, ref):
        occ = ccs.occluded(h, ccs.rays_to_device(r.soa()))
        torch.cuda.synchronize()
        assert np.array_equal(occ.cpu().numpy().astype(bool), rf["pid"] != MISS)
    # the learned proposal reorders the search only
    p = ccs.ccs_proposal_create(seed=9)
    rd = ccs.rays_to_device(rays[1].soa())
    out = ccs.alloc_hits(rays[1].n)
    ccs.ccs_intersect_learned(handles[1].handle, p, rd, rays[1].n, out, ccs.make_opts(), 0.0)
    torch.cuda.synchronize()
    same(ccs.hits_to_numpy(out), ref[1], "learned")
    ccs.ccs_proposal_destroy(p)
    # screen-space termination under local frames against the oracle
    sp = 3e-3
    g = run(handles[1], rays[1], pixel_spread=sp)
    o = oracle.intersect(scenes[1].P, scenes[1].types, rays[1].soa(), L=8, flags=True, spread=sp, local=True)
    ok = o["flags"] == 0
    assert np.array_equal(g["pid"][ok], o["pid"][ok])
    hit = ok & (o["pid"] != MISS)
    assert (np.abs(g["t"][hit] - o["t"][hit]) <= 1e-4 * np.abs(o["t"][hit])).all()
    for h in handles:
        h.close()


def test_benchmark_step_in_its_tuned_configuration_sampled():
    """The benchmark's step as bench.py times it: the 1920 x 1080 primary batch and its compacted diffuse
    batch on the local-frame scene, each with the options the autotuner picks (the primary batch as an
    image, so the work order may rank its tiles).  Sampled rays against the oracle under the same frames,
    and every hit identical to the default launch."""
    s = sg.config_scene(2)
    cam = sg.pinhole_rays(1920, 1080)
    sc = ccs.Scene(s.P, s.types, local=True)
    prim = ccs.rays_to_device(cam.soa())
    ref_p = ccs.hits_to_numpy(ccs.intersect(sc, prim, ccs.make_opts()))
    hp = ccs.intersect(sc, prim, ccs.make_opts())
    planes = ccs.gen_diffuse(sc, prim, hp, seed=1, leaf_depth=8, offset_abs=1e-4)
    torch.cuda.synchronize()
    act = (planes[7] >= planes[6]).nonzero().squeeze(1)
    diff = [p.index_select(0, act).contiguous() for p in planes]
    nd = int(act.numel())
    ref_d = ccs.hits_to_numpy(ccs.intersect(sc, diff, ccs.make_opts()))
    got = {}
    for name, rays, n, width in (("primary", prim, cam.n, 1920), ("diffuse", diff, nd, 0)):
        h = ccs.alloc_hits(n)
        best, _, _ = ccs.ccs_autotune(sc.handle, rays, n, h, ccs.make_opts(image_width=width), reps=1)
        out = ccs.alloc_hits(n)
        for t in out:
            t.fill_(-7)
        ccs.ccs_intersect(sc.handle, rays, n, out, best)
        torch.cuda.synchronize()
        assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
        got[name] = ccs.hits_to_numpy(out)
    same(got["primary"], ref_p, "primary, tuned")
    same(got["diffuse"], ref_d, "diffuse, tuned")
    hit_idx = np.nonzero(ref_p["pid"] != MISS)[0]
    pick = np.unique(np.concatenate([RNG.choice(cam.n, 1500, replace=False), RNG.choice(hit_idx, 1500, replace=False)]))
    o = oracle.intersect(s.P, s.types, cam.subset(pick).soa(), L=8, flags=True, local=True)
    compare({k: v[pick] for k, v in got["primary"].items()}, o, 8, max_flagged_frac=0.03)
    dsoa = [p.cpu().numpy() for p in diff]
    dpick = RNG.choice(nd, 3000, replace=False)
    o = oracle.intersect(s.P, s.types, [a[dpick] for a in dsoa], L=8, flags=True, local=True)
    compare({k: v[dpick] for k, v in got["diffuse"].items()}, o, 8, max_flagged_frac=0.05)
    sc.close()
