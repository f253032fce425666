"""Any-hit (shadow-ray) query through the C ABI: occlusion bit-exact against the closest-hit kernel's
hit/miss, parity with the FP64 oracle, the shadow-ray generator against the oracle's, less work than the
closest hit, and the edge cases."""
import numpy as np
import pytest

import oracle
from oracle.raygen import shadow_rays
from paper_1811_03510_gb300 import ccs, scenegen as sg
from parity import MISS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
LIGHT = (2.0, 3.0, 4.0)


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_03510_gb300 import build_ext
    build_ext.build()
    oracle.build()
    torch.cuda.set_device(0)


def closest_and_occluded(sc, r, **kw):
    rays = ccs.rays_to_device(r.soa())
    hits = ccs.intersect(sc, rays, ccs.make_opts(**kw))
    occ = ccs.occluded(sc, rays, ccs.make_opts(**kw))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    return ccs.hits_to_numpy(hits), occ.cpu().numpy()


def two_spheres():
    """The 1536-patch sphere and a 96-patch sphere of radius 0.35 between it and the light (casts a shadow
    on the lit, camera-facing side)."""
    big, small = sg.config_scene(2), sg.config_scene(1)
    ldir = np.array(LIGHT) / np.linalg.norm(LIGHT)
    P2 = (small.P.astype(np.float64) * 0.35 + 1.6 * ldir).astype(np.float32)
    return sg.Scene(np.concatenate([big.P, P2]), np.concatenate([big.types, small.types]), "two spheres")


def shadow_from_primary(s, w, h):
    cam = sg.pinhole_rays(w, h)
    sc = ccs.Scene(s.P, s.types)
    prim = ccs.rays_to_device(cam.soa())
    hp = ccs.intersect(sc, prim, ccs.make_opts())
    planes = ccs.gen_shadow(sc, prim, hp, LIGHT)
    torch.cuda.synchronize()
    act = (planes[7] >= planes[6]).nonzero().squeeze(1)
    sh = [p.index_select(0, act).cpu().numpy() for p in planes]
    return sc, sg.Rays(np.stack(sh[:3], 1), np.stack(sh[3:6], 1), sh[6], sh[7])


@pytest.mark.parametrize("which", ["cfg1_primary", "cfg2_random", "gregory_ring", "shadow"])
def test_occluded_equals_closest_hit_exists(which):
    if which == "cfg1_primary":
        s, r = sg.config_scene(1), sg.pinhole_rays(64, 64)
        sc = ccs.Scene(s.P, s.types)
    elif which == "cfg2_random":
        s, r = sg.config_scene(2), sg.random_rays(40000, seed=8)
        sc = ccs.Scene(s.P, s.types)
    elif which == "gregory_ring":
        s, r = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True), sg.random_rays(30000, seed=9, target=1.0)
        sc = ccs.Scene(s.P, s.types)
    else:
        sc, r = shadow_from_primary(two_spheres(), 480, 270)
    for kw in (dict(), dict(cache_slots=0, bvh_burst=1), dict(block_threads=64, refill=1, vote=12)):
        g, occ = closest_and_occluded(sc, r, **kw)
        assert np.array_equal(occ.astype(bool), g["pid"] != MISS), (which, kw)
    assert occ.sum() > 100 and (occ == 0).sum() > 100
    sc.close()


def test_occluded_matches_oracle():
    s = two_spheres()
    sc, r = shadow_from_primary(s, 320, 180)
    _, occ = closest_and_occluded(sc, r)
    o = oracle.occluded(s.P, s.types, r.soa(), L=8, flags=True)
    clear = (o["flags"] & 4) == 0   # hit/miss cannot flip under the FP32 error model
    assert clear.mean() > 0.99
    assert np.array_equal(occ[clear], o["occluded"][clear])
    assert o["occluded"].sum() > 100
    sc.close()


def test_shadow_generator_matches_oracle_generator():
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    cam = sg.pinhole_rays(160, 90)
    o = oracle.intersect(s.P, s.types, cam.soa(), L=8)
    sc = ccs.Scene(s.P, s.types)
    rays = ccs.rays_to_device(cam.soa())
    hits = [torch.from_numpy(np.where(o["pid"] != MISS, o["t"], np.inf).astype(np.float32)).cuda(),
            torch.from_numpy(o["u"]).cuda(), torch.from_numpy(o["v"]).cuda(),
            torch.from_numpy(o["pid"].view(np.int32)).cuda()]
    got = [p.cpu().numpy() for p in ccs.gen_shadow(sc, rays, hits, LIGHT)]
    torch.cuda.synchronize()
    ref = shadow_rays(s.P, s.types, cam.soa(), o, LIGHT)
    act = ref[7] >= ref[6]
    assert act.sum() > 1000
    # the lit test compares a normal with a light direction: allow disagreement only at grazing light
    agree = (got[7] >= got[6]) == act
    assert agree.mean() > 0.999
    both = act & (got[7] >= got[6])
    for k in range(8):
        np.testing.assert_allclose(got[k][both], ref[k][both], atol=2e-5, rtol=1e-5)
    sc.close()


def test_any_hit_does_no_more_work_than_closest_hit():
    sc, r = shadow_from_primary(two_spheres(), 480, 270)
    rays = ccs.rays_to_device(r.soa())
    c1 = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device="cuda")
    c2 = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device="cuda")
    ccs.intersect(sc, rays, ccs.make_opts(counters=c1))
    ccs.occluded(sc, rays, ccs.make_opts(counters=c2))
    torch.cuda.synchronize()
    a = dict(zip(ccs.COUNTER_NAMES, c1.cpu().tolist()))
    b = dict(zip(ccs.COUNTER_NAMES, c2.cpu().tolist()))
    for k in ("bvh_nodes", "bezier_splits", "gregory_splits", "leaves", "pairs"):
        assert b[k] <= a[k], (k, a, b)
    assert b["leaves"] < a["leaves"]   # an occluded ray stops at its first leaf
    sc.close()


def test_any_hit_edge_cases():
    s = sg.config_scene(1)
    r = sg.pinhole_rays(40, 40)
    o, d, tmin, tmax = r.o.copy(), r.d.copy(), r.tmin.copy(), r.tmax.copy()
    o[0, 0] = np.nan
    d[1, 2] = np.nan
    tmin[2], tmax[2] = 5.0, 1.0
    tmax[3:300] = 0.5
    rr = sg.Rays(o, d, tmin, tmax)
    sc = ccs.Scene(s.P, s.types)
    g, occ = closest_and_occluded(sc, rr)
    assert (occ[:300] == 0).all()
    assert np.array_equal(occ.astype(bool), g["pid"] != MISS)
    # zero rays: no launch, no error
    ccs.ccs_occluded(sc.handle, ccs.rays_to_device(r.soa()), 0, torch.zeros(1, dtype=torch.uint8, device="cuda"))
    # iteration cap: status latched, capped rays report 0, context usable
    occ_cap = ccs.occluded(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(iter_cap=3))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_ERR_TRAVERSAL_LIMIT
    assert (occ_cap.cpu().numpy() == 0).all()
    g2, occ2 = closest_and_occluded(sc, r)
    assert np.array_equal(occ2.astype(bool), g2["pid"] != MISS)
    sc.close()
    empty = ccs.Scene(s.P[:0], s.types[:0])
    _, occ = closest_and_occluded(empty, r)
    assert (occ == 0).all()
    empty.close()
