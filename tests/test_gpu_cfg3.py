"""The 393,216-patch cube-sphere (128 x 128 quads per face, noise 0.1 with 5 octaves): full-size launches
(3840 x 2160 primary rays, autotuned), sampled against the oracle; diffuse and mirror secondary rays
generated from oracle hits checked in full; full-size secondary generations run on the device."""
import numpy as np
import pytest

import oracle
from oracle.raygen import diffuse_rays
from paper_1811_03510_gb300 import ccs, scenegen as sg
from parity import MISS, compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_03510_gb300 import build_ext
    build_ext.build()
    oracle.build()
    torch.cuda.set_device(0)
    s = sg.config_scene(3)
    sc = ccs.Scene(s.P, s.types)
    yield s, sc
    sc.close()


def test_full_size_primary_sampled_and_secondaries(big):
    s, sc = big
    assert s.n == 393216
    cam = sg.pinhole_rays(3840, 2160)
    rays = ccs.rays_to_device(cam.soa())
    hits = ccs.alloc_hits(cam.n)
    best, ms, _ = ccs.ccs_autotune(sc.handle, rays, cam.n, hits, ccs.make_opts(), reps=1)
    ccs.ccs_intersect(sc.handle, rays, cam.n, hits, best)
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    g = ccs.hits_to_numpy(hits)
    hit_idx = np.nonzero(g["pid"] != MISS)[0]
    assert 0.1 < len(hit_idx) / cam.n < 0.3
    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([rng.choice(cam.n, 1500, replace=False), rng.choice(hit_idx, 1500, replace=False)]))
    sub = cam.subset(pick)
    o = oracle.intersect(s.P, s.types, sub.soa(), L=8, flags=True)
    compare({k: v[pick] for k, v in g.items()}, o, 8)
    # secondary rays from the oracle's hits of the sample, intersected by both sides
    for mirror in (False, True):
        sec = diffuse_rays(s.P, s.types, sub.soa(), o, seed=1, mirror=mirror)
        act = sec[7] >= sec[6]
        sr = [a[act] for a in sec]
        n = int(act.sum())
        hs = ccs.alloc_hits(n)
        ccs.ccs_intersect(sc.handle, ccs.rays_to_device(sr), n, hs, best)
        torch.cuda.synchronize()
        os_ = oracle.intersect(s.P, s.types, sr, L=8, flags=True)
        compare(ccs.hits_to_numpy(hs), os_, 8)
    # full-size generations on the device (one slot per pixel, inactive slots miss)
    for gen in (lambda: ccs.gen_diffuse(sc, rays, hits, seed=1), lambda: ccs.gen_mirror(sc, rays, hits)):
        planes = gen()
        h2 = ccs.alloc_hits(cam.n)
        ccs.ccs_intersect(sc.handle, planes, cam.n, h2, best)
        torch.cuda.synchronize()
        assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
        g2 = ccs.hits_to_numpy(h2)
        inactive = g["pid"] == MISS
        assert (g2["pid"][inactive] == MISS).all()


@pytest.mark.parametrize("pairs", [False, True])
def test_full_size_local_frames_sampled(big, pairs):
    """The same launch with the sub-domain boxes in the patches' local frames (Sec. 3.4), sampled against
    the oracle under the same frames, with its secondary rays.  Leaf cells of these small patches are
    about 5e-5 wide; a pair's ray is anchored at its entry into the patch box (its origin formed in FP64),
    so the FP32 error no longer grows with the 3 units to the camera and at most 2% of the sampled rays
    are ambiguous, as with boxes in world axes; every other ray must agree.  Both engines."""
    s, _ = big
    sc = ccs.Scene(s.P, s.types, local=True)
    cam = sg.pinhole_rays(3840, 2160)
    rays = ccs.rays_to_device(cam.soa())
    hits = ccs.alloc_hits(cam.n)
    ccs.ccs_intersect(sc.handle, rays, cam.n, hits, ccs.make_opts(pairs=pairs))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    g = ccs.hits_to_numpy(hits)
    hit_idx = np.nonzero(g["pid"] != MISS)[0]
    rng = np.random.default_rng(4)
    pick = np.unique(np.concatenate([rng.choice(cam.n, 1500, replace=False), rng.choice(hit_idx, 1500, replace=False)]))
    sub = cam.subset(pick)
    o = oracle.intersect(s.P, s.types, sub.soa(), L=8, flags=2, local=True)
    rep = compare({k: v[pick] for k, v in g.items()}, o, 8, max_flagged_frac=0.02)
    print("local frames, 393,216 patches:", rep)
    assert rep["hits"] - rep["flagged"] > 1400
    sec = diffuse_rays(s.P, s.types, sub.soa(), o, seed=2)
    act = sec[7] >= sec[6]
    sr = [a[act] for a in sec]
    n = int(act.sum())
    hs = ccs.alloc_hits(n)
    ccs.ccs_intersect(sc.handle, ccs.rays_to_device(sr), n, hs, ccs.make_opts(pairs=pairs))
    torch.cuda.synchronize()
    compare(ccs.hits_to_numpy(hs), oracle.intersect(s.P, s.types, sr, L=8, flags=True, local=True), 8,
            max_flagged_frac=0.02)
    sc.close()


def test_full_size_four_wide_bvh_and_work_order_equal_binary(big):
    """The 3840 x 2160 primary launch on the 393,216-patch scene, local frames: a 4-wide BVH (19-level
    binary tree collapsed) and the work order over the image's tiles give the binary launch's hits bit
    for bit."""
    s, _ = big
    cam = sg.pinhole_rays(3840, 2160)
    rays = ccs.rays_to_device(cam.soa())
    out = {}
    for width in (2, 4):
        sc = ccs.Scene(s.P, s.types, local=True, bvh_width=width)
        for order in (False, True):
            hits = ccs.alloc_hits(cam.n)
            ccs.ccs_intersect(sc.handle, rays, cam.n, hits, ccs.make_opts(order=order, image_width=3840))
            torch.cuda.synchronize()
            assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
            out[(width, order)] = ccs.hits_to_numpy(hits)
        sc.close()
    ref = out[(2, False)]
    assert (ref["pid"] != MISS).mean() > 0.1
    for key, g in out.items():
        for k in ("t", "u", "v", "pid"):
            assert np.array_equal(g[k], ref[k]), (key, k)
