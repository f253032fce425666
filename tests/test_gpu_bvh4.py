"""4-wide BVH (ccs_bvh_params.width = 4; a wider BVH is named as future work in Sec. 4).  The answer does
not depend on the hierarchy over the patches, so every hit must be bit-identical to the binary BVH's,
which the FP64 oracle pins: across launch options, both thread layouts, local and world frames, the
any-hit, screen-space, learned and work-order paths, refits after a deformation, and batches."""
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


def run(sc, r, **kw):
    hits = ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(**kw))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    return ccs.hits_to_numpy(hits)


def same(a, b, what):
    for k in ("t", "u", "v", "pid"):
        assert np.array_equal(a[k], b[k]), (what, k)


def test_four_wide_matches_oracle():
    s, r = sg.config_scene(2), sg.random_rays(20000, seed=61)
    sc = ccs.Scene(s.P, s.types, bvh_width=4)
    rep = compare(run(sc, r), oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True), 8)
    assert rep["hits"] > 500
    sc.close()


@pytest.mark.parametrize("local", [False, True])
def test_four_wide_hits_equal_binary_across_launch_options(local):
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(30000, seed=62)
    two = ccs.Scene(s.P, s.types, local=local)
    four = ccs.Scene(s.P, s.types, local=local, bvh_width=4)
    ref = run(two, r)
    assert (ref["pid"] != MISS).sum() > 1000
    for kw in [{}, dict(block_threads=32), dict(cache_slots=0, refill=1), dict(vote=16, bvh_burst=2),
               dict(bvh_burst=16, refill=16), dict(min_blocks=4), dict(lanes_per_ray=3),
               dict(lanes_per_ray=3, cache_slots=0, blocks_per_sm=6), dict(order=True),
               dict(order=True, image_width=173)]:
        same(run(four, r, **kw), ref, kw)
    two.close()
    four.close()


def test_four_wide_primary_image_and_query_modes():
    s = sg.config_scene(2)
    cam = sg.pinhole_rays(960, 540)
    two = ccs.Scene(s.P, s.types, local=True)
    four = ccs.Scene(s.P, s.types, local=True, bvh_width=4)
    same(run(four, cam, order=True, image_width=960), run(two, cam), "primary")
    spread = 2.0 * np.tan(np.radians(30.0)) / 540
    same(run(four, cam, pixel_spread=spread), run(two, cam, pixel_spread=spread), "screen space")
    rays = ccs.rays_to_device(cam.soa())
    assert torch.equal(ccs.occluded(four, rays), ccs.occluded(two, rays))
    p = ccs.ccs_proposal_create(seed=3)
    outs = []
    for sc in (two, four):
        out = ccs.alloc_hits(cam.n)
        ccs.ccs_intersect_learned(sc.handle, p, rays, cam.n, out, ccs.make_opts(), 0.0)
        torch.cuda.synchronize()
        outs.append(ccs.hits_to_numpy(out))
    same(outs[1], outs[0], "learned")
    ccs.ccs_proposal_destroy(p)
    two.close()
    four.close()


def test_four_wide_refit_after_deformation_and_single_patch():
    s = sg.config_scene(2)
    r = sg.random_rays(20000, seed=63)
    four = ccs.Scene(s.P, s.types, bvh_width=4)
    Q = s.P + 0.03 * np.sin(3.0 * s.P + 1.0).astype(np.float32)
    q = [torch.from_numpy(np.ascontiguousarray(Q[..., c]).reshape(-1)).cuda() for c in range(3)]
    ccs.ccs_scene_update_points(four.handle, *q)
    ccs.ccs_bvh_refit(four.handle)
    torch.cuda.synchronize()
    fresh = ccs.Scene(Q, s.types)   # binary BVH built on the deformed points
    same(run(four, r), run(fresh, r), "refit")
    four.close()
    fresh.close()
    one4 = ccs.Scene(s.P[:1], s.types[:1], bvh_width=4)
    one2 = ccs.Scene(s.P[:1], s.types[:1])
    rr = sg.random_rays(3000, seed=5, radius=2.0)
    same(run(one4, rr), run(one2, rr), "one patch")
    one4.close()
    one2.close()


def test_four_wide_batches_and_mixed_widths():
    scenes = [sg.make_scene(n, 0.02 * k, 3, k + 1) for k, n in enumerate([2, 5, 3])]
    rays = [sg.pinhole_rays(64, 48), sg.random_rays(4001, seed=3), sg.random_rays(517, seed=4)]
    two = [ccs.Scene(x.P, x.types) for x in scenes]
    four = [ccs.Scene(x.P, x.types, bvh_width=4) for x in scenes]
    ref = [run(h, r) for h, r in zip(two, rays)]
    hits = [ccs.alloc_hits(r.n) for r in rays]
    ccs.ccs_intersect_batched(four, [ccs.rays_to_device(r.soa()) for r in rays], hits, ccs.make_opts())
    torch.cuda.synchronize()
    for h, rf in zip(hits, ref):
        same(ccs.hits_to_numpy(h), rf, "batched")
    with pytest.raises(ccs.CcsError):
        ccs.ccs_intersect_batched([two[0], four[1]], [ccs.rays_to_device(r.soa()) for r in rays[:2]], hits[:2],
                                  ccs.make_opts())
    for h in two + four:
        h.close()


def test_four_wide_trace_export_runs_and_keeps_the_hits():
    """The trace export (a pair's features and its best leaf's depth-3 cell) on a 4-wide BVH: same hits as
    the binary tree, one exported row per pair that found a leaf, labels within the 64 depth-3 cells."""
    s = sg.config_scene(2)
    r = sg.random_rays(20000, seed=64)
    two = ccs.Scene(s.P, s.types)
    four = ccs.Scene(s.P, s.types, bvh_width=4)
    rays = ccs.rays_to_device(r.soa())
    hits = ccs.alloc_hits(r.n)
    cap = 4 * r.n
    feat = torch.zeros(cap, 24, device="cuda")
    lab = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ccs.ccs_trace_export(four.handle, rays, r.n, hits, ccs.make_opts(), feat, lab, cap, cnt)
    torch.cuda.synchronize()
    same(ccs.hits_to_numpy(hits), run(two, r), "export")
    k = int(cnt.item())
    assert k >= int((ccs.hits_to_numpy(hits)["pid"] != MISS).sum()) > 500
    assert (lab[:k].cpu().numpy() < 64).all() and torch.isfinite(feat[:k]).all()
    two.close()
    four.close()


def test_scene_with_both_trees_and_per_launch_width():
    """CCS_BVH_BOTH: one scene holds the binary and the 4-wide tree; each launch picks one (bvh_width), the
    tuner may pick either, a refit updates both, and asking a one-tree scene for the other width fails."""
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(30000, seed=65)
    both = ccs.Scene(s.P, s.types, local=True, bvh_width="both")
    two = ccs.Scene(s.P, s.types, local=True)
    ref = run(two, r)
    for w in (0, 2, 4):
        same(run(both, r, bvh_width=w), ref, ("width", w))
    same(run(both, r, bvh_width=4, order=True, lanes_per_ray=3), ref, "width 4, order, groups")
    # a binary launch whose work-order estimate walks the scene's 4-wide tree
    same(run(both, r, bvh_width=2, order=True), ref, "width 2, order")
    rays = ccs.rays_to_device(r.soa())
    h = ccs.alloc_hits(r.n)
    best, _, trials = ccs.ccs_autotune(both.handle, rays, r.n, h, ccs.make_opts(), reps=1)
    assert {o.bvh_width for o, _ in trials} >= {0, 4}
    same(run(both, r, **ccs.opts_dict(best)), ref, "tuned")
    # a deformation and one refit: both trees follow
    Q = s.P + 0.03 * np.sin(3.0 * s.P + 1.0).astype(np.float32)
    q = [torch.from_numpy(np.ascontiguousarray(Q[..., c]).reshape(-1)).cuda() for c in range(3)]
    ccs.ccs_scene_update_points(both.handle, *q)
    ccs.ccs_bvh_refit(both.handle)
    torch.cuda.synchronize()
    fresh = ccs.Scene(Q, s.types, local=True)
    ref2 = run(fresh, r)
    for w in (2, 4):
        same(run(both, r, bvh_width=w), ref2, ("refit", w))
        same(run(both, r, bvh_width=w, order=True), ref2, ("refit, order", w))
    with pytest.raises(ccs.CcsError):
        run(two, r, bvh_width=4)
    with pytest.raises(ccs.CcsError):   # batches need one tree per scene
        ccs.ccs_intersect_batched([both], [rays], [ccs.alloc_hits(r.n)], ccs.make_opts())
    for sc in (both, two, fresh):
        sc.close()
