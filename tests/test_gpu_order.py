"""Work order (CCS_TRACE_ORDER): a pre-pass ranks tiles of rays by the candidate patches their sampled
rays enter, and the work queue hands out the costliest tiles first.  Only the processing order changes:
every hit must be bit-identical to the launch without it, on images (with ragged edges and a partial
last row), on batches that are not images, through the host-buffer entry and in the any-hit query."""
import numpy as np
import pytest

from paper_1811_03510_gb300 import ccs, scenegen as sg
from parity import MISS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_03510_gb300 import build_ext
    build_ext.build()
    torch.cuda.set_device(0)


def run(sc, rays, **kw):
    d = ccs.rays_to_device(rays.soa())
    hits = ccs.alloc_hits(rays.n)
    for h in hits:   # a ray the queue never hands out would keep this
        h.fill_(-7)
    ccs.ccs_intersect(sc.handle, d, rays.n, hits, ccs.make_opts(**kw))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    return ccs.hits_to_numpy(hits)


def same(a, b, what):
    for k in ("t", "u", "v", "pid"):
        assert np.array_equal(a[k], b[k]), (what, k)


@pytest.mark.parametrize("local", [False, True])
def test_image_order_keeps_every_hit(local):
    s = sg.config_scene(2)
    r = sg.pinhole_rays(1920, 1080)
    sc = ccs.Scene(s.P, s.types, local=local)
    ref = run(sc, r)
    assert (ref["pid"] != MISS).mean() > 0.1
    for kw in (dict(order=True, image_width=1920), dict(order=True), dict(order=True, image_width=1920, vote=16,
                                                                           block_threads=96, lanes_per_ray=3)):
        same(run(sc, r, **kw), ref, kw)
    sc.close()


@pytest.mark.parametrize("w,n", [(333, 333 * 77 + 100), (37, 37 * 5), (1, 1000), (4096, 5000), (64, 63), (1 << 30, 1000)])
def test_ragged_images_and_tiny_batches(w, n):
    """Widths not a multiple of the tile, a partial last row, one-pixel-wide images, fewer rays than one
    row or one tile, and a width far beyond the batch (one partial row)."""
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(n, seed=w + n, target=1.0)
    sc = ccs.Scene(s.P, s.types, local=True)
    ref = run(sc, r)
    same(run(sc, r, order=True, image_width=w), ref, ("image", w, n))
    same(run(sc, r, order=True), ref, ("runs", n))
    sc.close()


def test_order_on_diffuse_batch_and_single_patch_scene():
    s = sg.config_scene(2)
    cam = sg.pinhole_rays(480, 270)
    sc = ccs.Scene(s.P, s.types, local=True)
    rays = ccs.rays_to_device(cam.soa())
    hits = ccs.intersect(sc, rays, ccs.make_opts())
    planes = ccs.gen_diffuse(sc, rays, hits, seed=3)
    torch.cuda.synchronize()
    act = (planes[7] >= planes[6]).nonzero().squeeze(1)
    diff = sg.Rays(*[torch.stack([planes[k].index_select(0, act) for k in range(a, a + 3)], 1).cpu().numpy()
                     for a in (0, 3)], planes[6].index_select(0, act).cpu().numpy(),
                   planes[7].index_select(0, act).cpu().numpy())
    same(run(sc, diff, order=True), run(sc, diff), "diffuse")
    sc.close()
    one = ccs.Scene(s.P[:1], s.types[:1])
    r = sg.random_rays(3000, seed=5, radius=2.0)
    same(run(one, r, order=True), run(one, r), "one patch")
    one.close()


def test_order_through_host_path_and_any_hit():
    s = sg.config_scene(2)
    r = sg.pinhole_rays(1920, 1080).subset(np.arange(1920 * 1000 + 17))   # two chunks on tile rows, partial last row
    sc = ccs.Scene(s.P, s.types, local=True)
    ref = run(sc, r)
    planes = [np.ascontiguousarray(a) for a in r.soa()]
    out = [np.full(r.n, -7, np.float32) for _ in range(3)] + [np.zeros(r.n, np.uint32)]
    for opts in (ccs.make_opts(order=True, image_width=1920), ccs.make_opts(order=True)):
        ccs.ccs_intersect_host(sc.handle, [a.ctypes.data for a in planes], r.n, [a.ctypes.data for a in out], opts)
        got = dict(t=out[0], u=out[1], v=out[2], pid=out[3])
        same(got, ref, "host")
    occ_ref = ccs.occluded(sc, ccs.rays_to_device(r.soa()))
    occ = ccs.occluded(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(order=True, image_width=1920))
    torch.cuda.synchronize()
    assert torch.equal(occ, occ_ref)
    assert np.array_equal(occ.cpu().numpy().astype(bool), ref["pid"] != MISS)
    sc.close()


def test_autotuner_keeps_image_width_and_may_choose_order():
    s = sg.config_scene(2)
    r = sg.pinhole_rays(640, 360)
    sc = ccs.Scene(s.P, s.types, local=True)
    rays = ccs.rays_to_device(r.soa())
    hits = ccs.alloc_hits(r.n)
    best, ms, trials = ccs.ccs_autotune(sc.handle, rays, r.n, hits, ccs.make_opts(image_width=640), reps=1)
    assert best.image_width == 640 and ms > 0
    assert any(o.flags & ccs.CCS_TRACE_ORDER for o, _ in trials)
    same(run(sc, r, **ccs.opts_dict(best)), run(sc, r), "tuned")
    sc.close()
