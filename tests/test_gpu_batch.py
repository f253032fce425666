"""Batched scenes through the C ABI: one persistent launch over many scenes' rays, batched update and
refit, CUDA-graph capture.  Hits must be bit-identical to per-scene launches, and agree with the oracle."""
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


def planes_of(P):
    return [torch.from_numpy(np.ascontiguousarray(P[..., c]).reshape(-1)).cuda() for c in range(3)]


@pytest.fixture(scope="module")
def batch_inputs():
    scenes = [sg.make_scene(n, 0.02 * (k % 3), 3, k + 1, gregory_ring=(k == 2)) for k, n in enumerate([2, 3, 5, 8, 4])]
    rays = [sg.pinhole_rays(96, 64), sg.random_rays(5000, seed=1), sg.pinhole_rays(1, 1), sg.random_rays(7000, seed=2),
            sg.pinhole_rays(80, 80)]
    rays[2] = sg.Rays(rays[2].o[:0], rays[2].d[:0], rays[2].tmin[:0], rays[2].tmax[:0])   # a scene without rays
    return scenes, rays


def per_scene(scenes, rays, opts=None):
    out = []
    for s, r in zip(scenes, rays):
        sc = ccs.Scene(s.P, s.types)
        if r.n:
            h = ccs.intersect(sc, ccs.rays_to_device(r.soa()), opts or ccs.make_opts())
            torch.cuda.synchronize()
            out.append(ccs.hits_to_numpy(h))
        else:
            out.append(None)
        sc.close()
    return out


def test_batched_launch_equals_per_scene_launches(batch_inputs):
    scenes, rays = batch_inputs
    ref = per_scene(scenes, rays)
    handles = [ccs.Scene(s.P, s.types) for s in scenes]
    rdev = [ccs.rays_to_device(r.soa()) if r.n else ccs.rays_to_device(sg.pinhole_rays(1, 1).soa()) for r in rays]
    hits = [ccs.alloc_hits(max(r.n, 1)) for r in rays]
    b = ccs.ccs_batch_create(handles, rdev, hits, n_rays=[r.n for r in rays])
    ccs.ccs_batch_run(b, ccs.CCS_BATCH_INTERSECT, ccs.make_opts())
    assert ccs.ccs_batch_sync_status(b) == ccs.CCS_OK
    for k, r in enumerate(rays):
        if not r.n:
            continue
        g = ccs.hits_to_numpy(hits[k])
        for key in ("t", "u", "v", "pid"):
            assert np.array_equal(g[key][:r.n], ref[k][key]), (k, key)
    ccs.ccs_batch_destroy(b)
    for h in handles:
        h.close()


def test_one_shot_batched_entry(batch_inputs):
    scenes, rays = batch_inputs
    keep = [k for k, r in enumerate(rays) if r.n]
    ref = per_scene([scenes[k] for k in keep], [rays[k] for k in keep])
    handles = [ccs.Scene(scenes[k].P, scenes[k].types) for k in keep]
    rdev = [ccs.rays_to_device(rays[k].soa()) for k in keep]
    hits = [ccs.alloc_hits(rays[k].n) for k in keep]
    ccs.ccs_intersect_batched(handles, rdev, hits, ccs.make_opts(block_threads=64, chunk=64))
    for j, k in enumerate(keep):
        g = ccs.hits_to_numpy(hits[j])
        assert np.array_equal(g["pid"], ref[j]["pid"]) and np.array_equal(g["t"], ref[j]["t"])
    for h in handles:
        h.close()


def test_batched_update_refit_and_graph_replay(batch_inputs):
    """Frames of deformed points: graph(update + refit + intersect) == per-scene fresh builds, every frame."""
    scenes, rays = batch_inputs
    keep = [k for k, r in enumerate(rays) if r.n]
    scenes = [scenes[k] for k in keep]
    rays = [rays[k] for k in keep]
    handles = [ccs.Scene(s.P, s.types) for s in scenes]
    rdev = [ccs.rays_to_device(r.soa()) for r in rays]
    hits = [ccs.alloc_hits(r.n) for r in rays]
    b = ccs.ccs_batch_create(handles, rdev, hits)
    frames = [[planes_of(sg.deform(s.P, f, 4, seed=7 + i)) for i, s in enumerate(scenes)] for f in range(3)]
    stages = ccs.CCS_BATCH_UPDATE | ccs.CCS_BATCH_REFIT | ccs.CCS_BATCH_INTERSECT
    for i in range(len(scenes)):
        ccs.ccs_batch_set_points(b, i, *frames[0][i])
    ccs.ccs_batch_capture(b, stages, ccs.make_opts())
    for f in range(3):
        torch.cuda.synchronize()
        for i in range(len(scenes)):
            ccs.ccs_batch_set_points(b, i, *frames[f][i])
        ccs.ccs_batch_launch(b)
        assert ccs.ccs_batch_sync_status(b) == ccs.CCS_OK
        deformed = [sg.Scene(sg.deform(s.P, f, 4, seed=7 + i), s.types, "d") for i, s in enumerate(scenes)]
        ref = per_scene(deformed, rays)
        for k in range(len(scenes)):
            g = ccs.hits_to_numpy(hits[k])
            for key in ("t", "u", "v", "pid"):
                assert np.array_equal(g[key], ref[k][key]), (f, k, key)
        if f == 2:   # and against the oracle on the last frame of one scene
            o = oracle.intersect(deformed[1].P, deformed[1].types, rays[1].soa(), L=8, flags=True)
            compare(ccs.hits_to_numpy(hits[1]), o, 8)
    ccs.ccs_batch_destroy(b)
    for h in handles:
        h.close()
