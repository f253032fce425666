"""Screen-space termination (Sec. 3.3, pixel_spread > 0) through the C ABI: parity with the FP64 oracle
under the same rule, the exact relations to the fixed-depth answer of the same kernel, less work, and
hits independent of the launch options."""
import numpy as np
import pytest

import oracle
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
    oracle.build()
    torch.cuda.set_device(0)


def pixel(height, fov_deg=60.0):
    return 2.0 * np.tan(np.radians(fov_deg) / 2) / height


def run(sc, r, counters=False, **kw):
    cnt = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device="cuda") if counters else None
    hits = ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(counters=cnt, **kw))
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    g = ccs.hits_to_numpy(hits)
    return (g, dict(zip(ccs.COUNTER_NAMES, cnt.cpu().tolist()))) if counters else g


def compare_screen(g, o, rel_t=1e-4, max_flagged=0.03):
    """Unflagged rays: same hit/miss and patch, t within rel_t, u and v within the extent of the oracle's
    leaf node (a neighbouring level differs from it by at most half of it)."""
    ok = o["flags"] == 0
    gh, oh = g["pid"] != MISS, o["pid"] != MISS
    assert (ok & (gh != oh)).sum() == 0
    both = ok & gh & oh
    assert (g["pid"][both] != o["pid"][both]).sum() == 0
    t = o["t"][both]
    assert (np.abs(g["t"][both] - t) <= rel_t * np.abs(t)).all()
    lev = o["level"][both].astype(np.int64)
    eu, ev = 2.0 ** -((lev + 1) // 2), 2.0 ** -(lev // 2)
    assert (np.abs(g["u"][both] - o["u"][both]) <= eu * (1 + 1e-6)).all()
    assert (np.abs(g["v"][both] - o["v"][both]) <= ev * (1 + 1e-6)).all()
    assert (~ok).mean() <= max_flagged, (~ok).mean()
    return int(both.sum())


@pytest.mark.parametrize("which", ["cfg1_64", "cfg2_320x180", "gregory_random"])
def test_screen_space_matches_oracle(which):
    if which == "cfg1_64":
        s, r, sp = sg.config_scene(1), sg.pinhole_rays(64, 64), pixel(64)
    elif which == "cfg2_320x180":
        s, r, sp = sg.config_scene(2), sg.pinhole_rays(320, 180), pixel(180)
    else:
        s, r, sp = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True), sg.random_rays(20000, seed=13), 3e-3
    sc = ccs.Scene(s.P, s.types)
    g = run(sc, r, pixel_spread=sp)
    o = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True, spread=sp)
    n = compare_screen(g, o)
    assert n > 500
    assert (o["level"][o["pid"] != MISS] < 16).mean() > 0.5   # the rule does terminate early here
    sc.close()


def test_screen_space_coarsens_the_fixed_depth_answer_exactly():
    s = sg.config_scene(2)
    r = sg.pinhole_rays(480, 270)
    sc = ccs.Scene(s.P, s.types)
    fixed, cf = run(sc, r, counters=True)
    ss, cs = run(sc, r, counters=True, pixel_spread=pixel(270))
    fh, sh = fixed["pid"] != MISS, ss["pid"] != MISS
    assert (sh | ~fh).all()                                   # a fixed-depth hit stays a hit
    both = fh & sh
    assert (ss["t"][both] <= fixed["t"][both]).all()          # an ancestor box is entered no later
    assert cs["bezier_splits"] + cs["gregory_splits"] < 0.8 * (cf["bezier_splits"] + cf["gregory_splits"])
    # a spread of zero is the fixed-depth kernel
    z = run(sc, r, pixel_spread=0.0)
    for k in ("t", "u", "v", "pid"):
        assert np.array_equal(z[k], fixed[k])
    sc.close()


def test_screen_space_hits_do_not_depend_on_launch_options():
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    r = sg.random_rays(30000, seed=23)
    sc = ccs.Scene(s.P, s.types)
    ref = run(sc, r, pixel_spread=2e-3)
    for kw in [dict(block_threads=32), dict(cache_slots=0, refill=1), dict(vote=16, bvh_burst=2), dict(chunk=1024),
               dict(lanes_per_ray=3)]:
        g = run(sc, r, pixel_spread=2e-3, **kw)
        for k in ("t", "u", "v", "pid"):
            assert np.array_equal(g[k], ref[k]), (kw, k)
    sc.close()


def test_pixel_spread_is_validated():
    s = sg.config_scene(1)
    sc = ccs.Scene(s.P, s.types)
    r = sg.pinhole_rays(4, 4)
    for bad in (-1e-3, 2.0, float("nan")):
        with pytest.raises(ccs.CcsError):
            ccs.intersect(sc, ccs.rays_to_device(r.soa()), ccs.make_opts(pixel_spread=bad))
    sc.close()
