"""Shadow rays and the any-hit query of the oracle, pinned to geometry and to brute force."""
import numpy as np

import oracle
from oracle.raygen import shadow_rays
from paper_1811_03510_gb300 import scenegen as sg

MISS = 0xFFFFFFFF


def test_shadow_rays_reach_the_light_from_the_offset_surface_point():
    s = sg.config_scene(1)
    cam = sg.pinhole_rays(48, 48)
    o = oracle.intersect(s.P, s.types, cam.soa(), L=8)
    light = (2.0, 3.0, 4.0)
    r = shadow_rays(s.P, s.types, cam.soa(), o, light, L=8)
    act = r[7] >= r[6]
    hit = o["pid"] != MISS
    assert act.sum() > 200 and not act[~hit].any()
    org = np.stack(r[:3], 1).astype(np.float64)
    d = np.stack(r[3:6], 1).astype(np.float64)
    # unit directions that end at the light after tmax
    assert np.allclose(np.linalg.norm(d[act], axis=1), 1.0, atol=1e-6)
    end = org[act] + r[7][act, None].astype(np.float64) * d[act]
    assert np.allclose(end, np.array(light)[None], atol=1e-5)
    # the origin sits off the surface point of the hit cell, on the side of the incoming ray
    for i in np.nonzero(act)[0][:50]:
        f, fu, fv = oracle.patch_frame(s.P[o["pid"][i]].astype(float), bool(s.types[o["pid"][i]]), float(o["u"][i]),
                                       float(o["v"][i]))
        nrm = np.cross(fu, fv)
        nrm /= np.linalg.norm(nrm)
        if nrm @ cam.d[i] > 0:
            nrm = -nrm
        off = org[i] - f
        assert np.linalg.norm(np.cross(off, nrm)) < 1e-5 * max(1.0, np.linalg.norm(off))   # along the normal
        assert off @ nrm > 0
        assert (np.array(light) - org[i]) @ nrm > 0   # lit side only
    # slots whose light is behind the surface get no ray: with the light inside the sphere, none is lit
    r_in = shadow_rays(s.P, s.types, cam.soa(), o, (0.0, 0.0, 0.0), L=8)
    assert not (r_in[7] >= r_in[6]).any()


def test_occluded_is_brute_force_any_leaf():
    """On a few patches and rays, occluded == some patch has a leaf hit by exhaustive leaf enumeration."""
    s = sg.config_scene(1)
    sel = [0, 5, 40, 41]
    P, T = s.P[sel], s.types[sel]
    rng = np.random.default_rng(3)
    c = P.reshape(-1, 3).mean(0)
    n = 120
    org = c + rng.normal(size=(n, 3)) * 2.0
    tgt = P[rng.integers(0, len(sel), n)].mean(1) + 0.2 * rng.normal(size=(n, 3))
    d = (tgt - org).astype(np.float32)
    tmax = np.where(rng.random(n) < 0.3, 0.5, np.inf).astype(np.float32)   # some rays end short of the patches
    rays = [org[:, 0].astype(np.float32), org[:, 1].astype(np.float32), org[:, 2].astype(np.float32),
            d[:, 0], d[:, 1], d[:, 2], np.zeros(n, np.float32), tmax]
    occ = oracle.occluded(P, T, rays, L=3)["occluded"]
    brute = np.zeros(n, np.uint8)
    for i in range(n):
        ray8 = np.array([r[i] for r in rays], dtype=np.float64)
        for k in range(len(sel)):
            if oracle.intersect_patch(P[k].astype(np.float64), bool(T[k]), ray8, 3, brute=True)[0]:
                brute[i] = 1
                break
    assert np.array_equal(occ, brute)
    assert 10 < occ.sum() < n - 10
