"""Pins of the oracle's secondary-ray generator (oracle/raygen.py) against its published definitions:
PCG32's published first outputs, the cosine-weighted hemisphere (mean cosine 2/3, unit directions on the
side the ray came from), the law of reflection, and the offset of the origin along the normal by
offset_abs + 2 * 2^-L * L1(patch box diagonal).  CPU only."""
import numpy as np

import oracle
from oracle import raygen

MISS = 0xFFFFFFFF


def rotation(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def flat_scene(Q=np.eye(3)):
    """One Bezier patch: the square [-1, 1]^2 of the plane z = 0 (u along x, v along y), rotated by Q."""
    g = np.zeros((20, 3), np.float32)
    for j in range(4):
        for i in range(4):
            g[4 * j + i] = Q @ np.array([2 * i / 3 - 1, 2 * j / 3 - 1, 0.0])
    g[16:] = g[[5, 6, 9, 10]]
    return g[None], np.zeros(1, np.uint8)


def head_on_rays(n, seed, from_below=False, Q=np.eye(3)):
    """Rays along the square's normal (-z in its frame, +z from below) onto random points of it."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-0.9, 0.9, size=(n, 2))
    z0, dz = (-3.0, 1.0) if from_below else (3.0, -1.0)
    o = np.stack([xy[:, 0], xy[:, 1], np.full(n, z0)], 1) @ Q.T
    d = np.tile(Q @ np.array([0.0, 0.0, dz]), (n, 1))
    planes = [*o.T, *d.T, np.zeros(n), np.full(n, np.inf)]
    return [np.ascontiguousarray(p, np.float32) for p in planes]


def test_pcg32_published_first_outputs():
    """pcg32_srandom_r(42, 54) then two pcg32_random_r calls: the reference demo's first two outputs."""
    assert raygen.pcg32_pair(42, 54) == (0xA15C02B7, 0x7B47F409)


def test_diffuse_directions_are_cosine_weighted_on_the_incoming_side():
    """Head-on rays onto a flat square, in its own axes and tilted (a general normal exercises the whole
    tangent basis): unit directions on the incoming side with the moments of the cosine-weighted
    hemisphere, and no preferred tangent direction."""
    for Q in (np.eye(3), rotation([1.0, 2.0, 0.5], 1.1)):
        P, T = flat_scene(Q)
        for from_below in (False, True):
            rays = head_on_rays(6000, 3 + from_below, from_below, Q)
            hits = oracle.intersect(P, T, rays, L=8)
            assert (hits["pid"] == 0).all()
            sec = raygen.diffuse_rays(P, T, rays, hits, seed=9, L=8)
            d = np.stack(sec[3:6], 1).astype(np.float64) @ Q      # in the square's frame
            np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
            cos = d[:, 2] * (-1.0 if from_below else 1.0)         # the normal faces the incoming ray
            assert cos.min() >= -1e-6
            # cosine-weighted hemisphere: E[cos] = 2/3, E[cos^2] = 1/2, tangent components average to zero
            assert abs(cos.mean() - 2 / 3) < 0.01 and abs((cos ** 2).mean() - 0.5) < 0.01
            assert abs(d[:, 0].mean()) < 0.02 and abs(d[:, 1].mean()) < 0.02
            assert abs((d[:, 0] ** 2).mean() - 0.25) < 0.01 and abs((d[:, 1] ** 2).mean() - 0.25) < 0.01
            assert (sec[6] == 0).all() and np.isinf(sec[7]).all()


def test_origin_offset_along_the_normal():
    """Flat patch hit head-on: the surface point of the cell centre moved along the normal by
    offset_abs + 2 * 2^-L * L1(box diagonal); the square's box diagonal has L1 length 4."""
    P, T = flat_scene()
    L, off_abs = 6, 1e-3
    for from_below in (False, True):
        rays = head_on_rays(200, 5, from_below)
        hits = oracle.intersect(P, T, rays, L=L)
        for mirror in (False, True):
            sec = raygen.diffuse_rays(P, T, rays, hits, seed=1, L=L, offset_abs=off_abs, mirror=mirror)
            off = off_abs + 2.0 * 2.0 ** -L * 4.0
            np.testing.assert_allclose(sec[2], -off if from_below else off, rtol=1e-6)
            np.testing.assert_allclose(sec[0], 2.0 * hits["u"].astype(np.float64) - 1.0, atol=1e-6)
            np.testing.assert_allclose(sec[1], 2.0 * hits["v"].astype(np.float64) - 1.0, atol=1e-6)


def test_mirror_directions_obey_the_law_of_reflection():
    P, T = flat_scene()
    rng = np.random.default_rng(8)
    n = 300
    o = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5, 0.5, n), np.full(n, 2.0)], 1)
    d = np.stack([rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, n), -np.ones(n)], 1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = [np.ascontiguousarray(a, np.float32) for a in (*o.T, *d.T, np.zeros(n), np.full(n, np.inf))]
    hits = oracle.intersect(P, T, rays, L=8)
    assert (hits["pid"] == 0).all()
    sec = raygen.diffuse_rays(P, T, rays, hits, seed=1, L=8, mirror=True)
    r = np.stack(sec[3:6], 1).astype(np.float64)
    din = np.stack(rays[3:6], 1).astype(np.float64)
    np.testing.assert_allclose(r[:, :2], din[:, :2], atol=1e-7)      # tangent part kept
    np.testing.assert_allclose(r[:, 2], -din[:, 2], atol=1e-7)       # normal part reversed


def test_slots_without_a_hit_are_empty_rays():
    P, T = flat_scene()
    rays = head_on_rays(50, 2)
    rays[0] = rays[0] + np.float32(5.0)                              # every ray misses the square
    hits = oracle.intersect(P, T, rays, L=6)
    assert (hits["pid"] == MISS).all()
    for sec in (raygen.diffuse_rays(P, T, rays, hits, seed=1, L=6),
                raygen.shadow_rays(P, T, rays, hits, [0.0, 0.0, 5.0], L=6)):
        assert (sec[6] == 1).all() and (sec[7] == 0).all()
