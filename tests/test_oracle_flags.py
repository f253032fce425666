"""Pins of the oracle's parity flags (the FP32 error model that excludes rays whose answer FP32 cannot be
expected to reproduce): each bit is set on a ray built to need it and clear on rays well away from every
such case.  bit0 another patch may win, bit1 a far cell of the hit patch may win, bit2 hit/miss may flip,
bit3 t may leave the relative tolerance.  CPU only."""
import numpy as np

import oracle
from paper_1811_03510_gb300 import scenegen as sg

MISS = 0xFFFFFFFF


def plane_patch(xs, ys):
    """Affine patch of the plane z = 0 with control-point columns xs (along u) and rows ys (along v)."""
    g = np.zeros((20, 3), np.float32)
    for j in range(4):
        for i in range(4):
            g[4 * j + i] = (xs[i], ys[j], 0.0)
    g[16:] = g[[5, 6, 9, 10]]
    return g


YS = (-1.5, -0.5, 0.5, 1.5)
LEFT = plane_patch((-1.5, -1.0, -0.5, 0.0), YS)     # x in [-1.5, 0]
RIGHT = plane_patch((0.0, 0.5, 1.0, 1.5), YS)       # x in [0, 1.5]: shares the edge x = 0


def trace(P, xy, d=(0.0, 0.0, -1.0), z0=2.0, L=8):
    xy = np.asarray(xy, float)
    n = len(xy)
    planes = [xy[:, 0], xy[:, 1], np.full(n, z0), np.full(n, d[0]), np.full(n, d[1]), np.full(n, d[2]),
              np.zeros(n), np.full(n, np.inf)]
    planes = [np.ascontiguousarray(p, np.float32) for p in planes]
    return oracle.intersect(np.stack(P), np.zeros(len(P), np.uint8), planes, L=L, flags=True)


def test_rays_well_inside_one_patch_are_not_flagged():
    """Away from patch edges and from leaf-cell boundaries (on a boundary shared by two cells both boxes
    may shrink in FP32, and the model flags that too)."""
    o = trace([LEFT, RIGHT], [(-0.7, 0.3), (0.77, -0.2), (-1.1, 0.9), (0.3, 0.1)])
    assert (o["pid"] == [0, 1, 0, 1]).all() and (o["flags"] == 0).all()
    edge = trace([LEFT], [(-0.75, 0.3)])                  # u = 1/2, a cell boundary
    assert edge["pid"][0] == 0 and edge["flags"][0] & 4
    assert edge["flags"][0] & 2 == 0                        # the two cells are neighbours, not far apart


def test_shared_edge_flags_another_patch():
    """On the shared edge x = 0 both patches are entered at the same distance; a ray within the box
    error of the edge could go to either patch in FP32."""
    o = trace([LEFT, RIGHT], [(0.0, 0.3), (1e-7, 0.3), (-1e-7, -0.4)])
    assert (o["pid"] != MISS).all()
    assert (o["flags"] & 1).all()
    far = trace([LEFT, RIGHT], [(1e-3, 0.3), (-1e-3, -0.4)])
    assert (far["flags"] & 1 == 0).all()


def test_outline_flags_hit_or_miss():
    """On the outer edge x = 1.5 of a lone patch (and just outside it, within the box error) the ray may
    hit or miss in FP32; clearly outside it is an unflagged miss."""
    o = trace([RIGHT], [(1.5, 0.2), (1.5 + 2e-7, 0.2), (1.5 + 1e-3, 0.2)])
    assert o["pid"][0] == 0 and o["pid"][2] == MISS
    assert o["flags"][0] & 4 and o["flags"][1] & 4 and o["flags"][2] == 0


def test_folded_patch_flags_a_far_cell():
    """x(u) = 3u(1-u) (control columns 0, 1, 1, 0) folds the patch onto itself: the points u and 1 - u
    coincide, so a ray along -z enters two cells far apart at the same distance."""
    fold = plane_patch((0.0, 1.0, 1.0, 0.0), YS)
    x = 3 * 0.25 * 0.75 + 1e-4
    o = trace([fold], [(x, 0.2)])
    assert o["pid"][0] == 0 and o["flags"][0] & 2
    flat = trace([RIGHT], [(0.3 + 1e-4, 0.2)])
    assert flat["flags"][0] & 2 == 0


def test_grazing_ray_flags_its_distance():
    """A ray at a grazing angle enters the (error-inflated) leaf boxes much earlier than the exact one:
    its distance cannot be held to the relative tolerance."""
    d = np.array([1.0, 0.0, -2e-4])
    d /= np.linalg.norm(d)
    o = trace([RIGHT], [(-0.5, 0.2)], d=tuple(d), z0=2e-4)       # reaches z = 0 at x = 0.5
    assert o["pid"][0] == 0 and o["flags"][0] & 8
    steep = trace([RIGHT], [(0.5, 0.2)])
    assert steep["flags"][0] & 8 == 0


def test_flagged_rays_are_few_on_the_cube_sphere():
    """The flags exclude a small share of an image: silhouette and seam rays, not the bulk."""
    s = sg.config_scene(1)
    r = sg.pinhole_rays(64, 64)
    o = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True)
    hit = o["pid"] != MISS
    assert hit.sum() > 500 and (o["flags"] != 0).sum() <= 0.01 * r.n
