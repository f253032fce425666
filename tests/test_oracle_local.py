"""Local frames (Sec. 3.4) in the oracle: below the patch root, boxes are taken in each patch's own frame.
Pinned to closed forms (the frame of a plane, the exact distance to a tilted flat patch), to brute force,
and to watertightness at the shared boundaries of the closed cube-sphere."""
import numpy as np
import pytest

import oracle
from paper_1811_03510_gb300 import scenegen as sg

MISS = 0xFFFFFFFF
RNG = np.random.default_rng(2024)


def rotation(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def flat_square(a, Q=np.eye(3), c=np.zeros(3)):
    """Degree-elevated affine patch: the square [-a/2, a/2]^2 of the plane z = 0 (u along x, v along y),
    rotated by Q and moved to c."""
    g = np.zeros((20, 3))
    for j in range(4):
        for i in range(4):
            g[4 * j + i] = Q @ np.array([a * (i / 3 - 0.5), a * (j / 3 - 0.5), 0.0]) + c
    g[16:20] = g[[5, 6, 9, 10]]
    return g


def test_frame_of_a_plane_is_its_tangent_frame():
    Q = rotation([1.0, 2.0, 0.5], 0.7)
    R = oracle.local_frame(flat_square(1.0, Q, np.array([0.3, -0.2, 1.0])))
    # rows: u direction, v direction, normal of the plane (the columns of Q)
    np.testing.assert_allclose(R, Q.T, atol=1e-12)
    np.testing.assert_allclose(oracle.local_frame(flat_square(2.0)), np.eye(3), atol=1e-12)


@pytest.mark.parametrize("L", [4, 8, 12])
def test_tilted_flat_patch_is_hit_at_the_plane_distance(L):
    """In its own frame a flat patch has boxes of zero thickness, widened to the box-extension thickness
    tau = 2^-19 (1 + L1 distance of the origin from the patch's box centre): the leaf is entered tau / 2
    before the plane along its normal.  In world axes the tilted leaf boxes are entered earlier."""
    Q = rotation([1.0, 0.3, 0.0], np.pi / 4)
    c = np.array([0.1, -0.2, 0.3])
    g = flat_square(1.0, Q, c)
    centre = 0.5 * (g[:16].min(0) + g[:16].max(0))
    nrm = Q[:, 2]
    for k in range(30):
        x, y = RNG.uniform(-0.45, 0.45, 2)
        target = Q @ np.array([x, y, 0.0]) + c
        o = target + 3.0 * (nrm + 0.3 * RNG.normal(size=3))
        d = target - o
        ray = np.array([*o, *d, 0.0, np.inf])
        t_plane = ((c - o) @ nrm) / (d @ nrm)
        tau = 2.0 ** -19 * (1.0 + np.abs(o - centre).sum())
        t_exp = t_plane - 0.5 * tau / abs(d @ nrm)
        hit, t, _, _ = oracle.intersect_patch(g, False, ray, L, local=True)
        assert hit and abs(t - t_exp) <= 1e-12 * abs(t_plane)
        hw, tw, _, _ = oracle.intersect_patch(g, False, ray, L, local=False)
        assert hw and tw < t_exp - 1e-9


@pytest.mark.parametrize("greg", [False, True])
@pytest.mark.parametrize("spread", [0.0, 3e-2])
def test_pruned_search_equals_brute_force_in_local_frames(greg, spread):
    s = sg.config_scene(1)
    p = int(np.nonzero(s.types == (1 if greg else 0))[0][0])
    g = s.P[p].astype(np.float64)
    c = g.mean(0)
    n_hit = 0
    for k in range(120):
        o = c + RNG.normal(size=3) * 1.5
        f = oracle.patch_frame(g, greg, *RNG.uniform(0.02, 0.98, 2))[0]
        d = f + 0.01 * RNG.normal(size=3) - o
        ray = np.array([*o, *d, 0.0, np.inf])
        a = oracle.intersect_patch(g, greg, ray, 4, spread=spread, with_level=True, local=True)
        b = oracle.intersect_patch(g, greg, ray, 4, brute=True, spread=spread, with_level=True, local=True)
        assert a[0] == b[0]
        if a[0]:
            n_hit += 1
            assert a[1] == b[1] and a[2] == b[2] and a[4] == b[4], (k, a, b)
    assert n_hit > 40


def test_local_frames_keep_shared_boundaries_watertight():
    """Rays through points on shared patch boundaries of the closed cube-sphere always hit in local
    frames too (Sec. 3.4: false positives only)."""
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
    n = len(targets)
    rays = [np.ascontiguousarray(a, dtype=np.float32)
            for a in (o[:, 0], o[:, 1], o[:, 2], d[:, 0], d[:, 1], d[:, 2], np.zeros(n), np.full(n, np.inf))]
    out = oracle.intersect(s.P, s.types, rays, L=8, local=True)
    assert (out["pid"] != MISS).all()


def test_local_frames_agree_with_world_frames_away_from_edges():
    """Both frames bound the same surface with boxes around each leaf cell, so away from patch edges they
    report the same patch, at distances a few leaf-box sizes apart (divided by the sine of the angle
    between ray and surface, which lets the rare grazing ray differ by more)."""
    s = sg.config_scene(2)
    r = sg.pinhole_rays(160, 90)
    w = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True)
    l = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True, local=True)
    both = (w["pid"] != MISS) & (l["pid"] != MISS) & (w["flags"] == 0) & (l["flags"] == 0)
    assert both.sum() > 2000
    same = both & (w["pid"] == l["pid"])
    assert same.mean() / both.mean() > 0.97
    dt = np.abs(l["t"][same] - w["t"][same])
    assert np.percentile(dt, 99.5) < 1e-2 and dt.max() < 3e-2 and np.median(dt) < 1e-3


def test_frame_of_a_curved_patch_is_a_rotation():
    """The frame of a curved patch: orthonormal rows with determinant +1, z along the normal of the
    corner quad (the cross product of the diagonals p33 - p00 and p03 - p30), x in the plane of z and the
    u edge p30 - p00 on that edge's side (so y is orthogonal to the edge)."""
    for _ in range(40):
        g = RNG.normal(size=(20, 3))
        R = oracle.local_frame(g)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
        n = np.cross(g[15] - g[0], g[12] - g[3])
        np.testing.assert_allclose(R[2], n / np.linalg.norm(n), atol=1e-12)
        e = g[3] - g[0]
        assert abs(R[1] @ e) <= 1e-12 * np.linalg.norm(e) and R[0] @ e > 0


def _f32_fma(a, b, c):
    """FP32 fused multiply-add: a*b is exact in FP64 for FP32 inputs, one rounding of the sum to FP32."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum(a, b):
    """Knuth's TwoSum in FP32: a + b = s + err exactly."""
    a, b = np.float32(a), np.float32(b)
    s = np.float32(a + b)
    bb = np.float32(s - a)
    return s, np.float32(np.float32(a - np.float32(s - bb)) + np.float32(b - bb))


def _two_prod(a, b):
    """TwoProduct in FP32: a b = p + err exactly (the error of a product of two floats is a float)."""
    a, b = np.float32(a), np.float32(b)
    p = np.float32(a * b)
    return p, np.float32(np.float64(a) * np.float64(b) - np.float64(p))


def _anchored_coord(o, a, t, d):
    """(o - a) + t d as an unevaluated FP32 sum h + l, as the kernels form it."""
    sh, sl = _two_sum(o, -np.float32(a))
    ph, pl = _two_prod(t, d)
    hh, hl = _two_sum(sh, ph)
    return hh, np.float32(hl + np.float32(sl + pl))


def _rotate_coord(Rk, e):
    """Compensated dot product (Ogita, Rump and Oishi 2005, Dot2) of a frame row with e = h + l, one
    final rounding, as the kernels form it."""
    p = [_two_prod(Rk[j], e[j][0]) for j in range(3)]
    s1 = _two_sum(p[0][0], p[1][0])
    s2 = _two_sum(s1[0], p[2][0])
    c = np.float32(np.float32(p[0][1] + p[1][1]) + np.float32(s1[1] + np.float32(s2[1] + p[2][1])))
    c = _f32_fma(Rk[0], e[0][1], _f32_fma(Rk[1], e[1][1], _f32_fma(Rk[2], e[2][1], c)))
    return np.float32(s2[0] + c)


def test_anchored_ray_error_is_within_the_flag_model():
    """The FP32 path intersects a pair with the ray anchored at its entry into the patch box: origin
    e = (o - anchor) + te d formed by error-free FP32 transformations (TwoSum, TwoProduct), rotated into the
    patch frame by a compensated dot product (Dot2) and rounded once, direction R d in FP32; emulated here
    operation by operation.  Over the patch box that ray stays within 3e-7 (|e| + box diagonal) of the exact ray in the same
    frame, whatever the distance from the ray's own origin (here 3 and 300 scene units): the term the
    oracle's parity flags add to eps.  The FP32 transform without the anchor misses that bound by far."""
    s = sg.config_scene(2)
    P = s.P.astype(np.float32)
    worst, worst_plain = 0.0, 0.0
    for k, p in enumerate(RNG.choice(s.n, 300, replace=False)):
        g = P[p]
        pts = g[:20] if s.types[p] else g[:16]
        lo, hi = pts.min(0), pts.max(0)
        an = ((lo + hi).astype(np.float32) * np.float32(0.5)).astype(np.float32)
        R = oracle.local_frame(g.astype(np.float64)).astype(np.float32)
        target = (lo + (hi - lo) * RNG.uniform(0.2, 0.8, 3)).astype(np.float64)
        for dist in (3.0, 300.0):
            u = RNG.normal(size=3)
            u /= np.linalg.norm(u)
            o = (target + dist * u).astype(np.float32)
            d = (-u).astype(np.float32)
            te = np.float32(dist - np.linalg.norm(hi - lo))
            e = np.float64(te) * d.astype(np.float64) + (o.astype(np.float64) - an.astype(np.float64))
            ef = [_anchored_coord(o[c], an[c], te, d[c]) for c in range(3)]
            org = np.array([_rotate_coord(R[i], ef) for i in range(3)], np.float32)
            dl = np.array([_f32_fma(R[i, 0], d[0], _f32_fma(R[i, 1], d[1], np.float32(R[i, 2] * d[2])))
                           for i in range(3)], np.float32)
            # the exact ray in the same (rounded) frame, and the unanchored FP32 transform for comparison
            ex_o = R.astype(np.float64) @ (o.astype(np.float64) - an.astype(np.float64))
            ex_d = R.astype(np.float64) @ d.astype(np.float64)
            o3 = (o - an).astype(np.float32)
            plain = np.array([_f32_fma(R[i, 0], o3[0], _f32_fma(R[i, 1], o3[1], np.float32(R[i, 2] * o3[2])))
                              for i in range(3)], np.float32)
            diag = float(np.linalg.norm((hi - lo).astype(np.float64)))
            bound = 3e-7 * (float(np.linalg.norm(e)) + diag)
            for tp in (0.0, diag, 2.0 * diag):
                exact = ex_o + (float(te) + tp) * ex_d
                worst = max(worst, float(np.linalg.norm(org + tp * dl.astype(np.float64) - exact)) / bound)
                worst_plain = max(worst_plain, float(np.linalg.norm(plain + (float(te) + tp) * dl.astype(np.float64)
                                                                    - exact)) / bound)
    assert worst < 1.0, worst
    assert worst_plain > 10.0, worst_plain
