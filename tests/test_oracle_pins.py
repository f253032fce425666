"""Pins of the FP64 oracle against things other than itself: closed forms, textbook routines,
invariants the paper states, brute force and the paper's printed constants.  CPU only."""
from fractions import Fraction
import math
import os

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(1234)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers written from textbooks

def bern(t):
    s = 1 - t
    return np.array([s ** 3, 3 * t * s * s, 3 * t * t * s, t ** 3])


def bezier_point(p16, u, v):
    """Tensor-product Bernstein sum, p16[4*j + i] (i along u)."""
    P = np.asarray(p16).reshape(4, 4, 3)  # [j, i]
    return np.einsum("i,j,jic->c", bern(u), bern(v), P)


def decasteljau_curve(b, t):
    """Textbook de Casteljau at t: returns (left, right) control points."""
    b = [np.asarray(x, float) for x in b]
    left, right = [b[0]], [b[-1]]
    while len(b) > 1:
        b = [(1 - t) * b[k] + t * b[k + 1] for k in range(len(b) - 1)]
        left.append(b[0])
        right.append(b[-1])
    return left, right[::-1]


def restrict_curve(b, a, c):
    """Two-sided de Casteljau restriction of a Bezier curve to [a, c]: cut at a, keep the right part,
    then cut that at (c - a) / (1 - a), keep the left part."""
    _, r = decasteljau_curve(b, a)
    s = (c - a) / (1 - a) if a < 1 else 0.0
    l, _ = decasteljau_curve(r, s)
    return l


def restrict_patch(p16, u0, u1, v0, v1):
    P = np.asarray(p16, float).reshape(4, 4, 3)  # [j, i]
    Q = np.empty_like(P)
    for j in range(4):
        Q[j] = np.array(restrict_curve(list(P[j]), u0, u1))
    R = np.empty_like(P)
    for i in range(4):
        R[:, i] = np.array(restrict_curve(list(Q[:, i]), v0, v1))
    return R.reshape(16, 3)


def random_patch(scale=1.0):
    return RNG.normal(size=(16, 3)) * scale


def random_gregory():
    g = np.zeros((20, 3))
    g[:16] = random_patch()
    g[16:] = g[[5, 6, 9, 10]] + RNG.normal(size=(4, 3)) * 0.3
    return g


def random_domain():
    a, b = np.sort(RNG.uniform(0, 1, 2))
    c, d = np.sort(RNG.uniform(0, 1, 2))
    if b - a < 1e-3:
        b = min(1.0, a + 0.1)
    if d - c < 1e-3:
        d = min(1.0, c + 0.1)
    return a, b, c, d


def greg_h(k, u, v):
    """Reading A1 (Algorithm 2's convention): weight of p^u for inner point k = (1,1),(2,1),(1,2),(2,2)."""
    num, den = [(u, u + v), (1 - u, (1 - u) + v), (u, u + (1 - v)), (1 - u, (1 - u) + (1 - v))][k]
    return 0.5 if den == 0 else num / den


# ---------------------------------------------------------------- Bezier evaluation / crop / split

def test_planar_patch_closed_form():
    """Degree-elevated affine grid p_ij = A + (i/3) U + (j/3) V evaluates to A + uU + vV."""
    A, U, V = RNG.normal(size=(3, 3))
    p = np.array([A + (i / 3) * U + (j / 3) * V for j in range(4) for i in range(4)])
    for u, v in RNG.uniform(0, 1, size=(20, 2)):
        f, fu, fv, fuv = oracle.bezier_eval(p, u, v)
        np.testing.assert_allclose(f, A + u * U + v * V, atol=1e-13)
        np.testing.assert_allclose(fu, U, atol=1e-13)
        np.testing.assert_allclose(fv, V, atol=1e-13)
        np.testing.assert_allclose(fuv, 0, atol=1e-13)


def test_bezier_eval_matches_bernstein_sum_and_derivatives():
    p = random_patch()
    for u, v in RNG.uniform(0, 1, size=(20, 2)):
        f, fu, fv, fuv = oracle.bezier_eval(p, u, v)
        np.testing.assert_allclose(f, bezier_point(p, u, v), atol=1e-12)
        h = 1e-6
        np.testing.assert_allclose(fu, (bezier_point(p, u + h, v) - bezier_point(p, u - h, v)) / (2 * h), atol=1e-6)
        np.testing.assert_allclose(fv, (bezier_point(p, u, v + h) - bezier_point(p, u, v - h)) / (2 * h), atol=1e-6)
        fd = (bezier_point(p, u + h, v + h) - bezier_point(p, u + h, v - h) - bezier_point(p, u - h, v + h)
              + bezier_point(p, u - h, v - h)) / (4 * h * h)
        np.testing.assert_allclose(fuv, fd, atol=1e-3)


def test_crop_equals_two_sided_de_casteljau():
    """Sec. 3.1: Algorithm 1 is mathematically equivalent to de Casteljau cutting each side."""
    for _ in range(50):
        p = random_patch()
        D = random_domain()
        np.testing.assert_allclose(oracle.crop(p, *D), restrict_patch(p, *D), rtol=0, atol=1e-12)


def test_crop_of_full_domain_is_identity():
    p = random_patch()
    np.testing.assert_allclose(oracle.crop(p, 0, 1, 0, 1), p, atol=1e-14)


def test_split_is_textbook_de_casteljau_halves():
    p = random_patch()
    for axis in (0, 1):
        L, R = oracle.split(p, axis)
        D = ((0, .5, 0, 1), (.5, 1, 0, 1)) if axis == 0 else ((0, 1, 0, .5), (0, 1, .5, 1))
        np.testing.assert_allclose(L, restrict_patch(p, *D[0]), atol=1e-13)
        np.testing.assert_allclose(R, restrict_patch(p, *D[1]), atol=1e-13)


def test_convex_hull_contains_every_sub_patch():
    """Sec. 3.1: the AABB of the (cropped) control points bounds the (restricted) surface."""
    for _ in range(30):
        p = random_patch()
        D = random_domain()
        q = oracle.crop(p, *D)
        lo, hi = q.min(0), q.max(0)
        for a, b in RNG.uniform(0, 1, size=(200, 2)):
            f = bezier_point(p, D[0] + a * (D[1] - D[0]), D[2] + b * (D[3] - D[2]))
            assert np.all(f >= lo - 1e-12) and np.all(f <= hi + 1e-12)


# ---------------------------------------------------------------- Gregory patches

def test_gregory_with_equal_pairs_is_the_bezier_patch():
    """Sec. 3.2: p^u = p^v makes a Gregory patch a Bezier patch; bound d is exactly zero."""
    p = random_patch()
    g = np.zeros((20, 3))
    g[:16] = p
    g[16:] = p[[5, 6, 9, 10]]
    for u, v in list(RNG.uniform(0, 1, size=(20, 2))) + [(0, 0), (1, 0), (0, 1), (1, 1)]:
        f, _ = oracle.gregory_eval(g, u, v)
        assert np.array_equal(f, oracle.bezier_eval(p, u, v)[0])
    for _ in range(20):
        D = random_domain()
        q, d, lo, hi = oracle.calc_points_and_d(g, True, *D)
        assert np.all(d == 0.0)
        assert np.array_equal(lo, hi)
        np.testing.assert_allclose(q, oracle.crop(p, *D), atol=0)


def test_gregory_inner_points_follow_definition():
    """p_ij(u, v) = h p^u + (1 - h) p^v with h from reading A1; boundary weights reduce to one side."""
    g = random_gregory()
    pu, pv = g[[5, 6, 9, 10]], g[16:]
    for u, v in RNG.uniform(0.01, 0.99, size=(20, 2)):
        _, inner = oracle.gregory_eval(g, u, v)
        for k in range(4):
            h = greg_h(k, u, v)
            np.testing.assert_allclose(inner[k], h * pu[k] + (1 - h) * pv[k], atol=1e-13)
    # at v = 0 the (1,1) and (2,1) points take p^u, at u = 0 the (1,1) and (1,2) points take p^v
    _, inner = oracle.gregory_eval(g, 0.4, 0.0)
    np.testing.assert_allclose(inner[0], pu[0], atol=1e-14)
    np.testing.assert_allclose(inner[1], pu[1], atol=1e-14)
    _, inner = oracle.gregory_eval(g, 0.0, 0.4)
    np.testing.assert_allclose(inner[0], pv[0], atol=1e-14)
    np.testing.assert_allclose(inner[2], pv[2], atol=1e-14)


def test_gregory_inner_point_bounds_hold_on_domain():
    """Sec. 3.2: p^min(D) <= p_ij(u, v) <= p^max(D) for (u, v) in D."""
    for _ in range(30):
        g = random_gregory()
        D = random_domain()
        _, _, lo, hi = oracle.calc_points_and_d(g, True, *D)
        for a, b in RNG.uniform(0, 1, size=(200, 2)):
            u, v = D[0] + a * (D[1] - D[0]), D[2] + b * (D[3] - D[2])
            _, inner = oracle.gregory_eval(g, u, v)
            assert np.all(inner >= lo - 1e-12) and np.all(inner <= hi + 1e-12)


def test_gregory_surface_inside_lower_patch_plus_displacement():
    """Sec. 3.2: the box [min q, max q + d] of Algorithm 2 bounds the Gregory patch restricted to D."""
    for _ in range(40):
        g = random_gregory()
        D = random_domain()
        q, d, _, _ = oracle.calc_points_and_d(g, True, *D)
        assert np.all(d >= 0)
        lo, hi = q.min(0), q.max(0) + d
        for a, b in RNG.uniform(0, 1, size=(300, 2)):
            u, v = D[0] + a * (D[1] - D[0]), D[2] + b * (D[3] - D[2])
            f, _ = oracle.gregory_eval(g, u, v)
            assert np.all(f >= lo - 1e-12) and np.all(f <= hi + 1e-12), (D, f, lo, hi)


def test_gregory_displacement_vanishes_toward_domain_boundary():
    """Sec. 3.2: d(D) is zero in the critical cases where the domain touches u or v = 0 or 1."""
    g = random_gregory()
    for corner in [(0.0, 0.3), (0.3, 0.0), (1.0, 0.6), (0.6, 1.0)]:
        prev = np.inf
        for e in [2.0 ** -k for k in range(2, 20, 2)]:
            u0 = corner[0] - (e if corner[0] == 1.0 else 0.0)
            v0 = corner[1] - (e if corner[1] == 1.0 else 0.0)
            D = (u0, u0 + e, v0, v0 + e) if corner[0] in (0.0, 1.0) else (corner[0], corner[0] + e, v0, v0 + e)
            _, d, _, _ = oracle.calc_points_and_d(g, True, *D)
            m = d.max()
            assert m <= prev + 1e-15
            prev = m
        assert prev < 1e-5


def _frac(s):
    return float(Fraction(s))


def test_bernstein_maxima_golden():
    """Bernstein maxima used by the weight bounds (golden values from Sec. 3.2 / Algorithm 2), read back
    through d(D) of Gregory patches whose only differing pair is one of the four inner pairs."""
    rows = []
    with open(os.path.join(GOLDEN, "bernstein_maxima.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([_frac(x) for x in line.split()])
    base = np.zeros((20, 3))
    for t0, t1, b1, b2 in rows:
        # pair (1,1): d.x = wbar1(u) * wbar1(v over [0,1]) * (h11 range); v over [0,1] gives 4/9
        g = base.copy()
        g[5] = [1.0, 0, 0]
        hs = [greg_h(0, u, v) for u in (t0, t1) for v in (0.0, 1.0)]
        _, d, _, _ = oracle.calc_points_and_d(g, True, t0, t1, 0.0, 1.0)
        assert d[0] == pytest.approx(b1 * (4 / 9) * (max(hs) - min(hs)), rel=1e-12)
        # pair (2,1): d.x = wbar2(u) * wbar1(v)
        g = base.copy()
        g[6] = [1.0, 0, 0]
        hs = [greg_h(1, u, v) for u in (t0, t1) for v in (0.0, 1.0)]
        _, d, _, _ = oracle.calc_points_and_d(g, True, t0, t1, 0.0, 1.0)
        assert d[0] == pytest.approx(b2 * (4 / 9) * (max(hs) - min(hs)), rel=1e-12)
        # pair (1,2): weights wbar1(u) * wbar2(v); swap roles: u over [0,1] -> 4/9, v over [t0,t1] -> b2
        g = base.copy()
        g[9] = [1.0, 0, 0]
        hs = [greg_h(2, u, v) for u in (0.0, 1.0) for v in (t0, t1)]
        _, d, _, _ = oracle.calc_points_and_d(g, True, 0.0, 1.0, t0, t1)
        assert d[0] == pytest.approx((4 / 9) * b2 * (max(hs) - min(hs)), rel=1e-12)
        # pair (2,2): weights wbar2(u) * wbar2(v), once with u over [t0,t1] and once with v over it
        g = base.copy()
        g[10] = [1.0, 0, 0]
        hs = [greg_h(3, u, v) for u in (t0, t1) for v in (0.0, 1.0)]
        _, d, _, _ = oracle.calc_points_and_d(g, True, t0, t1, 0.0, 1.0)
        assert d[0] == pytest.approx(b2 * (4 / 9) * (max(hs) - min(hs)), rel=1e-12)
        hs = [greg_h(3, u, v) for u in (0.0, 1.0) for v in (t0, t1)]
        _, d, _, _ = oracle.calc_points_and_d(g, True, 0.0, 1.0, t0, t1)
        assert d[0] == pytest.approx((4 / 9) * b2 * (max(hs) - min(hs)), rel=1e-12)
        # sampled check that the golden maxima are maxima
        ts = np.linspace(t0, t1, 1001)
        assert np.max(3 * ts * (1 - ts) ** 2) == pytest.approx(b1, rel=1e-5)
        assert np.max(3 * ts ** 2 * (1 - ts)) == pytest.approx(b2, rel=1e-5)


# ---------------------------------------------------------------- intersection: closed forms

def _ray(o, d, tmin=0.0, tmax=np.inf):
    return np.array([*o, *d, tmin, tmax], float)


def test_planar_patch_hit_matches_ray_plane_solution():
    """Planar patch A + uU + vV: the closest leaf at depth 24 reproduces the analytic ray-plane hit."""
    L = 24
    for _ in range(40):
        A = RNG.normal(size=3)
        U, V = RNG.normal(size=(2, 3))
        p = np.array([A + (i / 3) * U + (j / 3) * V for j in range(4) for i in range(4)])
        g = np.zeros((20, 3))
        g[:16] = p
        g[16:] = p[[5, 6, 9, 10]]
        us, vs = RNG.uniform(0.05, 0.95, 2)
        target = A + us * U + vs * V
        o = target + RNG.normal(size=3) * 2
        d = (target - o) / np.linalg.norm(target - o)
        t_star = np.linalg.norm(target - o)
        for greg in (False, True):
            hit, t, cell, _ = oracle.intersect_patch(g, greg, _ray(o, d), L)
            assert hit
            cu, cv = cell & ((1 << L) - 1), cell >> L
            u, v = (cu + 0.5) / 2 ** L, (cv + 0.5) / 2 ** L
            scale = np.linalg.norm(U) + np.linalg.norm(V)
            n = np.cross(U, V)
            cosang = abs(np.dot(n, d)) / np.linalg.norm(n)
            tol_t = 4 * scale * 2.0 ** -L / max(cosang, 1e-3)
            assert abs(t - t_star) <= tol_t
            assert t <= t_star + 1e-12  # the box entry never lies behind the surface
            tol_uv = 2.0 ** -L * (1 + 4 / max(cosang, 1e-3))
            assert abs(u - us) <= tol_uv and abs(v - vs) <= tol_uv


def _ray_bilinear(o, d, P00, P10, P01, P11):
    """Closest root of o + t d = bilinear(u, v): eliminate t with two planes containing the ray,
    solve the quadratic in v, back-substitute (textbook ray/bilinear-patch intersection)."""
    d = d / np.linalg.norm(d)
    a = np.cross(d, [1.0, 0, 0]) if abs(d[0]) < 0.9 else np.cross(d, [0, 1.0, 0])
    a /= np.linalg.norm(a)
    b = np.cross(d, a)
    best = None
    for n in (a, b):
        pass
    # plane equations n.(X - o) = 0 for n in {a, b}: sum of bilinear terms
    def coeffs(n):
        c00 = n @ (P00 - o)
        c10 = n @ (P10 - P00)
        c01 = n @ (P01 - P00)
        c11 = n @ (P11 - P10 - P01 + P00)
        return c00, c10, c01, c11   # c00 + u c10 + v c01 + u v c11 = 0
    A0, A1, A2, A3 = coeffs(a)
    B0, B1, B2, B3 = coeffs(b)
    # u = -(A0 + v A2) / (A1 + v A3); substitute into the second
    qa = B2 * A3 - B3 * A2
    qb = B0 * A3 - B3 * A0 + B2 * A1 - B1 * A2
    qc = B0 * A1 - B1 * A0
    roots = []
    if abs(qa) < 1e-14:
        if abs(qb) > 1e-14:
            roots = [-qc / qb]
    else:
        disc = qb * qb - 4 * qa * qc
        if disc >= 0:
            s = math.sqrt(disc)
            roots = [(-qb - s) / (2 * qa), (-qb + s) / (2 * qa)]
    for v in roots:
        if not (-1e-12 <= v <= 1 + 1e-12):
            continue
        den = A1 + v * A3
        if abs(den) < 1e-14:
            continue
        u = -(A0 + v * A2) / den
        if not (-1e-12 <= u <= 1 + 1e-12):
            continue
        X = (1 - u) * (1 - v) * P00 + u * (1 - v) * P10 + (1 - u) * v * P01 + u * v * P11
        t = d @ (X - o)
        if t >= 0 and (best is None or t < best[0]):
            best = (t, u, v)
    return best


def test_bilinear_patch_hit_matches_analytic_solution():
    """Degree-elevated bilinear patch: the oracle's leaf agrees with the analytic ray/bilinear root."""
    L = 22
    checked = 0
    for _ in range(200):
        P00, P10, P01, P11 = RNG.normal(size=(4, 3))
        p = np.array([(1 - i / 3) * (1 - j / 3) * P00 + (i / 3) * (1 - j / 3) * P10 + (1 - i / 3) * (j / 3) * P01
                      + (i / 3) * (j / 3) * P11 for j in range(4) for i in range(4)])
        us, vs = RNG.uniform(0.1, 0.9, 2)
        target = (1 - us) * (1 - vs) * P00 + us * (1 - vs) * P10 + (1 - us) * vs * P01 + us * vs * P11
        o = target + RNG.normal(size=3) * 3
        d = (target - o) / np.linalg.norm(target - o)
        ref = _ray_bilinear(o, d, P00, P10, P01, P11)
        assert ref is not None
        g = np.zeros((20, 3))
        g[:16] = p
        g[16:] = p[[5, 6, 9, 10]]
        hit, t, cell, _ = oracle.intersect_patch(g, False, _ray(o, d), L)
        assert hit
        # the surface point at the leaf cell centre lies on the ray up to the leaf size
        cu, cv = cell & ((1 << L) - 1), cell >> L
        u, v = (cu + 0.5) / 2 ** L, (cv + 0.5) / 2 ** L
        fu = (1 - u) * (1 - v) * P00 + u * (1 - v) * P10 + (1 - u) * v * P01 + u * v * P11
        extent = np.linalg.norm(np.ptp(p, axis=0))
        # grazing hits are ill-conditioned in (u, v); compare where the surface faces the ray
        du_ = (1 - vs) * (P10 - P00) + vs * (P11 - P01)
        dv_ = (1 - us) * (P01 - P00) + us * (P11 - P10)
        n = np.cross(du_, dv_)
        if abs(n @ d) < 0.2 * np.linalg.norm(n):
            continue
        checked += 1
        assert abs(t - ref[0]) <= 8 * extent * 2.0 ** -L
        assert np.linalg.norm(fu - (o + t * d)) <= 16 * extent * 2.0 ** -L
        assert abs(u - ref[1]) <= 64 * 2.0 ** -L and abs(v - ref[2]) <= 64 * 2.0 ** -L
    assert checked > 50


# ---------------------------------------------------------------- traversal order vs brute force

@pytest.mark.parametrize("greg", [False, True])
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_dfs_equals_brute_force_all_leaves(greg, L):
    """The pruned, ordered DFS returns the minimum key over all leaves whose ancestor chain is hit."""
    agree = hits = 0
    for _ in range(120):
        g = random_gregory() if greg else np.concatenate([random_patch(), np.zeros((4, 3))])
        if not greg:
            g[16:] = g[[5, 6, 9, 10]]
        c = g[:16].mean(0)
        o = c + RNG.normal(size=3) * 3
        d = (c + RNG.normal(size=3) * 0.7) - o
        d /= np.linalg.norm(d)
        tmax = np.inf if RNG.uniform() < 0.7 else np.linalg.norm(c - o) * RNG.uniform(0.5, 1.2)
        r = _ray(o, d, 0.0, tmax)
        a = oracle.intersect_patch(g, greg, r, L, brute=False)
        b = oracle.intersect_patch(g, greg, r, L, brute=True)
        assert a[0] == b[0]
        if a[0]:
            hits += 1
            assert a[1] == b[1] and a[2] == b[2]
        agree += 1
    assert hits > 20


def test_scene_closest_hit_is_min_over_patches():
    """Scene-level answer (BVH + per-patch traversal) = lexicographic minimum of per-patch answers."""
    from paper_1811_03510_gb300 import scenegen as sg
    s = sg.config_scene(1)
    r = sg.random_rays(300, seed=5)
    out = oracle.intersect(s.P, s.types, r.soa(), L=5)
    for i in range(r.n):
        ray8 = np.array([*r.o[i], *r.d[i], r.tmin[i], r.tmax[i]], float)
        best = (np.inf, 0xFFFFFFFF, 2 ** 64 - 1)
        for p in range(s.n):
            h, t, cell, _ = oracle.intersect_patch(s.P[p].astype(float), bool(s.types[p]), ray8, 5)
            if h and (t, p, cell) < best:
                best = (t, p, cell)
        assert out["t"][i] == best[0]
        assert out["pid"][i] == best[1]
        assert out["cell"][i] == best[2]


def _square_grid():
    """The square [0,3]^2 of the plane z = 0 as a degree-elevated affine patch, p_ij = (i, j, 0): every
    de Casteljau midpoint of it is a dyadic rational, so the leaf boundaries fall exactly on u, v = k / 2^L."""
    g = np.zeros((20, 3))
    for j in range(4):
        for i in range(4):
            g[4 * j + i] = [i, j, 0.0]
    g[16:] = g[[5, 6, 9, 10]]
    return g


def test_equal_entry_distances_take_the_lowest_cell():
    """Sec. 3.3 records the closest leaf; where several leaves are entered at the same distance the key
    (t, patch, cell) takes the lowest cell index (v_cell 2^L + u_cell).  A ray along -z onto a leaf
    boundary of the flat square enters the two (or four) leaves that share it at exactly t = 2."""
    g = _square_grid()
    L = 8
    v_mid = 3 * 37.5 / 256        # inside v cell 37
    for greg in (False, True):
        hit, t, cell, _ = oracle.intersect_patch(g, greg, _ray([1.5, v_mid, 2.0], [0.0, 0.0, -1.0]), L)
        assert hit and t == 2.0 and cell == (37 << L) | 127          # u = 1/2: cells 127 and 128
        hit, t, cell, _ = oracle.intersect_patch(g, greg, _ray([1.5, 1.5, 2.0], [0.0, 0.0, -1.0]), L)
        assert hit and t == 2.0 and cell == (127 << L) | 127         # u = v = 1/2: four cells
        hit, t, cell, _ = oracle.intersect_patch(g, greg, _ray([0.75, 2.25, 2.0], [0.0, 0.0, -1.0]), L)
        assert hit and t == 2.0 and cell == (191 << L) | 63          # u = 1/4, v = 3/4


def test_equal_keys_across_patches_take_the_lowest_patch():
    """Copies of one patch are entered at the same distance in the same cell: the scene's answer is the
    copy with the lowest index (key order t, patch, cell)."""
    g = _square_grid().astype(np.float32)
    far = g + np.float32(10.0)                                          # a patch off the ray
    rays = [np.array([x], np.float32) for x in (1.5, 1.5, 2.0, 0.0, 0.0, -1.0, 0.0, np.inf)]
    for P, want in (([g, g], 0), ([far, g, g, g], 1), ([g, far, g], 0)):
        out = oracle.intersect(np.stack(P), np.zeros(len(P), np.uint8), rays, L=6)
        assert out["pid"][0] == want and out["t"][0] == 2.0
