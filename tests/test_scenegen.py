"""Checks of the synthetic scene generator (input recipe of the workloads).  CPU only."""
import numpy as np
import pytest

from paper_1811_03510_gb300 import scenegen as sg


def test_workload_patch_counts():
    s = sg.config_scene(1)
    assert s.n == 96 and np.bincount(s.types).tolist() == [72, 24]
    s = sg.config_scene(2)
    assert s.n == 1536 and np.bincount(s.types).tolist() == [1512, 24]
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    assert np.bincount(s.types).tolist() == [1440, 96]
    assert sg.batched_sizes()[0] == 4 and sg.batched_sizes()[-1] == 64 and len(sg.batched_sizes()) == 32


def test_corners_are_catmull_clark_limit_positions():
    """Patch corners equal the limit of repeated refinement (Halstead et al. 1993 mask)."""
    V, F = sg.cube_sphere(2)
    V, F = sg.catmull_clark(V, F)
    P, types = sg.patches_from_mesh(V, F)
    corner = {}
    for f in range(len(F)):
        for k, slot in enumerate((0, 3, 15, 12)):
            corner[F[f, k]] = P[f, slot]
    Vk, Fk = V, F
    errs = []
    for _ in range(7):
        Vk, Fk = sg.catmull_clark(Vk, Fk)   # original vertex ids keep their index
        errs.append(max(np.linalg.norm(Vk[v] - c) for v, c in corner.items()))
    assert errs[-1] < 1e-4
    assert all(b < a for a, b in zip(errs, errs[1:]))


def _boundary(P, f, k):
    """Boundary curve of face f along its edge k (corner k -> k+1) as 4 points."""
    slots = [(0, 1, 2, 3), (3, 7, 11, 15), (15, 14, 13, 12), (12, 8, 4, 0)][k]
    return P[f, list(slots)]


@pytest.mark.parametrize("n,amp", [(2, 0.0), (8, 0.05)])
def test_neighbouring_patches_share_boundary_points_bit_for_bit(n, amp):
    V, F = sg.cube_sphere(n, amp, 3, 1)
    V, F = sg.catmull_clark(V, F)
    P, _ = sg.patches_from_mesh(V, F)
    P = P.astype(np.float32)
    he = sg.HalfEdges.build(F, len(V))
    for h in range(len(he.src)):
        t = he.twin[h]
        a = _boundary(P, h // 4, h % 4)
        b = _boundary(P, t // 4, t % 4)[::-1]
        assert np.array_equal(a, b)


def _bspline_to_bezier():
    return np.array([[1, 4, 1, 0], [0, 4, 2, 0], [0, 2, 4, 0], [0, 1, 4, 1]], float) / 6.0


def test_regular_faces_are_bspline_patches_and_gregory_builder_reproduces_them():
    """On an all-valence-4 mesh every patch equals M P M^T of its 16-point neighbourhood, and the
    Gregory construction gives p^u = p^v = that Bezier inner point."""
    nu, nv = 9, 7
    V, F = sg.torus_grid(nu, nv)
    P, types = sg.patches_from_mesh(V, F)
    assert (types == sg.BEZIER).all()
    Pg, tg = sg.patches_from_mesh(V, F, gregory_everywhere=True)
    assert (tg == sg.GREGORY).all()
    M = _bspline_to_bezier()
    Vg = V.reshape(nu, nv, 3)
    for f in range(len(F)):
        i, j = divmod(f, nv)
        G = np.array([[Vg[(i - 1 + a) % nu, (j - 1 + b) % nv] for b in range(4)] for a in range(4)])  # [a(u), b(v)]
        B = np.einsum("ca,db,abk->cdk", M, M, G)   # [c(u), d(v)]
        ref = np.array([B[c, d] for d in range(4) for c in range(4)])
        np.testing.assert_allclose(P[f, :16], ref, atol=1e-12)
        np.testing.assert_allclose(Pg[f, :16], ref, atol=1e-12)
        np.testing.assert_allclose(Pg[f, 16:], ref[[5, 6, 9, 10]], atol=1e-12)


def test_gregory_patches_have_distinct_pairs_on_the_cube_sphere():
    s = sg.config_scene(1)
    g = s.P[s.types == sg.GREGORY]
    diff = np.abs(g[:, [5, 6, 9, 10]] - g[:, 16:]).max(axis=(1, 2))
    assert (diff > 1e-3).all()


def test_pinhole_rays():
    r = sg.pinhole_rays(64, 48)
    assert r.n == 64 * 48
    np.testing.assert_allclose(np.linalg.norm(r.d, axis=1), 1, atol=1e-6)
    # centre rays look down -z, top-left pixel points up and left
    assert r.d[0, 0] < 0 and r.d[0, 1] > 0 and r.d[0, 2] < 0
    vfov = 2 * np.degrees(np.arctan(np.abs(r.d[:, 1] / r.d[:, 2]).max()))
    assert 58.5 < vfov < 60.0   # pixel centres sit half a pixel inside the frustum edge


def test_value_noise_range_and_determinism():
    p = np.random.default_rng(0).normal(size=(5000, 3))
    a = sg.value_noise(p, 3, 7)
    b = sg.value_noise(p, 3, 7)
    c = sg.value_noise(p, 3, 8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= -1 and a.max() <= 1 and a.std() > 0.05


def test_deformation_moves_shared_points_identically():
    s = sg.config_scene(1)
    P1 = sg.deform(s.P, 3, 8, seed=1)
    V, F = sg.cube_sphere(2)
    V, F = sg.catmull_clark(V, F)
    he = sg.HalfEdges.build(F, len(V))
    for h in range(len(he.src)):
        t = he.twin[h]
        assert np.array_equal(_boundary(P1, h // 4, h % 4), _boundary(P1, t // 4, t % 4)[::-1])
    assert 0.0 < np.abs(P1 - s.P).max() <= 0.0200001
