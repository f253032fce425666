"""Screen-space termination in the oracle (Sec. 3.3): a node made by a split is a leaf once the L1
length of its box diagonal is below spread / 2 times its entry distance.  Pinned to a closed form on a
flat patch, to brute force over the whole tree, and to the fixed-depth answer it coarsens."""
import numpy as np
import pytest

import oracle
from paper_1811_03510_gb300 import scenegen as sg

MISS = 0xFFFFFFFF


def flat_square(a):
    """Degree-elevated affine patch: the square [-a/2, a/2]^2 in the plane z = 0, u along x, v along y."""
    g = np.zeros((20, 3))
    for j in range(4):
        for i in range(4):
            g[4 * j + i] = (a * (i / 3 - 0.5), a * (j / 3 - 0.5), 0.0)
    g[16:20] = g[[5, 6, 9, 10]]
    return g


def expected_level(a, spread, D, L):
    """First split level whose node (a 2^-su x 2^-sv block of the square) has an L1 diagonal below
    spread / 2 * D; the box of a flat patch has no extent along z."""
    for lev in range(1, 2 * L + 1):
        su, sv = (lev + 1) // 2, lev // 2
        if a * (2.0 ** -su + 2.0 ** -sv) < 0.5 * spread * D:
            return lev
    return 2 * L


@pytest.mark.parametrize("spread", [1e-3, 4e-3, 2e-2, 0.09])
def test_flat_patch_terminates_at_the_closed_form_level(spread):
    a, D, L = 1.0, 5.0, 8
    g = flat_square(a)
    rng = np.random.default_rng(int(spread * 1e4))
    lev_exp = expected_level(a, spread, D, L)
    # no level's node size lies at the threshold, so rounding cannot decide
    thr = 0.5 * spread * D
    for lev in range(1, lev_exp + 1):
        su, sv = (lev + 1) // 2, lev // 2
        assert abs(a * (2.0 ** -su + 2.0 ** -sv) - thr) > 1e-6 * thr
    su, sv = (lev_exp + 1) // 2, lev_exp // 2
    for _ in range(40):
        x, y = rng.uniform(-0.49, 0.49, 2) * a
        ray = np.array([x, y, D, 0.0, 0.0, -1.0, 0.0, np.inf])
        hit, t, cell, _, lev = oracle.intersect_patch(g, False, ray, L, spread=spread, with_level=True)
        assert hit and abs(t - D) < 1e-12
        assert lev == lev_exp
        # the recorded cell is the lowest cell of the node that contains the hit point
        cu, cv = cell & ((1 << L) - 1), cell >> L
        u, v = x / a + 0.5, y / a + 0.5
        assert cu == int(u * 2 ** su) << (L - su) and cv == int(v * 2 ** sv) << (L - sv)


def test_coarse_leaf_reports_the_centre_of_its_domain():
    """A screen-space leaf above the fixed depth is a block of 2^-su x 2^-sv in (u, v), su = ceil(level/2)
    splits along u and sv = floor(level/2) along v; the hit reports the centre of that block.  Odd and even
    termination levels both occur below."""
    a, D, L = 1.0, 5.0, 8
    g = flat_square(a).astype(np.float32)
    rng = np.random.default_rng(77)
    levels = set()
    for spread in (1e-3, 4e-3, 2e-2, 0.09):
        lev = expected_level(a, spread, D, L)
        levels.add(lev % 2)
        su, sv = (lev + 1) // 2, lev // 2
        xy = rng.uniform(-0.49, 0.49, size=(50, 2)) * a
        n = len(xy)
        rays = [xy[:, 0], xy[:, 1], np.full(n, D), np.zeros(n), np.zeros(n), -np.ones(n), np.zeros(n),
                np.full(n, np.inf)]
        rays = [np.ascontiguousarray(r, np.float32) for r in rays]
        out = oracle.intersect(g[None], np.zeros(1, np.uint8), rays, L=L, spread=spread)
        u = rays[0].astype(np.float64) / a + 0.5
        v = rays[1].astype(np.float64) / a + 0.5
        want_u = (np.floor(u * 2 ** su) + 0.5) / 2 ** su
        want_v = (np.floor(v * 2 ** sv) + 0.5) / 2 ** sv
        assert (out["pid"] == 0).all()
        np.testing.assert_array_equal(out["u"], want_u.astype(np.float32))
        np.testing.assert_array_equal(out["v"], want_v.astype(np.float32))
    assert levels == {0, 1}


@pytest.mark.parametrize("greg", [False, True])
@pytest.mark.parametrize("L", [3, 5])
def test_pruned_search_equals_brute_force_with_screen_leaves(greg, L):
    s = sg.config_scene(1)
    p = int(np.nonzero(s.types == (1 if greg else 0))[0][0])
    g = s.P[p].astype(np.float64)
    c = g.mean(0)
    rng = np.random.default_rng(7 + L + 10 * greg)
    n_hit = 0
    for k in range(150):
        o = c + rng.normal(size=3) * 1.5
        f = oracle.patch_frame(g, greg, *rng.uniform(0.02, 0.98, 2))[0]   # aim at a surface point
        d = f + 0.01 * rng.normal(size=3) - o
        ray = np.array([*o, *d, 0.0, np.inf])
        spread = [0.0, 3e-3, 3e-2, 0.3][k % 4]
        a = oracle.intersect_patch(g, greg, ray, L, spread=spread, with_level=True)
        b = oracle.intersect_patch(g, greg, ray, L, brute=True, spread=spread, with_level=True)
        assert a[0] == b[0]
        if a[0]:
            n_hit += 1
            assert a[1] == b[1] and a[2] == b[2] and a[4] == b[4], (k, a, b)
    assert n_hit > 50


def test_screen_leaves_only_coarsen_the_fixed_depth_answer():
    s = sg.config_scene(1)
    r = sg.pinhole_rays(64, 64)
    L = 8
    fixed = oracle.intersect(s.P, s.types, r.soa(), L=L)
    spread = 2.0 * np.tan(np.radians(30.0)) / 64   # one pixel of the 64 x 64 camera
    ss = oracle.intersect(s.P, s.types, r.soa(), L=L, spread=spread)
    fh, sh = fixed["pid"] != MISS, ss["pid"] != MISS
    assert (sh | ~fh).all()                    # every fixed-depth hit is still a hit
    both = fh & sh
    assert (ss["t"][both] <= fixed["t"][both]).all()   # a coarser box is entered no later
    assert (ss["level"][sh] < 2 * L).mean() > 0.9      # the camera's pixels are much larger than a cell
    assert (fixed["level"][fh] == 2 * L).all()
    # the recorded leaf satisfies the rule: its diagonal spans less than half a pixel at its entry
    assert (ss["level"][sh] >= 1).all()
