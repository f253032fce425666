"""Seeded synthetic inputs: Catmull-Clark cube-spheres as Bezier/Gregory patch arrays, and camera rays.

This module produces the patch arrays and ray batches that both the CUDA path and the oracle consume.
It holds none of the ray/patch intersection arithmetic (no bounds, no subdivision, no hit tests).

Scene recipe (the paper's meshes are proprietary; cube-spheres stand in for them):
  * cube base mesh with n x n quads per face, vertices projected to the unit sphere and optionally
    displaced radially by amp * (octave value noise, seed s);
  * one Catmull-Clark refinement (Catmull & Clark 1978), which isolates the 8 valence-3 vertices;
  * every refined face becomes one patch (Sec. 3 takes regular patches as bicubic Bezier patches and
    irregular ones as Gregory patches, produced in the paper by OpenSubdiv's feature-adaptive
    subdivision).  Faces whose four corners have valence 4 are uniform bicubic B-spline patches,
    converted to Bezier form; faces touching an extraordinary vertex become Gregory patches.

Patch construction (our own, since the paper takes the patches from OpenSubdiv):
  * corner points are Catmull-Clark limit positions (Halstead et al. 1993 vertex mask);
  * boundary control points come from per-half-edge tables built from the limit tangent mask,
    scaled so that a valence-4 vertex reproduces the B-spline -> Bezier conversion exactly; every
    patch reads the same table entry for a shared edge, so neighbouring patches share boundary
    control points bit for bit (C0, watertight input);
  * interior points of regular faces are the B-spline -> Bezier inner points; Gregory patches get a
    pair (p^u, p^v) per inner point from a local cross-boundary twist estimate that equals the
    B-spline inner point when the vertex is regular.

Control-point layout handed to the library (20 slots per patch, SoA planes x, y, z):
  slots 0..15 = 4x4 grid, slot 4*j + i with i along u and j along v, corner p_00 at (u, v) = (0, 0);
  for Gregory patches slots 5, 6, 9, 10 ((i, j) = (1,1), (2,1), (1,2), (2,2)) hold p^u and slots
  16..19 hold p^v in the same order; Bezier patches repeat their inner points in slots 16..19.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BEZIER = 0
GREGORY = 1

# Grid slots of the four inner points, in the order (1,1), (2,1), (1,2), (2,2).
INNER_SLOTS = (5, 6, 9, 10)


# --------------------------------------------------------------------------------------------
# Hashing and value noise
# --------------------------------------------------------------------------------------------

def _pcg_hash(x: np.ndarray) -> np.ndarray:
    """32-bit PCG-style integer hash (RXS-M-XS output of one LCG step), Jarzynski & Olano 2020."""
    x = np.asarray(x, dtype=np.uint32)
    with np.errstate(over="ignore"):
        state = x * np.uint32(747796405) + np.uint32(2891336453)
        word = ((state >> ((state >> np.uint32(28)) + np.uint32(4))) ^ state) * np.uint32(277803737)
        return (word >> np.uint32(22)) ^ word


def _lattice(ix, iy, iz, seed: int) -> np.ndarray:
    """Value in [-1, 1] at integer lattice points."""
    h = _pcg_hash(np.uint32(seed & 0xFFFFFFFF))
    h = _pcg_hash(np.asarray(iz, dtype=np.int64).astype(np.uint32) ^ h)
    h = _pcg_hash(np.asarray(iy, dtype=np.int64).astype(np.uint32) ^ h)
    h = _pcg_hash(np.asarray(ix, dtype=np.int64).astype(np.uint32) ^ h)
    return (h.astype(np.float64) / 4294967295.0) * 2.0 - 1.0


def value_noise(p: np.ndarray, octaves: int, seed: int, base_freq: float = 2.0) -> np.ndarray:
    """Octave value noise in [-1, 1]: smoothstep trilinear lattice noise, frequency x2 and amplitude
    x1/2 per octave, normalised by the amplitude sum."""
    p = np.asarray(p, dtype=np.float64)
    total = np.zeros(p.shape[0])
    amp, freq, norm = 1.0, base_freq, 0.0
    for o in range(octaves):
        q = p * freq
        i0 = np.floor(q).astype(np.int64)
        f = q - i0
        s = f * f * (3.0 - 2.0 * f)
        acc = np.zeros(p.shape[0])
        for dz in (0, 1):
            wz = s[:, 2] if dz else 1.0 - s[:, 2]
            for dy in (0, 1):
                wy = s[:, 1] if dy else 1.0 - s[:, 1]
                for dx in (0, 1):
                    wx = s[:, 0] if dx else 1.0 - s[:, 0]
                    acc += wx * wy * wz * _lattice(i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz, seed + 1013 * o)
        total += amp * acc
        norm += amp
        amp *= 0.5
        freq *= 2.0
    return total / norm


# --------------------------------------------------------------------------------------------
# Meshes
# --------------------------------------------------------------------------------------------

def cube_sphere(n: int, amp: float = 0.0, octaves: int = 3, seed: int = 1):
    """Closed quad mesh: cube with n x n quads per face, projected to the unit sphere, radius
    1 + amp * noise.  Faces are counter-clockwise seen from outside.  Returns (V [nv,3] f64, F [nf,4])."""
    pts, quads = [], []
    base = 0
    a = np.arange(n + 1)
    A, B = np.meshgrid(a, a, indexing="ij")  # A along first tangent, B along second
    for axis in range(3):
        k1, k2 = (axis + 1) % 3, (axis + 2) % 3
        for sign in (1, -1):
            P = np.zeros((n + 1, n + 1, 3), dtype=np.int64)
            P[..., axis] = sign * n
            if sign > 0:
                P[..., k1] = 2 * A - n
                P[..., k2] = 2 * B - n
            else:
                P[..., k1] = 2 * B - n
                P[..., k2] = 2 * A - n
            pts.append(P.reshape(-1, 3))
            idx = base + (A * (n + 1) + B)
            q = np.stack([idx[:-1, :-1], idx[1:, :-1], idx[1:, 1:], idx[:-1, 1:]], axis=-1).reshape(-1, 4)
            quads.append(q)
            base += (n + 1) * (n + 1)
    pts = np.concatenate(pts)
    quads = np.concatenate(quads)
    m = 2 * n + 1
    key = (pts[:, 0] + n) * m * m + (pts[:, 1] + n) * m + (pts[:, 2] + n)
    _, first, inv = np.unique(key, return_index=True, return_inverse=True)
    V = pts[first].astype(np.float64)
    F = inv[quads]
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    if amp != 0.0:
        V *= (1.0 + amp * value_noise(V, octaves, seed))[:, None]
    return V, F.astype(np.int64)


def torus_grid(nu: int, nv: int, R: float = 1.0, r: float = 0.35):
    """Closed all-valence-4 quad mesh (torus), used to check regular-patch construction."""
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    th = 2 * np.pi * i / nu
    ph = 2 * np.pi * j / nv
    V = np.stack([(R + r * np.cos(ph)) * np.cos(th), (R + r * np.cos(ph)) * np.sin(th), r * np.sin(ph)], -1)
    V = V.reshape(-1, 3)
    idx = lambda a, b: (a % nu) * nv + (b % nv)
    F = np.stack([idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)], -1).reshape(-1, 4)
    return V, F.astype(np.int64)


@dataclass
class HalfEdges:
    """Half-edge h = 4*f + k runs from F[f,k] to F[f,(k+1)%4]."""
    F: np.ndarray
    src: np.ndarray
    dst: np.ndarray
    twin: np.ndarray
    nv: int

    @staticmethod
    def build(F: np.ndarray, nv: int) -> "HalfEdges":
        src = F.reshape(-1)
        dst = np.roll(F, -1, axis=1).reshape(-1)
        key = src.astype(np.int64) * nv + dst
        order = np.argsort(key)
        skey = key[order]
        rkey = dst.astype(np.int64) * nv + src
        pos = np.searchsorted(skey, rkey)
        if np.any(pos >= len(skey)) or np.any(skey[np.minimum(pos, len(skey) - 1)] != rkey):
            raise ValueError("mesh is not a closed 2-manifold")
        twin = order[pos]
        return HalfEdges(F, src, dst, twin, nv)

    def next(self, h):
        return (h // 4) * 4 + (h % 4 + 1) % 4

    def prev(self, h):
        return (h // 4) * 4 + (h % 4 + 3) % 4

    def face(self, h):
        return h // 4


def catmull_clark(V: np.ndarray, F: np.ndarray):
    """One Catmull-Clark refinement step of a closed quad mesh (Catmull & Clark 1978)."""
    nv, nf = len(V), len(F)
    he = HalfEdges.build(F, nv)
    a, b = he.src, he.dst
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    ekey = lo.astype(np.int64) * nv + hi
    ukeys, eid = np.unique(ekey, return_inverse=True)
    ne = len(ukeys)
    fp = V[F].mean(axis=1)
    fh = np.arange(4 * nf) // 4
    # each undirected edge has two half-edges; sum their faces' points and endpoints
    esum = np.zeros((ne, 3))
    np.add.at(esum, eid, fp[fh])
    ev = np.zeros((ne, 3))
    np.add.at(ev, eid, V[a])  # both directions -> a + b once each
    ep = (esum + ev) / 4.0
    val = np.bincount(a, minlength=nv).astype(np.float64)
    Q = np.zeros((nv, 3))
    np.add.at(Q, a, fp[fh])
    Q /= val[:, None]
    R = np.zeros((nv, 3))
    np.add.at(R, a, 0.5 * (V[a] + V[b]))
    R /= val[:, None]
    vp = (Q + 2.0 * R + (val[:, None] - 3.0) * V) / val[:, None]
    NV = np.concatenate([vp, ep, fp])
    e_of = eid.reshape(nf, 4)
    newF = np.empty((nf, 4, 4), dtype=np.int64)
    for k in range(4):
        newF[:, k, 0] = F[:, k]
        newF[:, k, 1] = nv + e_of[:, k]
        newF[:, k, 2] = nv + ne + np.arange(nf)
        newF[:, k, 3] = nv + e_of[:, (k + 3) % 4]
    return NV, newF.reshape(-1, 4)


# --------------------------------------------------------------------------------------------
# Patches
# --------------------------------------------------------------------------------------------

def _vertex_rings(he: HalfEdges, maxval: int = 16):
    """For every vertex: valence, and for every outgoing half-edge its index j in the CCW ring.
    Returns (valence [nv], ring_he [nv, maxval] outgoing half-edges, ring_idx [4*nf])."""
    nv = he.nv
    nh = len(he.src)
    out = np.full(nv, -1, dtype=np.int64)
    out[he.src[::-1]] = np.arange(nh)[::-1]
    ring = np.full((nv, maxval), -1, dtype=np.int64)
    ring_idx = np.full(nh, -1, dtype=np.int64)
    h = out.copy()
    valence = np.zeros(nv, dtype=np.int64)
    active = np.ones(nv, dtype=bool)
    for j in range(maxval):
        ring[active, j] = h[active]
        ring_idx[h[active]] = j
        valence[active] += 1
        h = np.where(active, he.twin[he.prev(h)], h)
        active &= h != out
        if not active.any():
            break
    if active.any():
        raise ValueError("valence above %d" % maxval)
    return valence, ring, ring_idx


def limit_and_edge_tables(V: np.ndarray, he: HalfEdges):
    """Limit position per vertex and Bezier edge control point per outgoing half-edge.

    Limit position (Halstead et al. 1993): (n^2 v + 4 sum e_k + sum f_k) / (n (n + 5)), e_k the
    edge neighbours and f_k the face-opposite vertices of the n quads around v.
    Tangent along ring direction j: T_j = sum_k A_n cos(2 pi (k-j)/n) e_k
    + (cos(2 pi (k-j)/n) + cos(2 pi (k-j+1)/n)) f_k, A_n = 1 + cos(2pi/n) + cos(pi/n) sqrt(2 (9 + cos(2pi/n))).
    Edge point = p + T_j / (3 K_n) with K_n = n (A_n/2 + 1 + cos(2 pi/n)), which makes the valence-4
    case equal to the B-spline -> Bezier boundary point."""
    valence, ring, ring_idx = _vertex_rings(he)
    nv = len(V)
    maxval = ring.shape[1]
    valid = ring >= 0
    rh = np.where(valid, ring, 0)
    E = V[he.dst[rh]]                      # edge neighbours e_k
    D = V[he.dst[he.next(rh)]]             # face-opposite vertices f_k
    E = np.where(valid[..., None], E, 0.0)
    D = np.where(valid[..., None], D, 0.0)
    n = valence.astype(np.float64)
    limit = (n[:, None] ** 2 * V + 4.0 * E.sum(1) + D.sum(1)) / (n * (n + 5.0))[:, None]
    c1 = np.cos(2 * np.pi / n)
    A = 1.0 + c1 + np.cos(np.pi / n) * np.sqrt(2.0 * (9.0 + c1))
    K = n * (A / 2.0 + 1.0 + c1)
    nh = len(he.src)
    edge = np.zeros((nh, 3))
    h_all = np.arange(nh)
    v_of = he.src
    j_of = ring_idx
    k = np.arange(maxval)[None, :]
    nn = n[v_of][:, None]
    ang = 2 * np.pi * (k - j_of[:, None]) / nn
    ang1 = 2 * np.pi * (k - j_of[:, None] + 1) / nn
    we = A[v_of][:, None] * np.cos(ang)
    wf = np.cos(ang) + np.cos(ang1)
    kv = valid[v_of]
    we = np.where(kv, we, 0.0)
    wf = np.where(kv, wf, 0.0)
    T = np.einsum("hk,hkc->hc", we, E[v_of]) + np.einsum("hk,hkc->hc", wf, D[v_of])
    edge[h_all] = limit[v_of] + T / (3.0 * K[v_of])[:, None]
    return valence, limit, edge


def patches_from_mesh(V: np.ndarray, F: np.ndarray, gregory_everywhere: bool = False):
    """Bezier/Gregory patch per face of a closed quad mesh.

    Returns (P [nf, 20, 3] float64, types [nf] uint8).  A face is Bezier when its four corners
    have valence 4 (and gregory_everywhere is False), Gregory otherwise."""
    nv, nf = len(V), len(F)
    he = HalfEdges.build(F, nv)
    valence, limit, edge = limit_and_edge_tables(V, he)
    P = np.zeros((nf, 20, 3))
    f = np.arange(nf)
    c = F  # corners c0..c3
    # corners
    P[:, 0] = limit[c[:, 0]]
    P[:, 3] = limit[c[:, 1]]
    P[:, 15] = limit[c[:, 2]]
    P[:, 12] = limit[c[:, 3]]
    h = 4 * f[:, None] + np.arange(4)[None, :]  # h[:,k] = c_k -> c_{k+1}
    tw = he.twin[h]
    P[:, 1] = edge[h[:, 0]]
    P[:, 2] = edge[tw[:, 0]]
    P[:, 7] = edge[h[:, 1]]
    P[:, 11] = edge[tw[:, 1]]
    P[:, 14] = edge[h[:, 2]]
    P[:, 13] = edge[tw[:, 2]]
    P[:, 8] = edge[h[:, 3]]
    P[:, 4] = edge[tw[:, 3]]

    # regular (B-spline) inner points: (4 c_k + 2 c_{k+1} + 2 c_{k-1} + c_{k+2}) / 9
    def bs_inner(k):
        return (4 * V[c[:, k]] + 2 * V[c[:, (k + 1) % 4]] + 2 * V[c[:, (k + 3) % 4]] + V[c[:, (k + 2) % 4]]) / 9.0

    # Gregory interior point paired with the boundary edge {c, x} of face f:
    # e(c->x) + r/3, r = 2/3 (centroid f - centroid g) + 1/3 (mid(c,y) - mid(c,z)), where g is the
    # face across the edge, y the other neighbour of c in f, z the other neighbour of c in g.
    cent = V[F].mean(axis=1)

    def interior(k, toward_next):
        ck = V[c[:, k]]
        if toward_next:
            hce = h[:, k]                      # c -> c_{k+1}, in f
            g = he.face(he.twin[hce])
            y = V[c[:, (k + 3) % 4]]
            z = V[he.dst[he.next(he.twin[hce])]]
            e = edge[hce]
        else:
            hp = h[:, (k + 3) % 4]             # c_{k-1} -> c, in f
            g = he.face(he.twin[hp])           # twin = c -> c_{k-1}, in g
            y = V[c[:, (k + 1) % 4]]
            z = V[he.src[he.prev(he.twin[hp])]]
            e = edge[he.twin[hp]]
        r = (2.0 / 3.0) * (cent[f] - cent[g]) + (1.0 / 3.0) * (0.5 * (ck + y) - 0.5 * (ck + z))
        return e + r / 3.0

    irregular = (valence[F] != 4).any(axis=1)
    greg = irregular | gregory_everywhere
    types = np.where(greg, GREGORY, BEZIER).astype(np.uint8)
    # inner slots (1,1)->5 corner 0, (2,1)->6 corner 1, (2,2)->10 corner 2, (1,2)->9 corner 3
    corner_of_slot = {5: 0, 6: 1, 10: 2, 9: 3}
    pv_slot = {5: 16, 6: 17, 9: 18, 10: 19}
    # p^u pairs with the u-edge: toward next at corners 0 and 2, toward previous at corners 1 and 3
    for slot, k in corner_of_slot.items():
        bs = bs_inner(k)
        pu = interior(k, toward_next=(k % 2 == 0))
        pvv = interior(k, toward_next=(k % 2 == 1))
        P[:, slot] = np.where(greg[:, None], pu, bs)
        P[:, pv_slot[slot]] = np.where(greg[:, None], pvv, bs)
    return P, types


# --------------------------------------------------------------------------------------------
# Scenes and rays
# --------------------------------------------------------------------------------------------

@dataclass
class Scene:
    P: np.ndarray       # [n, 20, 3] float32 control points (world space)
    types: np.ndarray   # [n] uint8
    name: str

    @property
    def n(self) -> int:
        return len(self.types)

    def soa(self):
        """(x, y, z) float32 planes of shape [n*20], contiguous."""
        P = np.ascontiguousarray(self.P, dtype=np.float32)
        return (np.ascontiguousarray(P[..., 0]).reshape(-1), np.ascontiguousarray(P[..., 1]).reshape(-1),
                np.ascontiguousarray(P[..., 2]).reshape(-1))


def make_scene(n: int, amp: float = 0.0, octaves: int = 3, seed: int = 1, gregory_ring: bool = False,
               name: str | None = None) -> Scene:
    V, F = cube_sphere(n, amp, octaves, seed)
    V2, F2 = catmull_clark(V, F)
    P, types = patches_from_mesh(V2, F2)
    if gregory_ring:
        # also represent regular faces that share a vertex with an irregular face as Gregory patches
        # with p^u = p^v (an identical surface): exercises Gregory/Bezier divergence
        he = HalfEdges.build(F2, len(V2))
        val, _, _ = limit_and_edge_tables(V2, he)
        irr_v = np.zeros(len(V2), dtype=bool)
        irr_v[F2[types == GREGORY].reshape(-1)] = True
        ring = irr_v[F2].any(axis=1)
        types = np.where(ring, GREGORY, types).astype(np.uint8)
    return Scene(P.astype(np.float32), types, name or f"cube-sphere n={n}")


def config_scene(k: int, seed: int = 1) -> Scene:
    """Scenes of the five workloads: 1 -> 2x2 per face, no noise (96 patches); 2 and 5 -> 8x8, amp 0.05,
    3 octaves (1536); 3 -> 128x128, amp 0.1, 5 octaves (393,216)."""
    if k == 1:
        return make_scene(2, 0.0, name="cfg1: 2x2/face cube-sphere, 96 patches")
    if k in (2, 5):
        return make_scene(8, 0.05, 3, seed, name=f"cfg2: 8x8/face cube-sphere, amp 0.05, seed {seed}")
    if k == 3:
        return make_scene(128, 0.1, 5, seed, name=f"cfg3: 128x128/face cube-sphere, amp 0.1, seed {seed}")
    raise ValueError(k)


def batched_sizes() -> list[int]:
    """Quads per cube face of the 32 scenes of the batched workload: 4 + round(60 k / 31)."""
    return [4 + int(round(60 * k / 31)) for k in range(32)]


def deform(P_rest: np.ndarray, frame: int, n_frames: int, seed: int, amp: float = 0.02) -> np.ndarray:
    """Per-frame sinusoidal control-point offsets, a function of the rest position so that shared
    boundary points move identically: p + amp * sin(w * p_rest + phi + 2 pi frame / F)."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(2.0, 6.0, size=3)
    phi = rng.uniform(0.0, 2 * np.pi, size=3)
    P = P_rest.astype(np.float64)
    off = amp * np.sin(w * P + phi + 2 * np.pi * frame / n_frames)
    return (P + off).astype(np.float32)


@dataclass
class Rays:
    o: np.ndarray      # [n, 3] float32
    d: np.ndarray      # [n, 3] float32
    tmin: np.ndarray   # [n] float32
    tmax: np.ndarray   # [n] float32

    @property
    def n(self) -> int:
        return len(self.tmin)

    def soa(self):
        """Eight contiguous float32 planes: ox, oy, oz, dx, dy, dz, tmin, tmax."""
        o = np.ascontiguousarray(self.o, dtype=np.float32)
        d = np.ascontiguousarray(self.d, dtype=np.float32)
        return [np.ascontiguousarray(o[:, 0]), np.ascontiguousarray(o[:, 1]), np.ascontiguousarray(o[:, 2]),
                np.ascontiguousarray(d[:, 0]), np.ascontiguousarray(d[:, 1]), np.ascontiguousarray(d[:, 2]),
                np.ascontiguousarray(self.tmin, dtype=np.float32), np.ascontiguousarray(self.tmax, dtype=np.float32)]

    def subset(self, idx) -> "Rays":
        return Rays(self.o[idx], self.d[idx], self.tmin[idx], self.tmax[idx])


def pinhole_rays(width: int, height: int, eye=(0.0, 0.0, 3.0), fov_deg: float = 60.0) -> Rays:
    """Pinhole camera looking down -z with +y up, vertical field of view fov_deg, one ray through each
    pixel centre, unit directions, tmin = 0, tmax = +inf.  Ray index = row * width + column."""
    j, i = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    th = math.tan(math.radians(fov_deg) / 2.0)
    aspect = width / height
    x = (2.0 * (i + 0.5) / width - 1.0) * th * aspect
    y = (1.0 - 2.0 * (j + 0.5) / height) * th
    d = np.stack([x, y, -np.ones_like(x)], -1).reshape(-1, 3)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(np.asarray(eye, dtype=np.float64), d.shape)
    n = d.shape[0]
    return Rays(o.astype(np.float32), d.astype(np.float32), np.zeros(n, np.float32), np.full(n, np.inf, np.float32))


def random_rays(n: int, seed: int, radius: float = 3.0, target: float = 1.1) -> Rays:
    """Rays from random points on a sphere of the given radius toward random points in a ball of radius
    `target`: incoherent directions, most of them crossing the scene."""
    rng = np.random.default_rng(seed)
    o = rng.normal(size=(n, 3))
    o *= radius / np.linalg.norm(o, axis=1, keepdims=True)
    t = rng.normal(size=(n, 3))
    t *= (target * rng.uniform(0, 1, size=(n, 1)) ** (1 / 3)) / np.linalg.norm(t, axis=1, keepdims=True)
    d = t - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return Rays(o.astype(np.float32), d.astype(np.float32), np.zeros(n, np.float32), np.full(n, np.inf, np.float32))


def concat_rays(rs: list[Rays]) -> Rays:
    return Rays(np.concatenate([r.o for r in rs]), np.concatenate([r.d for r in rs]),
                np.concatenate([r.tmin for r in rs]), np.concatenate([r.tmax for r in rs]))
