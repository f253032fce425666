"""Secondary rays from oracle hits, in FP64 (TEST INFRASTRUCTURE ONLY; written independently of the CUDA
generator from the same published definitions): origin = surface point of the hit cell centre offset
along the normal by offset_abs + 2 * 2^-L * L1(patch box diagonal) (Sec. 3.3 offsets by the L1 size of
the last box).  Diffuse: direction cosine-weighted from two PCG32 draws (O'Neill 2014,
pcg32_srandom_r(seed, i)) in the orthonormal basis of Duff et al. 2017.  Mirror: d - 2 (d.n) n.
Shadow (Sec. 4's one shadow ray per path): unit direction to a point light, tmax = its distance.
Slots without a hit (or, for shadow rays, with the light behind the surface) get tmin = 1, tmax = 0."""
import numpy as np

from . import patch_frame

_MULT = 6364136223846793005
_MASK = (1 << 64) - 1


def pcg32_pair(seed: int, seq: int):
    """First two outputs of pcg32 seeded with (initstate=seed, initseq=seq)."""
    inc = ((seq << 1) | 1) & _MASK
    state = 0

    def step(st):
        old = st
        st = (old * _MULT + inc) & _MASK
        xs = (((old >> 18) ^ old) >> 27) & 0xFFFFFFFF
        rot = old >> 59
        out = ((xs >> rot) | (xs << ((32 - rot) & 31))) & 0xFFFFFFFF
        return st, out

    state, _ = step(state)
    state = (state + seed) & _MASK
    state, _ = step(state)
    state, a = step(state)
    state, b = step(state)
    return a, b


def diffuse_rays(P, types, rays_soa, hits, seed: int, L: int = 8, offset_abs: float = 1e-4, mirror: bool = False):
    """rays_soa: the incoming rays (eight planes); hits: dict with pid, u, v.  Returns eight float32
    planes of diffuse rays (mirror=True: reflections d - 2 (d.n) n), one per slot."""
    n = len(hits["pid"])
    o = np.zeros((n, 3))
    d = np.zeros((n, 3))
    d[:, 2] = 1.0
    tmin = np.ones(n)
    tmax = np.zeros(n)
    din = np.stack([rays_soa[3], rays_soa[4], rays_soa[5]], 1).astype(np.float64)
    P = np.asarray(P, dtype=np.float32)
    for i in np.nonzero(np.asarray(hits["pid"]) != 0xFFFFFFFF)[0]:
        pid = int(hits["pid"][i])
        g = P[pid].astype(np.float64)
        greg = bool(types[pid])
        f, fu, fv = patch_frame(g, greg, float(hits["u"][i]), float(hits["v"][i]))
        nrm = np.cross(fu, fv)
        nrm /= np.linalg.norm(nrm)
        if nrm @ din[i] > 0:
            nrm = -nrm
        pts = g if greg else g[:16]
        l1 = np.ptp(pts, axis=0).sum()
        off = offset_abs + 2.0 * l1 * 2.0 ** -L
        o[i] = f + off * nrm
        tmin[i] = 0.0
        tmax[i] = np.inf
        if mirror:
            d[i] = din[i] - 2.0 * (din[i] @ nrm) * nrm
            continue
        a, b = pcg32_pair(seed, int(i))
        u1 = (a >> 8) / 16777216.0
        u2 = (b >> 8) / 16777216.0
        rr, phi = np.sqrt(u1), 2 * np.pi * u2
        lx, ly, lz = rr * np.cos(phi), rr * np.sin(phi), np.sqrt(max(0.0, 1 - u1))
        sg_ = 1.0 if nrm[2] >= 0 else -1.0
        aa = -1.0 / (sg_ + nrm[2])
        bb = nrm[0] * nrm[1] * aa
        b1 = np.array([1 + sg_ * nrm[0] ** 2 * aa, sg_ * bb, -sg_ * nrm[0]])
        b2 = np.array([bb, sg_ + nrm[1] ** 2 * aa, -nrm[1]])
        d[i] = lx * b1 + ly * b2 + lz * nrm
    planes = [o[:, 0], o[:, 1], o[:, 2], d[:, 0], d[:, 1], d[:, 2], tmin, tmax]
    return [np.ascontiguousarray(a, dtype=np.float32) for a in planes]


def _offset_origin(P, types, pid, u, v, din, L, offset_abs):
    """Surface point of (u, v), unit normal flipped against din, and the offset origin."""
    g = np.asarray(P, dtype=np.float32)[pid].astype(np.float64)
    greg = bool(types[pid])
    f, fu, fv = patch_frame(g, greg, float(u), float(v))
    nrm = np.cross(fu, fv)
    nrm /= np.linalg.norm(nrm)
    if nrm @ din > 0:
        nrm = -nrm
    pts = g if greg else g[:16]
    off = offset_abs + 2.0 * np.ptp(pts, axis=0).sum() * 2.0 ** -L
    return f, nrm, f + off * nrm


def shadow_rays(P, types, rays_soa, hits, light, L: int = 8, offset_abs: float = 1e-4):
    """Shadow rays toward the point light: eight float32 planes, one ray per slot."""
    n = len(hits["pid"])
    o = np.zeros((n, 3))
    d = np.zeros((n, 3))
    d[:, 2] = 1.0
    tmin = np.ones(n)
    tmax = np.zeros(n)
    din = np.stack([rays_soa[3], rays_soa[4], rays_soa[5]], 1).astype(np.float64)
    lp = np.asarray(light, dtype=np.float64)
    for i in np.nonzero(np.asarray(hits["pid"]) != 0xFFFFFFFF)[0]:
        _, nrm, org = _offset_origin(P, types, int(hits["pid"][i]), hits["u"][i], hits["v"][i], din[i], L, offset_abs)
        o[i] = org
        to_light = lp - org
        dist = np.linalg.norm(to_light)
        if dist > 0 and to_light @ nrm > 0:
            d[i] = to_light / dist
            tmin[i] = 0.0
            tmax[i] = dist
    planes = [o[:, 0], o[:, 1], o[:, 2], d[:, 0], d[:, 1], d[:, 2], tmin, tmax]
    return [np.ascontiguousarray(a, dtype=np.float32) for a in planes]
