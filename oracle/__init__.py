"""FP64 CPU oracle for ray / Bezier-Gregory patch closest-hit intersection (arXiv 1811.03510).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and by the CPU-baseline leg
of the benchmark, never by the library.  The C source (ccs_oracle.c) shares no code with the CUDA
path.  Every function takes plain numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccs_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libccs_oracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_U64 = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile ccs_oracle.c with gcc (plain C99, no FP contraction) if the library is missing or stale."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-std=gnu99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC,
                           "-lm", "-lpthread"])
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    """The compiled oracle.  CCS_ORACLE_LIB names another build of ccs_oracle.c to load instead: the
    planted-mistake test points it at copies of the source with one mistake each."""
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(os.environ.get("CCS_ORACLE_LIB") or build())
        _lib.orc_intersect.restype = ctypes.c_int
        _lib.orc_intersect_patch.restype = ctypes.c_int
        _lib.orc_num_cores.restype = ctypes.c_int
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def num_cores() -> int:
    return lib().orc_num_cores()


def intersect(P, types, rays_soa, L: int = 8, threads: int = 0, flags: bool | int = False, rel_t: float = 1e-4,
              eps: float = 5e-7, perturb: float = 1e-4, stats: bool = False, spread: float = 0.0,
              local: bool = False) -> dict:
    """Closest hit of every ray.  P: [n, 20, 3] float32 patch points, types [n] uint8, rays_soa: eight
    float32 arrays (ox, oy, oz, dx, dy, dz, tmin, tmax).  Returns t (f64, inf on miss), u, v (f32 cell
    centre), pid (u32, 0xFFFFFFFF on miss), cell (u64, v_cell * 2^L + u_cell); with flags 'flags' and 't2'
    under the FP32 error model (boxes within eps, far distances within 1 + 1e-6; bit0 another patch may
    win, bit1 a far cell of the patch may win, bit2 hit/miss may flip, bit3 t may leave rel_t; flags=2
    adds bit4, the origin perturbation test by +-perturb); with stats=True 'stats' [n, 5]
    (bvh nodes, Bezier expansions, Gregory expansions, leaves, pops) and 'threads'.
    spread > 0: screen-space termination (Sec. 3.3): a node made by a split is a leaf once the L1 length of
    its box diagonal is below spread / 2 times its entry distance (spread = radians per pixel of the ray);
    'level' gives the recorded leaf's tree level (2L at full depth), u, v the centre of its domain, and
    the flags also cover a termination test within FP32 error of its threshold.
    local=True: below the root, boxes are taken in each patch's local frame (Sec. 3.4; see local_frame);
    the root interval is still the world box's."""
    P = np.ascontiguousarray(P, dtype=np.float32)
    n = P.shape[0]
    x = np.ascontiguousarray(P[..., 0]).reshape(-1)
    y = np.ascontiguousarray(P[..., 1]).reshape(-1)
    z = np.ascontiguousarray(P[..., 2]).reshape(-1)
    types = np.ascontiguousarray(types, dtype=np.uint8)
    planes = [np.ascontiguousarray(a, dtype=np.float32) for a in rays_soa]
    m = planes[0].shape[0]
    out = dict(t=np.empty(m, np.float64), u=np.empty(m, np.float32), v=np.empty(m, np.float32),
               pid=np.empty(m, np.uint32), cell=np.empty(m, np.uint64))
    fl = np.zeros(m, np.uint8) if flags else None
    t2 = np.empty(m, np.float64) if flags else None
    st = np.zeros((m, 5), np.uint64) if stats else None
    level = np.zeros(m, np.uint8)
    nt = lib().orc_intersect(
        _p(x, _F), _p(y, _F), _p(z, _F), _p(types, _U8), ctypes.c_uint32(n),
        *[_p(a, _F) for a in planes], ctypes.c_uint32(m), ctypes.c_int(L), ctypes.c_int(threads),
        ctypes.c_int(int(flags)), ctypes.c_double(rel_t), ctypes.c_double(eps), ctypes.c_double(perturb),
        _p(out["t"], _D), _p(out["u"], _F), _p(out["v"], _F), _p(out["pid"], _U32), _p(out["cell"], _U64),
        _p(fl, _U8) if flags else None, _p(t2, _D) if flags else None, _p(st, _U64) if stats else None,
        ctypes.c_double(spread), _p(level, _U8), ctypes.c_int(int(local)))
    if nt < 0:
        raise ValueError("oracle rejected arguments (leaf depth out of range?)")
    out["threads"] = nt
    out["level"] = level
    if flags:
        out["flags"] = fl
        out["t2"] = t2
    if stats:
        out["stats"] = st
    return out


def occluded(P, types, rays_soa, L: int = 8, flags: bool | int = False, local: bool = False) -> dict:
    """Any-hit query of shadow rays (Sec. 4): a ray is occluded iff some leaf box of some patch has a
    non-empty nested interval inside [tmin, tmax] (the leaf condition of Algorithm 3), which is exactly when
    the closest-hit answer exists.  Returns occluded (u8) and, with flags, the FP32 error-model flags of the
    closest-hit query (bit 2: hit/miss may flip)."""
    o = intersect(P, types, rays_soa, L=L, flags=flags, local=local)
    out = {"occluded": (o["pid"] != 0xFFFFFFFF).astype(np.uint8)}
    if flags:
        out["flags"] = o["flags"]
    return out


def intersect_patch(g, greg: bool, ray8, L: int, brute: bool = False, spread: float = 0.0, with_level: bool = False,
                    local: bool = False):
    """Single (ray, patch) query; g [20, 3] f64, ray8 = (ox, oy, oz, dx, dy, dz, tmin, tmax).
    Returns (hit, t, cell, stats5), and the leaf level with with_level (spread: as in intersect)."""
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    r = np.ascontiguousarray(ray8, dtype=np.float64)
    t = ctypes.c_double()
    c = ctypes.c_uint64()
    st = np.zeros(5, np.uint64)
    lv = ctypes.c_int()
    h = lib().orc_intersect_patch(_p(g, _D), ctypes.c_int(int(greg)), _p(r, _D), ctypes.c_int(L),
                                  ctypes.c_int(int(brute)), ctypes.byref(t), ctypes.byref(c), _p(st, _U64),
                                  ctypes.c_double(spread), ctypes.byref(lv), ctypes.c_int(int(local)))
    if h < 0:
        raise ValueError("bad leaf depth")
    if with_level:
        return bool(h), t.value, c.value, st, lv.value
    return bool(h), t.value, c.value, st


def local_frame(g20):
    """Rows (x, y, z) of a patch's local frame (Sec. 3.4): z along the normal of the corner quad (the
    cross product of its diagonals), x along its u edge made orthogonal to z, y = z x x."""
    g = np.ascontiguousarray(g20, dtype=np.float64).reshape(-1)
    out = np.zeros(9)
    lib().orc_local_frame(_p(g, _D), _p(out, _D))
    return out.reshape(3, 3)


def bezier_eval(p16, u: float, v: float):
    """(f, f_u, f_v, f_uv) of a Bezier patch, p16 [16, 3]."""
    p = np.ascontiguousarray(p16, dtype=np.float64).reshape(-1)
    out = np.empty(12)
    lib().orc_bezier_eval(_p(p, _D), ctypes.c_double(u), ctypes.c_double(v), _p(out, _D))
    return out.reshape(4, 3)


def crop(p16, u0, u1, v0, v1):
    """Algorithm 1: control points of the patch restricted to [u0,u1] x [v0,v1]."""
    p = np.ascontiguousarray(p16, dtype=np.float64).reshape(-1)
    q = np.empty(48)
    lib().orc_crop(_p(p, _D), *[ctypes.c_double(a) for a in (u0, u1, v0, v1)], _p(q, _D))
    return q.reshape(16, 3)


def split(p16, axis: int):
    """de Casteljau halves at 1/2 along axis (0 = u, 1 = v)."""
    p = np.ascontiguousarray(p16, dtype=np.float64).reshape(-1)
    a = np.empty(48)
    b = np.empty(48)
    lib().orc_split(_p(p, _D), ctypes.c_int(axis), _p(a, _D), _p(b, _D))
    return a.reshape(16, 3), b.reshape(16, 3)


def gregory_eval(g20, u: float, v: float):
    """(f(u, v), inner points p_ij(u, v) [4, 3]) of a Gregory patch."""
    g = np.ascontiguousarray(g20, dtype=np.float64).reshape(-1)
    f = np.empty(3)
    inner = np.empty(12)
    lib().orc_gregory_eval(_p(g, _D), ctypes.c_double(u), ctypes.c_double(v), _p(f, _D), _p(inner, _D))
    return f, inner.reshape(4, 3)


def patch_frame(g20, greg: bool, u: float, v: float):
    """(f, f_u, f_v) of the (Gregory-reduced) patch at (u, v)."""
    g = np.ascontiguousarray(g20, dtype=np.float64).reshape(-1)
    out = np.empty(9)
    lib().orc_patch_frame(_p(g, _D), ctypes.c_int(int(greg)), ctypes.c_double(u), ctypes.c_double(v), _p(out, _D))
    return out.reshape(3, 3)


def calc_points_and_d(g20, greg: bool, u0, u1, v0, v1):
    """Algorithm 2: (q [16, 3], d [3], pmin [4, 3], pmax [4, 3])."""
    g = np.ascontiguousarray(g20, dtype=np.float64).reshape(-1)
    q = np.empty(48)
    d = np.empty(3)
    lo = np.zeros(12)
    hi = np.zeros(12)
    lib().orc_calc_points_and_d(_p(g, _D), ctypes.c_int(int(greg)), *[ctypes.c_double(a) for a in (u0, u1, v0, v1)],
                                _p(q, _D), _p(d, _D), _p(lo, _D), _p(hi, _D))
    return q.reshape(16, 3), d, lo.reshape(4, 3), hi.reshape(4, 3)


def child_boxes(g20, greg: bool, level: int, pu: int, pv: int):
    """(lo_L, hi_L, lo_R, hi_R) of the two children of node (level, pu, pv), positions at scale 2^52."""
    g = np.ascontiguousarray(g20, dtype=np.float64).reshape(-1)
    out = np.empty(12)
    lib().orc_child_boxes(_p(g, _D), ctypes.c_int(int(greg)), ctypes.c_int(level), ctypes.c_uint64(pu),
                          ctypes.c_uint64(pv), _p(out, _D))
    return out.reshape(4, 3)
