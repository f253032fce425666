"""Python binding of libccs (include/ccs.h): argument marshalling only, every step runs in the CUDA
library.  Device buffers are passed as torch tensors (their data_ptr()) or raw integer addresses;
streams as torch.cuda.Stream or raw handles.  There is no fallback: if libccs.so is missing, every
call raises."""
from __future__ import annotations

import ctypes
import os

from . import build_ext

CCS_OK = 0
CCS_ERR_INVALID_ARG = 1
CCS_ERR_CUDA = 2
CCS_ERR_OOM = 3
CCS_ERR_TRAVERSAL_LIMIT = 4
CCS_ERR_NOT_BUILT = 5
CCS_BEZIER = 0
CCS_GREGORY = 1
CCS_TRACE_COUNT = 1
CCS_TRACE_ORDER = 2
CCS_TRACE_HOST_MAPPED = 4
CCS_TRACE_PAIRS = 8
CCS_BVH_BOTH = 6
CCS_NUM_COUNTERS = 23
COUNTER_NAMES = ("bvh_nodes", "bezier_splits", "gregory_splits", "leaves", "backtracks", "redescent_levels",
                 "pruned_siblings", "pairs",
                 # schedule of the warps (depends on the launch options)
                 "warp_iters", "resident_rays", "split_rays", "split_iters", "gregory_rays", "gregory_iters",
                 "leaf_rays", "leaf_iters", "bvh_rays", "bvh_iters", "bvh_burst_steps", "refills",
                 # timeline of one launch (device-clock ns; the first two bitwise inverted, see timeline())
                 "start_ns_inv", "queue_empty_ns_inv", "end_ns")
NUM_WORK_COUNTERS = 8


def timeline(c: dict) -> dict:
    """Launch timeline from the counters of one counting launch: total time, and the drain (from the moment
    a warp first found the work queue empty to the last warp's exit), in microseconds."""
    m = (1 << 64) - 1
    start = ~(c["start_ns_inv"] & m) & m
    empty = ~(c["queue_empty_ns_inv"] & m) & m
    end = c["end_ns"] & m
    return {"launch_us": (end - start) / 1e3, "drain_us": (end - empty) / 1e3}
MISS = 0xFFFFFFFF

_STATUS = {0: "CCS_OK", 1: "CCS_ERR_INVALID_ARG", 2: "CCS_ERR_CUDA", 3: "CCS_ERR_OOM",
           4: "CCS_ERR_TRAVERSAL_LIMIT", 5: "CCS_ERR_NOT_BUILT"}


class CcsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class ccs_rays(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("ox", "oy", "oz", "dx", "dy", "dz", "tmin", "tmax")]


class ccs_hits(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("t", "u", "v", "patch_id")]


class ccs_trace_opts(ctypes.Structure):
    _fields_ = [("leaf_depth", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("refill", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("bvh_burst", ctypes.c_uint32), ("cache_slots", ctypes.c_uint32), ("min_blocks", ctypes.c_uint32),
                ("vote", ctypes.c_uint32), ("lanes_per_ray", ctypes.c_uint32), ("iter_cap", ctypes.c_uint32),
                ("pixel_spread", ctypes.c_float),
                ("flags", ctypes.c_uint32), ("counters", ctypes.c_void_p), ("image_width", ctypes.c_uint32),
                ("bvh_width", ctypes.c_uint32), ("host_chunk", ctypes.c_uint32)]


class ccs_autotune_trial(ctypes.Structure):
    _fields_ = [("opts", ccs_trace_opts), ("ms", ctypes.c_float)]


class ccs_bvh_params(ctypes.Structure):
    _fields_ = [("bins", ctypes.c_uint32), ("width", ctypes.c_uint32)]


_lib = None

# name -> argtypes; every function returns ccs_status (int) except ccs_last_error
_SIGS = {
    "ccs_scene_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p],
    "ccs_scene_update_points": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "ccs_scene_destroy": [ctypes.c_void_p],
    "ccs_bvh_build": [ctypes.c_void_p, ctypes.POINTER(ccs_bvh_params)],
    "ccs_bvh_refit": [ctypes.c_void_p, ctypes.c_void_p],
    "ccs_intersect": [ctypes.c_void_p, ctypes.POINTER(ccs_rays), ctypes.c_uint32, ctypes.POINTER(ccs_hits),
                      ctypes.POINTER(ccs_trace_opts), ctypes.c_void_p],
    "ccs_intersect_host": [ctypes.c_void_p, ctypes.POINTER(ccs_rays), ctypes.c_uint32, ctypes.POINTER(ccs_hits),
                           ctypes.POINTER(ccs_trace_opts), ctypes.c_void_p],
    "ccs_intersect_host_batches": [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ccs_rays),
                                   ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ccs_hits),
                                   ctypes.POINTER(ctypes.POINTER(ccs_trace_opts)), ctypes.c_void_p],
    "ccs_scene_sync_status": [ctypes.c_void_p, ctypes.c_void_p],
    "ccs_gen_diffuse": [ctypes.c_void_p, ctypes.POINTER(ccs_rays), ctypes.POINTER(ccs_hits), ctypes.c_uint32,
                        ctypes.c_uint64, ctypes.c_uint32, ctypes.c_float, ctypes.POINTER(ccs_rays), ctypes.c_void_p],
    "ccs_autotune": [ctypes.c_void_p, ctypes.POINTER(ccs_rays), ctypes.c_uint32, ctypes.POINTER(ccs_hits),
                     ctypes.POINTER(ccs_trace_opts), ctypes.c_uint32, ctypes.POINTER(ccs_trace_opts),
                     ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ccs_autotune_trial), ctypes.c_uint32,
                     ctypes.POINTER(ctypes.c_uint32), ctypes.c_void_p],
    "ccs_batch_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint32,
                         ctypes.POINTER(ccs_rays), ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ccs_hits)],
    "ccs_batch_set_points": [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "ccs_batch_run": [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ccs_trace_opts), ctypes.c_void_p],
    "ccs_batch_capture": [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ccs_trace_opts)],
    "ccs_batch_launch": [ctypes.c_void_p, ctypes.c_void_p],
    "ccs_batch_sync_status": [ctypes.c_void_p, ctypes.c_void_p],
    "ccs_batch_destroy": [ctypes.c_void_p],
    "ccs_intersect_batched": [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ccs_rays), ctypes.POINTER(ctypes.c_uint32),
                              ctypes.POINTER(ccs_hits), ctypes.c_uint32, ctypes.POINTER(ccs_trace_opts),
                              ctypes.c_void_p],
    "ccs_intersect_batched_noalloc": [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ccs_rays),
                                      ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ccs_hits), ctypes.c_uint32,
                                      ctypes.POINTER(ccs_trace_opts), ctypes.c_void_p],
    "ccs_proposal_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint64],
    "ccs_proposal_destroy": [ctypes.c_void_p],
    "ccs_proposal_set_params": [ctypes.c_void_p, ctypes.c_void_p],
    "ccs_proposal_get_params": [ctypes.c_void_p, ctypes.c_void_p],
    "ccs_proposal_save": [ctypes.c_void_p, ctypes.c_char_p],
    "ccs_proposal_load": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_char_p],
    "ccs_proposal_grad": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_void_p],
    "ccs_proposal_train_step": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_float,
                                ctypes.c_void_p, ctypes.c_void_p],
    "ccs_proposal_infer": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_void_p, ctypes.c_void_p],
    "ccs_trace_export": [ctypes.c_void_p, ctypes.POINTER(ccs_rays), ctypes.c_uint32, ctypes.POINTER(ccs_hits),
                         ctypes.POINTER(ccs_trace_opts), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                         ctypes.c_void_p, ctypes.c_void_p],
    "ccs_intersect_learned": [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ccs_rays), ctypes.c_uint32,
                              ctypes.POINTER(ccs_hits), ctypes.POINTER(ccs_trace_opts), ctypes.c_float,
                              ctypes.c_void_p],
    "ccs_gen_mirror": [ctypes.c_void_p, ctypes.POINTER(ccs_rays), ctypes.POINTER(ccs_hits), ctypes.c_uint32,
                       ctypes.c_uint32, ctypes.c_float, ctypes.POINTER(ccs_rays), ctypes.c_void_p],
    "ccs_scene_info": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)],
    "ccs_occluded": [ctypes.c_void_p, ctypes.POINTER(ccs_rays), ctypes.c_uint32, ctypes.c_void_p,
                     ctypes.POINTER(ccs_trace_opts), ctypes.c_void_p],
    "ccs_gen_shadow": [ctypes.c_void_p, ctypes.POINTER(ccs_rays), ctypes.POINTER(ccs_hits), ctypes.c_uint32,
                       ctypes.POINTER(ctypes.c_float), ctypes.c_uint32, ctypes.c_float, ctypes.POINTER(ccs_rays),
                       ctypes.c_void_p],
}


def lib_path() -> str:
    return build_ext.LIB


def lib():
    """Load libccs.so (built by build_ext.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        path = build_ext.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libccs.so not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.ccs_last_error.argtypes = []
        L.ccs_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def declared_symbols():
    """Names of the functions declared in include/*.h."""
    import glob
    import re
    names = []
    for h in sorted(glob.glob(os.path.join(build_ext.INCLUDE, "*.h"))):
        src = open(h).read()
        names += re.findall(r"^\s*(?:ccs_status|const char \*)\s*(ccs_\w+)\s*\(", src, flags=re.M)
    return names


def _check(status: int):
    if status != CCS_OK:
        raise CcsError(status, lib().ccs_last_error().decode())


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int:
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


CCS_CACHE_DEFAULT = 0xFFFFFFFF


def make_opts(leaf_depth=8, block_threads=0, blocks_per_sm=0, refill=0, chunk=0, bvh_burst=0,
              cache_slots=CCS_CACHE_DEFAULT, min_blocks=0, vote=0, lanes_per_ray=0, iter_cap=0,
              counters=None, pixel_spread=0.0, order=False, image_width=0, host_chunk=0,
              host_mapped=False, bvh_width=0, pairs=False) -> ccs_trace_opts:
    """ccs_trace_opts with the fields of include/ccs.h (0: the library's default).  counters: a device
    int64 tensor of CCS_NUM_COUNTERS entries (sets CCS_TRACE_COUNT); order: CCS_TRACE_ORDER over tiles of
    an image of width image_width (0: runs of 32 rays; the pair engine's candidate pass also takes 8 x 4
    pixel tiles of it when the width is a multiple of 8); host_mapped: CCS_TRACE_HOST_MAPPED; pairs:
    CCS_TRACE_PAIRS (the pair engine)."""
    o = ccs_trace_opts()
    o.leaf_depth = leaf_depth
    o.block_threads = block_threads
    o.blocks_per_sm = blocks_per_sm
    o.refill = refill
    o.chunk = chunk
    o.bvh_burst = bvh_burst
    o.min_blocks = min_blocks
    o.vote = vote
    o.lanes_per_ray = lanes_per_ray
    o.cache_slots = cache_slots
    o.iter_cap = iter_cap
    o.pixel_spread = pixel_spread
    o.flags = ((CCS_TRACE_COUNT if counters is not None else 0) | (CCS_TRACE_ORDER if order else 0)
               | (CCS_TRACE_HOST_MAPPED if host_mapped else 0) | (CCS_TRACE_PAIRS if pairs else 0))
    o.counters = _ptr(counters) if counters is not None else None
    o.image_width = image_width
    o.host_chunk = host_chunk
    o.bvh_width = bvh_width
    return o


def rays_struct(planes) -> ccs_rays:
    return ccs_rays(*[_ptr(p) for p in planes])


def hits_struct(planes) -> ccs_hits:
    return ccs_hits(*[_ptr(p) for p in planes])


# ------------------------------------------------------------------ entry points (same names as the C ABI)

CCS_SCENE_DEVICE_PTRS = 1
CCS_SCENE_LOCAL_FRAMES = 2


def ccs_scene_create(x, y, z, types, n_patches: int, device_ptrs: bool, stream=None, local: bool = False) -> int:
    h = ctypes.c_void_p()
    flags = (CCS_SCENE_DEVICE_PTRS if device_ptrs else 0) | (CCS_SCENE_LOCAL_FRAMES if local else 0)
    _check(lib().ccs_scene_create(ctypes.byref(h), _ptr(x), _ptr(y), _ptr(z), _ptr(types), n_patches, flags,
                                  _stream(stream)))
    return h.value


def ccs_scene_update_points(scene: int, x, y, z, stream=None):
    _check(lib().ccs_scene_update_points(scene, _ptr(x), _ptr(y), _ptr(z), _stream(stream)))


def ccs_scene_destroy(scene: int):
    _check(lib().ccs_scene_destroy(scene))


def ccs_bvh_build(scene: int, bins: int = 16, width: int = 2):
    p = ccs_bvh_params(bins, width)
    _check(lib().ccs_bvh_build(scene, ctypes.byref(p)))


def ccs_bvh_refit(scene: int, stream=None):
    _check(lib().ccs_bvh_refit(scene, _stream(stream)))


def ccs_intersect(scene: int, rays, n: int, hits, opts: ccs_trace_opts | None = None, stream=None):
    r = rays if isinstance(rays, ccs_rays) else rays_struct(rays)
    h = hits if isinstance(hits, ccs_hits) else hits_struct(hits)
    _check(lib().ccs_intersect(scene, ctypes.byref(r), n, ctypes.byref(h), ctypes.byref(opts) if opts else None,
                               _stream(stream)))


def ccs_intersect_host(scene: int, rays, n: int, hits, opts: ccs_trace_opts | None = None, stream=None):
    r = rays if isinstance(rays, ccs_rays) else rays_struct(rays)
    h = hits if isinstance(hits, ccs_hits) else hits_struct(hits)
    _check(lib().ccs_intersect_host(scene, ctypes.byref(r), n, ctypes.byref(h),
                                    ctypes.byref(opts) if opts else None, _stream(stream)))


def ccs_intersect_host_batches(scene: int, rays_list, n_list, hits_list, opts_list=None, stream=None):
    """Several host batches through one copy/trace pipeline; opts_list entries may be None (defaults)."""
    nb = len(rays_list)
    R = (ccs_rays * nb)(*[r if isinstance(r, ccs_rays) else rays_struct(r) for r in rays_list])
    H = (ccs_hits * nb)(*[h if isinstance(h, ccs_hits) else hits_struct(h) for h in hits_list])
    N = (ctypes.c_uint32 * nb)(*[int(x) for x in n_list])
    O = None
    if opts_list is not None:
        O = (ctypes.POINTER(ccs_trace_opts) * nb)(*[ctypes.pointer(o) if o is not None else None
                                                     for o in opts_list])
    _check(lib().ccs_intersect_host_batches(scene, nb, R, N, H, O, _stream(stream)))


def ccs_gen_diffuse(scene: int, in_rays, hits, n: int, seed: int, leaf_depth: int, offset_abs: float, out_rays,
                    stream=None):
    r = in_rays if isinstance(in_rays, ccs_rays) else rays_struct(in_rays)
    h = hits if isinstance(hits, ccs_hits) else hits_struct(hits)
    o = out_rays if isinstance(out_rays, ccs_rays) else rays_struct(out_rays)
    _check(lib().ccs_gen_diffuse(scene, ctypes.byref(r), ctypes.byref(h), n, seed, leaf_depth, offset_abs,
                                 ctypes.byref(o), _stream(stream)))


def ccs_gen_mirror(scene: int, in_rays, hits, n: int, leaf_depth: int, offset_abs: float, out_rays, stream=None):
    r = in_rays if isinstance(in_rays, ccs_rays) else rays_struct(in_rays)
    h = hits if isinstance(hits, ccs_hits) else hits_struct(hits)
    o = out_rays if isinstance(out_rays, ccs_rays) else rays_struct(out_rays)
    _check(lib().ccs_gen_mirror(scene, ctypes.byref(r), ctypes.byref(h), n, leaf_depth, offset_abs, ctypes.byref(o),
                                _stream(stream)))


def gen_mirror(scene: "Scene", rays_dev, hits, leaf_depth: int = 8, offset_abs: float = 1e-4, stream=None):
    """Mirror rays for every slot (inactive slots have tmin > tmax); returns eight device planes."""
    import torch
    n = int(rays_dev[0].numel())
    o = torch.empty(3 * n, dtype=torch.float32, device=rays_dev[0].device)
    d = torch.empty(3 * n, dtype=torch.float32, device=rays_dev[0].device)
    tmin = torch.empty(n, dtype=torch.float32, device=rays_dev[0].device)
    tmax = torch.empty(n, dtype=torch.float32, device=rays_dev[0].device)
    planes = [o[:n], o[n:2 * n], o[2 * n:], d[:n], d[n:2 * n], d[2 * n:], tmin, tmax]
    ccs_gen_mirror(scene.handle, rays_dev, hits, n, leaf_depth, offset_abs, planes, stream)
    return planes


def ccs_occluded(scene: int, rays, n: int, occluded, opts: ccs_trace_opts | None = None, stream=None):
    """Any-hit query: occluded (n device bytes) = 1 where the ray enters a leaf box within [tmin, tmax]."""
    r = rays if isinstance(rays, ccs_rays) else rays_struct(rays)
    _check(lib().ccs_occluded(scene, ctypes.byref(r), n, _ptr(occluded), ctypes.byref(opts) if opts else None,
                              _stream(stream)))


def ccs_gen_shadow(scene: int, in_rays, hits, n: int, light, leaf_depth: int, offset_abs: float, out_rays,
                   stream=None):
    r = in_rays if isinstance(in_rays, ccs_rays) else rays_struct(in_rays)
    h = hits if isinstance(hits, ccs_hits) else hits_struct(hits)
    o = out_rays if isinstance(out_rays, ccs_rays) else rays_struct(out_rays)
    lp = (ctypes.c_float * 3)(*[float(x) for x in light])
    _check(lib().ccs_gen_shadow(scene, ctypes.byref(r), ctypes.byref(h), n, lp, leaf_depth, offset_abs,
                                ctypes.byref(o), _stream(stream)))


def gen_shadow(scene: "Scene", rays_dev, hits, light, leaf_depth: int = 8, offset_abs: float = 1e-4, stream=None):
    """Shadow rays toward the point light for every slot (inactive slots have tmin > tmax)."""
    import torch
    n = int(rays_dev[0].numel())
    o = torch.empty(3 * n, dtype=torch.float32, device=rays_dev[0].device)
    d = torch.empty(3 * n, dtype=torch.float32, device=rays_dev[0].device)
    tmin = torch.empty(n, dtype=torch.float32, device=rays_dev[0].device)
    tmax = torch.empty(n, dtype=torch.float32, device=rays_dev[0].device)
    planes = [o[:n], o[n:2 * n], o[2 * n:], d[:n], d[n:2 * n], d[2 * n:], tmin, tmax]
    ccs_gen_shadow(scene.handle, rays_dev, hits, n, light, leaf_depth, offset_abs, planes, stream)
    return planes


def occluded(scene: "Scene", rays_dev, opts: ccs_trace_opts | None = None, stream=None):
    """Allocate the byte plane and run the any-hit query; returns a uint8 device tensor."""
    import torch
    n = int(rays_dev[0].numel())
    out = torch.empty(n, dtype=torch.uint8, device=rays_dev[0].device)
    ccs_occluded(scene.handle, rays_dev, n, out, opts, stream)
    return out


def gen_diffuse(scene: "Scene", rays_dev, hits, seed: int, leaf_depth: int = 8, offset_abs: float = 1e-4,
                stream=None):
    """Diffuse rays for every slot (inactive slots have tmin > tmax); returns eight device planes."""
    import torch
    n = int(rays_dev[0].numel())
    o = torch.empty(3 * n, dtype=torch.float32, device=rays_dev[0].device)
    d = torch.empty(3 * n, dtype=torch.float32, device=rays_dev[0].device)
    tmin = torch.empty(n, dtype=torch.float32, device=rays_dev[0].device)
    tmax = torch.empty(n, dtype=torch.float32, device=rays_dev[0].device)
    planes = [o[:n], o[n:2 * n], o[2 * n:], d[:n], d[n:2 * n], d[2 * n:], tmin, tmax]
    ccs_gen_diffuse(scene.handle, rays_dev, hits, n, seed, leaf_depth, offset_abs, planes, stream)
    return planes


def ccs_autotune(scene: int, rays, n: int, hits, base: ccs_trace_opts | None = None, reps: int = 3, stream=None,
                 max_trials: int = 256):
    """Returns (best opts, best ms, list of (opts, ms) trials)."""
    r = rays if isinstance(rays, ccs_rays) else rays_struct(rays)
    h = hits if isinstance(hits, ccs_hits) else hits_struct(hits)
    best = ccs_trace_opts()
    ms = ctypes.c_float()
    tr = (ccs_autotune_trial * max_trials)()
    nt = ctypes.c_uint32()
    _check(lib().ccs_autotune(scene, ctypes.byref(r), n, ctypes.byref(h), ctypes.byref(base) if base else None, reps,
                              ctypes.byref(best), ctypes.byref(ms), tr, max_trials, ctypes.byref(nt), _stream(stream)))
    trials = [(tr[i].opts, tr[i].ms) for i in range(min(nt.value, max_trials))]
    return best, ms.value, trials


CCS_BATCH_UPDATE = 1
CCS_BATCH_REFIT = 2
CCS_BATCH_INTERSECT = 4


def _batch_arrays(scenes, rays_list, hits_list):
    n = len(scenes)
    sc = (ctypes.c_void_p * n)(*[s if isinstance(s, int) else s.handle for s in scenes])
    r = (ccs_rays * n)(*[x if isinstance(x, ccs_rays) else rays_struct(x) for x in rays_list])
    h = (ccs_hits * n)(*[x if isinstance(x, ccs_hits) else hits_struct(x) for x in hits_list])
    cnt = (ctypes.c_uint32 * n)(*[int(x[0].numel()) if not isinstance(x, ccs_rays) else 0 for x in rays_list])
    return sc, r, cnt, h


def ccs_batch_create(scenes, rays_list, hits_list, n_rays=None) -> int:
    sc, r, cnt, h = _batch_arrays(scenes, rays_list, hits_list)
    if n_rays is not None:
        cnt = (ctypes.c_uint32 * len(scenes))(*n_rays)
    b = ctypes.c_void_p()
    _check(lib().ccs_batch_create(ctypes.byref(b), sc, len(scenes), r, cnt, h))
    return b.value


def ccs_batch_set_points(batch: int, scene_index: int, x, y, z):
    _check(lib().ccs_batch_set_points(batch, scene_index, _ptr(x), _ptr(y), _ptr(z)))


def ccs_batch_run(batch: int, stages: int, opts: ccs_trace_opts | None = None, stream=None):
    _check(lib().ccs_batch_run(batch, stages, ctypes.byref(opts) if opts else None, _stream(stream)))


def ccs_batch_capture(batch: int, stages: int, opts: ccs_trace_opts | None = None):
    _check(lib().ccs_batch_capture(batch, stages, ctypes.byref(opts) if opts else None))


def ccs_batch_launch(batch: int, stream=None):
    _check(lib().ccs_batch_launch(batch, _stream(stream)))


def ccs_batch_sync_status(batch: int, stream=None) -> int:
    st = lib().ccs_batch_sync_status(batch, _stream(stream))
    if st not in (CCS_OK, CCS_ERR_TRAVERSAL_LIMIT):
        _check(st)
    return st


def ccs_batch_destroy(batch: int):
    _check(lib().ccs_batch_destroy(batch))


def ccs_intersect_batched(scenes, rays_list, hits_list, opts: ccs_trace_opts | None = None, stream=None):
    sc, r, cnt, h = _batch_arrays(scenes, rays_list, hits_list)
    _check(lib().ccs_intersect_batched(sc, r, cnt, h, len(scenes), ctypes.byref(opts) if opts else None,
                                       _stream(stream)))


CCS_NOALLOC_MAX_SCENES = 256


def ccs_intersect_batched_noalloc(scenes, rays_list, hits_list, opts: ccs_trace_opts | None = None, stream=None):
    """Allocation-free batched closest hit: scratch in the library's static device array."""
    sc, r, cnt, h = _batch_arrays(scenes, rays_list, hits_list)
    _check(lib().ccs_intersect_batched_noalloc(sc, r, cnt, h, len(scenes), ctypes.byref(opts) if opts else None,
                                               _stream(stream)))


CCS_PROPOSAL_PARAMS = 9920
CCS_PROPOSAL_FEATURES = 24
CCS_PROPOSAL_CELLS = 64


def ccs_proposal_create(seed: int = 1) -> int:
    h = ctypes.c_void_p()
    _check(lib().ccs_proposal_create(ctypes.byref(h), seed))
    return h.value


def ccs_proposal_destroy(p: int):
    _check(lib().ccs_proposal_destroy(p))


def ccs_proposal_set_params(p: int, params):
    import numpy as np
    a = np.ascontiguousarray(params, dtype=np.float32)
    assert a.size == CCS_PROPOSAL_PARAMS
    _check(lib().ccs_proposal_set_params(p, a.ctypes.data))


def ccs_proposal_get_params(p: int):
    import numpy as np
    a = np.empty(CCS_PROPOSAL_PARAMS, np.float32)
    _check(lib().ccs_proposal_get_params(p, a.ctypes.data))
    return a


def ccs_proposal_save(p: int, path: str):
    _check(lib().ccs_proposal_save(p, path.encode()))


def ccs_proposal_load(path: str) -> int:
    h = ctypes.c_void_p()
    _check(lib().ccs_proposal_load(ctypes.byref(h), path.encode()))
    return h.value


def ccs_proposal_grad(p: int, features, labels, batch: int, grad, loss=None, stream=None):
    _check(lib().ccs_proposal_grad(p, _ptr(features), _ptr(labels), batch, _ptr(grad), _ptr(loss), _stream(stream)))


def ccs_proposal_train_step(p: int, features, labels, batch: int, lr: float, loss=None, stream=None):
    _check(lib().ccs_proposal_train_step(p, _ptr(features), _ptr(labels), batch, lr, _ptr(loss), _stream(stream)))


def ccs_proposal_infer(p: int, features, n: int, logits=None, cells=None, pmax=None, stream=None):
    _check(lib().ccs_proposal_infer(p, _ptr(features), n, _ptr(logits), _ptr(cells), _ptr(pmax), _stream(stream)))


def ccs_trace_export(scene: int, rays, n: int, hits, opts, features, labels, capacity: int, count, stream=None):
    r = rays if isinstance(rays, ccs_rays) else rays_struct(rays)
    h = hits if isinstance(hits, ccs_hits) else hits_struct(hits)
    _check(lib().ccs_trace_export(scene, ctypes.byref(r), n, ctypes.byref(h), ctypes.byref(opts) if opts else None,
                                  _ptr(features), _ptr(labels), capacity, _ptr(count), _stream(stream)))


def ccs_intersect_learned(scene: int, proposal: int, rays, n: int, hits, opts=None, min_confidence: float = 0.0,
                          stream=None):
    r = rays if isinstance(rays, ccs_rays) else rays_struct(rays)
    h = hits if isinstance(hits, ccs_hits) else hits_struct(hits)
    _check(lib().ccs_intersect_learned(scene, proposal, ctypes.byref(r), n, ctypes.byref(h),
                                       ctypes.byref(opts) if opts else None, min_confidence, _stream(stream)))


def opts_dict(o: ccs_trace_opts) -> dict:
    d = {k: int(getattr(o, k)) for k in ("leaf_depth", "block_threads", "blocks_per_sm", "refill", "chunk",
                                          "bvh_burst", "cache_slots", "min_blocks", "vote", "lanes_per_ray",
                                          "image_width", "host_chunk", "bvh_width")}
    d["order"] = bool(o.flags & CCS_TRACE_ORDER)
    d["pairs"] = bool(o.flags & CCS_TRACE_PAIRS)
    return d


def ccs_scene_sync_status(scene: int, stream=None) -> int:
    """Returns CCS_OK or CCS_ERR_TRAVERSAL_LIMIT (does not raise for the latter)."""
    st = lib().ccs_scene_sync_status(scene, _stream(stream))
    if st not in (CCS_OK, CCS_ERR_TRAVERSAL_LIMIT):
        _check(st)
    return st


def ccs_scene_info(scene: int):
    a, b = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().ccs_scene_info(scene, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ccs_last_error() -> str:
    return lib().ccs_last_error().decode()


# ------------------------------------------------------------------ small conveniences over the entry points

class Scene:
    """Owns a ccs_scene handle built from host arrays P [n, 20, 3] float32 and types [n] uint8; local=True
    takes the sub-domain boxes in each patch's own frame (CCS_SCENE_LOCAL_FRAMES); bvh_width 2, 4 or
    "both" (CCS_BVH_BOTH: launches choose with make_opts(bvh_width=...))."""

    def __init__(self, P, types, bins: int = 16, stream=None, local: bool = False, bvh_width: int = 2):
        import numpy as np
        P = np.ascontiguousarray(P, dtype=np.float32)
        self.n = int(P.shape[0])
        x = np.ascontiguousarray(P[..., 0]).reshape(-1)
        y = np.ascontiguousarray(P[..., 1]).reshape(-1)
        z = np.ascontiguousarray(P[..., 2]).reshape(-1)
        t = np.ascontiguousarray(types, dtype=np.uint8)
        self.local = bool(local)
        self.handle = ccs_scene_create(x.ctypes.data, y.ctypes.data, z.ctypes.data, t.ctypes.data, self.n, False,
                                       stream, local=self.local)
        self.bvh_width = CCS_BVH_BOTH if bvh_width == "both" else int(bvh_width)
        ccs_bvh_build(self.handle, bins, self.bvh_width)

    def close(self):
        if self.handle:
            ccs_scene_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rays_to_device(rays_soa, device="cuda"):
    """Eight host float32 planes -> list of contiguous device tensors."""
    import numpy as np
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device) for a in rays_soa]


def alloc_hits(n: int, device="cuda"):
    import torch
    return [torch.empty(n, dtype=torch.float32, device=device), torch.empty(n, dtype=torch.float32, device=device),
            torch.empty(n, dtype=torch.float32, device=device), torch.empty(n, dtype=torch.int32, device=device)]


def hits_to_numpy(hits):
    import numpy as np
    t, u, v, p = [h.cpu().numpy() for h in hits]
    return dict(t=t, u=u, v=v, pid=p.view(np.uint32))


def intersect(scene: Scene, rays_dev, opts: ccs_trace_opts | None = None, stream=None):
    """Allocate hit planes and intersect device rays; returns the four hit tensors (pid as int32 bits)."""
    n = int(rays_dev[0].numel())
    hits = alloc_hits(n, rays_dev[0].device)
    ccs_intersect(scene.handle, rays_dev, n, hits, opts, stream)
    return hits
