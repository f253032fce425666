"""Benchmark: closest-hit MRays/s of the 1536-patch cube-sphere workload (8x8 quads per face, radial noise
amplitude 0.05 with 3 octaves, one Catmull-Clark refinement; 1920x1080 pinhole primary rays plus one
generation of cosine-weighted diffuse rays from their hits; leaf depth 8; FP32).

One step = one closest-hit launch over the primary batch plus one over the diffuse batch, inputs resident
on the device, L2 flushed (256 MB write) before every timed step.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ccs|reference] [--variant plain]
Under torchrun every rank runs its own copy of the workload (rays are independent; no collective on the
data path) and rank 0 reports the whole-job rate over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "closest-hit MRays/s (primary, diffuse) & % FP32 roofline, learned/batched vs plain"
UNIT = "MRays/s"
WORKLOAD = "cfg2: 1536-patch cube-sphere (8x8/face, noise 0.05, 3 oct, seed 1), 1920x1080 primary + diffuse, L=8"

# FP32 operations per unit of work that the method itself performs (the roofline of the traversal):
OPS_BVH_NODE = 34        # two slab tests
OPS_SPLIT_BEZIER = 360   # de Casteljau split 144 + two 16-point boxes 180 + two slabs 34 + order 2
OPS_SPLIT_GREGORY = 360 + 1130   # + Algorithm 2 bounds and Algorithm 1 crop of the lower patch
OPS_PAIR_FRAME = 24              # local frames: the ray rotated into the patch frame (2 x 9 + 3 inverses + 3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ccs", choices=["ccs", "reference"])
    ap.add_argument("--variant", default="all", choices=["all", "plain", "batched", "learned"])
    ap.add_argument("--train-seeds", type=int, default=15,
                    help="scenes (seeds 2..) whose traces train the proposal (until 4.5 M traces: 4 M to train on, "
                         "the rest held out)")
    ap.add_argument("--frames", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default launch options (profiling runs)")
    ap.add_argument("--opts-primary", default=None,
                    help='launch options of the primary batch as JSON (e.g. {"block_threads": 96, "order": true}), '
                         "instead of the tuner's (profiling runs)")
    ap.add_argument("--opts-diffuse", default=None, help="the same for the diffuse batch")
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--boxes", default="local", choices=["local", "world"],
                    help="sub-domain boxes in each patch's frame (Sec. 3.4) or in world axes")
    ap.add_argument("--bvh-width", default="both", choices=["2", "4", "both"],
                    help="children per BVH node; both: the binary and the 4-wide tree, the tuner picks per batch")
    return ap.parse_args()


def bvh_arg(args):
    return "both" if args.bvh_width == "both" else int(args.bvh_width)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        out.update(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


def build_workload(width, height, seed=1):
    from paper_1811_03510_gb300 import scenegen as sg
    s = sg.config_scene(2, seed=seed)
    r = sg.pinhole_rays(width, height)
    return s, r


def max_over_ranks(t: float, device=None) -> float:
    """The slowest rank's time: the whole job ends when its last replica does (barrier-bracketed timing).
    Works with gloo (CPU tensor) and nccl (device tensor); a single process returns t."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t)
    x = torch.tensor([float(t)], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def whole_job_rate(rays_per_step: int, steps: int, t_slowest: float, world: int) -> float:
    """MRays/s of the whole job: every rank traces its own replica of the step (weak scaling)."""
    return rays_per_step * world * steps / t_slowest / 1e6


def engine_of(o) -> str:
    from paper_1811_03510_gb300 import ccs
    d = ccs.opts_dict(o)
    return "pairs" if d["pairs"] and d["lanes_per_ray"] != 3 else ("ray+order" if d["order"] else "ray")


def kernels_per_launch(o) -> int:
    """Kernels of this library one ccs_intersect launches: the pair engine's candidate and subdivision passes;
    the work order's three kernels and k_intersect; or k_intersect alone."""
    return {"pairs": 2, "ray+order": 4, "ray": 1}[engine_of(o)]


def schedule_summary(c: dict, lanes_per_ray: int, engine: str = "ray") -> dict:
    """Warp schedule from the kernel's schedule counters.  Ray-persistent kernel: rays resident per warp
    iteration, and for each step kind the share of iterations that run it and the rays taking part when it
    runs.  Pair engine: lanes per warp iteration in a subdivision step, helping with a handed-over subtree,
    waiting for helpers or idle; the candidate lists and the fallback."""
    from paper_1811_03510_gb300 import ccs
    if engine == "pairs":   # slots 8..17 of the pair engine's counting launch
        v = [c[ccs.COUNTER_NAMES[k]] for k in range(ccs.CCS_NUM_COUNTERS)]
        it = max(1, v[12])
        out = {"engine": "pairs", "warp_iters": v[12], "split_lanes_per_iter": v[13] / it,
               "helper_lanes_per_iter": v[14] / it, "waiting_lanes_per_iter": v[15] / it,
               "idle_lanes_per_iter": v[16] / it, "subtrees_handed_over": v[11], "candidates": v[8],
               "candidates_culled_by_root_box": v[17], "rays_with_dropped_candidates": v[9],
               "walks_for_dropped_candidates": v[10]}
        out.update(ccs.timeline(c))
        return out
    it = max(1, c["warp_iters"])
    rpw = 10 if lanes_per_ray == 3 else 32
    out = {"warp_iters": c["warp_iters"], "rays_per_warp": rpw, "resident_per_iter": c["resident_rays"] / it}
    for k in ("split", "gregory", "leaf", "bvh"):
        runs = c[k + "_iters"]
        out[k + "_iter_frac"] = runs / it
        out[k + "_rays_per_run"] = c[k + "_rays"] / runs if runs else 0.0
    out["bvh_steps_per_run"] = c["bvh_burst_steps"] / max(1, c["bvh_iters"])
    from paper_1811_03510_gb300 import ccs
    out.update(ccs.timeline(c))   # of the counting launch, which runs slower than the timed one
    return out


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("traverse.cuh", "intersect_impl.cuh", "intersect.cu", "intersect4.cu", "order.cu", "order_plan.h",
              "learned.cuh", "ccs_internal.h", "pairs.cuh", "pairs.cu", "pairs_launch.cuh", "pairs_plain.cu"):
        with open(os.path.join(ROOT, "paper_1811_03510_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic() -> tuple:
    """DRAM bytes per primary and diffuse launch of the dominant kernel (the pair engine's subdivision pass,
    under ncu's cold cache) from the committed ncu summary, if it was taken on the current kernel sources
    (else None: the counters describe another kernel)."""
    path = os.path.join(ROOT, "profiles", "k_pairs_cfg2_dram.md")
    try:
        text = open(path).read()
    except OSError:
        return None, None
    import re
    m_hash = re.search(r"kernel sources sha256\[:16\]: ([0-9a-f]{16})", text)
    m_p = re.search(r"primary launch: dram bytes (\d+)", text)
    m_d = re.search(r"diffuse launch: dram bytes (\d+)", text)
    if not (m_hash and m_p and m_d) or m_hash.group(1) != kernel_source_hash():
        return None, path
    return (int(m_p.group(1)), int(m_d.group(1))), path


def measured_share() -> tuple:
    """Share of the subdivision pass (both batches) in the step's kernel time, from the committed ncu launch
    list, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "k_pairs_cfg2_launches.md")
    try:
        text = open(path).read()
    except OSError:
        return None, None
    import re
    m_hash = re.search(r"kernel sources sha256\[:16\]: ([0-9a-f]{16})", text)
    m = re.search(r"k_pairs share of the step: ([0-9.]+)", text)
    if not (m_hash and m) or m_hash.group(1) != kernel_source_hash():
        return None, path
    return float(m.group(1)), path


def measured_issue() -> tuple:
    """Thread-instruction issue of the primary launch over the FP32 lane peak (all instructions, and FADD/FMUL/FFMA
    alone) from the committed full ncu capture, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "k_pairs_cfg2_960x540_ncu.md")
    try:
        text = open(path).read()
    except OSError:
        return None, None
    import re
    m_hash = re.search(r"kernel sources sha256\[:16\]: ([0-9a-f]{16})", text)
    m = re.search(r"thread instruction issue / FP32 lanes: ([0-9.]+) \(FADD, FMUL, FFMA: ([0-9.]+)\)", text)
    if not (m_hash and m) or m_hash.group(1) != kernel_source_hash():
        return None, path
    return (float(m.group(1)), float(m.group(2))), path


def fp32_peak_ops(n_sm: int, mhz: float) -> float:
    """FP32 issue peak: SMs x 128 FP32 lanes x SM clock (one FMA, add, mul or min/max = one op)."""
    return n_sm * 128 * mhz * 1e6


def run_reference(args, rank, world):
    """The oracle (FP64 C, explicit stack, all host cores) timed on bounded samples of the workload."""
    import oracle
    out = {"impl": "reference", "metric": METRIC, "unit": UNIT, "higher_is_better": True}
    if rank != 0:
        return None
    s, r = build_workload(args.width, args.height)
    # diffuse rays of the reference arm come from the oracle's own primary hits
    from oracle.raygen import diffuse_rays
    stride = 8
    sub = r.subset(np.arange(0, r.n, stride))
    o = oracle.intersect(s.P, s.types, sub.soa(), L=8, local=args.boxes == "local")
    d = diffuse_rays(s.P, s.types, sub.soa(), o, seed=1)
    act = d[7] >= d[6]
    dsub = [a[act] for a in d]
    n_step = sub.n + int(act.sum())
    times = []
    threads = 0
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        a = oracle.intersect(s.P, s.types, sub.soa(), L=8, local=args.boxes == "local")
        b = oracle.intersect(s.P, s.types, dsub, L=8, local=args.boxes == "local")
        dt = time.perf_counter() - t0
        threads = a["threads"]
        if k >= args.warmup:
            times.append(dt)
    T = float(np.sum(times))
    value = n_step * args.steps / T / 1e6
    out.update(value=value, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
               ms_per_step=1e3 * T / args.steps, scaling="weak", vs_baseline=None, dtype="f64",
               data="synthetic", config={"workload": WORKLOAD, "boxes": args.boxes,
                                         "sample": f"every {stride}th primary ray "
                                         f"({sub.n}) + its {int(act.sum())} diffuse rays per step"},
               cpu_baseline={"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"every {stride}th primary ray + its diffuse rays, {n_step} rays per step"},
               e2e={"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
    return out


WORKLOAD_BATCHED = ("batched: 32 cube-spheres with 4..64 quads/face (24 n^2 patches each, 1.13M total), 8 frames of "
                    "sinusoidal control-point offsets (amp 0.02), 512x512 primary + diffuse rays per scene, L=8")


def run_batched(args, dev, stream, world):
    """Per frame: update + refit + closest hit of all 32 scenes, as one CUDA-graph replay of the batch
    (one launch per stage over all scenes) versus the same calls scene by scene."""
    import torch
    from paper_1811_03510_gb300 import ccs, scenegen as sg
    sizes = sg.batched_sizes()
    scenes = [sg.make_scene(n, 0.0, name=f"n={n}") for n in sizes]
    one = 2 if args.bvh_width == "both" else int(args.bvh_width)   # batches need one tree per scene
    handles = [ccs.Scene(s.P, s.types, local=args.boxes == "local", bvh_width=one) for s in scenes]
    cam = sg.pinhole_rays(512, 512)
    prim = ccs.rays_to_device(cam.soa(), dev)
    opts = ccs.make_opts(leaf_depth=8)
    rays, hits, n_prim, n_diff = [], [], 0, 0
    for sc in handles:
        hp = ccs.alloc_hits(cam.n, dev)
        ccs.ccs_intersect(sc.handle, prim, cam.n, hp, opts, stream)
        d = ccs.gen_diffuse(sc, prim, hp, seed=1, leaf_depth=8, stream=stream)
        torch.cuda.synchronize()
        act = (d[7] >= d[6]).nonzero().squeeze(1)
        rays.append([torch.cat([p, q.index_select(0, act)]).contiguous() for p, q in zip(prim, d)])
        hits.append(ccs.alloc_hits(int(rays[-1][0].numel()), dev))
        n_prim += cam.n
        n_diff += int(act.numel())
    # frames: deformed control points, a function of the rest position (device, FP32)
    gen = torch.Generator().manual_seed(1)
    w = (torch.rand(3, generator=gen) * 4 + 2).to(dev)
    phi = (torch.rand(3, generator=gen) * 6.283185307179586).to(dev)
    rest = [torch.from_numpy(s.P).to(dev) for s in scenes]
    frames = []
    for f in range(args.frames):
        fr = []
        for P in rest:
            Q = P + 0.02 * torch.sin(w * P + phi + 6.283185307179586 * f / args.frames)
            fr.append([Q[..., c].contiguous().reshape(-1) for c in range(3)])
        frames.append(fr)
    if not args.no_autotune:   # launch options tuned on the largest scene's rays (the batch has no work order)
        big = max(range(len(handles)), key=lambda i: scenes[i].n)
        opts, _, _ = ccs.ccs_autotune(handles[big].handle, rays[big], int(rays[big][0].numel()), hits[big], opts,
                                      reps=2, stream=stream)
        opts.flags &= ~ccs.CCS_TRACE_ORDER
    b = ccs.ccs_batch_create(handles, rays, hits)
    stages = ccs.CCS_BATCH_UPDATE | ccs.CCS_BATCH_REFIT | ccs.CCS_BATCH_INTERSECT
    for i in range(len(handles)):
        ccs.ccs_batch_set_points(b, i, *frames[0][i])
    if not args.no_autotune:
        # the largest scene alone is a smaller launch than the batch: its choice and the same with other
        # refill thresholds are timed on the batch's own frame, and the fastest serves both arms
        cands = [opts] + [ccs.make_opts(**{**ccs.opts_dict(opts), "refill": r}) for r in (8, 24) if r != opts.refill]
        best_t = None
        for c in cands:
            ccs.ccs_batch_capture(b, stages, c)
            ts = []
            for k in range(4):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ccs.ccs_batch_launch(b, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            t = sorted(ts[1:])[1]
            if best_t is None or t < best_t:
                best_t, best_o = t, c
        opts = best_o
    ccs.ccs_batch_capture(b, stages, opts)

    def batched_frame(f):
        for i in range(len(handles)):
            ccs.ccs_batch_set_points(b, i, *frames[f][i])
        ccs.ccs_batch_launch(b, stream)

    def plain_frame(f):
        for i, sc in enumerate(handles):
            ccs.ccs_scene_update_points(sc.handle, *frames[f][i], stream)
            ccs.ccs_bvh_refit(sc.handle, stream)
            ccs.ccs_intersect(sc.handle, rays[i], int(rays[i][0].numel()), hits[i], opts, stream)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    for name, fn in (("plain", plain_frame), ("batched", batched_frame)):
        for k in range(args.warmup):
            fn(k % args.frames)
        torch.cuda.synchronize()
        times = []
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(k % args.frames)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        res[name] = times
        if name == "plain":
            ref = [[h.clone() for h in hh] for hh in hits]
    assert ccs.ccs_batch_sync_status(b, stream) == ccs.CCS_OK
    last = (args.steps - 1) % args.frames
    plain_frame(last)
    torch.cuda.synchronize()
    ref = [[h.clone() for h in hh] for hh in hits]
    batched_frame(last)
    torch.cuda.synchronize()
    identical = all(torch.equal(a, c) for hh, rr in zip(hits, ref) for a, c in zip(hh, rr))
    ccs.ccs_batch_destroy(b)
    for h in handles:
        h.close()
    n_step = n_prim + n_diff
    T_b, T_p = sum(res["batched"]), sum(res["plain"])
    return {"rays_per_frame": n_step, "primary_rays": n_prim, "diffuse_rays": n_diff,
            "batched_mrays_s": n_step * args.steps / T_b / 1e6, "plain_mrays_s": n_step * args.steps / T_p / 1e6,
            "batched_ms_per_frame": 1e3 * T_b / args.steps, "plain_ms_per_frame": 1e3 * T_p / args.steps,
            "speedup": T_p / T_b, "identical_hits": bool(identical),
            "launches_per_frame": {"batched": 1, "plain": 3 * len(handles)},
            "launch_opts": ccs.opts_dict(opts)}


LIGHT = (2.0, 3.0, 4.0)


def run_shadow(args, dev, stream, flush):
    """Shadow rays (Sec. 4: one per path) from the primary hits toward a point light, traced as an any-hit
    query and, for comparison, as a closest-hit query.  The scene is the benchmark sphere plus a 96-patch
    sphere of radius 0.35 between it and the light, so that some rays are occluded."""
    import torch
    from paper_1811_03510_gb300 import ccs, scenegen as sg
    big, small = sg.config_scene(2), sg.config_scene(1)
    ldir = np.array(LIGHT) / np.linalg.norm(LIGHT)
    P = np.concatenate([big.P, (small.P.astype(np.float64) * 0.35 + 1.6 * ldir).astype(np.float32)])
    T = np.concatenate([big.types, small.types])
    sc = ccs.Scene(P, T, local=args.boxes == "local", bvh_width=bvh_arg(args))
    cam = sg.pinhole_rays(args.width, args.height)
    prim = ccs.rays_to_device(cam.soa(), dev)
    hp = ccs.intersect(sc, prim, ccs.make_opts(), stream)
    planes = ccs.gen_shadow(sc, prim, hp, LIGHT, stream=stream)
    torch.cuda.synchronize()
    act = (planes[7] >= planes[6]).nonzero().squeeze(1)
    rays = [p.index_select(0, act).contiguous() for p in planes]
    n = int(act.numel())
    occ = torch.empty(n, dtype=torch.uint8, device=dev)
    hits = ccs.alloc_hits(n, dev)
    out = {"scene": "1536-patch sphere + 96-patch occluder sphere (r 0.35) toward the light", "light": LIGHT,
           "rays": n}
    for name, call in (("any_hit", lambda o: ccs.ccs_occluded(sc.handle, rays, n, occ, o, stream)),
                       ("closest_hit", lambda o: ccs.ccs_intersect(sc.handle, rays, n, hits, o, stream))):
        opts = ccs.make_opts()
        for _ in range(max(3, args.warmup)):
            call(opts)
        tot = 0.0
        for k in range(args.steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call(opts)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        out[name + "_mrays_s"] = n * args.steps / tot / 1e3
    torch.cuda.synchronize()
    g = ccs.hits_to_numpy(hits)
    o = occ.cpu().numpy()
    out["occluded_frac"] = float(o.mean())
    out["identical_to_closest_hit"] = bool(np.array_equal(o.astype(bool), g["pid"] != 0xFFFFFFFF))
    out["speedup"] = out["any_hit_mrays_s"] / out["closest_hit_mrays_s"]
    sc.close()
    return out


def run_screen(args, dev, stream, scene, prim, n_prim, flush, opts_p):
    """Primary rays with screen-space termination (Sec. 3.3) at the camera's pixel size, against the fixed
    leaf depth of the benchmark, on the same rays and launch options.  Both arms run the ray-persistent
    kernel: the pair engine has no screen-space mode, so its flag is cleared for both."""
    import torch
    from paper_1811_03510_gb300 import ccs
    spread = 2.0 * np.tan(np.radians(30.0)) / args.height   # 60 degree vertical field of view
    base = ccs.opts_dict(opts_p)
    base["pairs"] = False
    out = {"pixel_spread": spread, "engine": "ray-persistent (both arms)"}
    hits = ccs.alloc_hits(n_prim, dev)
    for name, sp in (("fixed_depth", 0.0), ("screen_space", spread)):
        opts = ccs.make_opts(**base, pixel_spread=sp)
        for _ in range(max(3, args.warmup)):
            ccs.ccs_intersect(scene.handle, prim, n_prim, hits, opts, stream)
        tot = 0.0
        for k in range(args.steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ccs.ccs_intersect(scene.handle, prim, n_prim, hits, opts, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        c = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device=dev)
        ccs.ccs_intersect(scene.handle, prim, n_prim, hits, ccs.make_opts(**base, pixel_spread=sp, counters=c), stream)
        torch.cuda.synchronize()
        v = dict(zip(ccs.COUNTER_NAMES, c.cpu().tolist()))
        out[name + "_mrays_s"] = n_prim * args.steps / tot / 1e3
        out[name + "_splits"] = v["bezier_splits"] + v["gregory_splits"]
    out["speedup"] = out["screen_space_mrays_s"] / out["fixed_depth_mrays_s"]
    return out


def run_large(args, dev, stream, flush, n_sm):
    """The 393,216-patch cube-sphere (128 x 128 quads per face, noise 0.1, 5 octaves) with 3840 x 2160
    primary rays and the diffuse and mirror generations from their hits (active slots), each tuned, on binary
    and on 4-wide BVHs: MRays/s, the fraction of the FP32 issue peak and BVH nodes per ray (Sec. 4: larger
    models are dominated by the traversal of the hierarchy)."""
    import torch
    from paper_1811_03510_gb300 import ccs, scenegen as sg
    s = sg.config_scene(3)
    cam = sg.pinhole_rays(3840, 2160)
    prim = ccs.rays_to_device(cam.soa(), dev)
    out = {"patches": int(s.n), "primary_rays": cam.n}
    reps = max(3, args.steps // 4)
    for width in (2, 4):
        sc = ccs.Scene(s.P, s.types, local=args.boxes == "local", bvh_width=width)
        hp = ccs.intersect(sc, prim, ccs.make_opts(), stream)
        gens = {"primary": (prim, cam.n, 3840)}
        for name, planes in (("diffuse", ccs.gen_diffuse(sc, prim, hp, seed=1, leaf_depth=8, offset_abs=1e-4,
                                                         stream=stream)),
                             ("mirror", ccs.gen_mirror(sc, prim, hp, leaf_depth=8, offset_abs=1e-4, stream=stream))):
            torch.cuda.synchronize()
            act = (planes[7] >= planes[6]).nonzero().squeeze(1)
            gens[name] = ([p.index_select(0, act).contiguous() for p in planes], int(act.numel()), 0)
        res = {}
        for name, (rays, n, iw) in gens.items():
            h = ccs.alloc_hits(n, dev)
            best, _, _ = ccs.ccs_autotune(sc.handle, rays, n, h, ccs.make_opts(image_width=iw), reps=1, stream=stream)
            for _ in range(2):
                ccs.ccs_intersect(sc.handle, rays, n, h, best, stream)
            tot = 0.0
            for k in range(reps):
                flush.fill_(float(k))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ccs.ccs_intersect(sc.handle, rays, n, h, best, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1) / 1e3
            ops, cc = alg_ops_of(sc, rays, n, h, stream, dev)
            res[name + "_rays"] = n
            res[name + "_mrays_s"] = n * reps / tot / 1e6
            res[name + "_roofline_frac"] = ops * reps / tot / fp32_peak_ops(n_sm, 2070.0)
            res[name + "_bvh_nodes_per_ray"] = cc["bvh_nodes"] / n
            res[name + "_engine"] = engine_of(best)
        out[f"bvh{width}"] = res
        sc.close()
    return out


def alg_ops_of(scene, rays, n, hits, stream, dev) -> tuple:
    """Algorithmic FP32 ops of one launch, from a counting launch of the ray-persistent kernel (binary BVH,
    default options): BVH nodes, Bezier and Gregory splits, the local-frame ray per pair."""
    import torch
    from paper_1811_03510_gb300 import ccs
    c = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device=dev)
    ccs.ccs_intersect(scene.handle, rays, n, hits, ccs.make_opts(leaf_depth=8, counters=c), stream)
    torch.cuda.synchronize()
    v = dict(zip(ccs.COUNTER_NAMES, c.cpu().tolist()))
    ops = (v["bvh_nodes"] * OPS_BVH_NODE + v["bezier_splits"] * OPS_SPLIT_BEZIER + v["gregory_splits"] * OPS_SPLIT_GREGORY
           + (v["pairs"] * OPS_PAIR_FRAME if scene.local else 0))
    return ops, v


def run_world_step(args, dev, stream, s, prim, n_prim, diff, n_diff, flush, n_sm):
    """The benchmark step (the same primary and diffuse rays) on a scene whose sub-domain boxes are in world
    axes, launch options tuned per batch: MRays/s and the fraction of the FP32 issue peak."""
    import torch
    from paper_1811_03510_gb300 import ccs
    sc = ccs.Scene(s.P, s.types, local=False, bvh_width=bvh_arg(args))
    out, ops, t_tot = {}, 0.0, 0.0
    for name, rays, n, width in (("primary", prim, n_prim, args.width), ("diffuse", diff, n_diff, 0)):
        h = ccs.alloc_hits(n, dev)
        best = ccs.make_opts(leaf_depth=8)
        if not args.no_autotune:
            best, _, _ = ccs.ccs_autotune(sc.handle, rays, n, h, ccs.make_opts(leaf_depth=8, image_width=width),
                                          reps=2, stream=stream)
        for _ in range(max(3, args.warmup)):
            ccs.ccs_intersect(sc.handle, rays, n, h, best, stream)
        tot = 0.0
        for k in range(args.steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ccs.ccs_intersect(sc.handle, rays, n, h, best, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1) / 1e3
        o, _ = alg_ops_of(sc, rays, n, h, stream, dev)
        ops += o * args.steps
        t_tot += tot
        out[name + "_mrays_s"] = n * args.steps / tot / 1e6
        out[name + "_engine"] = engine_of(best)
    sc.close()
    out["step_mrays_s"] = (n_prim + n_diff) * args.steps / t_tot / 1e6
    out["roofline_frac"] = ops / t_tot / fp32_peak_ops(n_sm, 2070.0)
    return out


def run_frames(args, dev, stream, s, prim, n_prim, diff, n_diff, flush):
    """The same rays with sub-domain boxes in world axes and in each patch's frame (Sec. 3.4), default
    launch options for both: MRays/s and subdivision steps."""
    import torch
    from paper_1811_03510_gb300 import ccs
    out = {}
    for name, local in (("world", False), ("local", True)):
        sc = ccs.Scene(s.P, s.types, local=local, bvh_width=bvh_arg(args))
        res = {}
        for kind, rays, n in (("primary", prim, n_prim), ("diffuse", diff, n_diff)):
            hits = ccs.alloc_hits(n, dev)
            opts = ccs.make_opts()
            for _ in range(max(3, args.warmup)):
                ccs.ccs_intersect(sc.handle, rays, n, hits, opts, stream)
            tot = 0.0
            for k in range(args.steps):
                flush.fill_(float(k))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ccs.ccs_intersect(sc.handle, rays, n, hits, opts, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            c = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device=dev)
            ccs.ccs_intersect(sc.handle, rays, n, hits, ccs.make_opts(counters=c), stream)
            torch.cuda.synchronize()
            v = dict(zip(ccs.COUNTER_NAMES, c.cpu().tolist()))
            res[kind + "_mrays_s"] = n * args.steps / tot / 1e3
            res[kind + "_splits"] = v["bezier_splits"] + v["gregory_splits"]
            res[kind + "_backtracks"] = v["backtracks"]
        out[name] = res
        sc.close()
    out["speedup_primary"] = out["local"]["primary_mrays_s"] / out["world"]["primary_mrays_s"]
    out["speedup_diffuse"] = out["local"]["diffuse_mrays_s"] / out["world"]["diffuse_mrays_s"]
    return out


def run_learned(args, dev, stream, scene, s, prim, diff, opts_p, opts_d):
    """Train the proposal on traces of scenes with other seeds (GPU export + GPU training), then time the
    learned traversal against the plain one on this workload's primary and diffuse batches."""
    import torch
    from paper_1811_03510_gb300 import ccs, scenegen as sg
    t_setup = time.perf_counter()
    cap = 4_500_000   # 4 M (ray, patch, hit cell) traces to train on, one tenth more held out
    feat = torch.empty(cap, 24, device=dev)
    lab = torch.empty(cap, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    n_tr = 0
    cam = sg.pinhole_rays(args.width, args.height)
    cam_d = ccs.rays_to_device(cam.soa(), dev)
    for seed in range(2, 2 + args.train_seeds):
        st = sg.config_scene(2, seed=seed)
        sct = ccs.Scene(st.P, st.types, local=args.boxes == "local", bvh_width=bvh_arg(args))
        hp = ccs.alloc_hits(cam.n, dev)
        room = cap - n_tr
        if room <= 0:
            break
        ccs.ccs_trace_export(sct.handle, cam_d, cam.n, hp, ccs.make_opts(), feat[n_tr:], lab[n_tr:], room, cnt, stream)
        d = ccs.gen_diffuse(sct, cam_d, hp, seed=seed, stream=stream)
        torch.cuda.synchronize()
        n_tr += min(int(cnt.item()), room)
        act = (d[7] >= d[6]).nonzero().squeeze(1)
        dd = [q.index_select(0, act).contiguous() for q in d]
        room = cap - n_tr
        if room > 0 and act.numel():
            hd = ccs.alloc_hits(int(act.numel()), dev)
            ccs.ccs_trace_export(sct.handle, dd, int(act.numel()), hd, ccs.make_opts(), feat[n_tr:], lab[n_tr:], room,
                                 cnt, stream)
            torch.cuda.synchronize()
            n_tr += min(int(cnt.item()), room)
        sct.close()
    n_val = max(n_tr // 10, 1)
    perm = torch.randperm(n_tr, device=dev, generator=torch.Generator(device=dev).manual_seed(1))
    feat, lab = feat[:n_tr][perm].contiguous(), lab[:n_tr][perm].contiguous()
    prop = ccs.ccs_proposal_create(seed=1)
    B, epochs, lr = 8192, 3, 2e-3
    loss = torch.zeros(1, device=dev)
    n_fit = n_tr - n_val
    steps = 0
    t_train = time.perf_counter()
    for ep in range(epochs):
        for i0 in range(0, n_fit - B + 1, B):
            ccs.ccs_proposal_train_step(prop, feat[n_val + i0:], lab[n_val + i0:], B, lr * (0.5 ** ep), loss, stream)
            steps += 1
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    cells = torch.empty(n_val, dtype=torch.uint8, device=dev)
    ccs.ccs_proposal_infer(prop, feat[:n_val], n_val, None, cells, None, stream)
    torch.cuda.synchronize()
    acc = (cells == lab[:n_val]).float().mean().item()
    t_setup = time.perf_counter() - t_setup
    # timing: plain (tuned) against learned, both on the test seed's batches
    res = {"train_traces": n_tr - n_val, "val_traces": n_val, "train_steps": steps, "train_s": t_train,
           "final_train_loss": loss.item(), "val_top1": acc, "setup_s": t_setup}
    nb = {"primary": (prim, int(prim[0].numel()), opts_p), "diffuse": (diff, int(diff[0].numel()), opts_d)}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    lopts = ccs.make_opts(leaf_depth=8, cache_slots=0)
    for name, (rays, n, op) in nb.items():
        hp, hl = ccs.alloc_hits(n, dev), ccs.alloc_hits(n, dev)
        out = {}
        for label, fn in (("plain", lambda: ccs.ccs_intersect(scene.handle, rays, n, hp, op, stream)),
                          ("learned", lambda: ccs.ccs_intersect_learned(scene.handle, prop, rays, n, hl, lopts, 0.0,
                                                                        stream)),
                          ("learned_conf0.3", lambda: ccs.ccs_intersect_learned(scene.handle, prop, rays, n, hl, lopts,
                                                                                0.3, stream))):
            for _ in range(args.warmup):
                fn()
            ts = []
            for k in range(args.steps):
                flush.fill_(float(k))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            out[label + "_mrays_s"] = n * args.steps / sum(ts) / 1e6
        out["identical_hits"] = bool(all(torch.equal(a, b) for a, b in zip(hp, hl)))
        c_p = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device=dev)
        c_l = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device=dev)
        ccs.ccs_intersect(scene.handle, rays, n, hp, ccs.make_opts(leaf_depth=8, cache_slots=0, counters=c_p), stream)
        ccs.ccs_intersect_learned(scene.handle, prop, rays, n, hl, ccs.make_opts(leaf_depth=8, counters=c_l), 0.0,
                                  stream)
        torch.cuda.synchronize()
        cp, cl = dict(zip(ccs.COUNTER_NAMES, c_p.tolist())), dict(zip(ccs.COUNTER_NAMES, c_l.tolist()))
        out["splits_plain"] = cp["bezier_splits"] + cp["gregory_splits"]
        out["splits_learned"] = cl["bezier_splits"] + cl["gregory_splits"]
        out["backtracks_plain"], out["backtracks_learned"] = cp["backtracks"], cl["backtracks"]
        out["speedup"] = out["learned_mrays_s"] / out["plain_mrays_s"]
        # the most any proposal can gain: the same search started with the final best distance (tmax set to
        # the plain answer's distance, inclusive, so the hits stay the same), plain launch options
        seeded = list(rays)
        seeded[7] = torch.where(hp[3] != -1, hp[0], rays[7]).contiguous()
        hs = ccs.alloc_hits(n, dev)
        ts = []
        for k in range(args.warmup + args.steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ccs.ccs_intersect(scene.handle, seeded, n, hs, op, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= args.warmup:
                ts.append(e0.elapsed_time(e1) / 1e3)
        c_s = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device=dev)
        ccs.ccs_intersect(scene.handle, seeded, n, hs, ccs.make_opts(leaf_depth=8, cache_slots=0, counters=c_s), stream)
        torch.cuda.synchronize()
        cs = dict(zip(ccs.COUNTER_NAMES, c_s.tolist()))
        out["bound_seeded_best"] = {"mrays_s": n * args.steps / sum(ts) / 1e6,
                                    "splits": cs["bezier_splits"] + cs["gregory_splits"],
                                    "identical_hits": bool(all(torch.equal(a, b) for a, b in zip(hp, hs))),
                                    "time_speedup_bound": (n * args.steps / sum(ts) / 1e6) / out["plain_mrays_s"]}
        res[name] = out
    ccs.ccs_proposal_destroy(prop)
    return res


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ccs" else "gloo"
        dist.init_process_group(backend)
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    from paper_1811_03510_gb300 import build_ext, ccs

    torch.cuda.set_device(local)
    build_ext.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    if args.variant == "batched":
        out = run_batched(args, dev, stream, world)
        res = {"metric": METRIC, "value": out["batched_mrays_s"] * world, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["batched_ms_per_frame"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic", "config": {"workload": WORKLOAD_BATCHED, "variant": "batched",
                                               "l2": "flushed (256 MB write) before every timed frame"},
               "batched": out, "gpu_launches": 3 * args.steps}
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    s, r = build_workload(args.width, args.height)
    scene = ccs.Scene(s.P, s.types, local=args.boxes == "local", bvh_width=bvh_arg(args))
    prim = ccs.rays_to_device(r.soa(), dev)
    n_prim = r.n
    opts = ccs.make_opts(leaf_depth=8)
    hits_p = ccs.alloc_hits(n_prim, dev)
    ccs.ccs_intersect(scene.handle, prim, n_prim, hits_p, opts, stream)
    # diffuse generation on the device from the primary hits, compacted to the active slots (setup)
    dplanes = ccs.gen_diffuse(scene, prim, hits_p, seed=1, leaf_depth=8, offset_abs=1e-4, stream=stream)
    torch.cuda.synchronize()
    active = (dplanes[7] >= dplanes[6]).nonzero().squeeze(1)
    diff = [p.index_select(0, active).contiguous() for p in dplanes]
    n_diff = int(active.numel())
    hits_d = ccs.alloc_hits(n_diff, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        ccs.ccs_intersect(scene.handle, prim, n_prim, hits_p, opts_p, stream)
        ccs.ccs_intersect(scene.handle, diff, n_diff, hits_d, opts_d, stream)

    # launch options from the autotuner (answer-preserving knobs), separately for each batch
    tuned = {"primary": opts, "diffuse": opts}
    # the primary batch is an image (the work order may rank its 8 x 8 pixel tiles), the diffuse one is not
    for name, rays, n, h, width in (("primary", prim, n_prim, hits_p, args.width), ("diffuse", diff, n_diff, hits_d, 0)):
        if args.no_autotune:
            break
        if (args.opts_primary if name == "primary" else args.opts_diffuse):
            continue
        best, ms, _ = ccs.ccs_autotune(scene.handle, rays, n, h, ccs.make_opts(leaf_depth=8, image_width=width), reps=2,
                                       stream=stream)
        tuned[name] = best
    for name, arg in (("primary", args.opts_primary), ("diffuse", args.opts_diffuse)):
        if arg:
            tuned[name] = ccs.make_opts(**{"leaf_depth": 8, **json.loads(arg)})
    opts_p, opts_d = tuned["primary"], tuned["diffuse"]

    # algorithmic work per launch from the traversal counters (separate, untimed launches)
    counts = {}
    for name, rays, n, h in (("primary", prim, n_prim, hits_p), ("diffuse", diff, n_diff, hits_d)):
        c = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device=dev)
        ccs.ccs_intersect(scene.handle, rays, n, h, ccs.make_opts(leaf_depth=8, counters=c), stream)
        torch.cuda.synchronize()
        counts[name] = dict(zip(ccs.COUNTER_NAMES, c.cpu().tolist()))
    alg_ops = {k: v["bvh_nodes"] * OPS_BVH_NODE + v["bezier_splits"] * OPS_SPLIT_BEZIER
               + v["gregory_splits"] * OPS_SPLIT_GREGORY + (v["pairs"] * OPS_PAIR_FRAME if scene.local else 0)
               for k, v in counts.items()}
    # schedule of the warps under the chosen options (counting launches of the same configuration)
    sched = {}
    for name, rays, n, h, o in (("primary", prim, n_prim, hits_p, opts_p), ("diffuse", diff, n_diff, hits_d, opts_d)):
        c = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device=dev)
        ccs.ccs_intersect(scene.handle, rays, n, h, ccs.make_opts(**ccs.opts_dict(o), counters=c), stream)
        torch.cuda.synchronize()
        sched[name] = schedule_summary(dict(zip(ccs.COUNTER_NAMES, c.cpu().tolist())), o.lanes_per_ray, engine_of(o))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        ccs.ccs_intersect(scene.handle, prim, n_prim, hits_p, opts_p, stream)
        ev[k][1].record(stream)
        ccs.ccs_intersect(scene.handle, diff, n_diff, hits_d, opts_d, stream)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    t_prim = sum(a.elapsed_time(b) for a, b, _ in ev) / 1e3
    t_diff = sum(b.elapsed_time(c) for _, b, c in ev) / 1e3
    T = t_prim + t_diff
    if world > 1:
        import torch.distributed as dist
        T = max_over_ranks(T, dev)
        dist.barrier()
    st = ccs.ccs_scene_sync_status(scene.handle, stream)
    assert st == ccs.CCS_OK, "traversal limit reached"

    rays_per_step = n_prim + n_diff
    value = whole_job_rate(rays_per_step, args.steps, T, world)

    # the same two batches on two streams at once (each launch takes its own work-queue head): the diffuse
    # launch fills the SMs that the primary launch frees while its last rays finish.  Reported beside
    # the step, not as its value: a renderer overlaps independent batches this way.
    side = torch.cuda.Stream(dev)
    ov = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        side.wait_event(e0)
        ccs.ccs_intersect(scene.handle, prim, n_prim, hits_p, opts_p, stream)
        ccs.ccs_intersect(scene.handle, diff, n_diff, hits_d, opts_d, side)
        stream.wait_stream(side)
        e1.record(stream)
        torch.cuda.synchronize()
        ov.append(e0.elapsed_time(e1) / 1e3)
    overlapped = whole_job_rate(rays_per_step, args.steps, max_over_ranks(sum(ov), dev), world)

    # end to end through the host-buffer entry point: pinned host rays in, hits out, every step
    # each batch's ray planes are the rows of one pinned block, and so are its hit planes
    host_p = list(torch.stack([p.cpu() for p in prim]).pin_memory())
    host_d = list(torch.stack([p.cpu() for p in diff]).pin_memory())
    out_p = list(torch.empty(4, n_prim, dtype=torch.float32).pin_memory())
    out_d = list(torch.empty(4, n_diff, dtype=torch.float32).pin_memory())
    # (one pipeline: both batches through ccs_intersect_host_batches, the diffuse batch's copies and
    # launches overlapping the end of the primary one; staged: one ccs_intersect_host call per batch, copies
    # through device buffers in chunks overlapping the traversal; mapped: one call per batch, the launch
    # reads rays and writes hits through the page-locked memory's device mapping)
    # (the plane pointers go into the C structs once, as a caller that traces the same buffers every frame
    # would keep them)
    rs_p, rs_d = ccs.rays_struct(host_p), ccs.rays_struct(host_d)
    hs_p, hs_d = ccs.hits_struct(out_p), ccs.hits_struct(out_d)
    e2e = {}
    for name, mapped, one in (("one_pipeline", False, True), ("staged_copies", False, False), ("mapped", True, False)):
        op = ccs.make_opts(**ccs.opts_dict(opts_p), host_mapped=mapped)
        od = ccs.make_opts(**ccs.opts_dict(opts_d), host_mapped=mapped)

        def step():
            if one:
                ccs.ccs_intersect_host_batches(scene.handle, [rs_p, rs_d], [n_prim, n_diff], [hs_p, hs_d],
                                               [op, od], stream)
            else:
                ccs.ccs_intersect_host(scene.handle, rs_p, n_prim, hs_p, op, stream)
                ccs.ccs_intersect_host(scene.handle, rs_d, n_diff, hs_d, od, stream)
        for _ in range(2):
            step()
        te = []
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step()
            te.append(time.perf_counter() - t0)
        e2e[name] = whole_job_rate(rays_per_step, args.steps, max_over_ranks(sum(te), dev), world)
        # the host path gives the device-resident step's hits, bit for bit
        for outs, dev_h in ((out_p, hits_p), (out_d, hits_d)):
            for a, b in zip(outs, dev_h):
                assert torch.equal(a.view(torch.int32), b.cpu().view(torch.int32)), f"{name}: hits differ"
    e2e_value = e2e["one_pipeline"]

    # the same step with the sub-domain boxes in world axes (Algorithm 3 as printed, without Sec. 3.4's local
    # frames), tuned the same way: the plain method's own rate and roofline fraction beside the headline
    world_step = None
    if scene.local and args.variant == "all":
        world_step = run_world_step(args, dev, stream, s, prim, n_prim, diff, n_diff, flush, n_sm)

    traffic, traffic_src = measured_traffic()
    issue, issue_src = measured_issue()
    share, share_src = measured_share()
    # the dominant kernel alone: the subdivision steps (Bezier and Gregory splits, the local-frame ray per
    # pair) over its share of the event-timed step, when the pair engine runs both batches
    kernel_roof = None
    if share and engine_of(opts_p) == "pairs" and engine_of(opts_d) == "pairs":
        ops_k = sum(v["bezier_splits"] * OPS_SPLIT_BEZIER + v["gregory_splits"] * OPS_SPLIT_GREGORY
                    + (v["pairs"] * OPS_PAIR_FRAME if scene.local else 0) for v in counts.values())
        t_k = share * T / args.steps
        kernel_roof = {"kernel": "k_pairs (subdivision pass, primary + diffuse)", "achieved": ops_k / t_k / 1e12,
                       "frac": ops_k / t_k / fp32_peak_ops(n_sm, 2070.0), "unit": "Top/s (FP32)",
                       "time_share": share, "share_source": os.path.relpath(share_src, ROOT),
                       "per": "its algorithmic ops over its share (ncu launch list) of the event-timed step"}
    peak_max = fp32_peak_ops(n_sm, 2070.0)
    ops_step = alg_ops["primary"] + alg_ops["diffuse"]
    achieved = ops_step * args.steps / T
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "primary_rays": n_prim, "diffuse_rays": n_diff, "leaf_depth": 8,
                   "boxes": ("local frames (Sec. 3.4)" if scene.local else "world axes"),
                   "bvh_width": args.bvh_width,
                   "variant": args.variant, "l2": "flushed (256 MB write) before every timed step",
                   "launch_opts": {"primary": ccs.opts_dict(opts_p), "diffuse": ccs.opts_dict(opts_d),
                                   "chosen_by": "given" if (args.opts_primary or args.opts_diffuse) else
                                   "defaults" if args.no_autotune else "ccs_autotune (answer-preserving knobs)"},
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "overlapped_batches_mrays_s": overlapped,
        "primary_mrays_s": n_prim * args.steps / t_prim / 1e6,
        "diffuse_mrays_s": n_diff * args.steps / t_diff / 1e6,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_max / 1e12, "unit": "Top/s (FP32)",
                     "frac": achieved / peak_max,
                     "traffic": (traffic[0] + traffic[1]) / 2 if traffic else None,
                     "per": "step (both batches, every kernel of the chosen engines, event-timed)",
                     "note": "algorithmic FP32 ops (BVH node 34, Bezier split 360, Gregory split 1490, local-frame "
                             "ray 24 per pair) / event-timed step time; peak = SMs x 128 lanes x 2070 MHz "
                             "(nominal FP32 issue; no FP32 figure in the measured peaks)",
                     "op_counts": "work counters of a counting launch of the ray-persistent kernel on the binary "
                                  "BVH with default options: the method's work with best-distance pruning (the "
                                  "pair engine's candidate pass visits more BVH nodes, not credited)",
                     "traffic_per": "launch of the dominant kernel (the pair engine's subdivision pass), mean of "
                                    "the primary and diffuse batches",
                     "traffic_source": ({"file": os.path.relpath(traffic_src, ROOT), "kernel_sources_sha16":
                                         kernel_source_hash(), "matches": bool(traffic)} if traffic_src else None),
                     "algorithmic_bytes_per_launch": 48 * rays_per_step / 2,
                     "frac_at_measured_clock": (achieved / fp32_peak_ops(n_sm, ck["sm_mhz"])) if ck["sm_mhz"] else None,
                     "dominant_kernel": kernel_roof,
                     "issue_frac_ncu": ({"all_instructions": issue[0], "fadd_fmul_ffma": issue[1],
                                         "source": os.path.relpath(issue_src, ROOT),
                                         "kernel_sources_sha16": kernel_source_hash(),
                                         "per": "thread instructions per cycle / (SMs x 128 lanes), the dominant "
                                                "kernel of one 960x540 primary launch under ncu"} if issue else None)},
        "world_axes": world_step,
        "counters": counts,
        "schedule": sched,
        "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"],
                   "samples": ck["samples"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 32 * rays_per_step,
                "d2h_bytes_per_step": 16 * rays_per_step,
                "transfer": "ccs_intersect_host_batches on page-locked planes: both batches through one pipeline "
                            "of copies staged through device buffers in chunks that overlap the traversal; wall "
                            "clock per step including the call's synchronisation",
                "separate_calls_value": e2e["staged_copies"], "mapped_value": e2e["mapped"]},
        # this library's kernels per step: the pair engine's four, the work order's three and k_intersect, or
        # k_intersect alone, per batch as the tuner chose
        "gpu_launches": args.steps * sum(kernels_per_launch(o) for o in (opts_p, opts_d)),
        "engine": {"primary": engine_of(opts_p), "diffuse": engine_of(opts_d)},
    }
    if args.variant in ("all", "learned"):
        res["learned"] = run_learned(args, dev, stream, scene, s, prim, diff, opts_p, opts_d)
    if args.variant == "all":
        b = run_batched(args, dev, stream, world)
        res["batched"] = b
        res["shadow"] = run_shadow(args, dev, stream, flush)
        res["screen_space"] = run_screen(args, dev, stream, scene, prim, n_prim, flush, opts_p)
        res["frames"] = run_frames(args, dev, stream, s, prim, n_prim, diff, n_diff, flush)
        res["large_scene"] = run_large(args, dev, stream, flush, n_sm)
    if rank == 0 and not args.no_cpu_baseline:
        # the FP64 oracle on all host cores over the same step, repeated until about 10 s of CPU work
        import oracle
        dh = [p.cpu().numpy() for p in diff]
        loc = args.boxes == "local"
        reps, t0 = 0, time.perf_counter()
        while True:
            o = oracle.intersect(s.P, s.types, r.soa(), L=8, local=loc)
            oracle.intersect(s.P, s.types, dh, L=8, local=loc)
            reps += 1
            dt = time.perf_counter() - t0
            if dt >= 10.0:
                break
        res["cpu_baseline"] = {"value": reps * rays_per_step / dt / 1e6, "unit": UNIT, "cores": o["threads"],
                               "kind": "oracle", "sample": f"the full step ({n_prim} primary + {n_diff} diffuse rays), "
                               f"{reps} times, FP64 oracle, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(res), flush=True)
    scene.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
