#!/usr/bin/env python
"""Frame benchmark of the GB300 ray tracer.

One step = one frame of the medium workload (64 instances of 4 procedural
meshes, 157,964 unique triangles, 1920x1080, 4 point lights, max depth 4):
seeded per-instance motion, a full TLAS rebuild (float64 instance inverses,
Arvo boxes, Morton codes, radix sort, Karras hierarchy, refit), then the
Whitted render (ray generation, closest-hit traversal, shading and queue
compaction, any-hit shadow traversal with accumulation) into an RGBA32F
image.  The four BLAS are built once per scene (their build time is reported
in config.blas_build_ms).

value  = traced rays (closest-hit + shadow) per second over all ranks, inputs
         resident in HBM, L2 flushed (256 MiB write) before every timed frame.
e2e    = the same frames with the instance transforms copied host->device from
         pinned memory and the image copied back to pinned memory, inside the
         timed region.
--impl reference runs the float64 CPU oracle on the same frames.

Multi-GPU (torchrun): replicas, each rank renders its own frames; value is
the sum of all ranks' rays over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenegen as g  # noqa: E402

METRIC = "Mrays/s closest-hit at 1 GB300 vs plain path & oracle; p50/p99 frame latency"
WORKLOAD = ("medium: 64 instances of 4 procedural meshes (UV sphere 80x40, icosphere s5, cube, 256^2 heightfield; "
            "157,964 unique tris) with seeded affine transforms in a 100^3 box, materials diffuse/mirror/glass "
            "60/20/20%, 4 point lights, 1920x1080, max_depth 4; per frame seeded motion + full TLAS rebuild + render")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU baseline budget (wall seconds)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--compressed", action="store_true",
                   help="trace with the compressed 8-wide BVH (default: the float32 binary BVH, faster here)")
    p.add_argument("--workload", default="medium", choices=["medium", "large", "serve"],
                   help="medium: the render frame (default); large: incoherent closest/any-hit queries; "
                        "serve: the continuous-batching render server alone")
    p.add_argument("--requests", type=int, default=400, help="serving: requests in the Poisson stream")
    p.add_argument("--no-serving", action="store_true", help="medium: skip the serving measurement")
    p.add_argument("--inflight", type=int, default=4,
                   help="medium: frames in flight (scene contexts sharing the BLAS, one stream each)")
    p.add_argument("--no-pair", action="store_true",
                   help="trace each level's (server: step's) shadow rays and the next one's closest-hit rays in separate launches")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------- clocks

REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    """nvidia-smi samples every 50 ms during the timed region."""

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="rg_clocks_", suffix=".csv")
        os.close(fd)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        with open(self.path) as f:
            out = summarize_clocks(f)
        os.unlink(self.path)
        return out


def summarize_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen Active
    in nvidia-smi CSV lines (clocks.sm, clocks.max.sm, power.draw, active
    mask, then the four reasons); malformed lines are skipped, None if none
    is left."""
    sm, smax, reasons = [], [], set()
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 8:
            continue
        try:
            sm.append(float(f[0]))
            smax.append(float(f[1]))
        except ValueError:
            continue
        for name, v in zip(REASONS, f[4:8]):
            if v.lower() == "active":
                reasons.add(name)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


# ---------------------------------------------------------------- helpers

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def code_sha(*paths):
    """Hash of source files' code: // comments, trailing spaces and blank
    lines removed (a comment edit leaves the kernels, and their counters, as
    they were)."""
    lines = []
    for path in paths:
        for line in open(path).read().splitlines():
            code = re.sub(r"//.*$", "", line).rstrip()
            if code.strip():
                lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


TRAVERSAL_SOURCES = [os.path.join(ROOT, "paper_2001_09792_gb300", "csrc", f)
                     for f in ("traverse.cuh", "trace.cu", "api.cu")]


def traffic_record():
    """DRAM bytes per traversal launch of the medium frame (the frame's
    closest-hit, pair and shadow launches, averaged) from the committed ncu
    summary, valid only while the traversal code (traverse.cuh, trace.cu) and
    the launch sequence of a frame (api.cu) are unchanged."""
    path = os.path.join(ROOT, "profiles", "trace_pair_medium.md")
    try:
        txt = open(path).read()
        sha = code_sha(*TRAVERSAL_SOURCES)
        m = re.search(r"dram_bytes_per_traversal_launch:\s*([0-9.]+)", txt)
        s = re.search(r"traversal_code_sha256_16:\s*([0-9a-f]+)", txt)
        if m and s and s.group(1) == sha:
            return float(m.group(1))
    except OSError:
        pass
    return None


def l2_record(compressed):
    """L2 figures of one traversal launch of the medium frame, read from the
    committed ncu summary (a capture, not measured by this run): L2 and L1
    sector hit rates and, for the binary BVH, L2 throughput in % of peak."""
    name = "trace8_medium.md" if compressed else "trace_pair_medium.md"
    try:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    m = re.search(r"^\| L2 / L1 sector hit rate \| ([0-9.]+) % / ([0-9.]+) %", txt, flags=re.M)
    if not m:
        return None
    out = {"l2_sector_hit_pct": float(m.group(1)), "l1_sector_hit_pct": float(m.group(2))}
    t = re.search(r"^\| L2 \(lts\) throughput, % of peak \| ([0-9.]+) %", txt, flags=re.M)
    if t:
        out["l2_throughput_pct_of_peak"] = float(t.group(1))
    out["source"] = f"ncu capture of one traversal launch (profiles/{name}), not this run"
    return out


def path_flag(args):
    import paper_2001_09792_gb300 as rg
    return ((rg.RG_SCENE_COMPRESSED if args.compressed else 0)
            | (rg.RG_SCENE_NO_PAIR if getattr(args, "no_pair", False) else 0))


def node_bytes(args):
    return 80 if args.compressed else 64


def kernel_name(args, where):
    if where == "render":
        return ("k_trace8 closest-hit and any-hit, compressed 8-wide BVH (render)" if args.compressed
                else "k_trace_warp / k_trace_pair closest-hit and any-hit, binary float32 BVH (render)")
    return (f"k_trace8 closest-hit, compressed 8-wide BVH ({where})" if args.compressed
            else f"k_trace closest-hit, binary float32 BVH ({where})")


def frame_motions(scene, n):
    return [g.motion(scene.M, k) for k in range(n)]


# ---------------------------------------------------------------- native arm

def run_native(args, world, rank, local):
    import torch
    import paper_2001_09792_gb300 as rg
    from paper_2001_09792_gb300 import _build

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()

    s = g.medium_scene()
    W, H, D = s.width, s.height, s.max_depth
    n_frames = args.warmup + args.steps
    motions = frame_motions(s, n_frames)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gs = rg.GpuScene(s, flags=rg.RG_SCENE_TIMING | path_flag(args))
    torch.cuda.synchronize()
    blas_build_ms = (time.perf_counter() - t0) * 1e3  # four BLAS + first TLAS, host-timed incl. uploads
    blas_build = blas_build_rate(s)
    blas_ids = [gs.blas[m] for m in s.mesh_id]
    inst_host = [rg.pack_instances(M, blas_ids, s.material_id) for M in motions]
    inst_dev = [torch.from_numpy(x).cuda() for x in inst_host]
    img = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > 129 MB L2
    cam = rg.make_camera(s.camera)
    stream = torch.cuda.current_stream()

    # F frame contexts over the same BLAS (rg_scene_create_shared), one stream
    # each: frame k renders on context k mod F, so the next frame's first,
    # throughput-bound levels fill the latency-bound last levels of the one
    # before it
    F = max(1, args.inflight)
    ctxs = [gs] + [gs.shared() for _ in range(F - 1)]
    streams = [stream] + [torch.cuda.Stream() for _ in range(F - 1)]
    imgs_f = [img] + [torch.empty_like(img) for _ in range(F - 1)]

    def frame(q, k):
        st_q = streams[q]
        with torch.cuda.stream(st_q):
            rg.rg_tlas_build(ctxs[q].h, inst_dev[k], stream=st_q)
            rg.rg_render(ctxs[q].h, cam, W, H, D, out=imgs_f[q], stream=st_q)

    for k in range(args.warmup):
        for q in range(F):
            frame(q, k)
    torch.cuda.synchronize()

    # algorithmic work per closest-hit ray: one counting frame on a second scene
    with rg.GpuScene(s, flags=rg.RG_SCENE_COUNT | path_flag(args)) as gc:
        rg.rg_tlas_build(gc.h, torch.from_numpy(inst_host[args.warmup]).cuda())
        rg.rg_reset_stats(gc.h)
        rg.rg_render(gc.h, cam, W, H, D)
        cst = rg.rg_get_stats(gc.h)

    def timed(nf):
        """args.steps frames, nf in flight; the L2 flush (on the frame's
        stream) before each frame is inside the one timed region.  Returns
        rays, wall seconds, per-frame ms (its stream, flush excluded) and the
        contexts' statistics."""
        for c in ctxs[:nf]:
            rg.rg_sync(c.h)
            rg.rg_reset_stats(c.h)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e_start = torch.cuda.Event(enable_timing=True)
        e_end = torch.cuda.Event(enable_timing=True)
        e_start.record(stream)
        for q in range(1, nf):
            streams[q].wait_event(e_start)
        per = []
        for k in range(args.warmup, n_frames):
            q = (k - args.warmup) % nf
            with torch.cuda.stream(streams[q]):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(streams[q])
                frame(q, k)
                e1.record(streams[q])
            per.append((e0, e1))
        for q in range(1, nf):
            stream.wait_stream(streams[q])
        e_end.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        stats = [rg.rg_get_stats(c.h) for c in ctxs[:nf]]
        rays = sum(x["closest_rays"] + x["shadow_rays"] for x in stats)
        return rays, e_start.elapsed_time(e_end) / 1e3, [a.elapsed_time(b) for a, b in per], stats

    clocks = ClockSampler(gpu_index(local))
    clocks.start()
    for k in range(args.warmup):             # settle after the sampler starts
        for q in range(F):
            frame(q, k)
    torch.cuda.synchronize()
    # one frame at a time (also the kernels' roofline); the first such pass of a
    # process has measured slow at times, so it runs twice and the second counts
    timed(1)
    rays1, wall1, ms, stats1 = timed(1)
    if F > 1:
        rays, total_s, ms_f, stats_f = timed(F)
    else:
        rays, total_s, ms_f, stats_f = rays1, wall1, ms, stats1
    clk = clocks.stop()
    st = stats1[0]

    # FXAA of the frame (Sec. 2.1 post-processing), timed alone, L2 flushed before each launch
    fx_out = torch.empty_like(img)
    fx_ms = []
    for k in range(23):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rg.rg_fxaa(img, out=fx_out)
        e1.record(stream)
        if k >= 3:
            fx_ms.append((e0, e1))
    torch.cuda.synchronize()
    fxaa_ms = statistics.median(a.elapsed_time(b) for a, b in fx_ms)

    # e2e: host instance transforms in, host image out, through the same calls;
    # frames back to back with the readback of frame k overlapping frame k+1
    # (two device images, a copy stream), timed as one region from the first
    # copy-in to the last readback, the L2 flush before each frame included
    e2e = None
    if not args.no_e2e:
        pin_in = [torch.from_numpy(x).pin_memory() for x in inst_host]
        nb = max(F, 2)
        pin_out = [torch.empty((H, W, 4), dtype=torch.float32).pin_memory() for _ in range(nb)]
        out_dev = imgs_f + [torch.empty_like(img) for _ in range(nb - F)]
        dev_in = [torch.empty_like(inst_dev[0]) for _ in range(F)]
        copy_stream = torch.cuda.Stream()
        freed = [None] * nb
        for c in ctxs:
            rg.rg_sync(c.h)
            rg.rg_reset_stats(c.h)
        torch.cuda.synchronize()
        e_start = torch.cuda.Event(enable_timing=True)
        e_end = torch.cuda.Event(enable_timing=True)
        e_start.record(stream)
        for q in range(1, F):
            streams[q].wait_event(e_start)
        for k in range(args.warmup, n_frames):
            q = (k - args.warmup) % F          # context and stream
            b = (k - args.warmup) % nb         # device image and pinned readback buffer
            st_q = streams[q]
            if freed[b] is not None:
                st_q.wait_event(freed[b])      # image b's previous readback is done
            with torch.cuda.stream(st_q):
                flush.zero_()
                dev_in[q].copy_(pin_in[k], non_blocking=True)
                rg.rg_tlas_build(ctxs[q].h, dev_in[q], stream=st_q)
                rg.rg_render(ctxs[q].h, cam, W, H, D, out=out_dev[b], stream=st_q)
                rendered = torch.cuda.Event()
                rendered.record(st_q)
            copy_stream.wait_event(rendered)
            with torch.cuda.stream(copy_stream):
                pin_out[b].copy_(out_dev[b], non_blocking=True)
                freed[b] = torch.cuda.Event()
                freed[b].record(copy_stream)
        for q in range(1, F):
            stream.wait_stream(streams[q])
        stream.wait_stream(copy_stream)
        e_end.record(stream)
        torch.cuda.synchronize()
        e2e_rays = sum(rg.rg_get_stats(c.h)["closest_rays"] + rg.rg_get_stats(c.h)["shadow_rays"] for c in ctxs)
        e2e = (e2e_rays, e_start.elapsed_time(e_end) / 1e3, inst_host[0].nbytes, W * H * 16)

    # aggregate over ranks: the slowest rank's time, every rank's rays
    (total_s_all, e2e_s_all), (rays_all, e2e_rays_all) = reduce_over_ranks(
        [total_s, e2e[1] if e2e else 0.0], [float(rays), float(e2e[0]) if e2e else 0.0], "cuda")
    if e2e:
        e2e = (e2e_rays_all, e2e_s_all, e2e[2], e2e[3])

    if rank == 0:
        peak, peak_kind = measured_peaks()
        # the traversal launches of the timed frames (closest-hit alone for the
        # camera rays, shadow + next level's closest-hit pairs, shadow alone for
        # the last level): the algorithmic bytes of all their rays over their
        # summed device time
        cr, sr = max(cst["closest_rays"], 1), max(cst["shadow_rays"], 1)
        nb = node_bytes(args)
        bytes_per_ray = 32 + 16 + nb * cst["node_visits"] / cr + 48 * cst["tri_tests"] / cr + 80 * cst["inst_entries"] / cr
        bytes_per_shadow = (32 + 16 + nb * cst["any_node_visits"] / sr + 48 * cst["any_tri_tests"] / sr
                            + 80 * cst["any_inst_entries"] / sr)
        trav_ms = st["trace_ms"] + st["any_ms"] + st["pair_ms"]
        trav_launches = max(st["trace_launches"] + st["any_launches"] + st["pair_launches"], 1)
        trav_bytes = bytes_per_ray * st["closest_rays"] + bytes_per_shadow * st["shadow_rays"]
        launch_ms = trav_ms / trav_launches
        rays_per_launch = (st["closest_rays"] + st["shadow_rays"]) / trav_launches
        achieved = trav_bytes / trav_launches / (launch_ms / 1e3) / 1e9
        tr = None if args.compressed else traffic_record()
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": None if tr is None else round(tr),
                    "kernel": kernel_name(args, "render"), "peak_kind": peak_kind,
                    "algorithmic_bytes_per_launch": round(trav_bytes / trav_launches),
                    "algorithmic_bytes_per_closest_ray": round(bytes_per_ray, 1),
                    "algorithmic_bytes_per_shadow_ray": round(bytes_per_shadow, 1),
                    "launches_per_frame": round(trav_launches / args.steps, 2),
                    "nodes_per_ray": round(cst["node_visits"] / cr, 2), "tris_per_ray": round(cst["tri_tests"] / cr, 2),
                    "inst_per_ray": round(cst["inst_entries"] / cr, 3), "avg_launch_ms": round(launch_ms, 4),
                    "traversal_share_of_frame": round(trav_ms / sum(ms), 3),
                    "shares": {"closest_alone": round(st["trace_ms"] / sum(ms), 3),
                               "shadow_closest_pairs": round(st["pair_ms"] / sum(ms), 3),
                               "shadow_alone": round(st["any_ms"] / sum(ms), 3)},
                    "shadow_nodes_per_ray": round(cst["any_node_visits"] / sr, 2),
                    "shadow_inst_per_ray": round(cst["any_inst_entries"] / sr, 3),
                    "shadow_tris_per_ray": round(cst["any_tri_tests"] / sr, 2),
                    "l2": l2_record(args.compressed)}
        def pcts(x):
            xs = sorted(x)
            return round(xs[len(xs) // 2], 3), round(xs[min(len(xs) - 1, math.ceil(0.99 * len(xs)) - 1)], 3)
        p50, p99 = pcts(ms_f)
        p50_1, p99_1 = pcts(ms)
        out = {
            "metric": METRIC,
            "value": round(rays_all / total_s_all / 1e6, 2),
            "unit": "Mrays/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(total_s_all * 1e3 / args.steps, 3),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic (seeded procedural scene, random-free shading)",
            "config": {"workload": WORKLOAD, "width": W, "height": H, "max_depth": D, "lights": 4,
                       "instances": s.n_instances, "instanced_tris": s.instanced_tris(),
                       "rays_per_step": round(rays / args.steps), "closest_rays_per_step": round(st["closest_rays"] / args.steps),
                       "shadow_rays_per_step": round(st["shadow_rays"] / args.steps),
                       "closest_mrays_s": round(st["closest_rays"] / max(rays1, 1) * rays / total_s / 1e6, 2),
                       "frames_in_flight": F,
                       "p50_ms": p50, "p99_ms": p99,
                       "one_in_flight": {"value": round(rays1 / wall1 / 1e6, 2), "ms_per_step": round(wall1 * 1e3 / args.steps, 3),
                                         "p50_ms": p50_1, "p99_ms": p99_1,
                                         "note": "the same frames one at a time; the roofline's launch times are taken here"},
                       "latency": "per frame, from its TLAS build to its image on its stream (with frames in flight, "
                                  "the frames share the GPU)",
                       "blas_build_ms": round(blas_build_ms, 2), "blas_build": blas_build,
                       "l2": "flushed before each frame (256 MiB write on the frame's stream, inside the timed region)",
                       "fxaa": {"ms": round(fxaa_ms, 4), "gbs": round(W * H * 32 / (fxaa_ms / 1e3) / 1e9, 1),
                                "bytes_per_pixel": 32, "note": "k_fxaa_luma + k_fxaa on the frame, timed alone, not in the step"},
                       "parallelism": f"replicas x{world}", "bvh": "compressed 8-wide" if args.compressed else "binary float32"},
            "roofline": roofline,
            "gpu_launches": int(stats_f[0]["kernel_launches"]),
        }
        if clk:
            out["clocks"] = clk
        if e2e:
            out["e2e"] = {"value": round(e2e[0] / e2e[1] / 1e6, 2), "unit": "Mrays/s",
                          "h2d_bytes_per_step": int(e2e[2]), "d2h_bytes_per_step": int(e2e[3]),
                          "note": f"frames back to back, {F} in flight (one scene context and stream each), "
                                  "each image read back on a copy stream while later frames render; one timed "
                                  "region incl. L2 flushes"}
        if world == 1 and not args.no_serving:
            out["serving"] = run_serving(args.requests, pair=not args.no_pair)
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(s, motions[args.warmup:], args.cpu_seconds)
        print(json.dumps(out), flush=True)
    gs.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


SERVE_WORKLOAD = ("serve: Poisson arrivals at 200 req/s over 8 resident scenes (the tiny scene + 7 medium-style "
                  "scenes), resolution uniform over 320x240 / 640x480 / 1280x720 / 1920x1080 / 3840x2160, max_depth "
                  "uniform 1..8, seeded per-request instance motion (per-request TLAS refit)")


def pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, math.ceil(q * len(xs)) - 1))]


def run_serving(n_requests, admit_rays=0, pair=True):
    """The request stream through the continuous-batching server in real time,
    then the same stream one request at a time (rg_tlas_refit + rg_render each,
    in arrival order, against the same arrival clock).  Latency = arrival to
    the completion of the image on the device (host clock)."""
    import torch
    import paper_2001_09792_gb300 as rg

    scenes = g.serving_scenes()
    reqs = g.serving_requests(n_requests)
    gss = [rg.GpuScene(sc, flags=0 if pair else rg.RG_SCENE_NO_PAIR) for sc in scenes]
    trans = [g.motion(scenes[q["scene"]].M, q["motion_seed"]) for q in reqs]
    cams = [rg.make_camera(sc.camera) for sc in scenes]
    srv = rg.rg_server_create(admit_rays=admit_rays, flags=0 if pair else rg.RG_SERVER_NO_PAIR)
    try:
        for gsc in gss:
            rg.rg_server_add_scene(srv, gsc.h)
        scratch = torch.empty((1080, 1920, 4), device="cuda")
        cache = os.environ.get("RG_TUNE_CACHE", os.path.join(tempfile.gettempdir(), "rg_tuned_shapes.json"))
        tuned = rg.rg_server_autotune(srv, 1, scenes[1].camera, 1920, 1080, 4, scratch, cache_path=cache)
        del scratch
        # warm-up: one request of each scene through the server (graph captures)
        for k in range(len(scenes)):
            img = torch.empty((240, 320, 4), device="cuda")
            rg.rg_server_submit(srv, k, cams[k], 320, 240, 4, img)
            rg.rg_server_drain(srv)
        rg.rg_server_poll(srv, 64)
        base = rg.rg_server_get_stats(srv)
        torch.cuda.synchronize()
        imgs, lat, busy = {}, [], 0.0
        nxt = 0
        t0 = time.perf_counter()
        t_first = reqs[0]["arrival"]
        while len(lat) < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt]["arrival"] <= now:
                q = reqs[nxt]
                imgs[nxt] = torch.empty((q["height"], q["width"], 4), device="cuda")
                rg.rg_server_submit(srv, q["scene"], cams[q["scene"]], q["width"], q["height"], q["max_depth"],
                                    imgs[nxt], trans[nxt], tag=nxt)
                nxt += 1
            st = rg.rg_server_get_stats(srv)
            if st["active"] == 0 and st["pending"] == 0:
                time.sleep(max(0.0, reqs[nxt]["arrival"] - (time.perf_counter() - t0)))
                continue
            a = time.perf_counter()
            rg.rg_server_step(srv)
            b = time.perf_counter()
            busy += b - a
            for c in rg.rg_server_poll(srv, 256):
                lat.append(b - t0 - reqs[c["tag"]]["arrival"])
                del imgs[c["tag"]]
        t_end = time.perf_counter() - t0
        st = rg.rg_server_get_stats(srv)
        rays = (st["closest_rays"] - base["closest_rays"]) + (st["shadow_rays"] - base["shadow_rays"])
        steps = st["steps"] - base["steps"]
    finally:
        rg.rg_server_destroy(srv)

    # one request at a time through the plain path, against the same arrival clock
    for gsc in gss:
        rg.rg_reset_stats(gsc.h)
    seq_lat, seq_busy = [], 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, q in enumerate(reqs):
        wait = q["arrival"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        gsc = gss[q["scene"]]
        out = torch.empty((q["height"], q["width"], 4), device="cuda")
        a = time.perf_counter()
        gsc.refit(trans[k])
        rg.rg_render(gsc.h, cams[q["scene"]], q["width"], q["height"], q["max_depth"], out=out)
        torch.cuda.synchronize()
        b = time.perf_counter()
        seq_busy += b - a
        seq_lat.append(b - t0 - q["arrival"])
        del out
    seq_end = time.perf_counter() - t0
    seq_rays = 0
    for gsc in gss:
        s2 = rg.rg_get_stats(gsc.h)
        seq_rays += s2["closest_rays"] + s2["shadow_rays"]
        gsc.close()
    return {
        "workload": SERVE_WORKLOAD, "requests": len(reqs),
        "offered_req_s": round(len(reqs) / (reqs[-1]["arrival"] - t_first + 1e-9), 1),
        "p50_ms": round(pct(lat, 0.50) * 1e3, 2), "p99_ms": round(pct(lat, 0.99) * 1e3, 2),
        "mrays_s": round(rays / (t_end - t_first) / 1e6, 2), "busy_mrays_s": round(rays / busy / 1e6, 2),
        "rays": int(rays), "steps": int(steps), "ring_peak": int(st["ring_peak"]),
        "shapes": tuned,
        "one_at_a_time": {"p50_ms": round(pct(seq_lat, 0.50) * 1e3, 2), "p99_ms": round(pct(seq_lat, 0.99) * 1e3, 2),
                          "busy_mrays_s": round(seq_rays / seq_busy / 1e6, 2),
                          "mrays_s": round(seq_rays / (seq_end - t_first) / 1e6, 2), "rays": int(seq_rays)},
        "latency": "arrival to completion of the image on the device (host clock)",
    }


def reduce_over_ranks(max_vals, sum_vals, device):
    """MAX-reduce `max_vals` and SUM-reduce `sum_vals` over the ranks of the
    default process group (identity when there is none or one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(max_vals), list(sum_vals)
    t_max = torch.tensor(list(max_vals), dtype=torch.float64, device=device)
    t_sum = torch.tensor(list(sum_vals), dtype=torch.float64, device=device)
    dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    dist.all_reduce(t_sum, op=dist.ReduceOp.SUM)
    return t_max.tolist(), t_sum.tolist()


def gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        parts = [p.strip() for p in vis.split(",")]
        if local < len(parts) and parts[local].isdigit():
            return int(parts[local])
    return local


# ---------------------------------------------------------------- oracle arms

def blas_build_rate(scene, reps=3):
    """BLAS builds of the scene's meshes (LBVH: boxes, Morton codes, radix
    sort, Karras hierarchy, refit, bounding sphere), inputs already on the
    device, CUDA events around the builds; the median of `reps` builds."""
    import torch
    import paper_2001_09792_gb300 as rg
    meshes = [(torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda(),
               torch.from_numpy(np.ascontiguousarray(i, np.uint32).view(np.int32)).cuda()) for v, i in scene.meshes]
    tris = sum(int(i.shape[0]) for _, i in scene.meshes)
    ms = []
    for _ in range(reps + 1):
        h = rg.rg_scene_create()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for tv, ti in meshes:
            rg.rg_blas_build(h, tv, ti)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        rg.rg_scene_destroy(h)
    t = statistics.median(ms[1:])
    return {"ms": round(t, 3), "tris": tris, "mtris_s": round(tris / t / 1e3, 1),
            "note": "the four BLAS, median of 3 after one warm-up build, inputs resident"}


def oracle_frames(scene, motions, budget_s, min_frames=1):
    """Render whole frames with the float64 oracle until the budget is spent."""
    import oracle
    O = oracle.OracleScene(scene)
    rays = 0
    frames = 0
    t0 = time.perf_counter()
    per_frame = []
    for M in motions:
        f0 = time.perf_counter()
        O.set_instances(M, scene.mesh_id, scene.material_id)
        r = O.render(scene.camera, scene.width, scene.height, scene.max_depth)
        per_frame.append(time.perf_counter() - f0)
        rays += r["closest_rays"] + r["shadow_rays"]
        frames += 1
        if frames >= min_frames and time.perf_counter() - t0 >= budget_s:
            break
    return rays, time.perf_counter() - t0, frames, per_frame


def cpu_baseline(scene, motions, budget_s):
    import oracle
    cores = len(os.sched_getaffinity(0))
    rays, secs, frames, _ = oracle_frames(scene, motions, budget_s)
    # one thread, on a seeded eighth of one frame's pixels
    O = oracle.OracleScene(scene)
    O.set_instances(motions[0], scene.mesh_id, scene.material_id)
    n_px = scene.width * scene.height
    pix = np.sort(np.random.default_rng(7).choice(n_px, n_px // 8, replace=False)).astype(np.uint32)
    t0 = time.perf_counter()
    r = O.render(scene.camera, scene.width, scene.height, scene.max_depth, pixels=pix, threads=1)
    t1 = time.perf_counter() - t0
    one = (r["closest_rays"] + r["shadow_rays"]) / t1 / 1e6
    return {"value": round(rays / secs / 1e6, 3), "unit": "Mrays/s", "cores": cores, "kind": "oracle",
            "sample": f"{frames} whole frame(s) of the same workload (float64, {cores} threads), {secs:.1f} s",
            "one_thread": {"value": round(one, 3), "unit": "Mrays/s",
                           "sample": f"a seeded eighth of one frame's pixels, 1 thread, {t1:.1f} s"}}


def run_reference(args, world, rank, local):
    if rank != 0:
        return
    s = g.medium_scene()
    n_frames = args.warmup + args.steps
    motions = frame_motions(s, n_frames)
    # bounded sample per step: a seeded subset of the frame's pixels
    import oracle
    O = oracle.OracleScene(s)
    n_pix = s.width * s.height
    sample = max(1, n_pix // 8)
    rng = np.random.default_rng(7)
    times, rays = [], 0
    for k in range(n_frames):
        pix = np.sort(rng.choice(n_pix, sample, replace=False)).astype(np.uint32)
        t0 = time.perf_counter()
        O.set_instances(motions[k], s.mesh_id, s.material_id)
        r = O.render(s.camera, s.width, s.height, s.max_depth, pixels=pix)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            rays += r["closest_rays"] + r["shadow_rays"]
    total = sum(times)
    cores = len(os.sched_getaffinity(0))
    value = round(rays / total / 1e6, 3)
    ts = sorted(times)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded procedural scene)",
        "config": {"workload": WORKLOAD, "width": s.width, "height": s.height, "max_depth": s.max_depth,
                   "sample_pixels_per_step": sample, "p50_ms": round(ts[len(ts) // 2] * 1e3, 3),
                   "p99_ms": round(ts[-1] * 1e3, 3), "parallelism": "host threads"},
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": "Mrays/s",
                         "sample": f"{sample} seeded pixels of each 1920x1080 frame, float64, {cores} threads"},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


LARGE_WORKLOAD = ("large: 4096 instances of 16 procedural meshes (1,938,944 unique / ~60M instanced tris), per step "
                  "seeded motion + full TLAS rebuild + 16,777,216 closest-hit and 16,777,216 any-hit rays "
                  "(origins uniform in the scene box, directions uniform, any-hit length U(1,50))")


def run_native_large(args, world, rank, local):
    """Incoherent ray queries: per step a TLAS rebuild and one closest-hit and
    one any-hit launch of 2^24 rays each (inputs larger than L2)."""
    import torch
    import paper_2001_09792_gb300 as rg
    from paper_2001_09792_gb300 import _build

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    s = g.large_scene()
    n = 1 << 24
    closest, anyhit = g.large_rays(s, n)
    n_frames = args.warmup + args.steps
    gs = rg.GpuScene(s, flags=rg.RG_SCENE_TIMING | path_flag(args))
    blas_ids = [gs.blas[m] for m in s.mesh_id]
    inst_dev = [torch.from_numpy(rg.pack_instances(g.motion(s.M, k), blas_ids, s.material_id)).cuda()
                for k in range(min(n_frames, 8))]
    d_c, d_a = torch.from_numpy(closest).cuda(), torch.from_numpy(anyhit).cuda()
    h_c = torch.empty((n, 5), dtype=torch.int32, device="cuda")
    h_a = torch.empty((n, 5), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(k):
        rg.rg_tlas_build(gs.h, inst_dev[k % len(inst_dev)])
        rg.rg_trace_rays(gs.h, d_c, rg.RG_CLOSEST, h_c)
        rg.rg_trace_rays(gs.h, d_a, rg.RG_ANY, h_a)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    with rg.GpuScene(s, flags=rg.RG_SCENE_COUNT | path_flag(args)) as gc:
        rg.rg_tlas_build(gc.h, torch.from_numpy(rg.pack_instances(g.motion(s.M, 0), [gc.blas[m] for m in s.mesh_id],
                                                                  s.material_id)).cuda())
        rg.rg_reset_stats(gc.h)
        rg.rg_trace_rays(gc.h, d_c, rg.RG_CLOSEST | rg.RG_TRACE_STATS, h_c)
        cst = rg.rg_get_stats(gc.h)
    rg.rg_sync(gs.h)
    rg.rg_reset_stats(gs.h)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_index(local))
    clocks.start()
    ev = []
    for k in range(args.warmup, n_frames):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(k)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    st = rg.rg_get_stats(gs.h)
    rg.rg_sync(gs.h)
    rays = st["closest_rays"] + st["shadow_rays"]
    (total_s_all,), (rays_all,) = reduce_over_ranks([sum(ms) / 1e3], [float(rays)], "cuda")
    if rank == 0:
        peak, peak_kind = measured_peaks()
        cr = max(cst["closest_rays"], 1)
        bpr = 32 + 20 + node_bytes(args) * cst["node_visits"] / cr + 48 * cst["tri_tests"] / cr + 80 * cst["inst_entries"] / cr
        launch_ms = st["trace_ms"] / max(st["trace_launches"], 1)
        achieved = bpr * (st["closest_rays"] / max(st["trace_launches"], 1)) / (launch_ms / 1e3) / 1e9
        ms_sorted = sorted(ms)
        out = {"metric": METRIC, "value": round(rays_all / total_s_all / 1e6, 2), "unit": "Mrays/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_s_all * 1e3 / args.steps, 3),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded procedural scene and rays)",
               "config": {"workload": LARGE_WORKLOAD, "rays_per_step": 2 * n, "instances": s.n_instances,
                          "closest_mrays_s": round(st["closest_rays"] / (sum(ms) / 1e3) / 1e6, 2),
                          "closest_ms": round(launch_ms, 3), "any_ms": round(st["any_ms"] / max(st["any_launches"], 1), 3),
                          "refine_ms": round(st["refine_ms"] / max(st["refine_launches"], 1), 3),
                          "p50_ms": round(ms_sorted[len(ms) // 2], 3), "p99_ms": round(ms_sorted[-1], 3),
                          "l2": "inputs larger than L2 (2 x 512 MiB of rays, ~220 MB of BVH)",
                          "parallelism": f"replicas x{world}", "bvh": "compressed 8-wide" if args.compressed else "binary float32"},
               "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                            "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind,
                            "kernel": kernel_name(args, "rg_trace_rays"), "algorithmic_bytes_per_ray": round(bpr, 1),
                            "nodes_per_ray": round(cst["node_visits"] / cr, 2),
                            "tris_per_ray": round(cst["tri_tests"] / cr, 2),
                            "inst_per_ray": round(cst["inst_entries"] / cr, 3)},
               "gpu_launches": int(st["kernel_launches"])}
        if clk:
            out["clocks"] = clk
        print(json.dumps(out), flush=True)
    gs.close()


def run_native_serve(args, world, rank, local):
    import torch
    from paper_2001_09792_gb300 import _build

    torch.cuda.set_device(local)
    _build.build()
    if rank != 0:
        return
    r = run_serving(args.requests, pair=not args.no_pair)
    out = {"metric": "served Mrays/s and p50/p99 request latency (continuous batching) vs one request at a time",
           "value": r["mrays_s"], "unit": "Mrays/s", "n_gpus": 1, "steps": r["steps"], "warmup": len(g.serving_scenes()),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded procedural scenes and request stream)", "config": {"workload": SERVE_WORKLOAD},
           "serving": r}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank, local)
    elif args.workload == "large":
        run_native_large(args, world, rank, local)
    elif args.workload == "serve":
        run_native_serve(args, world, rank, local)
    else:
        run_native(args, world, rank, local)


if __name__ == "__main__":
    main()
