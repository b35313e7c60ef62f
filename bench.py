#!/usr/bin/env python
"""Benchmark of the GB300 ray tracer.

Default (--workload large): one step = the large query workload (4,096
instances of 16 procedural meshes, 1,938,944 unique / about 60M instanced
triangles): seeded per-instance motion, a full TLAS rebuild (float64 instance
inverses, Arvo boxes, Morton codes, sort, Karras hierarchy, refit), then
16,777,216 closest-hit rays (one rg_trace_rays launch: float32 traversal, then
the exact t, u, v of each hit) and 16,777,216 any-hit rays (one launch).
Inputs are larger than L2 (1 GiB of rays, about 400 MB of BVH).

value  = closest-hit rays per step / ms_per_step (the whole step: rebuild,
         closest-hit and any-hit launches), over all ranks.
e2e    = the same steps through rg_trace_rays with the rays in pinned host
         memory and the hit records copied back to it, copies inside the
         timed region (each kind's rays copied in while the other kind traces).
The line also carries the any-hit rate, the medium render frame (64
instances, 1920x1080, depth 4) and the serving stream as extra keys.
--impl reference runs the float64 CPU oracle on a seeded sample of each
step's rays.

Multi-GPU (torchrun): replicas, each rank runs its own steps; value is the
sum of all ranks' rays over the slowest rank's time.
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
LARGE_WORKLOAD = ("large: 4096 instances of 16 procedural meshes (1,938,944 unique / ~60M instanced tris), per step "
                  "seeded motion + full TLAS rebuild + 16,777,216 closest-hit and 16,777,216 any-hit rays "
                  "(origins uniform in the scene box, directions uniform, any-hit length U(1,50))")
MEDIUM_WORKLOAD = ("medium: 64 instances of 4 procedural meshes (UV sphere 80x40, icosphere s5, cube, 256^2 heightfield; "
                   "157,964 unique tris) with seeded affine transforms in a 100^3 box, materials diffuse/mirror/glass "
                   "60/20/20%, 4 point lights, 1920x1080, max_depth 4; per frame seeded motion + full TLAS rebuild + render")
WORKLOAD = LARGE_WORKLOAD
N_LARGE = 1 << 24
# e2e copy granularity: the step's rays of one kind (measured against 4M- and
# 8M-ray chunks: 1,043-1,080 against 1,020-1,027 and 951-1,062 Mrays/s; every
# chunk is a traversal launch with its own tail)
E2E_CHUNK = 1 << 24


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None, help="timed steps (default: large 20, medium 200)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU baseline budget (wall seconds)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--serial", action="store_true",
                   help="large workload: trace the step's two queries one after the other on one stream (default: "
                        "the any-hit query on a second stream, overlapping the closest-hit query)")
    p.add_argument("--compressed", action="store_true",
                   help="trace with the compressed 8-wide BVH (default: the float32 binary BVH, faster here)")
    p.add_argument("--workload", default="large", choices=["large", "medium", "serve"],
                   help="large: incoherent closest/any-hit queries (default); medium: the render frame; "
                        "serve: the continuous-batching render server alone")
    p.add_argument("--requests", type=int, default=400, help="serving: requests in the Poisson stream")
    p.add_argument("--lanes", type=int, default=0, help="serving: server lanes (0: the library's default)")
    p.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    p.add_argument("--tlas", default="sah", choices=["sah", "lbvh"],
                   help="large workload: TLAS hierarchy, binned SAH in one block (RG_SCENE_SAH_TLAS) or LBVH")
    p.add_argument("--blas", default="sah", choices=["sah", "lbvh"],
                   help="BLAS build of every scene: binned SAH (RG_BLAS_SAH, for trace speed) or LBVH (for build speed)")
    p.add_argument("--no-medium", action="store_true", help="large: skip the medium render frame")
    p.add_argument("--rays", type=int, default=N_LARGE, help="large: rays of each kind per step")
    p.add_argument("--inflight", type=int, default=4,
                   help="medium: frames in flight (scene contexts sharing the BLAS, one stream each)")
    p.add_argument("--no-pair", action="store_true",
                   help="trace each level's (server: step's) shadow rays and the next one's closest-hit rays in separate launches")
    a = p.parse_args(argv)
    if a.steps is None:
        a.steps = 200 if a.workload == "medium" else 20
    return a


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


def sm_max_mhz():
    """The maximum SM clock (MEASURED_PEAKS.json, else GB300's 2070 MHz)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        return 2070.0


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


def traffic_record(profile="trace_pair_medium.md", key="dram_bytes_per_traversal_launch"):
    """DRAM bytes per launch of a traversal kernel, from a committed ncu
    summary under profiles/ (default: the medium frame's five traversal
    launches, averaged), valid only while the traversal code (traverse.cuh,
    trace.cu) and the launch sequence (api.cu) are unchanged: the summary
    carries the hash of that code."""
    path = os.path.join(ROOT, "profiles", profile)
    try:
        txt = open(path).read()
        sha = code_sha(*TRAVERSAL_SOURCES)
        m = re.search(key + r":\s*([0-9.]+)", txt)
        s = re.search(r"traversal_code_sha256_16:\s*([0-9a-f]+)", txt)
        if m and s and s.group(1) == sha:
            return float(m.group(1))
    except OSError:
        pass
    return None


def profile_figure(profile, label):
    """A percentage from a table row '| label | x % ...' of a committed ncu
    summary (a capture, not measured by this run); None if absent."""
    try:
        txt = open(os.path.join(ROOT, "profiles", profile)).read()
    except OSError:
        return None
    m = re.search(r"^\| " + re.escape(label) + r" \| ([0-9.]+) %", txt, flags=re.M)
    return float(m.group(1)) if m else None


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


def blas_flag(args):
    import paper_2001_09792_gb300 as rg
    return rg.RG_BLAS_SAH if getattr(args, "blas", "sah") == "sah" else rg.RG_MORTON30


def tlas_flag(args):
    import paper_2001_09792_gb300 as rg
    return rg.RG_SCENE_SAH_TLAS if getattr(args, "tlas", "sah") == "sah" else 0


def bvh_label(args, tlas=False):
    return (("compressed 8-wide" if args.compressed else "binary float32") + ", BLAS "
            + ("binned SAH" if getattr(args, "blas", "sah") == "sah" else "LBVH")
            + ((", TLAS " + ("binned SAH" if getattr(args, "tlas", "sah") == "sah" else "LBVH")) if tlas else ""))


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


# ---------------------------------------------------------------- medium render frame

def run_medium(args, world, rank, local, embedded=False):
    """The medium render frame (--workload medium, or a key of the large
    line when embedded): frames with per-frame motion, TLAS rebuild and
    render, four in flight; also one at a time (the roofline's launch times
    come from that pass, where launches do not overlap).  Returns the line on
    rank 0."""
    import torch
    import paper_2001_09792_gb300 as rg

    s = g.medium_scene()
    W, H, D = s.width, s.height, s.max_depth
    n_frames = args.warmup + args.steps
    motions = frame_motions(s, n_frames)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gs = rg.GpuScene(s, flags=rg.RG_SCENE_TIMING | path_flag(args), morton_flags=blas_flag(args))
    torch.cuda.synchronize()
    blas_build_ms = (time.perf_counter() - t0) * 1e3  # four BLAS + first TLAS, host-timed incl. uploads
    blas_build = blas_build_rate(s)
    blas_build["sah"] = blas_build_rate(s, sah=True)
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
    with rg.GpuScene(s, flags=rg.RG_SCENE_COUNT | path_flag(args), morton_flags=blas_flag(args)) as gc:
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
    closest1 = stats1[0]["closest_rays"]
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

    closest_f = sum(x["closest_rays"] for x in stats_f)

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
        e2e_rays = sum(rg.rg_get_stats(c.h)["closest_rays"] for c in ctxs)
        e2e = (e2e_rays, e_start.elapsed_time(e_end) / 1e3, inst_host[0].nbytes, W * H * 16)

    # aggregate over ranks: the slowest rank's time, every rank's rays
    if embedded:
        total_s_all, e2e_s_all, rays_all, closest_all = total_s, (e2e[1] if e2e else 0.0), rays, closest_f
        e2e_rays_all = e2e[0] if e2e else 0.0
    else:
        (total_s_all, e2e_s_all), (rays_all, closest_all, e2e_rays_all) = reduce_over_ranks(
            [total_s, e2e[1] if e2e else 0.0], [float(rays), float(closest_f), float(e2e[0]) if e2e else 0.0], "cuda")
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
        prof = "trace8_medium.md" if args.compressed else "trace_pair_medium.md"
        # the BVH lives in L2: the traversal is bound by instruction issue, so the
        # counted bytes (mostly L1/L2 hits) over the HBM peak is no DRAM fraction;
        # the DRAM fraction is the captured traffic over the same launch time
        # issue-bound (the BVH lives in L2): warp instructions of a frame's
        # traversal launches (the committed capture, valid for the code it
        # hashes) over their event-timed duration, against SMs x 4 schedulers x
        # the maximum SM clock; the counted bytes and the captured DRAM bytes
        # over the same time are reported beside it
        ipf = None if args.compressed else traffic_record(prof, "warp_inst_per_frame")
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        issue_peak = sms * 4 * sm_max_mhz() * 1e6 / 1e9
        frame_trav_ms = trav_ms / args.steps
        ach_i = None if ipf is None else ipf / (frame_trav_ms / 1e3) / 1e9
        roofline = {"bound": "issue", "achieved": None if ach_i is None else round(ach_i, 1),
                    "peak": round(issue_peak, 1), "unit": "G warp-instructions/s",
                    "frac": None if ach_i is None else round(ach_i / issue_peak, 4),
                    "traffic": None if tr is None else round(tr),
                    "dram_frac": None if tr is None else round(tr / (launch_ms / 1e3) / 1e9 / peak, 4),
                    "counted_bytes": {"gbs": round(achieved, 1), "frac_of_hbm": round(achieved / peak, 4),
                                      "hbm_peak_gbs": peak, "hbm_peak_kind": peak_kind},
                    "peak_derivation": f"{sms} SMs x 4 warp schedulers x 1 instruction/cycle x {sm_max_mhz():.0f} MHz",
                    "warp_inst_per_frame": ipf,
                    "issue_slots_active_pct": profile_figure(prof, "issue slots active"),
                    "bound_note": "achieved: warp instructions of a frame's traversal launches (committed capture) over "
                                  "their event-timed time; counted_bytes: algorithmic bytes per launch over the launch "
                                  "time, served mostly by L1/L2; dram_frac: the captured DRAM bytes over the same time",
                    "timed_region": "the one-in-flight pass (config.one_in_flight.ms_per_step)",
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
            "value": round(closest_all / total_s_all / 1e6, 2),
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
            "config": {"workload": MEDIUM_WORKLOAD, "width": W, "height": H, "max_depth": D, "lights": 4,
                       "instances": s.n_instances, "instanced_tris": s.instanced_tris(),
                       "rays_per_step": round(rays / args.steps), "closest_rays_per_step": round(st["closest_rays"] / args.steps),
                       "shadow_rays_per_step": round(st["shadow_rays"] / args.steps),
                       "all_rays_mrays_s": round(rays_all / total_s_all / 1e6, 2),
                       "value_is": "closest-hit rays (camera, reflected, refracted) per second; shadow (any-hit) "
                                   "rays are counted in all_rays_mrays_s",
                       "frames_in_flight": F,
                       "p50_ms": p50, "p99_ms": p99,
                       "one_in_flight": {"value": round(closest1 / wall1 / 1e6, 2),
                                         "all_rays_mrays_s": round(rays1 / wall1 / 1e6, 2),
                                         "ms_per_step": round(wall1 * 1e3 / args.steps, 3),
                                         "p50_ms": p50_1, "p99_ms": p99_1,
                                         "note": "the same frames one at a time; the roofline's launch times are taken here"},
                       "latency": "per frame, from its TLAS build to its image on its stream (with frames in flight, "
                                  "the frames share the GPU)",
                       "blas_build_ms": round(blas_build_ms, 2), "blas_build": blas_build,
                       "l2": "flushed before each frame (256 MiB write on the frame's stream, inside the timed region)",
                       "fxaa": {"ms": round(fxaa_ms, 4), "gbs": round(W * H * 32 / (fxaa_ms / 1e3) / 1e9, 1),
                                "bytes_per_pixel": 32, "note": "k_fxaa_luma + k_fxaa on the frame, timed alone, not in the step"},
                       "parallelism": f"replicas x{world}", "bvh": bvh_label(args)},
            "roofline": roofline,
            "gpu_launches": int(stats_f[0]["kernel_launches"]),
        }
        if clk:
            out["clocks"] = clk
        if e2e:
            out["e2e"] = {"value": round(e2e[0] / e2e[1] / 1e6, 2), "unit": "Mrays/s (closest-hit)",
                          "h2d_bytes_per_step": int(e2e[2]), "d2h_bytes_per_step": int(e2e[3]),
                          "note": f"frames back to back, {F} in flight (one scene context and stream each), "
                                  "each image read back on a copy stream while later frames render; one timed "
                                  "region incl. L2 flushes"}
        if not embedded and world == 1 and not args.no_serving:
            out["serving"] = run_serving(args.requests, pair=not args.no_pair, lanes=args.lanes,
                                         blas_flags=blas_flag(args))
        if not embedded and world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"], ref = cpu_baseline(s, motions[args.warmup:], args.cpu_seconds)
            # the GPU's render and camera-ray records of the oracle's first frame
            rg.rg_tlas_build(gs.h, inst_dev[args.warmup])
            img0 = rg.rg_render(gs.h, cam, W, H, D)
            hits0 = rg.rg_trace_rays(gs.h, torch.from_numpy(ref["rays"]).cuda())
            rg.rg_sync(gs.h)
            out["error_vs_oracle"] = {
                "pixels": pixel_error_vs_oracle(img0.cpu().numpy(), ref["frame"]),
                "rays": hit_error_vs_oracle(rg.split_hits(hits0), ref["ray_ref"]),
                "bvh": bvh_label(args),
                "sample": f"the whole frame of the first timed motion, and {len(ref['rays']):,} seeded camera rays of "
                          "it traced as closest-hit queries (rg_trace_rays)"}
    for c in ctxs[1:]:
        c.close()
    gs.close()
    return out if rank == 0 else None


def run_native_medium(args, world, rank, local):
    import torch
    from paper_2001_09792_gb300 import _build

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    out = run_medium(args, world, rank, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------- large queries (default)

def ray_bytes(cst, node_b, any_hit):
    """Algorithmic bytes per ray of a counting pass: the ray (32 B), its hit
    record (20 B), node_b per BVH node fetched, 48 B per triangle tested (one
    axis order of the record) and 80 B per instance entered (the float32
    inverse rows and the BLAS pointers, root and ids)."""
    pre = "any_" if any_hit else ""
    r = max(cst["shadow_rays" if any_hit else "closest_rays"], 1)
    return (32 + 20 + node_b * cst[pre + "node_visits"] / r + 48 * cst[pre + "tri_tests"] / r
            + 80 * cst[pre + "inst_entries"] / r)


def large_counts(s, rg, torch, args, motion, d_c, d_a):
    """Node, triangle and instance counts per ray of the large query (a
    counting traversal on a second scene with the same motion)."""
    flags = rg.RG_SCENE_COUNT | path_flag(args) | tlas_flag(args)
    with rg.GpuScene(s, flags=flags, morton_flags=blas_flag(args)) as gc:
        rg.rg_tlas_build(gc.h, torch.from_numpy(rg.pack_instances(motion, [gc.blas[m] for m in s.mesh_id],
                                                                  s.material_id)).cuda())
        rg.rg_reset_stats(gc.h)
        rg.rg_trace_rays(gc.h, d_c, rg.RG_CLOSEST | rg.RG_TRACE_STATS)
        rg.rg_trace_rays(gc.h, d_a, rg.RG_ANY | rg.RG_TRACE_STATS)
        return rg.rg_get_stats(gc.h)


def large_e2e(rg, torch, gs, inst_host, closest, anyhit, steps, first, serial=False):
    """The large steps end to end: per step the instance transforms, the
    closest-hit rays and the any-hit rays are copied from pinned host memory
    and the hit records copied back to it, in chunks of E2E_CHUNK rays (by
    default one per kind) pipelined over a copy-in stream, the tracing stream
    and a copy-out stream.  Each kind has a ring of device buffers two steps
    deep, so a chunk's rays can be copied in while the previous step's chunk
    of the same kind is traced (a whole step of time for each copy).  One
    timed region over all steps.  As in the device-side steps, the any-hit rays
    are traced on a stream of their own during the closest-hit launch (unless
    serial), and a step's TLAS rebuild waits for the previous step's any-hit
    launch.  Returns (closest rays, seconds, H2D bytes per step, D2H bytes per
    step)."""
    n = closest.shape[0]
    pin_c = torch.from_numpy(closest).pin_memory()
    pin_a = torch.from_numpy(anyhit).pin_memory()
    pin_inst = [torch.from_numpy(x).pin_memory() for x in inst_host]
    out_c = torch.empty((n, 5), dtype=torch.int32).pin_memory()
    out_a = torch.empty((n, 5), dtype=torch.int32).pin_memory()
    C = min(E2E_CHUNK, n)
    chunks = (n + C - 1) // C
    ring = 2 * chunks   # buffers per kind
    d_rays = [[torch.empty((C, 8), dtype=torch.float32, device="cuda") for _ in range(ring)] for _ in range(2)]
    d_hits = [[torch.empty((C, 5), dtype=torch.int32, device="cuda") for _ in range(ring)] for _ in range(2)]
    d_inst = torch.empty_like(torch.from_numpy(inst_host[0])).cuda()
    s_in, s_run, s_out = torch.cuda.Stream(), torch.cuda.current_stream(), torch.cuda.Stream()
    s_run2 = s_run if serial else torch.cuda.Stream()  # the any-hit launches
    any_done = None
    traced = [[None] * ring for _ in range(2)]   # buffer's rays have been traced (it may be refilled)
    copied = [[None] * ring for _ in range(2)]   # buffer's hits have been copied out (it may be rewritten)
    rg.rg_sync(gs.h)
    rg.rg_reset_stats(gs.h)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_run)
    s_in.wait_event(e0)
    s_out.wait_event(e0)
    s_run2.wait_event(e0)
    for k in range(first, first + steps):
        with torch.cuda.stream(s_in):
            d_inst.copy_(pin_inst[k % len(pin_inst)], non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(s_in)
        s_run.wait_event(ready)
        if any_done is not None:
            s_run.wait_event(any_done)  # the previous any-hit launch reads the TLAS
        rg.rg_tlas_build(gs.h, d_inst, stream=s_run)
        inst_used = torch.cuda.Event()
        inst_used.record(s_run)
        s_run2.wait_event(inst_used)
        for kind, (host_in, host_out, flags) in enumerate(((pin_c, out_c, rg.RG_CLOSEST), (pin_a, out_a, rg.RG_ANY))):
            run = s_run if kind == 0 else s_run2
            for j, c0 in enumerate(range(0, n, C)):
                m = min(C, n - c0)
                b = ((k - first) * chunks + j) % ring
                with torch.cuda.stream(s_in):
                    if traced[kind][b] is not None:
                        s_in.wait_event(traced[kind][b])
                    d_rays[kind][b][:m].copy_(host_in[c0:c0 + m], non_blocking=True)
                    loaded = torch.cuda.Event()
                    loaded.record(s_in)
                run.wait_event(loaded)
                if copied[kind][b] is not None:
                    run.wait_event(copied[kind][b])
                rg.rg_trace_rays(gs.h, d_rays[kind][b][:m], flags, d_hits[kind][b], stream=run)
                traced[kind][b] = torch.cuda.Event()
                traced[kind][b].record(run)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(traced[kind][b])
                    host_out[c0:c0 + m].copy_(d_hits[kind][b][:m], non_blocking=True)
                    copied[kind][b] = torch.cuda.Event()
                    copied[kind][b].record(s_out)
        if not serial:
            any_done = torch.cuda.Event()
            any_done.record(s_run2)
        s_in.wait_event(inst_used)  # the next step's transforms overwrite d_inst
    s_run.wait_stream(s_run2)
    s_run.wait_stream(s_out)
    s_run.wait_stream(s_in)
    e1.record(s_run)
    torch.cuda.synchronize()
    closest_rays = rg.rg_get_stats(gs.h)["closest_rays"]
    h2d = inst_host[0].nbytes + closest.nbytes + anyhit.nbytes
    d2h = out_c.numel() * 4 + out_a.numel() * 4
    return closest_rays, e0.elapsed_time(e1) / 1e3, h2d, d2h


def hit_error_vs_oracle(h, ref):
    """Per-output error of closest-hit records against the float64 oracle:
    ids that differ (and how many of those the oracle flags), and for the hits
    whose ids agree the largest and 99th-percentile relative errors of t and of
    u, v (relative to max(|u|, 1e-3))."""
    miss = 0xFFFFFFFF
    id_diff = (h["inst"] != ref["inst"]) | (h["prim"] != ref["prim"])
    agree = ~id_diff & (ref["inst"] != miss)
    et = np.abs(h["t"][agree] - ref["t"][agree]) / np.abs(ref["t"][agree])
    eu = np.abs(h["u"][agree] - ref["u"][agree]) / np.maximum(np.abs(ref["u"][agree]), 1e-3)
    ev = np.abs(h["v"][agree] - ref["v"][agree]) / np.maximum(np.abs(ref["v"][agree]), 1e-3)
    q = lambda x, p: float(np.quantile(x, p)) if x.size else 0.0  # noqa: E731
    return {"rays": int(len(id_diff)), "hits": int(agree.sum()), "id_differ": int(id_diff.sum()),
            "id_differ_flagged": int((id_diff & ref["ambiguous"]).sum()), "flagged": int(ref["ambiguous"].sum()),
            "t_rel": {"max": q(et, 1.0), "p99": q(et, 0.99)}, "u_rel": {"max": q(eu, 1.0), "p99": q(eu, 0.99)},
            "v_rel": {"max": q(ev, 1.0), "p99": q(ev, 0.99)},
            "tolerance": "t 1e-5 relative; u, v 1e-5 relative to max(|u|, 1e-3); differing ids flagged, <= 1e-4"}


def oracle_prefix(O, rays, budget_s, chunk=65536, any_hit=False):
    """The oracle on a prefix of the rays, chunk by chunk until the budget is
    spent (at least one chunk); returns (rays traced, seconds, its records)."""
    outs, done, t0 = [], 0, time.perf_counter()
    while done < len(rays):
        outs.append(O.trace(rays[done:done + chunk], any_hit=any_hit))
        done = min(len(rays), done + chunk)
        if time.perf_counter() - t0 >= budget_s:
            break
    secs = time.perf_counter() - t0
    rec = {k: np.concatenate([o[k] for o in outs]) for k in outs[0]}
    return done, secs, rec


def run_native_large(args, world, rank, local):
    """The default benchmark line (see the module docstring)."""
    import torch
    import paper_2001_09792_gb300 as rg
    from paper_2001_09792_gb300 import _build

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    s = g.large_scene()
    n = args.rays
    closest, anyhit = g.large_rays(s, n)
    n_frames = args.warmup + args.steps
    motions = [g.motion(s.M, k) for k in range(min(n_frames, 8))]
    gs = rg.GpuScene(s, flags=rg.RG_SCENE_TIMING | path_flag(args) | tlas_flag(args), morton_flags=blas_flag(args))
    blas_ids = [gs.blas[m] for m in s.mesh_id]
    inst_host = [rg.pack_instances(M, blas_ids, s.material_id) for M in motions]
    inst_dev = [torch.from_numpy(x).cuda() for x in inst_host]
    d_c, d_a = torch.from_numpy(closest).cuda(), torch.from_numpy(anyhit).cuda()
    h_c = torch.empty((n, 5), dtype=torch.int32, device="cuda")
    h_a = torch.empty((n, 5), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    s_any = torch.cuda.Stream()

    def step(k, serial=args.serial):
        # the TLAS rebuild, then the closest-hit query (and its exact-attribute
        # pass) and the any-hit query; by default the any-hit query runs on a
        # second stream at the same time, and the step ends when both have
        rg.rg_tlas_build(gs.h, inst_dev[k % len(inst_dev)])
        if serial:
            rg.rg_trace_rays(gs.h, d_c, rg.RG_CLOSEST, h_c)
            rg.rg_trace_rays(gs.h, d_a, rg.RG_ANY, h_a)
            return
        built = torch.cuda.Event()
        built.record(stream)
        s_any.wait_event(built)
        rg.rg_trace_rays(gs.h, d_c, rg.RG_CLOSEST, h_c)
        rg.rg_trace_rays(gs.h, d_a, rg.RG_ANY, h_a, stream=s_any)
        done = torch.cuda.Event()
        done.record(s_any)
        stream.wait_event(done)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    cst = large_counts(s, rg, torch, args, motions[0], d_c, d_a)
    rg.rg_sync(gs.h)
    rg.rg_reset_stats(gs.h)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_index(local))
    clocks.start()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev = []
    e_start.record(stream)
    for k in range(args.warmup, n_frames):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(k)
        e1.record(stream)
        ev.append((e0, e1))
    e_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    wall = e_start.elapsed_time(e_end) / 1e3
    ms = [a.elapsed_time(b) for a, b in ev]
    st = rg.rg_get_stats(gs.h)
    rg.rg_sync(gs.h)
    last_motion = (n_frames - 1) % len(motions)
    gpu_hits = rg.split_hits(h_c[: min(n, 1 << 20)]) if rank == 0 else None
    st_serial = None
    if not args.serial:
        # each launch alone: a few steps with the queries one after the other
        # (outside the timed region; context for the overlapped launch times)
        rg.rg_reset_stats(gs.h)
        torch.cuda.synchronize()
        e_s0, e_s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_s0.record(stream)
        for k in range(3):
            step(n_frames + k, serial=True)
        e_s1.record(stream)
        torch.cuda.synchronize()
        st_serial = rg.rg_get_stats(gs.h)
        st_serial["step_ms"] = e_s0.elapsed_time(e_s1) / 3
        rg.rg_sync(gs.h)

    e2e = None
    if not args.no_e2e:
        e2e = large_e2e(rg, torch, gs, inst_host, closest, anyhit, args.steps, args.warmup, serial=args.serial)
    (wall_all, e2e_s_all), (closest_all, any_all, e2e_rays_all) = reduce_over_ranks(
        [wall, e2e[1] if e2e else 0.0], [float(st["closest_rays"]), float(st["shadow_rays"]),
                                         float(e2e[0]) if e2e else 0.0], "cuda")

    out = None
    if rank == 0:
        peak, peak_kind = measured_peaks()
        nb = node_bytes(args)
        bpr = ray_bytes(cst, nb, False)
        bpa = ray_bytes(cst, nb, True)
        c_launches = max(st["trace_launches"], 1)
        c_ms = st["trace_ms"] / c_launches
        a_ms = st["any_ms"] / max(st["any_launches"], 1)
        r_ms = st["refine_ms"] / max(st["refine_launches"], 1)
        c_bytes = bpr * n
        counted_gbs = c_bytes / (c_ms / 1e3) / 1e9
        alone = None  # each launch alone (the serialized steps after an overlapped timed region)
        if st_serial is not None:
            sc = st_serial["trace_ms"] / max(st_serial["trace_launches"], 1)
            sa = st_serial["any_ms"] / max(st_serial["any_launches"], 1)
            sr = st_serial["refine_ms"] / max(st_serial["refine_launches"], 1)
            alone = {"closest_launch_ms": round(sc, 3), "refine_ms": round(sr, 3), "any_launch_ms": round(sa, 3),
                     "tlas_rebuild_and_rest_ms": round(st_serial["step_ms"] - sc - sr - sa, 3),
                     "step_ms": round(st_serial["step_ms"], 3),
                     "note": "3 steps with the two queries one after the other, after the timed region"}
        q_c, q_r, q_a = (sc, sr, sa) if alone else (c_ms, r_ms, a_ms)
        prof = "trace_large_compressed.md" if args.compressed else "trace_large.md"
        tr = traffic_record(prof, "dram_bytes_per_closest_launch")
        ipr = traffic_record(prof, "warp_inst_per_closest_ray")
        ms_sorted = sorted(ms)
        step_ms = wall_all * 1e3 / args.steps
        # The traversal is bound by instruction issue and the latency of its
        # dependent loads, not by HBM (the captured DRAM traffic is a few % of
        # the counted bytes): achieved = warp instructions per launch (the
        # captured count per ray times the rays) over the event-timed launch;
        # peak = SMs x 4 schedulers x 1 warp instruction per cycle at the
        # maximum SM clock.
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        issue_peak = sms * 4 * sm_max_mhz() * 1e6 / 1e9
        achieved = None if ipr is None else ipr * n / (c_ms / 1e3) / 1e9
        achieved_alone = None if (ipr is None or alone is None) else ipr * n / (sc / 1e3) / 1e9
        roofline = {
            "bound": "issue", "achieved": None if achieved is None else round(achieved, 1), "peak": round(issue_peak, 1),
            "unit": "G warp-instructions/s", "frac": None if achieved is None else round(achieved / issue_peak, 4),
            "traffic": None if tr is None else round(tr),
            "dram_frac": None if tr is None else round(tr / (c_ms / 1e3) / 1e9 / peak, 4),
            "counted_bytes": {"gbs": round(counted_gbs, 1), "frac_of_hbm": round(counted_gbs / peak, 4),
                              "hbm_peak_gbs": peak, "hbm_peak_kind": peak_kind,
                              "note": "algorithmic bytes (nodes, triangles, instances, ray, hit) per launch over the "
                                      "launch time; served mostly from L1/L2"},
            "peak_derivation": f"{sms} SMs x 4 warp schedulers x 1 instruction/cycle x {sm_max_mhz():.0f} MHz",
            "warp_inst_per_ray": ipr, "kernel": kernel_name(args, "rg_trace_rays"),
            "per_launch": "one closest-hit traversal launch of 16,777,216 rays, timed by CUDA events around each "
                          "launch inside the timed steps; instructions per ray and DRAM bytes from the committed "
                          f"ncu capture (profiles/{prof}, valid for the traversal code it hashes)",
            "avg_launch_ms": round(c_ms, 4), "algorithmic_bytes_per_launch": round(c_bytes),
            "algorithmic_bytes_per_ray": round(bpr, 1),
            "nodes_per_ray": round(cst["node_visits"] / max(cst["closest_rays"], 1), 2),
            "tris_per_ray": round(cst["tri_tests"] / max(cst["closest_rays"], 1), 2),
            "inst_per_ray": round(cst["inst_entries"] / max(cst["closest_rays"], 1), 3),
            "any_hit": {"algorithmic_bytes_per_ray": round(bpa, 1), "avg_launch_ms": round(a_ms, 4),
                        "achieved_gbs": round(bpa * n / (a_ms / 1e3) / 1e9, 1),
                        "nodes_per_ray": round(cst["any_node_visits"] / max(cst["shadow_rays"], 1), 2)},
            "step_check": {"algorithmic_bytes_per_step": round(c_bytes + bpa * n),
                           "gbs_over_ms_per_step": round((c_bytes + bpa * n) / (step_ms / 1e3) / 1e9, 1)},
            "l2": profile_l2(prof)}
        ipa = traffic_record(prof, "warp_inst_per_any_ray")
        ipf = traffic_record(prof, "warp_inst_per_refine_launch")
        if ipr is not None and ipa is not None and ipf is not None:
            # every warp instruction of a step's two queries (the captured
            # counts) over the step time: the issue rate of the whole step
            step_inst = ipr * n + ipf + ipa * n
            roofline["step"] = {"warp_instructions": round(step_inst),
                                "achieved": round(step_inst / (step_ms / 1e3) / 1e9, 1),
                                "frac": round(step_inst / (step_ms / 1e3) / 1e9 / issue_peak, 4),
                                "note": "closest-hit, exact-attribute and any-hit launches' warp instructions (ncu) "
                                        "over ms_per_step (TLAS rebuild included, its instructions not counted)"}
        if alone:
            roofline["per_launch"] += ("; the timed steps trace the any-hit query on a second stream during the "
                                       "closest-hit launch, so avg_launch_ms includes the shared time")
            roofline["alone"] = {"avg_launch_ms": round(sc, 4),
                                 "achieved": None if achieved_alone is None else round(achieved_alone, 1),
                                 "frac": None if achieved_alone is None else round(achieved_alone / issue_peak, 4),
                                 "note": "the same launch with the GPU to itself (serialized steps after the timed "
                                         "region)"}
        out = {
            "metric": METRIC,
            "value": round(closest_all / wall_all / 1e6, 2),
            "unit": "Mrays/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(step_ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded procedural scene and rays)",
            "config": {
                "workload": LARGE_WORKLOAD, "instances": s.n_instances, "instanced_tris": s.instanced_tris(),
                "closest_rays_per_step": n, "any_hit_rays_per_step": n,
                "value_is": "closest-hit rays per step / ms_per_step (the step: TLAS rebuild, then the closest-hit "
                            "launch + exact-attribute pass and the any-hit launch, "
                            + ("one after the other)" if args.serial else "the any-hit launch on a second stream "
                               "at the same time)"),
                "closest_launch_ms": round(c_ms, 3), "refine_ms": round(r_ms, 3), "any_launch_ms": round(a_ms, 3),
                "closest_query_mrays_s": round(n / ((q_c + q_r) / 1e3) / 1e6, 2),
                "any_hit_mrays_s": round(n / (q_a / 1e3) / 1e6, 2),
                "all_rays_mrays_s": round((closest_all + any_all) / wall_all / 1e6, 2),
                "tlas_rebuild_and_rest_ms": (alone["tlas_rebuild_and_rest_ms"] if alone
                                             else round(step_ms - c_ms - r_ms - a_ms, 3)),
                "launches_alone": alone,
                "p50_ms": round(ms_sorted[len(ms) // 2], 3), "p99_ms": round(pct(ms, 0.99), 3),
                "latency": "per step (TLAS rebuild + both queries), CUDA events on the stream",
                "l2": "inputs larger than L2 (2 x 512 MiB of rays, about 400 MB of BVH and triangle records); "
                      "no flush",
                "parallelism": f"replicas x{world}", "bvh": bvh_label(args, tlas=True)},
            "roofline": roofline,
            "gpu_launches": int(st["kernel_launches"]),
        }
        if clk:
            out["clocks"] = clk
        if e2e:
            out["e2e"] = {"value": round(e2e_rays_all / e2e_s_all / 1e6, 2), "unit": "Mrays/s",
                          "h2d_bytes_per_step": int(e2e[2]), "d2h_bytes_per_step": int(e2e[3]),
                          "note": "rays in pinned host memory, hit records back to pinned host memory, each kind's rays "
                                  "copied in during the previous step and its hits copied out while the next launches "
                                  "trace (copy-in, trace, copy-out streams; the any-hit launches on a second trace "
                                  "stream unless --serial), one timed region"}
    if world == 1 and rank == 0:
        if not args.no_cpu_baseline:
            import oracle
            O = oracle.OracleScene(s)
            O.set_instances(motions[last_motion], s.mesh_id, s.material_id)
            k, secs, ref = oracle_prefix(O, closest, args.cpu_seconds)
            ka, secs_a, _ = oracle_prefix(O, anyhit, max(1.0, args.cpu_seconds / 4), any_hit=True)
            cores = len(os.sched_getaffinity(0))
            out["cpu_baseline"] = {
                "value": round(k / secs / 1e6, 4), "unit": "Mrays/s", "cores": cores, "kind": "oracle",
                "sample": f"the first {k:,} closest-hit rays of the step (float64, {cores} threads, {secs:.1f} s)",
                "any_hit": {"value": round(ka / secs_a / 1e6, 4), "unit": "Mrays/s",
                            "sample": f"the first {ka:,} any-hit rays ({secs_a:.1f} s)"}}
            m = min(k, len(gpu_hits["inst"]))
            out["error_vs_oracle"] = hit_error_vs_oracle({kk: v[:m] for kk, v in gpu_hits.items()},
                                                         {kk: v[:m] for kk, v in ref.items()})
            out["error_vs_oracle"]["sample"] = f"closest-hit records of the first {m:,} rays of the last timed step"
        gs.close()
        if not args.no_medium:
            out["medium"] = medium_summary(run_medium(args_for_medium(args), 1, 0, local, embedded=True))
        if not args.no_serving:
            out["serving"] = run_serving(args.requests, pair=not args.no_pair, lanes=args.lanes,
                                         blas_flags=blas_flag(args))
    else:
        gs.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def args_for_medium(args):
    a = argparse.Namespace(**vars(args))
    a.steps = 60
    a.no_cpu_baseline = True
    a.no_serving = True
    return a


def medium_summary(line):
    """The medium frame's line, kept as a key of the large line."""
    keep = ("value", "unit", "ms_per_step", "config", "roofline", "e2e", "clocks", "gpu_launches", "steps", "warmup")
    out = {k: line[k] for k in keep if k in line}
    out["workload"] = MEDIUM_WORKLOAD
    out["value_is"] = "closest-hit rays per second of the frames (four in flight)"
    return out


def profile_l2(profile):
    """L2 / L1 hit rates and L2 throughput of a captured traversal launch."""
    try:
        txt = open(os.path.join(ROOT, "profiles", profile)).read()
    except OSError:
        return None
    m = re.search(r"^\| L2 / L1 sector hit rate \| ([0-9.]+) % / ([0-9.]+) %", txt, flags=re.M)
    if not m:
        return None
    out = {"l2_sector_hit_pct": float(m.group(1)), "l1_sector_hit_pct": float(m.group(2)),
           "source": f"ncu capture (profiles/{profile}), not this run"}
    for label, key in (("L2 (lts) throughput, % of peak", "l2_throughput_pct_of_peak"),
                       ("DRAM throughput, % of peak", "dram_throughput_pct_of_peak"),
                       ("issue slots active", "issue_slots_active_pct")):
        v = profile_figure(profile, label)
        if v is not None:
            out[key] = v
    return out


SERVE_WORKLOAD = ("serve: Poisson arrivals at 200 req/s over 8 resident scenes (the tiny scene + 7 medium-style "
                  "scenes), resolution uniform over 320x240 / 640x480 / 1280x720 / 1920x1080 / 3840x2160, max_depth "
                  "uniform 1..8, seeded per-request instance motion (per-request TLAS refit)")


def pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, math.ceil(q * len(xs)) - 1))]


def run_serving(n_requests, admit_rays=0, pair=True, lanes=0, blas_flags=0):
    """The request stream through the continuous-batching server in real time,
    then the same stream one request at a time (rg_tlas_refit + rg_render each,
    in arrival order, against the same arrival clock).  Latency = arrival to
    the completion of the image on the device (host clock)."""
    import torch
    import paper_2001_09792_gb300 as rg

    scenes = g.serving_scenes()
    reqs = g.serving_requests(n_requests)
    gss = [rg.GpuScene(sc, flags=0 if pair else rg.RG_SCENE_NO_PAIR, morton_flags=blas_flags) for sc in scenes]
    trans = [g.motion(scenes[q["scene"]].M, q["motion_seed"]) for q in reqs]
    cams = [rg.make_camera(sc.camera) for sc in scenes]
    srv = rg.rg_server_create(admit_rays=admit_rays, flags=0 if pair else rg.RG_SERVER_NO_PAIR, lanes=lanes)
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
        "shapes": tuned, "lanes": lanes or 1,
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

def blas_build_rate(scene, reps=3, sah=False):
    """BLAS builds of the scene's meshes (LBVH: boxes, Morton codes, radix
    sort, Karras hierarchy, refit, bounding sphere; with sah the binned-SAH
    build, one host round trip per tree level), inputs already on the device,
    CUDA events around the builds; the median of `reps` builds."""
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
            rg.rg_blas_build(h, tv, ti, rg.RG_BLAS_SAH if sah else rg.RG_MORTON30)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        rg.rg_scene_destroy(h)
    t = statistics.median(ms[1:])
    return {"ms": round(t, 3), "tris": tris, "mtris_s": round(tris / t / 1e3, 1),
            "note": "the four BLAS, median of 3 after one warm-up build, inputs resident"}


def oracle_frames(scene, motions, budget_s, min_frames=1):
    """Render whole frames with the float64 oracle until the budget is spent;
    also returns the first frame's result (rgba, ambiguous flags)."""
    import oracle
    O = oracle.OracleScene(scene)
    rays = 0
    frames = 0
    t0 = time.perf_counter()
    per_frame = []
    first = None
    for M in motions:
        f0 = time.perf_counter()
        O.set_instances(M, scene.mesh_id, scene.material_id)
        r = O.render(scene.camera, scene.width, scene.height, scene.max_depth)
        per_frame.append(time.perf_counter() - f0)
        rays += r["closest_rays"] + r["shadow_rays"]
        frames += 1
        if first is None:
            first = r
        if frames >= min_frames and time.perf_counter() - t0 >= budget_s:
            break
    return rays, time.perf_counter() - t0, frames, per_frame, first


def cpu_baseline(scene, motions, budget_s, n_sample_rays=50_000):
    """The oracle on the medium frames (whole frames, all host cores; one
    thread on an eighth of a frame).  Also returns, for the error of the GPU
    path, the first frame's oracle image and the oracle's records of a seeded
    sample of that frame's camera rays (traced as closest-hit queries)."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    rays, secs, frames, _, first = oracle_frames(scene, motions, budget_s)
    # one thread, on a seeded eighth of one frame's pixels
    O = oracle.OracleScene(scene)
    O.set_instances(motions[0], scene.mesh_id, scene.material_id)
    n_px = scene.width * scene.height
    pix = np.sort(np.random.default_rng(7).choice(n_px, n_px // 8, replace=False)).astype(np.uint32)
    t0 = time.perf_counter()
    r = O.render(scene.camera, scene.width, scene.height, scene.max_depth, pixels=pix, threads=1)
    t1 = time.perf_counter() - t0
    one = (r["closest_rays"] + r["shadow_rays"]) / t1 / 1e6
    spix = np.sort(np.random.default_rng(8).choice(n_px, min(n_sample_rays, n_px), replace=False)).astype(np.uint32)
    cam_rays = np.zeros((len(spix), 8), np.float32)
    cam_rays[:, 0:3] = scene.camera["eye"]
    cam_rays[:, 4:7] = oracle.camera_dirs(scene.camera, scene.width, scene.height, spix)
    cam_rays[:, 7] = np.inf
    ray_ref = O.trace(cam_rays)
    out = {"value": round(rays / secs / 1e6, 3), "unit": "Mrays/s", "cores": cores, "kind": "oracle",
           "sample": f"{frames} whole frame(s) of the same workload (float64, {cores} threads), {secs:.1f} s",
           "one_thread": {"value": round(one, 3), "unit": "Mrays/s",
                          "sample": f"a seeded eighth of one frame's pixels, 1 thread, {t1:.1f} s"}}
    return out, {"frame": first, "rays": cam_rays, "ray_ref": ray_ref}


def pixel_error_vs_oracle(img, ref, tol=2e-3):
    """Per-pixel error of an RGBA32F image against the oracle's render: the
    largest and 99th-percentile absolute channel error over the pixels the
    oracle does not flag, and how many pixels exceed the tolerance (all must
    be flagged)."""
    img = np.asarray(img, np.float64).reshape(-1, 4)
    err = np.abs(img - ref["rgba"]).max(1)
    ok = ~ref["ambiguous"]
    over = err > tol
    return {"pixels": int(len(err)), "max": float(err[ok].max(initial=0.0)),
            "p99": float(np.quantile(err[ok], 0.99)) if ok.any() else 0.0,
            "over_tolerance": int(over.sum()), "over_tolerance_flagged": int((over & ~ok).sum()),
            "flagged": int((~ok).sum()), "tolerance": f"{tol} absolute per channel"}


def run_reference_medium(args, world, rank, local):
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
    times, rays, closest = [], 0, 0
    for k in range(n_frames):
        pix = np.sort(rng.choice(n_pix, sample, replace=False)).astype(np.uint32)
        t0 = time.perf_counter()
        O.set_instances(motions[k], s.mesh_id, s.material_id)
        r = O.render(s.camera, s.width, s.height, s.max_depth, pixels=pix)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            rays += r["closest_rays"] + r["shadow_rays"]
            closest += r["closest_rays"]
    total = sum(times)
    cores = len(os.sched_getaffinity(0))
    value = round(closest / total / 1e6, 3)
    ts = sorted(times)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded procedural scene)",
        "config": {"workload": MEDIUM_WORKLOAD, "width": s.width, "height": s.height, "max_depth": s.max_depth,
                   "sample_pixels_per_step": sample, "p50_ms": round(ts[len(ts) // 2] * 1e3, 3),
                   "p99_ms": round(ts[-1] * 1e3, 3), "parallelism": "host threads"},
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": "Mrays/s",
                         "sample": f"{sample} seeded pixels of each 1920x1080 frame, float64, {cores} threads"},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)



REF_SAMPLE = 65536


def run_reference_large(args, world, rank, local):
    """The oracle on the large workload, on the host cores: per step the
    step's motion (the oracle's instance BVH rebuilt), then a seeded sample of
    REF_SAMPLE closest-hit and REF_SAMPLE any-hit rays of the step's ray sets;
    value = closest-hit rays per second of the steps, as in the native arm."""
    if rank != 0:
        return
    import oracle
    s = g.large_scene()
    n = args.rays
    closest, anyhit = g.large_rays(s, n)
    n_frames = args.warmup + args.steps
    motions = [g.motion(s.M, k) for k in range(min(n_frames, 8))]
    O = oracle.OracleScene(s)
    rng = np.random.default_rng(7)
    times = []
    for k in range(n_frames):
        ic = np.sort(rng.choice(n, REF_SAMPLE, replace=False))
        ia = np.sort(rng.choice(n, REF_SAMPLE, replace=False))
        t0 = time.perf_counter()
        O.set_instances(motions[k % len(motions)], s.mesh_id, s.material_id)
        O.trace(closest[ic])
        O.trace(anyhit[ia], any_hit=True)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    cores = len(os.sched_getaffinity(0))
    value = round(REF_SAMPLE * len(times) / total / 1e6, 4)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded procedural scene and rays)",
        "config": {"workload": LARGE_WORKLOAD, "sample_closest_rays_per_step": REF_SAMPLE,
                   "sample_any_hit_rays_per_step": REF_SAMPLE, "p50_ms": round(pct(times, 0.5) * 1e3, 3),
                   "p99_ms": round(pct(times, 0.99) * 1e3, 3), "parallelism": "host threads"},
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": "Mrays/s",
                         "sample": f"per step: instance BVH rebuild, then {REF_SAMPLE} seeded closest-hit and "
                                   f"{REF_SAMPLE} any-hit rays of the 16,777,216 of each kind, float64, {cores} threads"},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_reference(args, world, rank, local):
    if args.workload == "medium":
        run_reference_medium(args, world, rank, local)
    else:
        run_reference_large(args, world, rank, local)


def run_native_serve(args, world, rank, local):
    import torch
    from paper_2001_09792_gb300 import _build

    torch.cuda.set_device(local)
    _build.build()
    if rank != 0:
        return
    r = run_serving(args.requests, pair=not args.no_pair, lanes=args.lanes, blas_flags=blas_flag(args))
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
        run_native_medium(args, world, rank, local)


if __name__ == "__main__":
    main()
