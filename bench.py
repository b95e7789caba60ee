#!/usr/bin/env python3
"""Benchmark: integrate + incremental mesh (+ refine + gc) per depth frame on one B300.

Workload: the seeded 6 x 4 x 3 m room with 20 random primitives, 640 x 480 float32
depth (fx = fy = 525), smooth random-walk trajectory, noise sigma = 0.0012 z^2 and 2 %
dropped pixels; voxel 8 mm, truncation 3.2 cm, 2^20 hash buckets (synthetic stand-in for
the RGB-D sequences of the paper's Sec. VI).  A step is one frame: vm_step =
integrate_depth + update_mesh(refine) + gc, replayed from a CUDA graph, depth already
resident in HBM.  L2 is flushed (256 MB write) before every timed frame; each frame is
timed with CUDA events on the volume's stream.

The same JSON line also reports the large workload ("large": the 20x20x4 m floor at 5 mm)
and the two forms the method grows into, measured on the same GPU: "batched" (32 independent scenes of uneven sizes, one frame each per tick, five
launches per tick from one CUDA graph, autotuned schedules, against the same scenes stepped
one after another) and "differentiable" (forward and backward of the 60-frame sphere orbit
with 50 leaf depth frames, against the plain path on the same frames).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vmesh|reference]
With N > 1 (torchrun, one rank per GPU) every rank runs an independent replica on its own
seeded scene (no data-path collective); value = frames of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "depth frames/s (integrate+incremental mesh) and voxels/s; % of HBM peak"
UNIT = "frames/s"
WORKLOAD = ("room 6x4x3 m, 20 primitives, 640x480 float32 depth, voxel 8 mm, trunc 3.2 cm, 2^20 buckets; "
            "per frame integrate + incremental mesh + refine + gc")
L2_FLUSH_BYTES = 256 << 20
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

# Algorithmic bytes per launch of the per-frame kernels (the minimum each must move;
# counts come from the library's device counters, per frame):
#   k_integrate  16 B per voxel of the collected blocks (d, W read + write) + 20 B per block
#   k_mesh       11 B per voxel of the update set (d, W read; type read; previous type
#                write; vertex flags read) + 9 B per changed cube (type write, run slot
#                read + write) + 52 B per emitted triangle (16 B record, 3 vertex slots,
#                3 reference-count updates) + 56 B per released triangle (record read +
#                write, 3 reference-count updates) + 36 B per refreshed vertex (slot read,
#                position + normal write) + 52 B per created vertex
#   k_alloc      4 B per depth pixel + 16 B hash bucket per collected block
#   k_gc_blocks  29 B per block pool slot ever used (key, epoch, counts, near flag)
BYTES_MODEL = {
    "k_integrate": lambda s: 16 * 512 * s["frame_blocks"] + 20 * s["frame_blocks"],
    "k_mesh": lambda s: (11 * 512 * s["update_blocks"] + 9 * s["changed"] + 52 * s["emitted"] + 56 * s["released"]
                         + 36 * s["refreshed"] + 52 * s["created"]),
    "k_alloc": lambda s: 4 * s["pixels"] + 16 * s["frame_blocks"],
    "k_gc_blocks": lambda s: 29 * s["high_water"],
}


# DRAM traffic of a kernel (dram__bytes_read.sum + dram__bytes_write.sum) relative to its byte
# model, from the ncu capture summarised in profiles/ (kernels unchanged since that capture
# only).  The capture runs a smaller launch (frames 30-31, ~785 update-set blocks); the
# reported traffic scales it to this run's mean launch by the byte model.
TRAFFIC_RATIO = {
    "k_mesh": (1.004, "ncu --set full of frames 30-31 (15.00 MB DRAM / 14.94 MB modelled), scaled by the byte model"),
}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    def __init__(self, gpu_index: int, out_path: str | None = None):
        self.gpu = gpu_index
        self.proc = None
        self.out_path = out_path

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + CLOCK_QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.2)
        return self

    def __exit__(self, *exc):
        self.text = ""
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.text, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.text = ""
        if self.out_path and self.text:
            with open(self.out_path, "w") as f:
                f.write(self.text)

    def summary(self):
        rows = [r.split(",") for r in self.text.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def reduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def scene_for(rank: int, frames: int):
    # rank 0 runs the canonical seeded room sequence; other replicas use their own seeds
    return synth.room_scene(num_frames=frames, seed=synth.SEED_BASE + 2 + 1000 * rank)


def oracle_frames(scene, frames, warmup=0):
    """Time the float32 oracle (single-threaded C) over `frames` after `warmup` frames."""
    import oracle

    V = oracle.Volume.from_config(scene.volume, prec="f32")
    K = (scene.fx, scene.fy, scene.cx, scene.cy)
    depths = [scene.depth(k) for k in range(warmup + frames)]
    poses = []
    for k in range(warmup + frames):
        T = scene.pose(k).astype(np.float32)
        Ti = synth.pose_inverse_f64(scene.pose(k)).astype(np.float32)
        poses.append((T.astype(np.float64), Ti.astype(np.float64)))
    voxels = 0
    t_total = 0.0
    for k in range(warmup + frames):
        t0 = time.perf_counter()
        V.integrate(depths[k], K, *poses[k])
        V.update_mesh(refine=True)
        V.gc()
        dt = time.perf_counter() - t0
        if k >= warmup:
            t_total += dt
            voxels += 512 * V.stats()["frame_blocks"]
    return frames / t_total, voxels / t_total, t_total


def run_reference(args, rank, world):
    if rank != 0:
        return
    n = args.warmup + args.steps
    scene = scene_for(0, n)
    fps, vps, secs = oracle_frames(scene, args.steps, args.warmup)
    sample = "frames %d..%d of the room sequence (after %d warm-up frames), integrate+update(refine)+gc each" % (
        args.warmup, n - 1, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 / fps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "impl": "float32 CPU oracle (plain single-threaded C)"},
        "voxels_per_s": vps,
        "cpu_baseline": {"value": fps, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": fps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def mesh_bytes(c):
    return BYTES_MODEL["k_mesh"](c)


def run_batched(args, stream, flush, peak):
    """The batched form (BASELINE config 5 reading): `--batch-scenes` independent room scenes of
    uneven sizes (floor plan scaled 1-3.5x, voxel 5-10 mm), one 640x480 frame of each per tick,
    five launches per tick replayed from one CUDA graph, schedules autotuned on the first 6
    warm-up ticks.  Against it: the same scenes and frames stepped one scene after another
    through vm_step (one graph per scene) on fresh volumes.  L2 flushed before every tick."""
    import torch

    from paper_1803_03949_b300 import Intrinsics, Scenes, Volume

    S, T, Wm, P = args.batch_scenes, args.batch_ticks, max(args.batch_warmup, 8), 5
    n = Wm + T + P
    scenes = synth.batch_scenes(S, n)
    dev = [torch.from_numpy(np.stack([sc.depth(k) for k in range(n)])).cuda() for sc in scenes]
    Ks = [Intrinsics(sc.W, sc.H, sc.fx, sc.fy, sc.cx, sc.cy) for sc in scenes]
    poses = []
    for sc in scenes:
        pp = []
        for k in range(n):
            T4 = sc.pose(k)
            pp.append((T4.astype(np.float32), synth.pose_inverse_f64(T4).astype(np.float32)))
        poses.append(pp)

    def tick_args(k):
        return [d[k] for d in dev], Ks, [pp[k] for pp in poses]

    def stat_sum(vols, key):
        return sum(v.stats()[key] for v in vols)

    def timed_ticks(step_tick, k0, k1):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k1 - k0)]
        for i, k in enumerate(range(k0, k1)):
            flush.fill_(k)
            evs[i][0].record(stream)
            step_tick(k)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    # batched
    vols = [Volume.from_config(sc.volume, stream=stream) for sc in scenes]
    batch = Scenes(vols)
    batch.tune(2)
    for k in range(Wm):
        batch.step_all(*tick_args(k), graph=True)
    torch.cuda.synchronize()
    c0, u0 = stat_sum(vols, "collected_blocks"), stat_sum(vols, "meshed_blocks")
    ms = timed_ticks(lambda k: batch.step_all(*tick_args(k), graph=True), Wm, Wm + T)
    c1, u1 = stat_sum(vols, "collected_blocks"), stat_sum(vols, "meshed_blocks")
    # per-kernel times on P more ticks (eager launches with events) and their work counters
    before = [v.stats() for v in vols]
    batch.profile(P)
    for k in range(Wm + T, n):
        flush.fill_(k)
        batch.step_all(*tick_args(k), graph=True)
    kms = batch.kernel_ms()
    after = [v.stats() for v in vols]
    work = dict(update_blocks=0, frame_blocks=0, changed=0, emitted=0, released=0, refreshed=0, created=0)
    for a0, a1 in zip(before, after):
        work["update_blocks"] += (a1["meshed_blocks"] - a0["meshed_blocks"]) % (1 << 32)
        work["frame_blocks"] += (a1["collected_blocks"] - a0["collected_blocks"]) % (1 << 32)
        work["changed"] += a1["changed_cubes"] - a0["changed_cubes"]
        work["emitted"] += a1["emitted_triangles"] - a0["emitted_triangles"]
        work["released"] += a1["released_triangles"] - a0["released_triangles"]
        work["refreshed"] += a1["refreshed_vertices"] - a0["refreshed_vertices"]
        work["created"] += a1["created_vertices"] - a0["created_vertices"]
    roof = {}
    for name, model in (("kb_mesh", mesh_bytes), ("kb_integrate", BYTES_MODEL["k_integrate"])):
        t_ms = kms[name] * kms["ticks"]
        if t_ms > 0:
            gbs = model(work) / (t_ms / 1000.0) / 1e9
            roof[name] = {"avg_launch_us": 1000.0 * kms[name], "achieved": gbs, "peak": peak, "unit": "GB/s",
                          "frac": gbs / peak, "bytes_per_launch": model(work) / kms["ticks"]}
    sched = batch.schedule()
    active = sorted(v.stats()["live_blocks"] for v in vols)
    for v in vols:
        v.check()
    batch.close()
    for v in vols:
        v.close()
    del vols
    torch.cuda.empty_cache()

    # the same scenes one after another through vm_step
    vols = [Volume.from_config(sc.volume, stream=stream) for sc in scenes]

    def seq_tick(k):
        for v, d, K, pp in zip(vols, dev, Ks, poses):
            v.step(d[k], K, *pp[k], refine=True, gc=True, graph=True)

    for k in range(Wm):
        seq_tick(k)
    torch.cuda.synchronize()
    ms_seq = timed_ticks(seq_tick, Wm, Wm + T)
    for v in vols:
        v.check()
        v.close()
    del vols, dev
    torch.cuda.empty_cache()
    tot, tot_seq = sum(ms) / 1000.0, sum(ms_seq) / 1000.0
    return {
        "workload": "%d room scenes (floor plan 6x4 m scaled 1-3.5x log-uniform, 3 m high, 20 primitives, "
                    "voxel 5-10 mm, trunc 4 voxels), 640x480 float32 depth, one frame of each per tick; "
                    "integrate + incremental mesh + refine + gc" % S,
        "scenes": S, "ticks": T, "warmup_ticks": Wm, "value": S * T / tot, "unit": "scene-frames/s",
        "ms_per_tick": 1000.0 * tot / T, "voxels_per_s": 512 * ((c1 - c0) % (1 << 32)) / tot,
        "mean_blocks_per_tick": ((c1 - c0) % (1 << 32)) / T, "mean_update_blocks_per_tick": ((u1 - u0) % (1 << 32)) / T,
        "launches_per_tick": 5, "graph": True, "l2": "flushed before every tick (256 MB write)",
        "sequential": {"value": S * T / tot_seq, "unit": "scene-frames/s", "ms_per_tick": 1000.0 * tot_seq / T,
                       "how": "the same frames through vm_step, one CUDA graph per scene, scenes one after another"},
        "speedup_vs_sequential": tot_seq / tot,
        "schedule": sched["schedule"], "tuned_ms_per_option": sched["tuned_ms"],
        "kernel_ms_per_tick": {k: v for k, v in kms.items() if k != "ticks"}, "profiled_ticks": kms["ticks"],
        "roofline": roof,
        "active_blocks": {"min": active[0], "median": active[len(active) // 2], "max": active[-1]},
    }


def run_large(args, stream, flush, peak):
    """The large workload (BASELINE config 3): the 20x20x4 m floor of 4x4 rooms, 640x480,
    voxel 5 mm, truncation 2 cm, 2^23 buckets; the first `--large-frames` frames after 10
    warm-up frames of the configuration's 2000-frame trajectory (the default keeps the
    benchmark within minutes; `--large-frames 1990` runs all of it), each
    frame integrate + update(refine) + gc from the frame graph, enqueued back to back, L2
    flushed before every frame.  A second pass on a fresh volume times every kernel with event
    nodes (k_mesh and k_integrate for their roofline, all five for the per-frame breakdown)."""
    import torch

    from paper_1803_03949_b300 import Intrinsics, Volume

    T, Wm = args.large_frames, 10
    n = Wm + T
    sc = synth.floor_scene()  # the configuration's 2000-frame trajectory, its first n frames
    vc = sc.volume
    if args.small_pools:  # the first few hundred frames fit; keeps profiling captures small
        import dataclasses

        vc = dataclasses.replace(vc, hash_buckets=1 << 20, max_blocks=1 << 18, max_vertices=1 << 23,
                                 max_triangles=1 << 24)
    dev = torch.from_numpy(np.stack([sc.depth(k) for k in range(n)])).cuda()
    K = Intrinsics(sc.W, sc.H, sc.fx, sc.fy, sc.cx, sc.cy)
    poses = []
    for k in range(n):
        T4 = sc.pose(k)
        poses.append((T4.astype(np.float32), synth.pose_inverse_f64(T4).astype(np.float32)))

    def run(timing):
        v = Volume.from_config(vc, stream=stream)
        for k in range(Wm):
            v.step(dev[k], K, *poses[k], refine=True, gc=True, graph=True)
        if timing:
            v.enable_timing(True)
        torch.cuda.synchronize()
        s0 = v.stats()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(T)]
        work = dict(update_blocks=0, frame_blocks=0, changed=0, emitted=0, released=0, refreshed=0, created=0)
        prev = s0
        for i, k in enumerate(range(Wm, n)):
            flush.fill_(k)
            evs[i][0].record(stream)
            v.step(dev[k], K, *poses[k], refine=True, gc=True, graph=True)
            evs[i][1].record(stream)
            if timing:  # per-frame work counters for the byte model
                st = v.stats()
                work["update_blocks"] += st["update_blocks"]
                work["frame_blocks"] += st["frame_blocks"]
                work["changed"] += st["changed_cubes"] - prev["changed_cubes"]
                work["emitted"] += st["emitted_triangles"] - prev["emitted_triangles"]
                work["released"] += st["released_triangles"] - prev["released_triangles"]
                work["refreshed"] += st["refreshed_vertices"] - prev["refreshed_vertices"]
                work["created"] += st["created_vertices"] - prev["created_vertices"]
                prev = st
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in evs]
        s1 = v.stats()
        kt = v.kernel_times() if timing else {}
        v.check()
        v.close()
        return ms, s0, s1, kt, work

    ms, s0, s1, _, _ = run(False)
    if args.only_large:  # one pass (profiling captures)
        kt, work = {}, {}
    else:
        _, _, _, kt, work = run(True)
    del dev
    torch.cuda.empty_cache()
    tot = sum(ms) / 1000.0
    collected = (s1["collected_blocks"] - s0["collected_blocks"]) % (1 << 32)
    roof = {}
    for name, model in (("k_mesh", mesh_bytes), ("k_integrate", BYTES_MODEL["k_integrate"])):
        t_ms, cnt = kt.get(name, (0.0, 0))
        if t_ms > 0:
            gbs = model(work) / (t_ms / 1000.0) / 1e9
            roof[name] = {"avg_launch_us": 1000.0 * t_ms / cnt, "achieved": gbs, "peak": peak, "unit": "GB/s",
                          "frac": gbs / peak, "bytes_per_launch": model(work) / max(cnt, 1)}
    return {
        "workload": "floor 20x20x4 m (4x4 rooms with doorways, 8 primitives each), 640x480 float32 depth, voxel 5 mm, "
                    "trunc 2 cm, 2^23 buckets; per frame integrate + incremental mesh + refine + gc",
        "frames": T, "warmup": Wm, "value": T / tot, "unit": "frames/s", "ms_per_step": 1000.0 * tot / T,
        "voxels_per_s": 512 * collected / tot, "mean_blocks_per_frame": collected / T,
        "live_blocks_at_end": s1["live_blocks"], "l2": "flushed before every frame (256 MB write)",
        "roofline": roof,
        "kernel_us_per_frame": {k: 1000.0 * t / max(c, 1) for k, (t, c) in kt.items()},
        "work_per_frame": dict({k: v / T for k, v in work.items()},
                               freed_vertices=(s1["freed_vertices"] - s0["freed_vertices"]) / T,
                               freed_blocks=(s1["freed_blocks"] - s0["freed_blocks"]) / T),
    }


def run_differentiable(args, stream):
    """The differentiable form (BASELINE config 4 reading): the sphere orbit extended to 60
    frames, frames 0-9 integrated as constants, frames 10-59 leaf tensors; forward = the 50
    recorded integrations + one full refined mesh + download, backward = loss.backward()
    (vertex -> TSDF -> depth kernels, 50 reverse steps).  Against it: the plain path on the
    same frames (50 integrations + full refined mesh + download).  CUDA events; median of 5."""
    import torch

    from paper_1803_03949_b300 import Intrinsics, Volume, diff_mesh

    sc = synth.sphere_scene(num_frames=60)
    K = Intrinsics(sc.W, sc.H, sc.fx, sc.fy, sc.cx, sc.cy)
    dev = [torch.from_numpy(sc.depth(k)).cuda() for k in range(60)]
    poses = []
    for k in range(60):
        T4 = sc.pose(k)
        poses.append((T4.astype(np.float32), synth.pose_inverse_f64(T4).astype(np.float32)))
    c = torch.tensor([0.0, 0.0, 0.3], device="cuda")

    def loss_fn(pos, nrm):
        r = pos - c
        dist = torch.linalg.norm(r, dim=1)
        sph = dist - 0.3 <= pos[:, 2]
        sdf = torch.where(sph, dist - 0.3, pos[:, 2])
        up = torch.zeros_like(pos)
        up[:, 2] = 1.0
        u = torch.where(sph[:, None], r / dist[:, None], up)
        return (sdf ** 2).mean() + 0.1 * (1.0 - (nrm * u).sum(1)).mean()

    plain, fwd, bwd, nverts = [], [], [], 0
    for rep in range(5):
        v = Volume.from_config(sc.volume, stream=stream)
        for k in range(10):
            v.integrate(dev[k], K, *poses[k])
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        for k in range(10, 60):
            v.integrate(dev[k], K, *poses[k])
        v.update_mesh(full=True, refine=True)
        m = v.download(device=True)
        e[1].record(stream)
        torch.cuda.synchronize()
        plain.append(e[0].elapsed_time(e[1]))
        v.close()
        v = Volume.from_config(sc.volume, stream=stream)
        for k in range(10):
            v.integrate(dev[k], K, *poses[k])
        leaves = [d.clone().requires_grad_(True) for d in dev[10:]]
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        e[0].record(stream)
        pos, nrm, tris, keys = diff_mesh(v, K, poses[10:], leaves, refine=True)
        e[1].record(stream)
        loss = loss_fn(pos, nrm)
        e[2].record(stream)
        loss.backward()
        e[3].record(stream)
        torch.cuda.synchronize()
        fwd.append(e[0].elapsed_time(e[1]))
        bwd.append(e[2].elapsed_time(e[3]))
        nverts = int(pos.shape[0])
        v.check()
        v.close()
    med = statistics.median
    return {
        "workload": "sphere orbit 320x240, 60 frames (0-9 constant, 10-59 leaf depth tensors), voxel 1 cm; "
                    "loss = mean sdf^2 + 0.1 mean(1 - n . grad sdf / |grad sdf|)",
        "plain_forward_ms": med(plain), "diff_forward_ms": med(fwd), "backward_ms": med(bwd),
        "forward_overhead": med(fwd) / med(plain), "backward_over_forward": med(bwd) / med(fwd),
        "vertices": nverts, "leaf_pixels": 50 * sc.W * sc.H,
        "timing": "CUDA events on the volume's stream, median of 5 runs, caches warm",
    }


def run_vmesh(args, rank, world, local):
    import torch

    from paper_1803_03949_b300 import Intrinsics, Volume

    torch.cuda.set_device(local)
    if args.only_large:
        if rank == 0:
            flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
            print(json.dumps({"large": run_large(args, torch.cuda.current_stream(), flush, load_peaks()[0])}), flush=True)
        return
    n = args.warmup + args.steps
    scene = scene_for(rank, n)
    H, W = scene.H, scene.W
    depth_host = torch.empty((n, H, W), dtype=torch.float32).pin_memory()
    for k in range(n):
        depth_host[k].copy_(torch.from_numpy(scene.depth(k)))
    depth_dev = depth_host.cuda()
    poses = []
    for k in range(n):
        T = scene.pose(k)
        poses.append((T.astype(np.float32), synth.pose_inverse_f64(T).astype(np.float32)))
    K = Intrinsics(W, H, scene.fx, scene.fy, scene.cx, scene.cy)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    graph = not args.no_graph
    vc = scene.volume
    if args.small_pools:  # same workload, smaller pool allocations (profiling captures)
        import dataclasses

        vc = dataclasses.replace(vc, max_blocks=1 << 15, max_vertices=1 << 21, max_triangles=1 << 22)

    def warm_up(vol, calibrate=False):
        """Frames 0..W-1, untimed.  With calibrate, every kernel is timed on frames 0..W-2
        (a per-kernel breakdown); the last warm-up frame captures the graph without events."""
        calib = {}
        if calibrate:
            vol.enable_timing(True)
        for f in range(args.warmup):
            if calibrate and f == args.warmup - 1:
                calib = vol.kernel_times()
                vol.enable_timing(False)
            vol.step(depth_dev[f], K, *poses[f], refine=True, gc=True, graph=graph)
        torch.cuda.synchronize()
        return calib

    def timed(vol, timing_kernels=()):
        """Frames W..W+K-1 one at a time, each bracketed by CUDA events on the volume's stream
        after a 256 MB L2 flush; returns per-frame ms, per-frame work counters and kernel
        times (the host reads the counters after every frame)."""
        if timing_kernels:
            vol.enable_timing(list(timing_kernels))
        ms, counters = [], []
        prev = vol.stats()
        for f in range(args.warmup, n):
            flush.fill_(f)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vol.step(depth_dev[f], K, *poses[f], refine=True, gc=True, graph=graph)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            st = vol.stats()
            counters.append(dict(frame_blocks=st["frame_blocks"], update_blocks=st["update_blocks"],
                                 changed=st["changed_cubes"] - prev["changed_cubes"],
                                 emitted=st["emitted_triangles"] - prev["emitted_triangles"],
                                 released=st["released_triangles"] - prev["released_triangles"],
                                 refreshed=st["refreshed_vertices"] - prev["refreshed_vertices"],
                                 created=st["created_vertices"] - prev["created_vertices"],
                                 high_water=st["block_high_water"], pixels=W * H))
            prev = st
        kt = vol.kernel_times() if timing_kernels else {}
        vol.check()
        return ms, counters, kt

    def streamed(vol, e2e=False):
        """Frames W..W+K-1 enqueued back to back, the host never waiting between frames (as
        a camera stream would run): per frame an L2 flush, then a CUDA-event pair around the
        frame alone.  Returns per-frame ms and the blocks collected / meshed over the run."""
        res_host = torch.empty(2, dtype=torch.int32).pin_memory()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        s0 = vol.stats()
        # hold the stream while the host enqueues the frames (about 0.5 ms of GPU time per
        # frame, outside every frame's event window), so that no window waits on the host: on
        # a shared host, enqueue jitter (and the clock sampler's driver queries) would
        # otherwise enter the timing
        torch.cuda._sleep(int(min(n - args.warmup, 2000) * 1000000))
        for i, f in enumerate(range(args.warmup, n)):
            flush.fill_(f)
            evs[i][0].record(stream)
            if e2e:
                # the frame from pinned host memory: the collection kernel reads it across the
                # host link (4 W H bytes) and keeps the device copy the later kernels read
                vol.step(depth_host[f], K, *poses[f], refine=True, gc=True, graph=graph)
                vol.mesh_size_async(res_host)
            else:
                vol.step(depth_dev[f], K, *poses[f], refine=True, gc=True, graph=graph)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in evs]
        s1 = vol.stats()
        vol.check()
        wrap = lambda d: d % (1 << 32)
        return ms, wrap(s1["collected_blocks"] - s0["collected_blocks"]), wrap(s1["meshed_blocks"] - s0["meshed_blocks"])

    # pass 1 -- the benchmark value: no event nodes inside the frame graph
    vol = Volume.from_config(vc, stream=stream)
    calib = warm_up(vol, calibrate=True)
    barrier(world)
    with ClockSampler(local, args.clock_csv if rank == 0 else None) as cs:
        ms, collected, meshed = streamed(vol)
        torch.cuda.synchronize()
    barrier(world)
    mem = vol.mesh_memory()
    vol.close()
    total_ms = sum(ms)
    max_ms = reduce_max(total_ms, world)
    value = world * args.steps / (max_ms / 1000.0)
    vps = 512 * collected / (total_ms / 1000.0)

    # the compact cube record on the same frames (value pass only): speed and memory
    import dataclasses

    volc = Volume.from_config(dataclasses.replace(vc, compact_edges=True), stream=stream)
    warm_up(volc)
    ms_c, _, _ = streamed(volc)
    mem_c = volc.mesh_memory()
    volc.close()
    compact = {"value": args.steps / (sum(ms_c) / 1000.0), "unit": UNIT, "cube_bytes": mem_c["cube_bytes"],
               "edge_records": mem_c["edge_records"], "bytes_in_use": mem_c["bytes_in_use"],
               "bytes_allocated": mem_c["bytes_allocated"]}

    # pass 2 -- kernel durations: the same frames on a fresh volume (identical, deterministic
    # work), with CUDA-event pairs around the two kernels the calibration ranked highest
    peak, peak_kind = load_peaks()
    ranked = sorted((k for k in calib if k in BYTES_MODEL and calib[k][1] > 0), key=lambda k: -calib[k][0])[:2]
    roof = None
    if ranked and not args.no_kernel_timing:
        vol2 = Volume.from_config(vc, stream=stream)
        warm_up(vol2)
        ms2, counters2, kt = timed(vol2, timing_kernels=ranked)
        vol2.close()
        main = {k: kt[k] for k in ranked if kt.get(k, (0, 0))[1] > 0}
        dom = max(main, key=lambda k: main[k][0])
        tot_ms_k, launches = main[dom]
        bytes_total = sum(BYTES_MODEL[dom](c) for c in counters2)
        achieved = bytes_total / (tot_ms_k / 1000.0) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": TRAFFIC_RATIO[dom][0] * bytes_total / max(launches, 1) if dom in TRAFFIC_RATIO else None,
                "traffic_source": TRAFFIC_RATIO[dom][1] if dom in TRAFFIC_RATIO else None,
                "bytes_per_launch": bytes_total / max(launches, 1),
                "avg_launch_us": 1000.0 * tot_ms_k / max(launches, 1),
                "timing": "CUDA events around the kernel, same frames replayed on a fresh volume"}
        for k in main:
            if k != dom:
                kb = sum(BYTES_MODEL[k](c) for c in counters2)
                roof["runner_up"] = {"kernel": k, "avg_launch_us": 1000.0 * main[k][0] / max(main[k][1], 1),
                                     "achieved": kb / (main[k][0] / 1000.0) / 1e9}
    # kernels per frame, counted on the calibration frames (every launch timed there)
    calib_frames = max(args.warmup - 1, 1)
    per_frame_launches = round(sum(v[1] for v in calib.values()) / calib_frames) if calib else None
    launches_total = per_frame_launches * args.steps if per_frame_launches else None

    # pass 3 -- end to end through the public API: pinned host depth -> device, step, result -> host
    vol3 = Volume.from_config(vc, stream=stream)
    warm_up(vol3)
    ms_e2e, _, _ = streamed(vol3, e2e=True)
    vol3.close()
    e2e_value = world * args.steps / (reduce_max(sum(ms_e2e), world) / 1000.0)

    if rank != 0:
        return
    cpu = None
    if not args.skip_cpu_baseline:
        nframes = min(args.cpu_frames, n)
        fps, cvps, secs = oracle_frames(scene_for(0, nframes), nframes)
        cpu = {"value": fps, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "frames 0..%d of the same room sequence, integrate+update(refine)+gc each (%.1f s)" % (
                   nframes - 1, secs), "voxels_per_s": cvps}
    kernel_ms = {k: round(v[0] / calib_frames, 5) for k, v in calib.items() if v[1] > 0}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames": "%d..%d" % (args.warmup, n - 1),
                   "graph": graph, "l2": "flushed before every timed frame (256 MB write)",
                   "submission": "frames enqueued back to back; per-frame CUDA events exclude the flush",
                   "parallelism": "replicas" if world > 1 else "single"},
        "voxels_per_s": vps,
        "mean_blocks_per_frame": collected / args.steps,
        "mean_update_blocks_per_frame": meshed / args.steps,
        "kernel_ms_per_frame_warmup": kernel_ms,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * W * H, "d2h_bytes_per_step": 8,
                "path": "vm_step on the depth frame in pinned host memory (read across the host link by the "
                        "collection kernel), then vm_mesh_size_async into pinned host memory, per frame"},
        "gpu_launches": launches_total,
        "clocks": cs.summary(),
        "mesh_memory": {
            "after_frames": n, "vertices": mem["vertices"], "triangles": mem["triangles"],
            "per_block_extraction_vertices": mem["block_vertices"], "loose_triangle_vertices": mem["loose_vertices"],
            "per_block_over_ours": mem["block_vertices"] / max(mem["vertices"], 1),
            "loose_over_ours": mem["loose_vertices"] / max(mem["vertices"], 1),
            "blocks": mem["blocks"], "cube_bytes": mem["cube_bytes"], "edge_records": mem["edge_records"],
            "paper_cube_bytes": 56,
            "paper_compact_cube_bytes": 24, "bytes_in_use": mem["bytes_in_use"],
            "bytes_allocated": mem["bytes_allocated"],
            "compact_layout": compact,
        },
    }
    if not args.skip_forms:
        line["large"] = run_large(args, stream, flush, peak)
        line["batched"] = run_batched(args, stream, flush, peak)
        line["differentiable"] = run_differentiable(args, stream)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["vmesh", "reference"], default="vmesh")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--small-pools", action="store_true", help="smaller pool allocations (ncu captures)")
    ap.add_argument("--no-kernel-timing", action="store_true",
                    help="time frames without per-kernel event nodes (no roofline)")
    ap.add_argument("--cpu-frames", type=int, default=200)
    ap.add_argument("--skip-forms", action="store_true", help="skip the batched and differentiable forms")
    ap.add_argument("--clock-csv", default=None, help="also write the clock samples of the timed pass to this CSV")
    ap.add_argument("--large-frames", type=int, default=300)
    ap.add_argument("--only-large", action="store_true", help="run only the large workload's plain pass")
    ap.add_argument("--batch-scenes", type=int, default=32)
    ap.add_argument("--batch-ticks", type=int, default=60)
    ap.add_argument("--batch-warmup", type=int, default=10)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_vmesh(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
