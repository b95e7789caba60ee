#!/usr/bin/env python3
"""Benchmark: integrate + incremental mesh + refine + gc per depth frame on one B300.

Headline workload (the largest single-GPU configuration): the seeded 20 x 20 x 4 m floor of
4 x 4 rooms with doorways and 8 primitives per room, 640 x 480 float32 depth (fx = fy = 525),
a serpentine trajectory of 2000 frames through the doorways, noise sigma = 0.0012 z^2, 2 %
dropped pixels and a 4.5 m sensor range; voxel 5 mm, truncation 2 cm, 2^23 hash buckets,
pools of 2^21 blocks, 2^26 vertices, 2^27 triangles (synthetic stand-in for the RGB-D
sequences of the paper's Sec. VI).  A step is one frame: vm_step = integrate_depth +
update_mesh(refine) + gc, replayed from a CUDA graph, depth already resident in HBM.  The
timed steps are frames W .. W+K-1 of the trajectory after W untimed warm-up frames.  L2 is
flushed (256 MB write) before every timed frame; each frame is timed with CUDA events on the
volume's stream.

The same JSON line reports, measured in the same run on the same GPU: the whole-frame
roofline (algorithmic bytes per frame over the frame time) beside the dominant kernel's, two
end-to-end figures through the public API (depth from pinned host memory and the mesh size
read back; the same plus the mesh compacted every frame, the "compress" step of Table I),
the float32 CPU oracle on a bounded sample of the same frames, "full_sequence" (all 2000
frames of the floor), "room" (the 6 x 4 x 3 m room at 8 mm, the previous headline), and the
two forms the method grows into: "batched" and "batched_small" (32 independent scenes of uneven
sizes, 4.5k-150k and 0.5k-21k active blocks, one frame each per tick over 500 ticks, five
launches per tick from one CUDA graph, against the same scenes stepped one after another) and
"differentiable" (forward and backward of the 60-frame sphere orbit with 50
leaf depth frames, against the plain path on the same frames).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vmesh|reference]
With N > 1 (torchrun, one rank per GPU) every rank runs an independent replica on its own
seeded floor (no data-path collective); value = frames of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import dataclasses
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
FLOOR_WORKLOAD = ("floor 20x20x4 m (4x4 rooms with doorways, 8 primitives each), 640x480 float32 depth, voxel 5 mm, "
                  "trunc 2 cm, 2^23 buckets; per frame integrate + incremental mesh + refine + gc")
ROOM_WORKLOAD = ("room 6x4x3 m, 20 primitives, 640x480 float32 depth, voxel 8 mm, trunc 3.2 cm, 2^20 buckets; "
                 "per frame integrate + incremental mesh + refine + gc")
FLOOR_FRAMES = 2000  # the floor trajectory's length; the timed frames are a window of it
NOMINAL_HBM_GBS = 8000.0  # HBM3e bandwidth quoted for B300 (the measured copy rate is the main denominator)
L2_FLUSH_BYTES = 256 << 20
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,clocks.mem")

# Algorithmic bytes per launch of the per-frame kernels (the minimum each must move; counts
# come from the library's device counters, per frame):
#   k_alloc       4 B per depth pixel + 16 B hash bucket per collected block
#   k_integrate   16 B per voxel of the collected blocks (d, W read + write) + 20 B per block
#   k_mesh        11 B per voxel of the update set (d, W read; type read; previous type
#                 write; vertex flags read) + 9 B per changed cube (type write, run slot read +
#                 write) + 28 B per emitted triangle (16 B record, 3 vertex slots) + 32 B per
#                 released triangle (record read + clear) + 8 B per reference-count update
#                 (read-modify-write of a 4-byte count; one per edge whose use changes) + 36 B per
#                 refreshed vertex (slot read, position + normal write) + 52 B per created vertex
#   k_gc_vertices 29 B per freed vertex (list entry, edge, count, edge slot, flag byte, block
#                 count, stack slot); the released runs' few bytes are left out (a lower bound)
#   k_gc_blocks   29 B per block pool slot ever used (key, epoch, counts, near flag)
BYTES_MODEL = {
    "k_alloc": lambda s: 4 * s["pixels"] + 16 * s["frame_blocks"],
    "k_integrate": lambda s: 16 * 512 * s["frame_blocks"] + 20 * s["frame_blocks"],
    "k_mesh": lambda s: (11 * 512 * s["update_blocks"] + 9 * s["changed"] + 28 * s["emitted"] + 32 * s["released"]
                         + 8 * s["refupd"] + 36 * s["refreshed"] + 52 * s["created"]),
    "k_gc_vertices": lambda s: 29 * s["freed_vertices"],
    "k_gc_blocks": lambda s: 29 * s["high_water"],
}
FRAME_KERNELS = ["k_alloc", "k_integrate", "k_mesh", "k_gc_vertices", "k_gc_blocks"]


def frame_bytes(c):
    return sum(BYTES_MODEL[k](c) for k in FRAME_KERNELS)


# DRAM traffic of a kernel (dram__bytes_read.sum + dram__bytes_write.sum) relative to its byte
# model, from the ncu captures summarised in profiles/, per workload (kernels unchanged since
# the capture only).  The reported traffic scales the ratio to this run's mean launch.
TRAFFIC_RATIO = {
    ("floor", "k_mesh"): (287.6 / 195.2, "profiles/k_mesh_floor640x480.md: one launch's dram bytes (frame 8, "
                          "15,287 update-set blocks) over its byte model, scaled to this run's mean launch"),
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
        rows = [r.split(",") for r in self.text.strip().splitlines() if r.count(",") >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "mem_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        mem = statistics.median(float(r[9]) for r in rows)  # the memory clock (boxes differ in HBM rate)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "mem_mhz": mem, "reasons": reasons,
                "samples": len(rows)}


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


def scene_for(rank: int, frames: int = FLOOR_FRAMES):
    """The headline workload of a replica: rank 0 runs the canonical seeded floor; other replicas
    use their own seeds.  The trajectory always has the configuration's 2000 frames (a shorter one
    would move the camera faster); runs use a window of it."""
    if frames > FLOOR_FRAMES:
        raise ValueError("the floor trajectory has %d frames" % FLOOR_FRAMES)
    return synth.floor_scene(num_frames=FLOOR_FRAMES, seed=synth.SEED_BASE + 3 + 1000 * rank)


def room_scene_for(rank: int, frames: int):
    return synth.room_scene(num_frames=frames, seed=synth.SEED_BASE + 2 + 1000 * rank)


def oracle_frames(scene, frames, warmup=0, budget_s=None):
    """Time the float32 oracle (single-threaded C) on frames warmup .. warmup + frames - 1 (after
    the untimed warm-up frames), stopping early once `budget_s` seconds of timed work have run
    (at least one frame).  Returns (frames/s, voxels/s, seconds, frames timed)."""
    import oracle

    V = oracle.Volume.from_config(scene.volume, prec="f32")
    K = (scene.fx, scene.fy, scene.cx, scene.cy)
    voxels = 0
    t_total = 0.0
    timed = 0
    for k in range(warmup + frames):
        d = scene.depth(k)
        T = scene.pose(k).astype(np.float32)
        Ti = synth.pose_inverse_f64(scene.pose(k)).astype(np.float32)
        t0 = time.perf_counter()
        V.integrate(d, K, T.astype(np.float64), Ti.astype(np.float64))
        V.update_mesh(refine=True)
        V.gc()
        dt = time.perf_counter() - t0
        if k >= warmup:
            t_total += dt
            timed += 1
            voxels += 512 * V.stats()["frame_blocks"]
            if budget_s is not None and t_total >= budget_s:
                break
    return timed / t_total, voxels / t_total, t_total, timed


def run_reference(args, rank, world):
    if rank != 0:
        return
    scene = scene_for(0)
    fps, vps, secs, timed = oracle_frames(scene, args.steps, args.warmup, budget_s=args.reference_seconds)
    sample = ("frames %d..%d of the floor sequence (after %d untimed warm-up frames), integrate+update(refine)+gc "
              "each, %.1f s%s" % (args.warmup, args.warmup + timed - 1, args.warmup, secs,
                                 "" if timed == args.steps else "; stopped after %d of the %d steps at the %.0f s budget"
                                 % (timed, args.steps, args.reference_seconds)))
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 / fps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": FLOOR_WORKLOAD, "impl": "float32 CPU oracle (plain single-threaded C)"},
        "voxels_per_s": vps,
        "cpu_baseline": {"value": fps, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": fps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def mesh_bytes(c):
    return BYTES_MODEL["k_mesh"](c)


BATCH_MIXES = {
    # the room recipe scaled 1-3.5x, voxel 5-10 mm: over 500 ticks the scenes grow to 4.5k-150k
    # active blocks (BASELINE config 5's 5k-200k)
    "mixed": dict(scale_range=(1.0, 3.5), voxel_mm=(5, 10)),
    # small rooms (scaled 0.5-1x, voxel 8-10 mm, 0.5k-21k active blocks): one frame of one scene
    # leaves most of the GPU idle, the case a batch is for
    "small": dict(scale_range=(0.5, 1.0), voxel_mm=(8, 10)),
}


def batch_frames(scenes, n, workers=16):
    """Every scene's frames 0..n-1 on the device, one (n, H, W) tensor per scene, rendered on
    host threads (the generator releases the interpreter lock) one scene at a time."""
    import concurrent.futures as cf

    import torch

    out = []
    with cf.ThreadPoolExecutor(workers) as ex:
        for sc in scenes:
            host = np.stack(list(ex.map(sc.depth, range(n))))
            out.append(torch.from_numpy(host).cuda())
            del host
    return out


def run_batched(args, stream, flush, peak, mix="mixed"):
    """The batched form (BASELINE config 5 reading): `--batch-scenes` independent room scenes of
    uneven sizes (BATCH_MIXES), one 640x480 frame of each per tick, five launches per tick
    replayed from one CUDA graph, schedules autotuned on the first 6 warm-up ticks, then
    `--batch-ticks` timed ticks.  Against it: the same scenes and frames stepped one scene after
    another through vm_step (one graph per scene) on fresh volumes.  L2 flushed before every tick.
    Also the empty tick: the same five-launch graph on fresh volumes with all-invalid depth, the
    fixed cost of the launch structure (what one persistent launch per tick could save at most)."""
    import torch

    from paper_1803_03949_b300 import Intrinsics, Scenes, Volume

    S, T, Wm, P = args.batch_scenes, args.batch_ticks, max(args.batch_warmup, 8), 5
    n = Wm + T + P
    scenes = synth.batch_scenes(S, n, **BATCH_MIXES[mix])
    dev = batch_frames(scenes, n)
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

    def active(vols):
        a = sorted(v.stats()["live_blocks"] for v in vols)
        return {"min": a[0], "median": a[len(a) // 2], "max": a[-1]}

    def timed_ticks(step_tick, k0, k1):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k1 - k0)]
        # hold the stream while the host enqueues the first ticks (~0.5 ms of GPU time per tick,
        # outside every tick's event window), so that no window waits on the host
        torch.cuda._sleep(int(min(k1 - k0, 200) * 1000000))
        for i, k in enumerate(range(k0, k1)):
            flush.fill_(k)
            evs[i][0].record(stream)
            step_tick(k)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    # the empty tick: fresh volumes, every pixel invalid
    vols = [Volume.from_config(sc.volume, stream=stream) for sc in scenes]
    batch = Scenes(vols)
    zero = [torch.zeros_like(d[0]) for d in dev]
    for k in range(3):
        batch.step_all(zero, Ks, [pp[k] for pp in poses], graph=True)
    ms_empty = timed_ticks(lambda k: batch.step_all(zero, Ks, [pp[k] for pp in poses], graph=True), 3, 23)
    batch.close()
    for v in vols:
        v.close()
    del vols, zero

    # batched
    vols = [Volume.from_config(sc.volume, stream=stream) for sc in scenes]
    batch = Scenes(vols)
    batch.tune(2)
    for k in range(Wm):
        batch.step_all(*tick_args(k), graph=True)
    torch.cuda.synchronize()
    act0 = active(vols)
    c0, u0 = stat_sum(vols, "collected_blocks"), stat_sum(vols, "meshed_blocks")
    ms = timed_ticks(lambda k: batch.step_all(*tick_args(k), graph=True), Wm, Wm + T)
    c1, u1 = stat_sum(vols, "collected_blocks"), stat_sum(vols, "meshed_blocks")
    act1 = active(vols)
    # per-kernel times on P more ticks (eager launches with events) and their work counters
    before = [v.stats() for v in vols]
    batch.profile(P)
    for k in range(Wm + T, n):
        flush.fill_(k)
        batch.step_all(*tick_args(k), graph=True)
    kms = batch.kernel_ms()
    after = [v.stats() for v in vols]
    work = dict(update_blocks=0, frame_blocks=0, changed=0, emitted=0, released=0, refreshed=0, created=0, refupd=0)
    for a0, a1 in zip(before, after):
        work["refupd"] += a1["reference_updates"] - a0["reference_updates"]
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
    mk = BATCH_MIXES[mix]
    empty_us = 1000.0 * float(np.median(ms_empty))
    return {
        "workload": "%d room scenes (floor plan 6x4 m scaled %g-%gx log-uniform, 3 m high, 20 primitives, "
                    "voxel %d-%d mm, trunc 4 voxels, 4.5 m sensor range), 640x480 float32 depth, one frame of each "
                    "per tick; integrate + incremental mesh + refine + gc"
                    % (S, mk["scale_range"][0], mk["scale_range"][1], mk["voxel_mm"][0], mk["voxel_mm"][1]),
        "scenes": S, "ticks": T, "warmup_ticks": Wm, "value": S * T / tot, "unit": "scene-frames/s",
        "ms_per_tick": 1000.0 * tot / T, "voxels_per_s": 512 * ((c1 - c0) % (1 << 32)) / tot,
        "mean_blocks_per_tick": ((c1 - c0) % (1 << 32)) / T, "mean_update_blocks_per_tick": ((u1 - u0) % (1 << 32)) / T,
        "launches_per_tick": 5, "graph": True, "l2": "flushed before every tick (256 MB write)",
        "sequential": {"value": S * T / tot_seq, "unit": "scene-frames/s", "ms_per_tick": 1000.0 * tot_seq / T,
                       "how": "the same frames through vm_step, one CUDA graph per scene, scenes one after another"},
        "speedup_vs_sequential": tot_seq / tot,
        "empty_tick": {"us": empty_us, "share_of_tick": empty_us / (1000.0 * 1000.0 * tot / T),
                       "how": "median of 20 ticks of the same five-launch graph on fresh volumes with all-invalid "
                              "depth: the launch structure's fixed cost, the most one persistent launch could save"},
        "schedule": sched["schedule"], "tuned_ms_per_option": sched["tuned_ms"],
        "kernel_ms_per_tick": {k: v for k, v in kms.items() if k != "ticks"}, "profiled_ticks": kms["ticks"],
        "roofline": roof,
        "active_blocks": {"timed_start": act0, "timed_end": act1},
    }


def run_differentiable(args, stream):
    """The differentiable form (BASELINE config 4 reading): the sphere orbit extended to 60
    frames, frames 0-9 integrated as constants, frames 10-59 leaf tensors; forward = the 50
    recorded integrations + one full refined mesh + download, backward = loss.backward()
    (vertex -> TSDF -> depth kernels, 50 reverse steps).  Against it: the plain path on the
    same frames (50 integrations + full refined mesh + download).  CUDA events; median of --diff-reps runs."""
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
    for rep in range(args.diff_reps):
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
        "timing": "CUDA events on the volume's stream, median of %d runs, caches warm" % args.diff_reps,
        "backward_over_forward_p10_p90": [float(x) for x in np.quantile(np.array(bwd) / np.array(fwd), [0.1, 0.9])],
    }




def measure(args, scene, vc, W, K, stream, flush, peak, peak_kind, world, rank, local, label, clocks=False,
            memory=False):
    """One workload's measurements over frames W .. W+K-1 after W warm-up frames (each pass on a
    fresh volume, the same frames, so the same deterministic work):
      pass 1 -- value: frames enqueued back to back, no event node inside the frame graph;
      pass 2 -- kernels: CUDA-event pairs around every kernel of the frame, per-frame work counters
                (the byte models); the dominant kernel's and the whole frame's rooflines;
      pass 3 -- e2e: depth copied from pinned host memory (a double buffer on a copy stream, the
                next frame's copy inside the current frame's window), the mesh size read back
                every frame;
      pass 4 -- e2e with compress: as pass 3, plus the whole mesh compacted into fresh device
                buffers every frame (vm_get_stats + vm_download_mesh_into)."""
    import torch

    from paper_1803_03949_b300 import Intrinsics, Volume

    n = W + K
    H, Wd = scene.H, scene.W
    depth_host = torch.empty((n, H, Wd), dtype=torch.float32).pin_memory()
    for k in range(n):
        depth_host[k].copy_(torch.from_numpy(scene.depth(k)))
    depth_dev = depth_host.cuda()
    poses = []
    for k in range(n):
        T = scene.pose(k)
        poses.append((T.astype(np.float32), synth.pose_inverse_f64(T).astype(np.float32)))
    Kc = Intrinsics(Wd, H, scene.fx, scene.fy, scene.cx, scene.cy)
    graph = not args.no_graph

    def warm_up(vol, calibrate=False):
        """Frames 0..W-1, untimed.  With calibrate, every kernel is timed on frames 0..W-2 (the
        launch count per frame); the last warm-up frame captures the graph without events."""
        calib = {}
        if calibrate:
            vol.enable_timing(True)
        for f in range(W):
            if calibrate and f == W - 1:
                calib = vol.kernel_times()
                vol.enable_timing(False)
            vol.step(depth_dev[f], Kc, *poses[f], refine=True, gc=True, graph=graph)
        torch.cuda.synchronize()
        return calib

    def streamed(vol, mode="device"):
        """Frames W..W+K-1 enqueued back to back, the host never waiting between frames (as a
        camera stream would run; mode 'compress' waits inside every frame for the mesh size):
        per frame an L2 flush, then a CUDA-event pair around the frame alone.  Returns per-frame
        ms, the blocks collected / meshed over the run and the bytes copied per frame."""
        res_host = torch.empty(2, dtype=torch.int32).pin_memory()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        s0 = vol.stats()
        if mode != "compress":
            # hold the stream while the host enqueues the frames (about 0.5 ms of GPU time per
            # frame, outside every frame's event window), so that no window waits on the host: on
            # a shared host, enqueue jitter (and the clock sampler's driver queries) would
            # otherwise enter the timing
            torch.cuda._sleep(int(min(K, 2000) * 1000000))
        d2h = 0
        if mode != "device":
            # end to end: every frame's depth crosses from pinned host memory into one of two device
            # buffers on a copy stream.  Frame f + 1's copy starts when frame f's window opens and
            # that window waits for it, so each window holds one compute and one copy (the first
            # window also its own frame's copy), as a camera pipeline overlaps them
            copy_stream = torch.cuda.Stream()
            bufs = [torch.empty((H, Wd), dtype=torch.float32, device="cuda") for _ in range(2)]
            copied = [torch.cuda.Event(), torch.cuda.Event()]

            def copy_in(f, slot, after):
                copy_stream.wait_event(after)  # the buffer's previous frame is done with it
                with torch.cuda.stream(copy_stream):
                    bufs[slot].copy_(depth_host[f], non_blocking=True)
                    copied[slot].record(copy_stream)
        for i, f in enumerate(range(W, n)):
            flush.fill_(f)
            evs[i][0].record(stream)
            if mode == "device":
                vol.step(depth_dev[f], Kc, *poses[f], refine=True, gc=True, graph=graph)
            else:
                if i == 0:
                    copy_in(f, 0, evs[i][0])
                if f + 1 < n:
                    copy_in(f + 1, (i + 1) % 2, evs[i][0])
                stream.wait_event(copied[i % 2])
                vol.step(bufs[i % 2], Kc, *poses[f], refine=True, gc=True, graph=graph)
                if mode == "host":
                    vol.mesh_size_async(res_host)
                    d2h = 8
                else:
                    # the statistics block (high-water marks that size the outputs, 41 x 128 B), then
                    # counts + on-device compaction in one call (the two 4-byte counts come back)
                    m = vol.download(device=True)
                    d2h = 41 * 128 + 8
                    del m
                if f + 1 < n:
                    stream.wait_event(copied[(i + 1) % 2])  # the next frame's copy ends in this window
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in evs]
        s1 = vol.stats()
        vol.check()
        wrap = lambda d: d % (1 << 32)
        return ms, wrap(s1["collected_blocks"] - s0["collected_blocks"]), wrap(
            s1["meshed_blocks"] - s0["meshed_blocks"]), d2h

    def timed_kernels(vol):
        """Frames W..W+K-1 one at a time with event-record nodes around every kernel; the host
        reads the work counters after every frame."""
        vol.enable_timing(FRAME_KERNELS)
        counters = []
        prev = vol.stats()
        for f in range(W, n):
            flush.fill_(f)
            vol.step(depth_dev[f], Kc, *poses[f], refine=True, gc=True, graph=graph)
            st = vol.stats()
            counters.append(dict(frame_blocks=st["frame_blocks"], update_blocks=st["update_blocks"],
                                 changed=st["changed_cubes"] - prev["changed_cubes"],
                                 emitted=st["emitted_triangles"] - prev["emitted_triangles"],
                                 released=st["released_triangles"] - prev["released_triangles"],
                                 refreshed=st["refreshed_vertices"] - prev["refreshed_vertices"],
                                 created=st["created_vertices"] - prev["created_vertices"],
                                 refupd=st["reference_updates"] - prev["reference_updates"],
                                 freed_vertices=st["freed_vertices"] - prev["freed_vertices"],
                                 freed_blocks=st["freed_blocks"] - prev["freed_blocks"],
                                 high_water=st["block_high_water"], pixels=Wd * H))
            prev = st
        kt = vol.kernel_times()
        vol.check()
        return counters, kt

    # pass 1 -- the value: no event nodes inside the frame graph
    vol = Volume.from_config(vc, stream=stream)
    calib = warm_up(vol, calibrate=True)
    barrier(world)
    cs = None
    if clocks:
        with ClockSampler(local, args.clock_csv if rank == 0 else None) as cs:
            ms, collected, meshed, _ = streamed(vol)
            torch.cuda.synchronize()
    else:
        ms, collected, meshed, _ = streamed(vol)
    barrier(world)
    mem = vol.mesh_memory() if memory else None
    vol.close()
    del vol
    total_ms = sum(ms)
    max_ms = reduce_max(total_ms, world)
    out = {
        "value": world * K / (max_ms / 1000.0), "unit": UNIT, "ms_per_step": max_ms / K,
        "voxels_per_s": 512 * collected / (total_ms / 1000.0),
        "mean_blocks_per_frame": collected / K, "mean_update_blocks_per_frame": meshed / K,
        "frames": "%d..%d" % (W, n - 1),
    }
    if cs is not None:
        out["clocks"] = cs.summary()
    if mem is not None:
        out["mesh_memory"] = mem
    calib_frames = max(W - 1, 1)
    out["launches_per_frame"] = round(sum(v[1] for v in calib.values()) / calib_frames) if calib else None

    # pass 2 -- kernel durations and the rooflines
    if not args.no_kernel_timing:
        vol = Volume.from_config(vc, stream=stream)
        warm_up(vol)
        counters, kt = timed_kernels(vol)
        vol.close()
        del vol
        kernels = {}
        for k in FRAME_KERNELS:
            t_ms, cnt = kt.get(k, (0.0, 0))
            if cnt <= 0:
                continue
            b = sum(BYTES_MODEL[k](c) for c in counters)
            kernels[k] = {"avg_launch_us": 1000.0 * t_ms / cnt, "bytes_per_launch": b / cnt,
                          "achieved": b / (t_ms / 1000.0) / 1e9, "frac": b / (t_ms / 1000.0) / 1e9 / peak}
        dom = max(kernels, key=lambda k: kernels[k]["avg_launch_us"])
        d = kernels[dom]
        tr = TRAFFIC_RATIO.get((label, dom))
        fb = sum(frame_bytes(c) for c in counters) / K
        frame_s = (total_ms / K) / 1000.0
        out["roofline"] = {
            "bound": "hbm", "kernel": dom, "achieved": d["achieved"], "peak": peak, "unit": "GB/s",
            "frac": d["achieved"] / peak, "peak_source": peak_kind,
            "traffic": tr[0] * d["bytes_per_launch"] if tr else None, "traffic_source": tr[1] if tr else None,
            "bytes_per_launch": d["bytes_per_launch"], "avg_launch_us": d["avg_launch_us"],
            "timing": "CUDA events around each kernel, same frames replayed on a fresh volume",
            "frame": {"bytes_per_frame": fb, "ms_per_frame": 1000.0 * frame_s, "achieved": fb / frame_s / 1e9,
                      "frac_measured": fb / frame_s / 1e9 / peak, "frac_nominal": fb / frame_s / 1e9 / NOMINAL_HBM_GBS,
                      "nominal_peak": NOMINAL_HBM_GBS,
                      "how": "sum of the frame kernels' byte models per frame over the value pass's mean frame time"},
            "kernels": kernels,
        }
        out["work_per_frame"] = {k: sum(c[k] for c in counters) / K for k in counters[0] if k != "pixels"}

    # pass 3 -- end to end through the public API: pinned host depth copied in, step, mesh size to the host
    if not args.no_e2e:
        vol = Volume.from_config(vc, stream=stream)
        warm_up(vol)
        ms3, _, _, d2h = streamed(vol, "host")
        vol.close()
        del vol
        out["e2e"] = {"value": world * K / (reduce_max(sum(ms3), world) / 1000.0), "unit": UNIT,
                      "h2d_bytes_per_step": 4 * Wd * H, "d2h_bytes_per_step": d2h,
                      "path": "per frame: the depth frame copied from pinned host memory into a device double "
                              "buffer on a copy stream (frame f + 1's copy overlaps frame f and ends inside frame f's "
                              "window), vm_step on it, then vm_mesh_size_async into pinned host memory"}
        # pass 4 -- the same with the mesh compacted on the device every frame
        vol = Volume.from_config(vc, stream=stream)
        warm_up(vol)
        ms4, _, _, d2h = streamed(vol, "compress")
        vol.close()
        del vol
        out["e2e_compress"] = {"value": world * K / (reduce_max(sum(ms4), world) / 1000.0), "unit": UNIT,
                               "h2d_bytes_per_step": 4 * Wd * H, "d2h_bytes_per_step": d2h,
                               "path": "as e2e, plus the live mesh compacted every frame into dense device arrays "
                                       "(vm_get_stats for the pools' high-water marks that size the outputs, "
                                       "then vm_download_mesh_into: counts, scan and compaction of positions, "
                                       "normals, triangles, edge keys and reference counts, one synchronisation)"}
    torch.cuda.empty_cache()
    return out


def run_full_sequence(args, stream, flush):
    """All frames of the floor trajectory after 10 warm-up frames, value pass only (frames enqueued
    back to back, L2 flushed before each, CUDA events around each)."""
    import torch

    from paper_1803_03949_b300 import Intrinsics, Volume

    sc = scene_for(0)
    n = min(args.full_frames, FLOOR_FRAMES)
    W = 10
    t0 = time.time()
    dev = torch.empty((n, sc.H, sc.W), dtype=torch.float32, device="cuda")
    for k in range(n):
        dev[k].copy_(torch.from_numpy(sc.depth(k)))
    render_s = time.time() - t0
    Kc = Intrinsics(sc.W, sc.H, sc.fx, sc.fy, sc.cx, sc.cy)
    poses = []
    for k in range(n):
        T = sc.pose(k)
        poses.append((T.astype(np.float32), synth.pose_inverse_f64(T).astype(np.float32)))
    vol = Volume.from_config(sc.volume, stream=stream)
    for k in range(W):
        vol.step(dev[k], Kc, *poses[k], refine=True, gc=True, graph=True)
    torch.cuda.synchronize()
    s0 = vol.stats()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n - W)]
    torch.cuda._sleep(int(min(n - W, 2000) * 1000000))
    for i, k in enumerate(range(W, n)):
        flush.fill_(k)
        evs[i][0].record(stream)
        vol.step(dev[k], Kc, *poses[k], refine=True, gc=True, graph=True)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    s1 = vol.stats()
    vol.check()
    vol.close()
    del dev, vol
    torch.cuda.empty_cache()
    tot = sum(ms) / 1000.0
    q = np.quantile(ms, [0.5, 0.99, 1.0])
    collected = (s1["collected_blocks"] - s0["collected_blocks"]) % (1 << 32)
    return {"workload": FLOOR_WORKLOAD, "frames": "%d..%d" % (W, n - 1), "value": (n - W) / tot, "unit": UNIT,
            "ms_per_step": 1000.0 * tot / (n - W), "frame_ms_p50_p99_max": [float(x) for x in q],
            "voxels_per_s": 512 * collected / tot, "mean_blocks_per_frame": collected / (n - W),
            "live_blocks_at_end": s1["live_blocks"], "live_vertices_at_end": s1["live_vertices"],
            "live_triangles_at_end": s1["live_triangles"], "rehashes": s1["rehashes"] - s0["rehashes"],
            "l2": "flushed before every frame (256 MB write)", "render_s": render_s}


def floor_config(args, sc):
    vc = sc.volume
    if args.small_pools:  # the first few hundred frames fit; keeps profiling captures small
        vc = dataclasses.replace(vc, hash_buckets=1 << 20, max_blocks=1 << 18, max_vertices=1 << 23,
                                 max_triangles=1 << 24)
    return vc


def run_vmesh(args, rank, world, local):
    import torch

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    peak, peak_kind = load_peaks()
    W, K = args.warmup, args.steps
    if W + K > FLOOR_FRAMES:
        raise SystemExit("--warmup + --steps must not exceed the floor's %d frames" % FLOOR_FRAMES)
    sc = scene_for(rank)
    vc = floor_config(args, sc)
    if args.only_room:  # the room's value pass alone (profiling captures)
        args.no_kernel_timing = True
        args.no_e2e = True
        rs = room_scene_for(rank, W + K)
        r = measure(args, rs, rs.volume, W, K, stream, flush, peak, peak_kind, world, rank, local, "room")
        if rank == 0:
            print(json.dumps({"room_value_only": r}), flush=True)
        return
    if args.only_headline:  # the headline's value pass alone (profiling captures)
        args.no_kernel_timing = True
        args.no_e2e = True
        r = measure(args, sc, vc, W, K, stream, flush, peak, peak_kind, world, rank, local, "floor")
        if rank == 0:
            print(json.dumps({"floor_value_only": r}), flush=True)
        return
    head = measure(args, sc, vc, W, K, stream, flush, peak, peak_kind, world, rank, local, "floor", clocks=True)
    if rank != 0:
        return
    cpu = None
    if not args.skip_cpu_baseline and world == 1:  # the CPU baseline is an N = 1 figure
        fps, cvps, secs, timed = oracle_frames(scene_for(0), FLOOR_FRAMES, budget_s=args.cpu_seconds)
        cpu = {"value": fps, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "frames 0..%d of the same floor sequence, integrate+update(refine)+gc each (%.1f s of "
                         "single-threaded work; the run stops at a %.0f s budget)" % (timed - 1, secs, args.cpu_seconds),
               "voxels_per_s": cvps}
    lpf = head.pop("launches_per_frame")
    line = {
        "metric": METRIC, "value": head.pop("value"), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": head.pop("ms_per_step"), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": FLOOR_WORKLOAD, "frames": head.pop("frames"), "graph": not args.no_graph,
                   "l2": "flushed before every timed frame (256 MB write)",
                   "submission": "frames enqueued back to back; per-frame CUDA events exclude the flush",
                   "parallelism": "replicas" if world > 1 else "single",
                   "pools": "blocks %d, vertices %d, triangles %d, buckets %d" % (
                       vc.max_blocks, vc.max_vertices, vc.max_triangles, vc.hash_buckets)},
        "roofline": head.pop("roofline", None),
        "cpu_baseline": cpu,
        "e2e": head.pop("e2e", None),
        "e2e_compress": head.pop("e2e_compress", None),
        "gpu_launches": lpf * K if lpf else None,
        "clocks": head.pop("clocks"),
    }
    line.update(head)  # voxels_per_s, mean blocks, work per frame
    # the other workloads and forms are single-GPU figures: with several ranks they would hold every
    # GPU while rank 0 alone ran them
    if not args.skip_forms and world == 1:
        if not args.skip_full_sequence:
            line["full_sequence"] = run_full_sequence(args, stream, flush)
        rs = room_scene_for(0, args.room_warmup + args.room_steps)
        room = measure(args, rs, rs.volume, args.room_warmup, args.room_steps, stream, flush, peak, peak_kind, 1, 0,
                       local, "room", memory=True)
        room["workload"] = ROOM_WORKLOAD
        mem = room.pop("mesh_memory")
        # the compact cube record on the same frames (value pass only): speed and memory
        a2 = argparse.Namespace(**vars(args))
        a2.no_kernel_timing, a2.no_e2e = True, True
        rc = measure(a2, rs, dataclasses.replace(rs.volume, compact_edges=True), args.room_warmup, args.room_steps,
                     stream, flush, peak, peak_kind, 1, 0, local, "room", memory=True)
        mem_c = rc["mesh_memory"]
        room["mesh_memory"] = {
            "after_frames": args.room_warmup + args.room_steps, "vertices": mem["vertices"],
            "triangles": mem["triangles"], "per_block_extraction_vertices": mem["block_vertices"],
            "loose_triangle_vertices": mem["loose_vertices"],
            "per_block_over_ours": mem["block_vertices"] / max(mem["vertices"], 1),
            "loose_over_ours": mem["loose_vertices"] / max(mem["vertices"], 1),
            "blocks": mem["blocks"], "cube_bytes": mem["cube_bytes"], "edge_records": mem["edge_records"],
            "paper_cube_bytes": 56, "paper_compact_cube_bytes": 24, "bytes_in_use": mem["bytes_in_use"],
            "bytes_allocated": mem["bytes_allocated"],
            "compact_layout": {"value": rc["value"], "unit": UNIT, "cube_bytes": mem_c["cube_bytes"],
                               "edge_records": mem_c["edge_records"], "bytes_in_use": mem_c["bytes_in_use"],
                               "bytes_allocated": mem_c["bytes_allocated"]},
        }
        if not args.skip_cpu_baseline:
            fps, cvps, secs, timed = oracle_frames(room_scene_for(0, args.room_cpu_frames), args.room_cpu_frames)
            room["cpu_baseline"] = {"value": fps, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "frames 0..%d of the room sequence (%.1f s)" % (timed - 1, secs),
                                    "voxels_per_s": cvps}
        line["room"] = room
        line["batched"] = run_batched(args, stream, flush, peak, "mixed")
        line["batched_small"] = run_batched(args, stream, flush, peak, "small")
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
    ap.add_argument("--small-pools", action="store_true", help="smaller floor pool allocations (ncu captures)")
    ap.add_argument("--no-kernel-timing", action="store_true",
                    help="time frames without per-kernel event nodes (no roofline)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the two end-to-end passes")
    ap.add_argument("--only-headline", action="store_true", help="run only the headline's value pass")
    ap.add_argument("--only-room", action="store_true", help="run only the room's value pass (--steps, --warmup)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="budget of the oracle's timed sample")
    ap.add_argument("--reference-seconds", type=float, default=150.0, help="budget of the reference arm's timing")
    ap.add_argument("--skip-forms", action="store_true",
                    help="skip the full sequence, the room and the batched and differentiable forms")
    ap.add_argument("--skip-full-sequence", action="store_true")
    ap.add_argument("--full-frames", type=int, default=FLOOR_FRAMES)
    ap.add_argument("--clock-csv", default=None, help="also write the clock samples of the timed pass to this CSV")
    ap.add_argument("--room-steps", type=int, default=300)
    ap.add_argument("--room-warmup", type=int, default=10)
    ap.add_argument("--room-cpu-frames", type=int, default=200)
    ap.add_argument("--batch-scenes", type=int, default=32)
    ap.add_argument("--batch-ticks", type=int, default=500)
    ap.add_argument("--batch-warmup", type=int, default=10)
    ap.add_argument("--diff-reps", type=int, default=21)
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
