"""CUDA path vs the float32 oracle, element by element on the same seeded inputs (C ABI).

Bar: collected block set, cube types (current and previous) and canonical triangle
topology bit-exact; TSDF and weights within 1e-5 absolute; vertex positions within
1e-5 x voxel size; normals within 1e-5 (unit vectors evaluated in the same float32 order).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import (compare_blocks, compare_mesh, gpu_mesh_canonical, gpu_volume, intrinsics, poses32,
                            run_frames)
from tests.meshutil import manifold_report, sphere_fill

pytestmark = pytest.mark.gpu


def _integrate_only(scene, frames, g, o):
    K = intrinsics(scene)
    for k in frames:
        d = scene.depth(k)
        Twc, Tcw = poses32(scene.pose(k))
        g.integrate(torch.from_numpy(d).cuda(), K, Twc, Tcw)
        o.integrate(d, (scene.fx, scene.fy, scene.cx, scene.cy), Twc.astype(np.float64), Tcw.astype(np.float64))


def test_sphere_workload_full_extraction_and_refine():
    """10 frames 320x240 of the sphere-on-ground orbit, then one full extraction and refine."""
    s = synth.sphere_scene()
    g, o = gpu_volume(s.volume), oracle.Volume.from_config(s.volume)
    _integrate_only(s, range(s.num_frames), g, o)
    g.check()
    st = compare_blocks(g.blocks(), o.blocks())
    assert st["blocks"] > 1000
    g.update_mesh(full=True)
    o.update_mesh(full=True)
    compare_mesh(g.download(), o.mesh(), s.volume.voxel_size)
    g.refine_mesh(full=True)
    o.refine_mesh(full=True)
    g.check()
    compare_blocks(g.blocks(), o.blocks())
    ms = compare_mesh(g.download(), o.mesh(), s.volume.voxel_size)
    assert ms["triangles"] > 100000


def test_small_room_incremental_every_frame():
    """Incremental integrate / update+refine / gc, compared after every frame."""
    s = synth.small_room_scene(num_frames=8)
    g, o = gpu_volume(s.volume), oracle.Volume.from_config(s.volume)

    def check(k):
        g.check()
        compare_blocks(g.blocks(), o.blocks())
        compare_mesh(g.download(), o.mesh(), s.volume.voxel_size)

    run_frames(s, range(8), gpu=g, orc=o, after_frame=check)
    assert g.stats()["freed_blocks"] > 0


@pytest.mark.parametrize("mode", ["calls", "step", "graph"])
def test_room_full_size_launch_configurations(mode):
    """640x480 room frames at full size through each launch configuration (the benchmark
    times 'graph': vm_step replayed from a CUDA graph with refine and gc)."""
    s = synth.room_scene(num_frames=5)
    g, o = gpu_volume(s.volume), oracle.Volume.from_config(s.volume)
    run_frames(s, range(5), gpu=g, orc=o, mode=mode)
    g.check()
    st = compare_blocks(g.blocks(), o.blocks())
    ms = compare_mesh(g.download(), o.mesh(), s.volume.voxel_size)
    assert st["blocks"] > 500 and ms["triangles"] > 20000
    stats = g.stats()
    nv, nt = g.mesh_counts()
    assert stats["live_vertices"] == nv and stats["live_triangles"] == nt


def test_separate_refine_equals_fused_refine():
    s = synth.small_room_scene(num_frames=6, seed=synth.SEED_BASE + 21)
    g1, g2 = gpu_volume(s.volume), gpu_volume(s.volume)
    o = oracle.Volume.from_config(s.volume)
    run_frames(s, range(6), gpu=g1, orc=o, separate_refine=True)
    run_frames(s, range(6), gpu=g2)
    compare_blocks(g1.blocks(), o.blocks())
    compare_mesh(g1.download(), o.mesh(), s.volume.voxel_size)
    _, t1 = gpu_mesh_canonical(g1.download())
    _, t2 = gpu_mesh_canonical(g2.download())
    np.testing.assert_array_equal(t1, t2)


def test_mixed_entry_points_keep_parity():
    """One 640x480 room volume (6 mm voxels) driven through every entry point in turn: graph
    steps, plain steps, separate calls, integrate-only frames (two collection calls before a mesh pass),
    repeated mesh passes without an integrate call between them (one of them full, more
    blocks than the grid has CTAs), and steps after them.  The integrate calls' numbering and
    the mesh pass's block hand-out counter must carry over every sequence; compared with the
    oracle after each frame."""
    import dataclasses

    s = synth.room_scene(num_frames=7, seed=synth.SEED_BASE + 23)
    vc = dataclasses.replace(s.volume, voxel_size=0.006, trunc=0.024)  # ~2k blocks after 5 frames
    g, o = gpu_volume(vc), oracle.Volume.from_config(vc)
    K = intrinsics(s)
    Ko = (s.fx, s.fy, s.cx, s.cy)
    plan = ["graph", "calls", "integrate", "integrate", "passes", "step", "graph"]
    full_blocks = 0
    for k, how in enumerate(plan):
        d = s.depth(k)
        Twc, Tcw = poses32(s.pose(k))
        dt = torch.from_numpy(d).cuda()
        o.integrate(d, Ko, Twc.astype(np.float64), Tcw.astype(np.float64))
        if how in ("graph", "step"):
            g.step(dt, K, Twc, Tcw, refine=True, gc=True, graph=(how == "graph"))
            o.update_mesh(refine=True)
            o.gc()
        elif how == "integrate":
            g.integrate(dt, K, Twc, Tcw)
        else:
            g.integrate(dt, K, Twc, Tcw)
            g.update_mesh(refine=True)
            o.update_mesh(refine=True)
            if how == "passes":  # a full pass and a refine-only pass over the same sets
                g.update_mesh(full=True, refine=True)
                o.update_mesh(full=True, refine=True)
                full_blocks = g.stats()["update_blocks"]
                g.refine_mesh()
                o.refine_mesh()
            g.gc()
            o.gc()
        g.check()
        compare_blocks(g.blocks(), o.blocks())
        if how != "integrate":
            compare_mesh(g.download(), o.mesh(), vc.voxel_size)
    assert full_blocks > 1184  # that pass handed out blocks beyond one per CTA of its grid


def test_ragged_image_with_invalid_pixels():
    """97 x 61 frames (not a multiple of the 64 x 16 tile or of 4), NaN / inf / negative /
    zero depths sprinkled in: such pixels are skipped identically on both sides."""
    s = synth.small_room_scene(num_frames=4, W=97, H=61, seed=synth.SEED_BASE + 31)
    rng = np.random.default_rng(5)

    def depth(k):
        d = s.depth(k).copy()
        m = rng.random(d.shape)
        d[m < 0.01] = np.nan
        d[(m >= 0.01) & (m < 0.02)] = np.inf
        d[(m >= 0.02) & (m < 0.03)] = -1.0
        d[(m >= 0.03) & (m < 0.04)] = 0.0
        return d

    frames = [depth(k) for k in range(4)]
    g, o = gpu_volume(s.volume), oracle.Volume.from_config(s.volume)
    run_frames(s, range(4), gpu=g, orc=o, depth_fn=lambda k: frames[k])
    g.check()
    compare_blocks(g.blocks(), o.blocks())
    compare_mesh(g.download(), o.mesh(), s.volume.voxel_size)


def test_empty_and_all_invalid_frames():
    s = synth.small_room_scene(num_frames=2)
    g = gpu_volume(s.volume)
    z = np.zeros((s.H, s.W), np.float32)
    run_frames(s, range(2), gpu=g, depth_fn=lambda k: z if k == 0 else np.full_like(z, np.nan))
    g.check()
    assert g.num_blocks() == 0
    assert g.mesh_counts() == (0, 0)
    m = g.download()
    assert m["pos"].shape == (0, 3) and m["tris"].shape == (0, 3)


@pytest.mark.parametrize("radius", [0.1, 0.173])
def test_analytic_sphere_fill(radius):
    l, mu = 0.01, 0.04
    vc = synth.VolumeConfig(voxel_size=l, trunc=mu, hash_buckets=1 << 12, max_blocks=1 << 12,
                            max_vertices=1 << 18, max_triangles=1 << 19)
    keys, tsdf, w = sphere_fill((0.013, -0.021, 0.007), radius, l, mu)
    g, o = gpu_volume(vc), oracle.Volume.from_config(vc)
    g.set_blocks(keys, tsdf.astype(np.float32), w.astype(np.float32))
    o.set_blocks(keys, tsdf.astype(np.float32).astype(np.float64), w)
    g.update_mesh(full=True)
    o.update_mesh(full=True)
    g.check()
    m = g.download()
    compare_mesh(m, o.mesh(), l)
    rep = manifold_report(m["tris"])
    assert rep["closed"] and rep["oriented"] and rep["euler"] == 2


def test_incremental_equals_full_extraction_on_gpu():
    s = synth.small_room_scene(num_frames=8)
    g = gpu_volume(s.volume)
    run_frames(s, range(8), gpu=g, refine=False)
    b = g.blocks()
    f = gpu_volume(s.volume)
    f.set_blocks(b["keys"], b["tsdf"], b["weight"])
    f.update_mesh(full=True)
    k1, t1 = gpu_mesh_canonical(g.download())
    k2, t2 = gpu_mesh_canonical(f.download())
    np.testing.assert_array_equal(t1, t2)
    np.testing.assert_array_equal(np.sort(k1), np.sort(k2))


def test_runs_are_deterministic():
    s = synth.small_room_scene(num_frames=6, seed=synth.SEED_BASE + 41)
    out = []
    for _ in range(2):
        g = gpu_volume(s.volume)
        run_frames(s, range(6), gpu=g, mode="graph")
        b = g.blocks()
        m = g.download()
        keys, tris = gpu_mesh_canonical(m)
        order = np.argsort(keys)
        out.append((b, keys[order], tris, m["pos"][order]))
    from tests.gpu_util import sorted_blocks

    b0, b1 = sorted_blocks(out[0][0]), sorted_blocks(out[1][0])
    for k in b0:
        np.testing.assert_array_equal(b0[k], b1[k])
    for a, b in zip(out[0][1:], out[1][1:]):
        np.testing.assert_array_equal(a, b)


def test_rehash_under_block_churn_keeps_parity():
    """A hash table small enough that recycled blocks' tombstones force rebuilds."""
    s = synth.small_room_scene(num_frames=10, seed=synth.SEED_BASE + 51)
    vc = s.volume
    import dataclasses

    small = dataclasses.replace(vc, hash_buckets=1 << 10)  # ~500 live blocks: rebuilds start at frame 2
    g, o = gpu_volume(small), oracle.Volume.from_config(vc)
    run_frames(s, range(10), gpu=g, orc=o)
    g.check()
    compare_blocks(g.blocks(), o.blocks())
    compare_mesh(g.download(), o.mesh(), vc.voxel_size)
    st = g.stats()
    assert st["freed_blocks"] > 0 and st["rehashes"] > 0


def test_large_floor_first_frames_match_oracle():
    """The 20x20x4 m floor at its full size (640x480, voxel 5 mm, 2^23 buckets) through the
    benchmark's launch configuration (vm_step from a CUDA graph): 6 frames against the oracle."""
    s = synth.floor_scene()  # the 2000-frame trajectory; its first frames
    g = gpu_volume(s.volume)
    o = oracle.Volume.from_config(s.volume, prec="f32")
    run_frames(s, range(6), gpu=g, orc=o, refine=True, gc=True, mode="graph")
    g.check()
    compare_blocks(g.blocks(), o.blocks())
    st = compare_mesh(g.download(), o.mesh(), s.volume.voxel_size)
    assert st["triangles"] > 50000


def test_large_floor_long_run_properties():
    """The first 600 frames of the floor (unrefined, with gc): the incremental mesh equals a full
    extraction of the final TSDF in a fresh volume (canonical topology, positions and normals
    bit-exact), every vertex is unique and its reference count equals its degree."""
    s = synth.floor_scene()  # the 2000-frame trajectory; its first 600 frames
    g = gpu_volume(s.volume)
    run_frames(s, range(600), gpu=g, refine=False, gc=True, mode="graph")
    g.check()
    st = g.stats()
    assert st["live_blocks"] > 200000
    b = g.blocks()
    f = gpu_volume(s.volume)
    f.set_blocks(b["keys"], b["tsdf"], b["weight"])
    f.update_mesh(full=True)
    f.check()
    gm, fm = g.download(), f.download()
    gk, gt = gpu_mesh_canonical(gm)
    fk, ft = gpu_mesh_canonical(fm)
    assert len(np.unique(gk)) == len(gk)
    np.testing.assert_array_equal(gt, ft)
    og, of = np.argsort(gk), np.argsort(fk)
    np.testing.assert_array_equal(gk[og], fk[of])
    np.testing.assert_array_equal(np.asarray(gm["pos"])[og], np.asarray(fm["pos"])[of])
    np.testing.assert_array_equal(np.asarray(gm["nrm"])[og], np.asarray(fm["nrm"])[of])
    deg = np.bincount(np.asarray(gm["tris"]).reshape(-1), minlength=len(gk))
    np.testing.assert_array_equal(np.asarray(gm["refcount"]), deg)
