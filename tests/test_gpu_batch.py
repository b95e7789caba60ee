"""Batched step (many independent scenes, one frame each per tick, five launches per tick):
every scene's state equals the oracle's on the same frames and the same scene stepped alone
through vm_step, with and without the tick graph and across autotuning ticks."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import compare_blocks, compare_mesh, gpu_volume, intrinsics, poses32, sorted_blocks

pytestmark = pytest.mark.gpu


def _scenes(frames):
    """Uneven scenes: image sizes 96x72 .. 640x480, voxels 8 mm .. 2 cm, different seeds."""
    return [
        synth.small_room_scene(num_frames=frames, seed=synth.SEED_BASE + 40),
        synth.small_room_scene(num_frames=frames, seed=synth.SEED_BASE + 41, W=97, H=61),
        synth.sphere_scene(num_frames=frames),
        synth.room_scene(num_frames=frames, seed=synth.SEED_BASE + 42, W=320, H=240),
        synth.room_scene(num_frames=frames),
    ]


def _run_batch(scenes, frames, graph=True, tune_rounds=0, schedule=None):
    import torch

    from paper_1803_03949_b300 import Scenes

    vols = [gpu_volume(s.volume) for s in scenes]
    b = Scenes(vols)
    if schedule is not None:
        b.set_schedule(schedule)
    if tune_rounds:
        b.tune(tune_rounds)
    Ks = [intrinsics(s) for s in scenes]
    for k in range(frames):
        depths = [torch.from_numpy(s.depth(k)).cuda() for s in scenes]
        b.step_all(depths, Ks, [poses32(s.pose(k)) for s in scenes], refine=True, gc=True, graph=graph)
    torch.cuda.synchronize()
    for v in vols:
        v.check()
    return b, vols


def _run_single(scene, frames):
    import torch

    v = gpu_volume(scene.volume)
    K = intrinsics(scene)
    for k in range(frames):
        v.step(torch.from_numpy(scene.depth(k)).cuda(), K, *poses32(scene.pose(k)), refine=True, gc=True, graph=True)
    v.check()
    return v


def _same_state(a, b):
    ba, bb = sorted_blocks(a.blocks()), sorted_blocks(b.blocks())
    for k in ba:
        np.testing.assert_array_equal(ba[k], bb[k], err_msg=k)
    ma, mb = a.download(), b.download()
    from tests.gpu_util import gpu_mesh_canonical

    ka, ta = gpu_mesh_canonical(ma)
    kb, tb = gpu_mesh_canonical(mb)
    np.testing.assert_array_equal(np.sort(ka), np.sort(kb))
    np.testing.assert_array_equal(ta, tb)
    oa, ob = np.argsort(ka), np.argsort(kb)
    np.testing.assert_array_equal(np.asarray(ma["pos"])[oa], np.asarray(mb["pos"])[ob])
    np.testing.assert_array_equal(np.asarray(ma["nrm"])[oa], np.asarray(mb["nrm"])[ob])
    sa, sb = a.stats(), b.stats()
    for k in ("live_blocks", "live_vertices", "live_triangles", "collected_blocks", "meshed_blocks", "freed_blocks"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])


def test_batch_equals_each_scene_alone_and_the_oracle():
    frames = 6
    scenes = _scenes(frames)
    b, vols = _run_batch(scenes, frames, graph=True)
    for s, v in zip(scenes, vols):
        _same_state(v, _run_single(s, frames))
    # the oracle on the two small scenes
    for s, v in list(zip(scenes, vols))[:2]:
        o = oracle.Volume.from_config(s.volume, prec="f32")
        K = (s.fx, s.fy, s.cx, s.cy)
        for k in range(frames):
            Twc, Tcw = poses32(s.pose(k))
            o.integrate(s.depth(k), K, Twc.astype(np.float64), Tcw.astype(np.float64))
            o.update_mesh(refine=True)
            o.gc()
        compare_blocks(v.blocks(), o.blocks())
        compare_mesh(v.download(), o.mesh(), s.volume.voxel_size)
    b.close()


@pytest.mark.parametrize("graph", [False, True])
def test_batch_with_autotuning_and_every_schedule_option(graph):
    """Tuning ticks run each kernel on every candidate option; the state afterwards, and
    under the least and most parallel fixed schedules, equals the scenes stepped alone."""
    frames = 7
    scenes = _scenes(frames)[:4]
    b, vols = _run_batch(scenes, frames, graph=graph, tune_rounds=2)
    sc = b.schedule()
    assert sc["schedule"]["alloc_pixels_per_thread"] in (1, 2, 4)
    assert all(min(t) > 0 for t in sc["tuned_ms"].values()), sc
    singles = [_run_single(s, frames) for s in scenes]
    for v, s1 in zip(vols, singles):
        _same_state(v, s1)
    for sched in ([1, 4, 4, 1, 2], [4, 12, 8, 4, 8]):
        b2, vols2 = _run_batch(scenes, frames, graph=graph, schedule=sched)
        for v, s1 in zip(vols2, singles):
            _same_state(v, s1)
        b2.close()
    b.close()


def test_batch_arguments_are_checked():
    import torch

    from paper_1803_03949_b300 import Scenes, VmeshError

    s = synth.small_room_scene(num_frames=1)
    v = gpu_volume(s.volume)
    with pytest.raises(VmeshError):
        Scenes([v, v])
    with pytest.raises(VmeshError):
        Scenes([])
    b = Scenes([v])
    with pytest.raises(VmeshError):
        b.set_schedule([3, 12, 7, 2, 8])  # 3 pixels per thread is not an option
    bad = intrinsics(s)
    bad.fx = -1.0
    with pytest.raises(VmeshError):
        b.step_all([torch.from_numpy(s.depth(0)).cuda()], [bad], [poses32(s.pose(0))])
    v.diff_begin(1)
    with pytest.raises(VmeshError):
        b.step_all([torch.from_numpy(s.depth(0)).cuda()], [intrinsics(s)], [poses32(s.pose(0))])
    v.diff_end()
    b.step_all([torch.from_numpy(s.depth(0)).cuda()], [intrinsics(s)], [poses32(s.pose(0))])
    v.check()
    b.close()


def test_batch_hash_rebuilds_under_block_churn():
    """Scenes whose hash tables are small enough that recycled blocks' tombstones force rebuilds
    (the batched vertex gc clears a scene's table with the whole grid, the batched block gc
    reinserts its live blocks), next to a scene with a large table that never rebuilds: each
    equals the scene stepped alone, and the small-table scene the oracle."""
    import dataclasses

    frames = 10
    s0 = synth.small_room_scene(num_frames=frames, seed=synth.SEED_BASE + 51)
    s1 = synth.small_room_scene(num_frames=frames, seed=synth.SEED_BASE + 52)
    s2 = synth.small_room_scene(num_frames=frames, seed=synth.SEED_BASE + 53)
    s0.volume = dataclasses.replace(s0.volume, hash_buckets=1 << 10)  # ~500 live blocks: rebuilds from frame 2
    s2.volume = dataclasses.replace(s2.volume, hash_buckets=1 << 11)
    scenes = [s0, s1, s2]
    b, vols = _run_batch(scenes, frames, graph=True)
    for s, v in zip(scenes, vols):
        _same_state(v, _run_single(s, frames))
    assert vols[0].stats()["rehashes"] > 0 and vols[0].stats()["freed_blocks"] > 0
    assert vols[1].stats()["rehashes"] == 0
    o = oracle.Volume.from_config(s0.volume, prec="f32")
    K = (s0.fx, s0.fy, s0.cx, s0.cy)
    for k in range(frames):
        Twc, Tcw = poses32(s0.pose(k))
        o.integrate(s0.depth(k), K, Twc.astype(np.float64), Tcw.astype(np.float64))
        o.update_mesh(refine=True)
        o.gc()
    compare_blocks(vols[0].blocks(), o.blocks())
    compare_mesh(vols[0].download(), o.mesh(), s0.volume.voxel_size)
    b.close()
