"""Depth frames passed in pinned host memory: the collection kernel reads them across the host
link and keeps the device copy the later kernels read.  The state after every frame equals the
same frames passed in device memory (plain calls, steps and graph replays); pageable host memory
is refused."""
import numpy as np
import pytest

import synth
from tests.gpu_util import compare_blocks, gpu_mesh_canonical, gpu_volume, intrinsics, poses32

pytestmark = pytest.mark.gpu


def _same(a, b):
    import torch

    torch.cuda.synchronize()
    compare_blocks(a.blocks(), b.blocks(), tol=0.0)
    ka, ta = gpu_mesh_canonical(a.download())
    kb, tb = gpu_mesh_canonical(b.download())
    np.testing.assert_array_equal(np.sort(ka), np.sort(kb))
    np.testing.assert_array_equal(ta, tb)


@pytest.mark.parametrize("mode", ["calls", "step", "graph"])
def test_pinned_host_depth_equals_device_depth(mode):
    import torch

    s = synth.room_scene(num_frames=4, W=320, H=240, seed=synth.SEED_BASE + 27)
    dev, host = gpu_volume(s.volume), gpu_volume(s.volume)
    K = intrinsics(s)
    for k in range(4):
        d = torch.from_numpy(s.depth(k))
        dh = d.pin_memory()
        dd = d.cuda()
        Twc, Tcw = poses32(s.pose(k))
        for v, depth in ((dev, dd), (host, dh)):
            if mode == "calls":
                v.integrate(depth, K, Twc, Tcw)
                v.update_mesh(refine=True)
                v.gc()
            else:
                v.step(depth, K, Twc, Tcw, refine=True, gc=True, graph=(mode == "graph"))
        host.check()
        _same(dev, host)
    # a larger frame after smaller ones grows the device copy
    s2 = synth.room_scene(num_frames=1, seed=synth.SEED_BASE + 28)
    d = torch.from_numpy(s2.depth(0))
    Twc, Tcw = poses32(s2.pose(0))
    dev.step(d.cuda(), intrinsics(s2), Twc, Tcw, refine=True, gc=True)
    host.step(d.pin_memory(), intrinsics(s2), Twc, Tcw, refine=True, gc=True)
    host.check()
    _same(dev, host)


def test_pageable_host_depth_is_refused():
    import torch

    from paper_1803_03949_b300 import VmeshError

    s = synth.small_room_scene(num_frames=1)
    v = gpu_volume(s.volume)
    Twc, Tcw = poses32(s.pose(0))
    with pytest.raises(VmeshError):
        v.step(torch.from_numpy(s.depth(0)), intrinsics(s), Twc, Tcw)
    with pytest.raises(VmeshError):
        v.integrate(torch.from_numpy(s.depth(0)), intrinsics(s), Twc, Tcw)
    v.check()
    assert v.num_blocks() == 0


@pytest.mark.parametrize("graph", [False, True])
def test_batched_step_with_pinned_host_depths(graph):
    import torch

    from paper_1803_03949_b300 import Scenes

    scenes = [synth.small_room_scene(num_frames=3, seed=synth.SEED_BASE + 50 + i) for i in range(3)]
    dev_vols = [gpu_volume(s.volume) for s in scenes]
    host_vols = [gpu_volume(s.volume) for s in scenes]
    bd, bh = Scenes(dev_vols), Scenes(host_vols)
    Ks = [intrinsics(s) for s in scenes]
    for k in range(3):
        frames = [torch.from_numpy(s.depth(k)) for s in scenes]
        poses = [poses32(s.pose(k)) for s in scenes]
        bd.step_all([f.cuda() for f in frames], Ks, poses, graph=graph)
        bh.step_all([f.pin_memory() for f in frames], Ks, poses, graph=graph)
    for a, b in zip(dev_vols, host_vols):
        b.check()
        _same(a, b)
    bd.close()
    bh.close()
