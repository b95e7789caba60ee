"""Failure handling on the GPU without faulting it: exhausted capacities end as a sticky
device status (no trap, no hang) and the volume stays usable for destruction; bad host
arguments are refused before anything is enqueued."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_1803_03949_b300 import VmeshError
from paper_1803_03949_b300.vmesh import Intrinsics, Volume, load_library, vm_params
from tests.gpu_util import gpu_volume, intrinsics, poses32, run_frames

pytestmark = pytest.mark.gpu

HASH_FULL, POOL_FULL, INVALID = 2, 3, 1


def _vol(**kw):
    s = synth.small_room_scene(num_frames=3)
    base = dict(voxel_size=s.volume.voxel_size, trunc=s.volume.trunc, hash_buckets=1 << 14, max_blocks=1 << 13,
                max_vertices=1 << 20, max_triangles=1 << 21)
    base.update(kw)
    return s, Volume(**base)


def test_hash_full_is_reported():
    s, g = _vol(hash_buckets=16)
    run_frames(s, range(2), gpu=g)
    assert g.last_error() == HASH_FULL
    g.close()


@pytest.mark.parametrize("kw", [dict(max_blocks=8), dict(max_vertices=100), dict(max_triangles=64)])
def test_pool_exhaustion_is_reported(kw):
    s, g = _vol(**kw)
    run_frames(s, range(2), gpu=g)
    assert g.last_error() == POOL_FULL
    g.close()


def test_bad_arguments_are_refused():
    s, g = _vol()
    K = intrinsics(s)
    Twc, Tcw = poses32(s.pose(0))
    d = torch.from_numpy(s.depth(0)).cuda()
    with pytest.raises(VmeshError) as e:
        g.integrate(None, K, Twc, Tcw)
    assert e.value.code == INVALID
    bad = Twc.copy()
    bad[0, 0] = np.nan
    with pytest.raises(VmeshError):
        g.integrate(d, K, bad, Tcw)
    with pytest.raises(VmeshError):
        g.integrate(d, Intrinsics(s.W, s.H, 0.0, s.fy, s.cx, s.cy), Twc, Tcw)
    with pytest.raises(VmeshError):
        g.integrate(d, Intrinsics(0, s.H, s.fx, s.fy, s.cx, s.cy), Twc, Tcw)
    with pytest.raises(VmeshError):  # a field of view too wide for the ray-slope limit
        g.integrate(d, Intrinsics(s.W, s.H, 0.5, s.fy, s.cx, s.cy), Twc, Tcw)
    assert g._lib.vm_update_mesh(g._h, 64) == INVALID
    assert g.last_error() == 0


@pytest.mark.parametrize("field,value", [("voxel_size", 0.0), ("trunc", -1.0), ("trunc", 1.0), ("hash_buckets", 1000),
                                         ("hash_buckets", 8), ("max_blocks", 0), ("max_blocks", (1 << 21) + 1),
                                         ("w_max", 0.5), ("flags", 2)])
def test_bad_params_are_refused(field, value):
    lib = load_library()
    p = vm_params(0.01, 0.04, 0.002, 255.0, 1 << 14, 1 << 10, 1 << 16, 1 << 16)
    setattr(p, field, value)
    h = ctypes.c_void_p()
    assert lib.vm_create_volume(ctypes.byref(p), None, ctypes.byref(h)) == INVALID
    assert not h.value
