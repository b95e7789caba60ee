"""vm_download_mesh_noalloc: the mesh download for callers that may not allocate device
memory (a caching allocator owning the free memory, a fixed budget set at start-up).

It is called through the C ABI twice in a row on the same volume and must give exactly
what vm_download_mesh gives (the same stable compaction, so the arrays match element by
element; positions and normals are copies, within the parity tolerance of 1e-5 and in
fact equal).  It also answers a size query, refuses outputs that are too small and
volumes whose pools exceed its static scratch.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import gpu_volume, run_frames

pytestmark = pytest.mark.gpu

INVALID = 1


def _noalloc(g, nv, nt, cap_v=None, cap_t=None, memory=None):
    """One call into caller-allocated outputs; with `memory` (a list), the device's free bytes
    and torch's allocated bytes just before and just after the call are appended to it."""
    dev = torch.device("cuda")
    out = dict(pos=torch.full((nv, 3), -7.0, device=dev), nrm=torch.full((nv, 3), -7.0, device=dev),
               tris=torch.full((nt, 3), -7, dtype=torch.int32, device=dev),
               keys=torch.zeros((nv,), dtype=torch.int64, device=dev),
               refcount=torch.full((nv,), -7, dtype=torch.int32, device=dev))
    n1, n2 = ctypes.c_int64(), ctypes.c_int64()
    torch.cuda.synchronize()
    before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated())
    rc = g._lib.vm_download_mesh_noalloc(g._h, out["pos"].data_ptr(), out["nrm"].data_ptr(), out["tris"].data_ptr(),
                                         out["keys"].data_ptr(), out["refcount"].data_ptr(),
                                         nv if cap_v is None else cap_v, nt if cap_t is None else cap_t,
                                         ctypes.byref(n1), ctypes.byref(n2))
    torch.cuda.synchronize()
    if memory is not None:
        memory.append((before, (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated())))
    return rc, (n1.value, n2.value), {k: v.cpu().numpy() for k, v in out.items()}


def _check_against_download(g, voxel):
    ref = {k: v.cpu().numpy() for k, v in g.download(device=True).items()}
    nv, nt = ref["pos"].shape[0], ref["tris"].shape[0]
    # size query: no outputs
    qv, qt = ctypes.c_int64(), ctypes.c_int64()
    assert g._lib.vm_download_mesh_noalloc(g._h, None, None, None, None, None, 0, 0, ctypes.byref(qv),
                                           ctypes.byref(qt)) == 0
    assert (qv.value, qt.value) == (nv, nt)
    memory = []
    for _ in range(2):  # two calls in a row share the static scratch
        rc, counts, out = _noalloc(g, nv, nt, memory=memory)
        assert rc == 0 and counts == (nv, nt)
        np.testing.assert_allclose(out["pos"], ref["pos"], rtol=0, atol=1e-5 * voxel)
        np.testing.assert_allclose(out["nrm"], ref["nrm"], rtol=0, atol=1e-5)
        np.testing.assert_array_equal(out["tris"], ref["tris"])
        np.testing.assert_array_equal(out["keys"], ref["keys"])
        np.testing.assert_array_equal(out["refcount"], ref["refcount"])
    # the second call (after the first one's one-time symbol lookup) takes no device memory:
    # neither the device's free bytes nor torch's allocated bytes move across it
    before, after = memory[1]
    assert after == before, (before, after)
    return nv, nt


def test_noalloc_download_matches_download_twice():
    s = synth.small_room_scene(num_frames=8, seed=synth.SEED_BASE + 61)
    g = gpu_volume(s.volume)
    run_frames(s, range(6), gpu=g, mode="graph")
    nv, nt = _check_against_download(g, s.volume.voxel_size)
    assert nv > 1000 and nt > 1000
    # the mesh changes with more frames; later calls follow it
    run_frames(s, range(6, 8), gpu=g, mode="graph")
    _check_against_download(g, s.volume.voxel_size)
    assert g.last_error() == 0


def test_noalloc_download_refuses_small_outputs_and_large_pools():
    s = synth.small_room_scene(num_frames=3, seed=synth.SEED_BASE + 62)
    g = gpu_volume(s.volume)
    run_frames(s, range(3), gpu=g)
    nv, nt = g.mesh_counts()
    rc, counts, out = _noalloc(g, nv, nt, cap_v=nv - 1)
    assert rc == INVALID and counts == (nv, nt)
    assert np.all(out["pos"] == -7.0) and np.all(out["tris"] == -7)
    import dataclasses

    # only the vertex pool is beyond the scratch's limit; the other pools stay small
    big = gpu_volume(dataclasses.replace(s.volume, max_vertices=(1 << 24) + 1, max_blocks=1 << 10,
                                         max_triangles=1 << 12, hash_buckets=1 << 12))
    try:
        n1, n2 = ctypes.c_int64(), ctypes.c_int64()
        assert big._lib.vm_download_mesh_noalloc(big._h, None, None, None, None, None, 0, 0, ctypes.byref(n1),
                                                 ctypes.byref(n2)) == INVALID
    finally:
        big.close()
