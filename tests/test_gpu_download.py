"""vm_download_mesh_into (the compaction into caller-allocated device buffers with capacities,
one synchronisation) against vm_download_mesh on the host and on the device, through the C ABI:
the same stable compaction element by element; capacities below the counts give
VM_ERR_INVALID_ARG with the counts and nothing written at or past a capacity; an empty mesh gives
zero counts."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import gpu_volume, run_frames

pytestmark = pytest.mark.gpu

INVALID = 1
SENTINEL = -7


def _buffers(nv, nt):
    dev = torch.device("cuda")
    return dict(pos=torch.full((nv, 3), float(SENTINEL), device=dev), nrm=torch.full((nv, 3), float(SENTINEL), device=dev),
                tris=torch.full((nt, 3), SENTINEL, dtype=torch.int32, device=dev),
                keys=torch.full((nv,), SENTINEL, dtype=torch.int64, device=dev),
                refcount=torch.full((nv,), SENTINEL, dtype=torch.int32, device=dev))


def _into(g, b, cap_v, cap_t):
    n1, n2 = ctypes.c_int64(), ctypes.c_int64()
    rc = g._lib.vm_download_mesh_into(g._h, b["pos"].data_ptr(), b["nrm"].data_ptr(), b["tris"].data_ptr(),
                                      b["keys"].data_ptr(), b["refcount"].data_ptr(), cap_v, cap_t, ctypes.byref(n1),
                                      ctypes.byref(n2))
    torch.cuda.synchronize()
    return rc, (n1.value, n2.value), {k: v.cpu().numpy() for k, v in b.items()}


def _volume(frames=6, seed=71):
    s = synth.small_room_scene(num_frames=frames, seed=synth.SEED_BASE + seed)
    g = gpu_volume(s.volume)
    run_frames(s, range(frames), gpu=g, mode="graph")
    return s, g


def test_into_matches_host_and_device_downloads():
    s, g = _volume()
    host = g.download()
    nv, nt = host["pos"].shape[0], host["tris"].shape[0]
    assert nv > 1000 and nt > 1000
    # vm_download_mesh with device buffers (on_device = 1)
    dev = _buffers(nv, nt)
    assert g._lib.vm_download_mesh(g._h, dev["pos"].data_ptr(), dev["nrm"].data_ptr(), dev["tris"].data_ptr(),
                                   dev["keys"].data_ptr(), dev["refcount"].data_ptr(), 1) == 0
    torch.cuda.synchronize()
    # the new entry point into larger buffers: exactly the counted prefix is written
    rc, counts, out = _into(g, _buffers(nv + 50, nt + 50), nv + 50, nt + 50)
    assert rc == 0 and counts == (nv, nt)
    for k in ("pos", "nrm", "tris", "keys", "refcount"):
        d = dev[k].cpu().numpy()
        np.testing.assert_array_equal(out[k][:d.shape[0]], d)
        np.testing.assert_array_equal(out[k][:d.shape[0]], host[k].astype(d.dtype) if k == "keys" else host[k])
        assert np.all(out[k][d.shape[0]:] == SENTINEL), k
    # the binding's device download takes this path
    m = g.download(device=True)
    np.testing.assert_array_equal(m["tris"].cpu().numpy(), host["tris"])
    np.testing.assert_array_equal(m["pos"].cpu().numpy(), host["pos"])
    assert g.last_error() == 0


def test_into_refuses_small_capacities_without_writing_past_them():
    s, g = _volume(seed=72)
    nv, nt = g.mesh_counts()
    cv, ct = nv // 2, nt // 3
    b = _buffers(nv, nt)
    rc, counts, out = _into(g, b, cv, ct)
    assert rc == INVALID and counts == (nv, nt)
    # nothing at or past a capacity is written
    for k in ("pos", "nrm", "keys", "refcount"):
        assert np.all(out[k][cv:] == SENTINEL), k
    assert np.all(out["tris"][ct:] == SENTINEL)
    # the prefix below the capacities is the compaction's
    host = g.download()
    np.testing.assert_array_equal(out["pos"][:cv], host["pos"][:cv])
    np.testing.assert_array_equal(out["refcount"][:cv], host["refcount"][:cv])
    # called again with the counts as capacities, it succeeds
    rc, counts, out = _into(g, _buffers(nv, nt), nv, nt)
    assert rc == 0 and counts == (nv, nt)
    np.testing.assert_array_equal(out["tris"], host["tris"])


def test_into_on_an_empty_volume():
    s = synth.small_room_scene(num_frames=1, seed=synth.SEED_BASE + 73)
    g = gpu_volume(s.volume)
    rc, counts, out = _into(g, _buffers(4, 4), 4, 4)
    assert rc == 0 and counts == (0, 0)
    assert np.all(out["pos"] == SENTINEL) and np.all(out["tris"] == SENTINEL)
    m = g.download(device=True)
    assert m["pos"].shape == (0, 3) and m["tris"].shape == (0, 3)
