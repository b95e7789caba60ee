"""The compact cube record (VM_PARAM_COMPACT_EDGES: one edge-record index per voxel, records
only for voxels that own a vertex): the same results as the oracle and as the default layout,
through the single-volume path, the frame graph, gc and the batched step."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import (compare_blocks, compare_mesh, gpu_mesh_canonical, gpu_volume, intrinsics, poses32,
                            run_frames, sorted_blocks)

pytestmark = pytest.mark.gpu


def _compact(vc):
    return dataclasses.replace(vc, compact_edges=True)


def _same_state(a, b):
    ba, bb = sorted_blocks(a.blocks()), sorted_blocks(b.blocks())
    for k in ba:
        np.testing.assert_array_equal(ba[k], bb[k], err_msg=k)
    ma, mb = a.download(), b.download()
    ka, ta = gpu_mesh_canonical(ma)
    kb, tb = gpu_mesh_canonical(mb)
    np.testing.assert_array_equal(ta, tb)
    oa, ob = np.argsort(ka), np.argsort(kb)
    np.testing.assert_array_equal(ka[oa], kb[ob])
    np.testing.assert_array_equal(np.asarray(ma["pos"])[oa], np.asarray(mb["pos"])[ob])
    np.testing.assert_array_equal(np.asarray(ma["nrm"])[oa], np.asarray(mb["nrm"])[ob])
    np.testing.assert_array_equal(np.asarray(ma["refcount"])[oa], np.asarray(mb["refcount"])[ob])


def test_sphere_full_extraction_matches_oracle():
    s = synth.sphere_scene()
    g, o = gpu_volume(_compact(s.volume)), oracle.Volume.from_config(s.volume)
    run_frames(s, range(s.num_frames), gpu=g, orc=o, refine=False, gc=False)
    g.update_mesh(full=True, refine=True)
    o.update_mesh(full=True, refine=True)
    g.check()
    compare_blocks(g.blocks(), o.blocks())
    assert compare_mesh(g.download(), o.mesh(), s.volume.voxel_size)["triangles"] > 100000
    assert g.mesh_memory()["cube_bytes"] == 19


def test_small_room_incremental_with_gc_matches_oracle():
    s = synth.small_room_scene(num_frames=8)
    g, o = gpu_volume(_compact(s.volume)), oracle.Volume.from_config(s.volume)

    def check(k):
        g.check()
        compare_blocks(g.blocks(), o.blocks())
        compare_mesh(g.download(), o.mesh(), s.volume.voxel_size)

    run_frames(s, range(8), gpu=g, orc=o, after_frame=check)
    assert g.stats()["freed_vertices"] > 0 and g.stats()["freed_blocks"] > 0


@pytest.mark.parametrize("which", ["room", "floor"])
def test_full_size_graph_equals_default_layout(which):
    """640x480 frames through vm_step graphs (the benchmark's launches): both layouts end in the
    same blocks, TSDF, types, canonical mesh, positions, normals and reference counts."""
    s = synth.room_scene(num_frames=40) if which == "room" else synth.floor_scene()
    n = 40 if which == "room" else 12
    a, b = gpu_volume(s.volume), gpu_volume(_compact(s.volume))
    run_frames(s, range(n), gpu=a, mode="graph")
    run_frames(s, range(n), gpu=b, mode="graph")
    a.check()
    b.check()
    _same_state(a, b)
    mb = b.mesh_memory()
    owners = len(np.unique(np.asarray(b.download()["keys"], np.uint64) >> np.uint64(2)))
    assert mb["edge_records"] == owners  # after the frame's gc: one record per owning voxel


def test_batched_step_with_compact_volumes():
    import torch

    from paper_1803_03949_b300 import Scenes, VmeshError

    scenes = [synth.small_room_scene(num_frames=6, seed=synth.SEED_BASE + 50 + i) for i in range(3)]
    vols = [gpu_volume(_compact(s.volume)) for s in scenes]
    with pytest.raises(VmeshError):  # one layout per batch
        Scenes([vols[0], gpu_volume(scenes[1].volume)])
    batch = Scenes(vols)
    Ks = [intrinsics(s) for s in scenes]
    for k in range(6):
        batch.step_all([torch.from_numpy(s.depth(k)).cuda() for s in scenes], Ks, [poses32(s.pose(k)) for s in scenes])
    torch.cuda.synchronize()
    for s, v in zip(scenes, vols):
        v.check()
        single = gpu_volume(s.volume)
        run_frames(s, range(6), gpu=single, mode="graph")
        _same_state(v, single)
    batch.close()
