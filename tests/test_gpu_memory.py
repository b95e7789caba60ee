"""Mesh memory counts on the GPU (Sec. VI-B): edge-owned vertices against a per-block
extraction and loose triangles, equal to the oracle's counts."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import gpu_volume, run_frames
from tests.meshutil import field_fill

pytestmark = pytest.mark.gpu


def _check_counts(g, o, after_gc):
    gm, om = g.mesh_memory(), o.mesh_memory()
    for k in ("vertices", "block_vertices", "loose_vertices", "triangles"):
        assert gm[k] == om[k], (k, gm[k], om[k])
    if g.params.flags:  # the compact cube record
        assert gm["cube_bytes"] == 19
        # one edge record per voxel owning a vertex: exactly the live vertices' owners after a gc
        # (before it, also voxels whose vertices await recycling and spares of lost claims)
        owners = len(np.unique(np.asarray(g.download()["keys"], np.uint64) >> np.uint64(2)))
        assert gm["edge_records"] == owners if after_gc else gm["edge_records"] >= owners, (gm["edge_records"], owners)
    else:
        assert gm["cube_bytes"] == 27 and gm["edge_records"] == 0
    assert 0 < gm["bytes_in_use"] < gm["bytes_allocated"]
    return gm


def test_plane_patch_closed_form():
    l, mu = 0.01, 0.04
    keys = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], np.int32)
    keys, tsdf, w = field_fill(keys, lambda p: p[..., 2] - 3.5 * l, l, mu)
    g = gpu_volume(synth.VolumeConfig(voxel_size=l, trunc=mu, hash_buckets=1 << 10, max_blocks=64,
                                      max_vertices=1 << 12, max_triangles=1 << 13))
    g.set_blocks(keys, tsdf, w)
    g.update_mesh(full=True)
    m = g.mesh_memory()
    assert (m["vertices"], m["block_vertices"], m["loose_vertices"], m["triangles"]) == (256, 289, 1350, 450)


def test_sphere_workload_counts_match_oracle():
    s = synth.sphere_scene()
    g = gpu_volume(s.volume)
    o = oracle.Volume.from_config(s.volume, prec="f32")
    run_frames(s, range(10), gpu=g, orc=o, refine=False, gc=False)
    g.update_mesh(full=True, refine=True)
    o.update_mesh(full=True, refine=True)
    m = _check_counts(g, o, after_gc=False)
    assert m["block_vertices"] > m["vertices"] and m["loose_vertices"] > 4 * m["vertices"]


@pytest.mark.parametrize("compact", [False, True])
def test_room_incremental_counts_match_oracle(compact):
    s = synth.room_scene(num_frames=12, W=320, H=240)
    g = gpu_volume(dataclasses.replace(s.volume, compact_edges=compact))
    o = oracle.Volume.from_config(s.volume, prec="f32")
    run_frames(s, range(12), gpu=g, orc=o, refine=True, gc=True, mode="graph")
    _check_counts(g, o, after_gc=True)
