"""Full-size, long runs against the float32 oracle, element by element, in the benchmark's
launch configuration (vm_step replayed from a CUDA graph, refine and gc every frame).

* The room (640x480, voxel 8 mm, 2^20 buckets) over 300 frames, compared after frames 25,
  100 and 300: by then the free stacks have handed recycled vertex ids, triangle runs and
  block slots back out many times (the pools' high-water marks stay below the totals
  created), so steady-state reuse is covered.
* The floor (640x480, voxel 5 mm, 2^23 buckets, 2^21-block pools), refined, over its first
  60 frames, compared after frames 30 and 60.

Bar as in test_gpu_parity: block set, cube types and canonical topology bit-exact, TSDF and
weights within 1e-5, positions within 1e-5 x voxel, normals within 1e-5, reference count ==
degree, no duplicate vertex.
"""
import pytest

import oracle
import synth
from tests.gpu_util import compare_blocks, compare_mesh, gpu_volume, run_frames

pytestmark = pytest.mark.gpu


def _run_and_compare(scene, frames, at):
    g = gpu_volume(scene.volume)
    o = oracle.Volume.from_config(scene.volume, prec="f32")
    seen = []

    def check(k):
        if k + 1 not in at:
            return
        g.check()
        sb = compare_blocks(g.blocks(), o.blocks())
        sm = compare_mesh(g.download(), o.mesh(), scene.volume.voxel_size)
        seen.append((k + 1, sb, sm, g.stats()))

    run_frames(scene, range(frames), gpu=g, orc=o, refine=True, gc=True, mode="graph", after_frame=check)
    assert [s[0] for s in seen] == sorted(at)
    return seen


def test_room_300_frames_match_oracle_with_pool_reuse():
    s = synth.room_scene(num_frames=310)  # the benchmark's room sequence
    seen = _run_and_compare(s, 300, (25, 100, 300))
    for n, sb, sm, st in seen:
        assert sb["blocks"] > 500 and sm["triangles"] > 50000, (n, sb, sm)
        assert st["freed_vertices"] > 0, n
    _, _, _, st = seen[-1]
    # recycled ids handed out again: fewer pool slots ever used than items ever created
    assert st["freed_blocks"] > 0 and st["block_high_water"] < st["new_blocks"], st
    assert st["vertex_high_water"] < st["created_vertices"], st
    assert st["triangle_high_water"] < st["emitted_triangles"], st


def test_floor_60_refined_frames_match_oracle():
    s = synth.floor_scene()  # the 2000-frame trajectory; its first 60 frames
    seen = _run_and_compare(s, 60, (30, 60))
    for n, sb, sm, st in seen:
        assert sb["blocks"] > 10000 and sm["triangles"] > 1000000, (n, sb, sm)
        assert st["freed_vertices"] > 0, n
    _, _, _, st = seen[-1]
    assert st["vertex_high_water"] < st["created_vertices"], st
    assert st["triangle_high_water"] < st["emitted_triangles"], st
