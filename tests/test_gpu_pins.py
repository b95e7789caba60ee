"""The CUDA path on the inputs of the oracle pins (tests/test_oracle_pins.py), through the C ABI.

* The per-pixel-coded depth frame: the GPU fuses every voxel from the same pixel as the
  float32 oracle (block set and TSDF bit-exact, weights equal), so the hand-computed
  nearest-pixel pick that pins the oracle pins the kernel too.
* The hand-built block-recycling cases: after each of the two gc calls (one before the
  pending mesh update, one after it) the GPU keeps exactly the blocks the oracle keeps.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import compare_blocks, gpu_volume
from tests.test_oracle_pins import CX, CY, EMPTY, FX, FY, H_IMG, W_IMG, _coded_frame, _rule_volume

pytestmark = pytest.mark.gpu


def _vc(l, mu):
    return synth.VolumeConfig(voxel_size=l, trunc=mu, hash_buckets=1 << 14, max_blocks=1 << 12,
                              max_vertices=1 << 16, max_triangles=1 << 17)


def test_coded_frame_fuses_the_same_pixels_as_the_oracle():
    from paper_1803_03949_b300 import Intrinsics

    l, mu = 0.01, 0.2
    g = gpu_volume(_vc(l, mu))
    o = oracle.Volume(l, mu, prec="f32")
    D = _coded_frame()
    I4 = np.eye(4, dtype=np.float32)
    g.integrate(torch.from_numpy(D).cuda(), Intrinsics(W_IMG, H_IMG, FX, FY, CX, CY), I4, I4)
    o.integrate(D, (FX, FY, CX, CY), np.eye(4), np.eye(4))
    g.check()
    st = compare_blocks(g.blocks(), o.blocks(), tol=0.0)
    assert st["tsdf_bit_exact"] and st["blocks"] > 300


def _alive(b):
    return {tuple(int(c) for c in k) for k in b["keys"]}


def test_gc_block_rule_cases_match_the_oracle():
    from paper_1803_03949_b300 import Intrinsics

    o, mu, blocks = _rule_volume("f32")
    g = gpu_volume(_vc(0.01, mu))

    def put(which):
        keys = np.array(which, np.int32).reshape(-1, 3)
        t = np.stack([blocks[tuple(k)][0] for k in which])
        w = np.stack([blocks[tuple(k)][1] for k in which])
        g.set_blocks(keys, t.astype(np.float32), w.astype(np.float32))
        o.set_blocks(keys, t.astype(np.float32).astype(np.float64), w)

    every = list(blocks)
    put(every)
    g.update_mesh(full=True)
    o.update_mesh(full=True)
    empty = torch.from_numpy(EMPTY).cuda()
    g.integrate(empty, Intrinsics(4, 4, 1.0, 1.0, 1.5, 1.5), np.eye(4, dtype=np.float32), np.eye(4, dtype=np.float32))
    o.integrate(EMPTY, (1.0, 1.0, 1.5, 1.5), np.eye(4), np.eye(4))
    put([(50, 0, 0), (60, 0, 0)])
    g.gc()
    o.gc()
    g.check()
    a1 = _alive(g.blocks())
    assert a1 == _alive(o.blocks())
    assert set(every) - a1 == {(0, 0, 0), (10, 0, 0)}
    g.update_mesh()
    o.update_mesh()
    g.gc()
    o.gc()
    g.check()
    a2 = _alive(g.blocks())
    assert a2 == _alive(o.blocks())
    assert a1 - a2 == {(59, 0, 0)}
    assert g.stats()["freed_blocks"] == 3
