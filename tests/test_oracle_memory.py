"""Pins of the oracle's mesh-memory counts (Sec. VI-B "Memory"): a plane crossing a 2 x 2
block patch, where every count has a closed form."""
import numpy as np

import oracle
from meshutil import field_fill


def test_plane_patch_vertex_counts():
    """Plane z = 3.5 voxels through blocks (0..1, 0..1, 0): cubes 0..14 in x and y are valid
    (cube 15 needs voxel 16, in a block that does not exist), so the plane has 15 x 15 cubes:
    16 x 16 edge-owned vertices and 2 x 15 x 15 triangles (Sec. VI-B: about 2 triangles per
    vertex).  A per-block extraction stores (cubes_x + 1)(cubes_y + 1) vertices per block:
    9 x 9 + 8 x 9 + 9 x 8 + 8 x 8 = 289; loose triangles store 3 x 450."""
    l, mu = 0.01, 0.04
    keys = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], np.int32)
    keys, tsdf, w = field_fill(keys, lambda p: p[..., 2] - 3.5 * l, l, mu)
    for prec in ("f32", "f64"):
        V = oracle.Volume(l, mu, prec=prec)
        V.set_blocks(keys, tsdf, w)
        V.update_mesh(full=True)
        m = V.mesh_memory()
        assert m == dict(vertices=256, block_vertices=289, loose_vertices=1350, triangles=450), m
        assert len(V.mesh()["vkeys"]) == 256


def test_single_block_sphere_has_no_copies():
    """A surface inside one block: the per-block extraction shares every vertex too."""
    l, mu = 0.01, 0.04
    keys = np.array([[0, 0, 0]], np.int32)
    c = np.array([3.6, 3.4, 3.5]) * l
    keys, tsdf, w = field_fill(keys, lambda p: np.linalg.norm(p - c, axis=-1) - 2.2 * l, l, mu)
    V = oracle.Volume(l, mu, prec="f64")
    V.set_blocks(keys, tsdf, w)
    V.update_mesh(full=True)
    m = V.mesh_memory()
    assert m["vertices"] == m["block_vertices"] == len(V.mesh()["vkeys"]) > 0
    assert m["loose_vertices"] == 3 * m["triangles"]
