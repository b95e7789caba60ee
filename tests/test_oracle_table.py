"""Pins of the oracle's marching-cubes table (Sec. V-B) against what the definition fixes.

* every sign-change edge carries a vertex and no other edge does (the meaning of T(t));
* at most 5 triangles per cube (Fig. 3 caption, Sec. IV);
* a shared face is cut identically, with opposite orientation, by both cubes (watertight);
* a lone negative (positive) corner is cut off by one triangle facing away from (towards) it;
* random fields with a positive border mesh into closed, consistently oriented surfaces whose
  enclosed volume is positive.
"""
import itertools

import numpy as np
import pytest

import oracle
from tests.meshutil import manifold_report, signed_volume

CORNER = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])
EDGE = np.array([[0, 1], [1, 2], [3, 2], [0, 3], [4, 5], [5, 6], [7, 6], [4, 7], [0, 4], [1, 5], [2, 6], [3, 7]])


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_table_builds_consistently(prec):
    assert oracle.table_ok(prec)


def test_vertices_exactly_on_sign_change_edges():
    n, t = oracle.mc_table()
    for code in range(256):
        neg = [(code >> k) & 1 for k in range(8)]
        crossing = {k for k in range(12) if neg[EDGE[k, 0]] != neg[EDGE[k, 1]]}
        used = set(t[code, : n[code]].reshape(-1).tolist())
        assert used == crossing, code


def test_at_most_five_triangles_and_trivial_codes():
    n, _ = oracle.mc_table()
    assert n.max() == 5
    assert n[0] == 0 and n[255] == 0
    for k in range(8):
        assert n[1 << k] == 1 and n[255 ^ (1 << k)] == 1


def _midpoint(e):
    return 0.5 * (CORNER[EDGE[e, 0]] + CORNER[EDGE[e, 1]])


def test_single_corner_orientation():
    n, t = oracle.mc_table()
    centre = np.array([0.5, 0.5, 0.5])
    for k in range(8):
        for code, sign in ((1 << k, 1.0), (255 ^ (1 << k), -1.0)):
            e = t[code, 0]
            p = [_midpoint(x) for x in e]
            normal = np.cross(p[1] - p[0], p[2] - p[0])
            # normal points from negative to positive: away from a lone negative corner
            assert sign * np.dot(normal, centre - CORNER[k]) > 0, (code, k)


def _boundary_segments(code, n, t, offset):
    """Directed boundary edges of a cube's patch, vertices named by global edge identity."""
    def gid(e):
        c = CORNER[EDGE[e, 0]] + offset
        axis = int(np.argmax(CORNER[EDGE[e, 1]] - CORNER[EDGE[e, 0]]))
        return (int(c[0]), int(c[1]), int(c[2]), axis)

    directed = []
    for tri in t[code, : n[code]]:
        g = [gid(x) for x in tri]
        directed += [(g[0], g[1]), (g[1], g[2]), (g[2], g[0])]
    s = set(directed)
    return {d for d in s if (d[1], d[0]) not in s}


def test_watertight_shared_faces():
    n, t = oracle.mc_table()
    for axis in range(3):
        off = np.zeros(3, int)
        off[axis] = 1
        a_face = [k for k in range(8) if CORNER[k, axis] == 1]
        b_of = {k: int(np.nonzero((CORNER == CORNER[k] - off).all(1))[0][0]) for k in a_face}

        def on_face(edge_gid):
            c = list(edge_gid[:3])
            return c[axis] == 1 and edge_gid[3] != axis

        for ca in range(256):
            sa = {g for g in _boundary_segments(ca, n, t, np.zeros(3, int)) if on_face(g[0]) and on_face(g[1])}
            for cb in range(256):
                if any(((ca >> k) & 1) != ((cb >> b_of[k]) & 1) for k in a_face):
                    continue
                sb = {g for g in _boundary_segments(cb, n, t, off) if on_face(g[0]) and on_face(g[1])}
                assert {(q, p) for (p, q) in sa} == sb, (axis, ca, cb)


def _plain_mesh_from_field(field, n, t):
    """Mesh a dense corner field (all corners valid) cube by cube, vertices welded by edge."""
    nx, ny, nz = field.shape
    vid = {}
    pos = []
    tris = []
    for z, y, x in itertools.product(range(nz - 1), range(ny - 1), range(nx - 1)):
        d = [field[x + c[0], y + c[1], z + c[2]] for c in CORNER]
        code = sum(1 << k for k in range(8) if d[k] < 0)
        for tri in t[code, : n[code]]:
            ids = []
            for e in tri:
                a, b = EDGE[e]
                pa = np.array([x, y, z]) + CORNER[a]
                pb = np.array([x, y, z]) + CORNER[b]
                key = (tuple(pa), tuple(pb))
                if key not in vid:
                    s = d[a] / (d[a] - d[b])
                    vid[key] = len(pos)
                    pos.append(pa + s * (pb - pa))
                ids.append(vid[key])
            tris.append(ids)
    return np.array(pos), np.array(tris)


@pytest.mark.parametrize("seed", range(6))
def test_random_fields_give_closed_oriented_surfaces(seed):
    n, t = oracle.mc_table()
    rng = np.random.default_rng(seed)
    field = rng.normal(size=(9, 9, 9))
    field[[0, -1], :, :] = 1.0
    field[:, [0, -1], :] = 1.0
    field[:, :, [0, -1]] = 1.0
    field[field == 0] = 1e-3
    pos, tris = _plain_mesh_from_field(field, n, t)
    rep = manifold_report(tris)
    assert rep["closed"] and rep["oriented"] and rep["degenerate"] == 0, rep
    assert signed_volume(pos, tris) > 0
