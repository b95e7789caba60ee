"""Comparison helpers shared by the tests: canonical mesh forms and manifold checks.

Nothing here computes the method; these functions only reorder and count what the
oracle or the CUDA path returned.

Canonical form: a vertex is named by its edge key (owner voxel coordinates biased by
2^19, 20 bits each, and the axis in the low 2 bits); a triangle by its three vertex keys
rotated so that the smallest key comes first (orientation kept); a mesh by the sorted
list of its triangles.  Raw pool indices never enter a comparison.
"""
from __future__ import annotations

import numpy as np

BIAS = 1 << 19


def key_decode(keys: np.ndarray):
    k = np.asarray(keys, np.uint64)
    g = np.stack([((k >> np.uint64(s)) & np.uint64(0xFFFFF)).astype(np.int64) - BIAS for s in (42, 22, 2)], axis=-1)
    return g, (k & np.uint64(3)).astype(np.int64)


def key_encode(g: np.ndarray, axis: np.ndarray) -> np.ndarray:
    g = np.asarray(g, np.int64) + BIAS
    return ((g[..., 0].astype(np.uint64) << np.uint64(42)) | (g[..., 1].astype(np.uint64) << np.uint64(22))
            | (g[..., 2].astype(np.uint64) << np.uint64(2)) | np.asarray(axis, np.uint64))


def canonical_triangles(tkeys: np.ndarray) -> np.ndarray:
    """(nt, 3) key triples -> rotated min-first, rows sorted lexicographically."""
    t = np.asarray(tkeys, np.uint64).reshape(-1, 3)
    if len(t) == 0:
        return t
    r = np.argmin(t, axis=1)
    idx = (r[:, None] + np.arange(3)[None, :]) % 3
    rot = np.take_along_axis(t, idx, axis=1)
    order = np.lexsort((rot[:, 2], rot[:, 1], rot[:, 0]))
    return rot[order]


def edge_incidence(tris: np.ndarray):
    """Directed-edge and undirected-edge counts of an indexed triangle list."""
    t = np.asarray(tris).reshape(-1, 3)
    a = np.concatenate([t[:, 0], t[:, 1], t[:, 2]])
    b = np.concatenate([t[:, 1], t[:, 2], t[:, 0]])
    directed = np.stack([a, b], 1)
    und = np.sort(directed, axis=1)
    u, cnt = np.unique(und, axis=0, return_counts=True)
    d, dcnt = np.unique(directed, axis=0, return_counts=True)
    return u, cnt, d, dcnt


def manifold_report(tris: np.ndarray) -> dict:
    """Closed, consistently oriented 2-manifold checks and the Euler characteristic."""
    t = np.asarray(tris).reshape(-1, 3)
    if len(t) == 0:
        return dict(closed=True, oriented=True, euler=0, V=0, E=0, F=0, degenerate=0)
    u, cnt, d, dcnt = edge_incidence(t)
    V = len(np.unique(t))
    E = len(u)
    F = len(t)
    degenerate = int(np.sum((t[:, 0] == t[:, 1]) | (t[:, 1] == t[:, 2]) | (t[:, 0] == t[:, 2])))
    return dict(closed=bool(np.all(cnt == 2)), oriented=bool(np.all(dcnt == 1)), euler=V - E + F, V=V, E=E, F=F,
                degenerate=degenerate)


def signed_volume(pos: np.ndarray, tris: np.ndarray) -> float:
    p = np.asarray(pos, np.float64)
    t = np.asarray(tris).reshape(-1, 3)
    a, b, c = p[t[:, 0]], p[t[:, 1]], p[t[:, 2]]
    return float(np.sum(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6.0)


def index_mesh(vkeys: np.ndarray, tkeys: np.ndarray):
    """Key-named triangles -> indices into the sorted unique vertex keys."""
    vk = np.asarray(vkeys, np.uint64)
    order = np.argsort(vk)
    idx = np.searchsorted(vk[order], np.asarray(tkeys, np.uint64).reshape(-1))
    return order[idx].reshape(-1, 3)


def sphere_fill(center, radius, voxel, trunc, pad_blocks=1):
    """Blocks covering a sphere with the exact SDF clamped to [-trunc, trunc], weight 1."""
    c = np.asarray(center, np.float64)
    lo = np.floor((c - radius - trunc) / voxel / 8).astype(int) - pad_blocks + 1
    hi = np.floor((c + radius + trunc) / voxel / 8).astype(int) + pad_blocks
    keys = np.array([[x, y, z] for z in range(lo[2], hi[2] + 1) for y in range(lo[1], hi[1] + 1)
                     for x in range(lo[0], hi[0] + 1)], np.int32)
    loc = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1)
    loc = loc.transpose(2, 1, 0, 3).reshape(512, 3)  # x fastest
    g = keys[:, None, :] * 8 + loc[None, :, :]
    p = g * voxel
    sdf = np.linalg.norm(p - c, axis=-1) - radius
    return keys, np.clip(sdf, -trunc, trunc), np.ones_like(sdf)


def field_fill(keys, fn, voxel, trunc):
    """Blocks `keys` filled with clip(fn(world points), -trunc, trunc), weight 1."""
    keys = np.asarray(keys, np.int32).reshape(-1, 3)
    loc = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1)
    loc = loc.transpose(2, 1, 0, 3).reshape(512, 3)
    g = keys[:, None, :] * 8 + loc[None, :, :]
    vals = fn(g * voxel)
    return keys, np.clip(vals, -trunc, trunc), np.ones(vals.shape)
