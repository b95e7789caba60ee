"""Pins of the oracle's gradients (differentiable path, Secs. V-A and V-C with topology held
fixed): central finite differences of the float64 oracle's own forward, and closed forms
for a fronto-parallel plane."""
import numpy as np
import pytest

import oracle
import synth
from meshutil import key_decode, sphere_fill


def _functional(n, seed):
    """A random linear loss L = sum(A * pos) + sum(B * nrm): its derivatives are A and B."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 3)), rng.standard_normal((n, 3))


def _loss(mesh, A, B, vkeys):
    assert np.array_equal(mesh["vkeys"], vkeys)  # same vertices (topology fixed)
    return float(np.sum(A * mesh["pos"]) + np.sum(B * mesh["nrm"]))


def test_vertex_gradient_matches_finite_differences_on_analytic_sphere():
    l, mu = 0.01, 0.04
    keys, tsdf, w = sphere_fill((0.013, -0.021, 0.007), 0.093, l, mu)
    V = oracle.Volume(l, mu, prec="f64")
    V.set_blocks(keys, tsdf, w)
    V.update_mesh(full=True)
    m0 = V.mesh()
    A, B = _functional(len(m0["vkeys"]), 7)
    V.diff_begin()
    V.grad_vertices(m0["vkeys"], A, B)
    G = V.grad_tsdf()
    bk = V.blocks()["keys"]
    nz = np.argwhere(np.abs(G) > 1e-9)
    rng = np.random.default_rng(3)
    pick = nz[rng.choice(len(nz), size=min(60, len(nz)), replace=False)]
    h = 1e-7
    checked = 0
    for b, i in pick:
        g = bk[b] * 8 + np.array([i % 8, (i // 8) % 8, i // 64])
        d = tsdf[np.flatnonzero((keys == bk[b]).all(1))[0], i]
        V.set_voxel(g, d + h)
        mp = V.mesh()
        V.set_voxel(g, d - h)
        mm = V.mesh()
        V.set_voxel(g, d)
        fd = (_loss(mp, A, B, m0["vkeys"]) - _loss(mm, A, B, m0["vkeys"])) / (2 * h)
        assert abs(fd - G[b, i]) <= 1e-5 * max(1.0, abs(G[b, i])), (g, fd, G[b, i])
        checked += 1
    assert checked >= 40
    # voxels no vertex reads have no gradient
    reads = set()
    g_v, ax = key_decode(m0["vkeys"])
    for gv, a in zip(g_v, ax):
        e = np.eye(3, dtype=np.int64)
        for off in [np.zeros(3, np.int64), e[a]] + [e[b] for b in range(3) if b != a] + [e[a] + e[b] for b in range(3) if b != a]:
            reads.add(tuple(gv + off))
    for b, i in np.argwhere(np.abs(G) > 0):
        g = tuple(bk[b] * 8 + np.array([i % 8, (i // 8) % 8, i // 64]))
        assert g in reads


def _run(scene, frames, leaf_from, depth_override=None, prec="f64"):
    V = oracle.Volume.from_config(scene.volume, prec=prec)
    K = (scene.fx, scene.fy, scene.cx, scene.cy)
    for k in range(frames):
        if k == leaf_from:
            V.diff_begin()
        d = scene.depth(k) if depth_override is None or k not in depth_override else depth_override[k]
        T = scene.pose(k)
        V.integrate(d, K, T, synth.pose_inverse_f64(T))
    V.update_mesh(full=True, refine=True)
    return V


def test_depth_gradient_matches_finite_differences():
    """h = 1e-4 m on sampled depth pixels of the leaf frames, skipping samples whose +-h runs
    change an integration decision (integrated set, truncation branch) or the topology."""
    s = synth.small_room_scene(num_frames=6)
    frames, leaf = 6, 3
    V = _run(s, frames, leaf)
    m0 = V.mesh()
    st0 = V.stats()
    A, B = _functional(len(m0["vkeys"]), 11)
    V.grad_vertices(m0["vkeys"], A, B)
    Gd = V.grad_depth(s.W, s.H)
    assert Gd.shape == (frames - leaf, s.H, s.W)
    flat = np.argwhere(np.abs(Gd) > 1e-6 * np.abs(Gd).max())
    rng = np.random.default_rng(5)
    pick = flat[rng.choice(len(flat), size=min(40, len(flat)), replace=False)]
    h = 1e-4
    checked = 0
    for f, v, u in pick:
        k = leaf + f
        base = s.depth(k).astype(np.float32)
        runs = []
        for sgn in (1, -1):
            d = base.copy()
            d[v, u] = np.float32(d[v, u] + sgn * h)
            Vp = _run(s, frames, leaf, {k: d})
            runs.append((Vp.mesh(), Vp.stats(), float(d[v, u]) - float(base[v, u])))
        (mp, sp, hp), (mm, sm, hm) = runs
        same = all(sp[x] == sm[x] == st0[x] for x in ("voxels_integrated", "truncated", "cells"))
        same = same and np.array_equal(mp["vkeys"], m0["vkeys"]) and np.array_equal(mm["vkeys"], m0["vkeys"])
        same = same and np.array_equal(mp["tkeys"], m0["tkeys"]) and np.array_equal(mm["tkeys"], m0["tkeys"])
        if not same:
            continue
        fd = (_loss(mp, A, B, m0["vkeys"]) - _loss(mm, A, B, m0["vkeys"])) / (hp - hm)
        g = Gd[f, v, u]
        assert abs(fd - g) <= 2e-3 * abs(g) + 1e-7 * np.abs(Gd).max(), (k, v, u, fd, g)
        checked += 1
    assert checked >= 20


def _plane_scene(frames):
    """Noise-free fronto-parallel plane at camera depth 0.503 m (between lattice planes),
    camera at the origin looking along +z (identity pose), 64 x 48 pixels."""
    W, H = 64, 48
    depth = np.full((H, W), 0.503, np.float32)
    K = (60.0, 60.0, 31.5, 23.5)
    return W, H, depth, K


def test_uniform_depth_shift_closed_form_on_plane():
    """A vertex on the plane moves by n_leaf / W per unit shift of every leaf depth pixel
    (d is the average of identical frames; the leaf frames carry n_leaf of W shares), so its
    depth gradients sum to n_leaf / W; a sideways position or a normal does not move."""
    W, H, depth, K = _plane_scene(4)
    l, mu = 0.01, 0.04
    T = np.eye(4)
    V = oracle.Volume(l, mu, prec="f64")
    for k in range(4):
        if k == 2:
            V.diff_begin()
        V.integrate(depth, K, T, T)
    V.update_mesh(full=True)
    m = V.mesh()
    g, ax = key_decode(m["vkeys"])
    assert np.all(ax == 2) and np.allclose(m["pos"][:, 2], 0.503, atol=1e-7)
    # interior vertices: well inside the image (projected |x|, |y| small)
    inner = np.flatnonzero((np.abs(m["pos"][:, 0]) < 0.1) & (np.abs(m["pos"][:, 1]) < 0.08))
    assert len(inner) > 50
    for j in inner[:: max(1, len(inner) // 12)]:
        for comp, expect in ((2, 0.5), (0, 0.0)):
            V2 = oracle.Volume(l, mu, prec="f64")
            for k in range(4):
                if k == 2:
                    V2.diff_begin()
                V2.integrate(depth, K, T, T)
            V2.update_mesh(full=True)
            gp = np.zeros_like(m["pos"])
            gp[j, comp] = 1.0
            V2.grad_vertices(m["vkeys"], gp, np.zeros_like(gp))
            Gd = V2.grad_depth(W, H)
            assert Gd.sum() == pytest.approx(expect, abs=1e-9)
        # the normal is (0, 0, -1) for every uniform shift: no depth gradient
        gn = np.zeros_like(m["nrm"])
        gn[j] = (0.3, -0.2, 0.7)
        V3 = oracle.Volume(l, mu, prec="f64")
        for k in range(4):
            if k == 2:
                V3.diff_begin()
            V3.integrate(depth, K, T, T)
        V3.update_mesh(full=True)
        V3.grad_vertices(m["vkeys"], np.zeros_like(gn), gn)
        assert abs(V3.grad_depth(W, H).sum()) < 1e-9


def test_tsdf_gradient_of_plane_vertex_is_the_interpolation_derivative():
    """p_z = z0 + l d0 / (d0 - d1) on a slope-1 field: dp/dd0 = -d1 / l, dp/dd1 = d0 / l."""
    W, H, depth, K = _plane_scene(1)
    l, mu = 0.01, 0.04
    T = np.eye(4)
    V = oracle.Volume(l, mu, prec="f64")
    V.integrate(depth, K, T, T)
    V.update_mesh(full=True)
    m = V.mesh()
    V.diff_begin()
    j = int(np.argmin(np.abs(m["pos"][:, 0]) + np.abs(m["pos"][:, 1])))
    gp = np.zeros_like(m["pos"])
    gp[j, 2] = 1.0
    V.grad_vertices(m["vkeys"], gp, np.zeros_like(gp))
    G = V.grad_tsdf()
    blk = V.blocks()
    (g0,), (a,) = key_decode(m["vkeys"][j:j + 1])
    assert a == 2

    def at(g):
        b = np.flatnonzero((blk["keys"] == np.floor_divide(g, 8)).all(1))[0]
        r = g - blk["keys"][b] * 8
        i = r[0] + 8 * r[1] + 64 * r[2]
        return blk["tsdf"][b, i], G[b, i]

    d0, G0 = at(g0)
    d1, G1 = at(g0 + np.array([0, 0, 1]))
    assert G0 == pytest.approx(-d1 / (d0 - d1) ** 2 * l, rel=1e-9)
    assert G1 == pytest.approx(d0 / (d0 - d1) ** 2 * l, rel=1e-9)
    assert G0 + G1 == pytest.approx(1.0, rel=1e-9)  # unit slope: a uniform d shift moves p by itself
    assert np.count_nonzero(G) == 2
