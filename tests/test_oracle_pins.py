"""Pins of two oracle rules whose mistakes no other pin would see.

* Nearest-pixel pick of the fusion (Sec. V-A, Eq. 2, pixel centres at integer coordinates):
  a depth frame whose value differs at every pixel (neighbours 1e-4 m apart) is fused once
  from the identity pose, so every fused voxel's TSDF names the pixel it sampled; the test
  computes that pixel by hand (the exact projection rounded to the nearest integer) and
  also checks the image bounds, the invalid-pixel skip, the -mu skip and the truncation at
  mu.  A projection that truncates instead of rounding, swaps fx and fy, or is off by one in
  cx or cy changes the TSDF of thousands of voxels by at least 1e-4 m.
* Block recycling (Sec. V-E, extended to blocks): hand-built volumes whose freed set follows
  from the rule by hand -- a block is freed iff it was not collected in the current epoch,
  is not kept for a pending update (gc before the mesh update), has no cube with triangles,
  has no voxel with W > 0 and d < mu, and none of its 7 lower neighbours has a cube with
  triangles.  Each case is built so that exactly one clause decides its fate.
"""
import numpy as np
import pytest

import oracle

# ------------------------------------------------------------------ nearest-pixel pick

W_IMG, H_IMG = 40, 30
FX, FY, CX, CY = 50.0, 47.0, 19.3, 14.6
STEP = 1e-4  # depth difference between neighbouring pixels (m)
INVALID = [(5, 7), (12, 30), (20, 3)]  # (row, column) pixels with depth 0, NaN, -1


def _coded_frame():
    u = np.arange(W_IMG)[None, :]
    v = np.arange(H_IMG)[:, None]
    D = (1.0 + STEP * (u + W_IMG * v)).astype(np.float32)
    D[INVALID[0]] = 0.0
    D[INVALID[1]] = np.nan
    D[INVALID[2]] = -1.0
    return D


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
def test_fusion_samples_the_nearest_pixel(prec, tol):
    l, mu = 0.01, 0.2
    V = oracle.Volume(l, mu, prec=prec)
    D = _coded_frame()
    I4 = np.eye(4)
    V.integrate(D, (FX, FY, CX, CY), I4, I4)
    b = V.blocks()
    keys, tsdf, wgt = b["keys"], b["tsdf"].reshape(-1), b["weight"].reshape(-1)
    loc = np.arange(512)
    g = (keys[:, None, :] * 8 + np.stack([loc % 8, (loc // 8) % 8, loc // 64], 1)[None]).reshape(-1, 3)
    p = g * l
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    # the exact projection, pixel centres at integer coordinates; the nearest pixel by hand
    us = FX * x / z + CX + 0.5
    vs = FY * y / z + CY + 0.5
    iu, iv = np.floor(us).astype(int), np.floor(vs).astype(int)
    # voxels whose pick, or image membership, is decided within 1e-3 px are left out
    fu, fv = us - iu, vs - iv
    clear = (z > 0) & (np.minimum(fu, 1 - fu) > 1e-3) & (np.minimum(fv, 1 - fv) > 1e-3)
    inside = (iu >= 0) & (iu < W_IMG) & (iv >= 0) & (iv < H_IMG)
    Dp = np.where(inside, D[np.clip(iv, 0, H_IMG - 1), np.clip(iu, 0, W_IMG - 1)].astype(np.float64), np.nan)
    valid = inside & np.isfinite(Dp) & (Dp > 0)
    sdf = Dp - z
    clear &= ~valid | (np.abs(sdf + mu) > 1e-5)
    fused = valid & (sdf >= -mu)
    c = clear
    # fused voxels: the TSDF of the hand-picked pixel, truncated at mu; the rest untouched
    np.testing.assert_array_equal(wgt[c & fused], 1.0)
    np.testing.assert_array_equal(wgt[c & ~fused], 0.0)
    np.testing.assert_allclose(tsdf[c & fused], np.minimum(sdf[c & fused], mu), rtol=0, atol=tol)
    np.testing.assert_array_equal(tsdf[c & ~fused], 0.0)
    # the workload exercises what the pin is about
    lin = c & fused & (sdf < mu - 1e-3)
    assert lin.sum() > 5000  # voxels whose TSDF names their pixel
    assert (lin & (fu >= 0.5)).sum() > 1000 and (lin & (fu < 0.5)).sum() > 1000
    assert (lin & (fv >= 0.5)).sum() > 1000 and (lin & (fv < 0.5)).sum() > 1000
    assert (c & fused & (sdf >= mu)).sum() > 1000  # truncated at mu
    assert (c & valid & (sdf < -mu)).sum() > 1000  # behind the surface: skipped
    assert (c & inside & ~valid & (z > 0.9) & (z < 1.3)).sum() > 10  # invalid pixels: skipped
    assert (c & ~inside).sum() > 1000  # outside the image: skipped


# ------------------------------------------------------------------ block recycling


def _rule_volume(prec):
    """The hand-built cases; returns (volume, mu as the build stores it, case table)."""
    l = 0.01
    mu = float(np.float32(0.04)) if prec == "f32" else 0.04
    V = oracle.Volume(l, mu, prec=prec)
    blocks = {}

    def put(key, tsdf, weight=1.0):
        t = np.full(512, tsdf, np.float64) if np.isscalar(tsdf) else np.asarray(tsdf, np.float64)
        blocks[tuple(key)] = (t, np.full(512, weight, np.float64))

    # A: every voxel observed at exactly d = mu (d >= mu is not near): freed
    put((0, 0, 0), mu)
    # B: nothing observed (W = 0, d = 0): freed
    put((10, 0, 0), 0.0, weight=0.0)
    # C: one voxel at d = mu / 2, no sign change anywhere: kept (near)
    t = np.full(512, mu)
    t[100] = 0.5 * mu
    put((20, 0, 0), t)
    # C2: one voxel one float step below mu: kept (near)
    t = np.full(512, mu)
    t[7] = float(np.nextafter(np.float32(mu), np.float32(0))) if prec == "f32" else np.nextafter(mu, 0.0)
    put((22, 0, 0), t)
    # D: the 8 blocks around one lattice corner, d = mu everywhere except d = -mu at that corner
    # (voxel 0 of the upper block): the corner block's cube (7,7,7) is the only cube of block
    # (30,0,0) with a triangle, and that triangle's three edges are owned by other blocks, so the
    # block owns no vertex and has no near voxel: kept because it has triangles
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                t = np.full(512, mu)
                if (dx, dy, dz) == (1, 1, 1):
                    t[0] = -mu
                put((30 + dx, dy, dz), t)
    # E: L has a sign change inside it (x < 4 negative), its +x neighbour U is far and has no
    # valid cube with a sign change and owns no vertex: U kept because its lower neighbour
    # L has triangles
    t = np.full(512, mu)
    t[(np.arange(512) % 8) < 4] = -0.5 * mu
    put((40, 0, 0), t)
    put((41, 0, 0), mu)
    # F: far, collected again in the current epoch: kept
    put((50, 0, 0), mu)
    # H: P far and collected again in the current epoch; its -x neighbour Q far: a gc before the
    # mesh update keeps Q (pending update set), the gc after it frees Q
    put((60, 0, 0), mu)
    put((59, 0, 0), mu)
    return V, mu, blocks


def _set(V, blocks, which):
    keys = np.array(which, np.int32).reshape(-1, 3)
    V.set_blocks(keys, np.stack([blocks[tuple(k)][0] for k in which]), np.stack([blocks[tuple(k)][1] for k in which]))


def _alive(V):
    return {tuple(int(c) for c in k) for k in V.blocks()["keys"]}


EMPTY = np.zeros((4, 4), np.float32)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_gc_block_rule_on_hand_built_volumes(prec):
    V, mu, blocks = _rule_volume(prec)
    every = list(blocks)
    _set(V, blocks, every)
    V.update_mesh(full=True)
    # the corner block of D has triangles, U has none, L has some (the construction holds)
    b = V.blocks()
    ntri = oracle.mc_table(prec)[0]
    tri = {tuple(int(c) for c in k): int(ntri[ce].sum()) for k, ce in zip(b["keys"], b["code_eff"])}
    assert tri[(30, 0, 0)] == 1 and tri[(31, 1, 1)] == 1 and tri[(41, 0, 0)] == 0 and tri[(40, 0, 0)] > 0
    assert tri[(0, 0, 0)] == 0 and tri[(20, 0, 0)] == 0
    # a frame without valid pixels starts the next epoch and collects nothing
    V.integrate(EMPTY, (1.0, 1.0, 1.5, 1.5), np.eye(4), np.eye(4))
    _set(V, blocks, [(50, 0, 0), (60, 0, 0)])  # collected in the new epoch, before its mesh update
    n1 = V.gc()
    after1 = _alive(V)
    freed1 = set(every) - after1
    assert freed1 == {(0, 0, 0), (10, 0, 0)}, sorted(freed1)
    assert n1 == 2
    V.update_mesh()
    n2 = V.gc()
    after2 = _alive(V)
    assert after1 - after2 == {(59, 0, 0)}, sorted(after1 - after2)
    assert n2 == 1
    # a further gc frees nothing
    assert V.gc() == 0
