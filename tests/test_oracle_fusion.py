"""Pins of the oracle's block collection (Sec. V-A, Eq. 1) and fusion (Sec. V-A, Eq. 2).

* the 3D DDA visits exactly the block cells a segment passes through (float64 brute force);
* every block near each observed surface point is collected (coverage);
* fusing fronto-parallel planes gives, per voxel, the arithmetic mean of the truncated
  plane distances over the frames that saw it (closed form), with the -mu skip rule;
* float32 and float64 builds agree on the block set for the sphere sequence.
"""
import numpy as np
import pytest

import oracle
import synth


def _cells_brute(A, B):
    """Cells whose closed box the segment A-B crosses with positive length (float64)."""
    A, B = np.asarray(A, float), np.asarray(B, float)
    lo = np.floor(np.minimum(A, B)).astype(int)
    hi = np.floor(np.maximum(A, B)).astype(int)
    d = B - A
    out = set()
    for x in range(lo[0], hi[0] + 1):
        for y in range(lo[1], hi[1] + 1):
            for z in range(lo[2], hi[2] + 1):
                t0, t1 = 0.0, 1.0
                for i, c in enumerate((x, y, z)):
                    if abs(d[i]) < 1e-300:
                        if not (c <= A[i] <= c + 1):
                            t0, t1 = 1.0, 0.0
                        continue
                    a, b = (c - A[i]) / d[i], (c + 1 - A[i]) / d[i]
                    t0, t1 = max(t0, min(a, b)), min(t1, max(a, b))
                if t1 - t0 > 1e-9:
                    out.add((x, y, z))
    return out


def test_dda_visits_exactly_the_crossed_cells():
    rng = np.random.default_rng(7)
    for _ in range(1500):
        A = rng.uniform(-6, 6, 3)
        B = A + rng.normal(size=3) * rng.uniform(0.1, 4.0)
        cells = oracle.dda(A, B, "f64")
        assert tuple(cells[0]) == tuple(np.floor(A).astype(int))
        assert tuple(cells[-1]) == tuple(np.floor(B).astype(int))
        steps = np.abs(np.diff(cells, axis=0)).sum(1)
        assert np.all(steps == 1)  # 6-connected walk
        assert len(cells) == np.abs(np.floor(B) - np.floor(A)).sum() + 1
        assert {tuple(c) for c in cells} == _cells_brute(A, B)


def test_dda_float32_walk_stays_on_the_segment():
    rng = np.random.default_rng(8)
    for _ in range(500):
        A = rng.uniform(-50, 50, 3).astype(np.float32).astype(np.float64)
        B = (A + rng.normal(size=3) * 2).astype(np.float32).astype(np.float64)
        cells = oracle.dda(A, B, "f32")
        assert np.all(np.abs(np.diff(cells, axis=0)).sum(1) == 1)
        # every visited cell lies within 1e-4 block units of the segment
        for c in cells:
            lo, hi = c - 1e-4, c + 1 + 1e-4
            d = B - A
            with np.errstate(divide="ignore", invalid="ignore"):
                ta, tb = (lo - A) / d, (hi - A) / d
            t0 = np.max(np.where(np.abs(d) > 0, np.minimum(ta, tb), -np.inf))
            t1 = np.min(np.where(np.abs(d) > 0, np.maximum(ta, tb), np.inf))
            assert max(t0, 0) <= min(t1, 1) + 1e-9


def _plane_frames(Ds, W=64, H=48, f=50.0):
    K = (f, f, (W - 1) / 2.0, (H - 1) / 2.0)
    return [np.full((H, W), D, np.float32) for D in Ds], K


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
@pytest.mark.parametrize("posed", [False, True])
def test_fusion_closed_form_fronto_parallel_planes(prec, tol, posed):
    l, mu = 0.01, 0.04
    Ds = [1.0, 1.013, 0.987, 1.021, 0.9935]
    frames, K = _plane_frames(Ds)
    if posed:
        a = 0.4
        R = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]]) @ \
            np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
        T_wc = np.eye(4)
        T_wc[:3, :3] = R
        T_wc[:3, 3] = [0.21, -0.13, 0.37]
    else:
        T_wc = np.eye(4)
    T_cw = synth.pose_inverse_f64(T_wc)
    if prec == "f32":
        T_wc = T_wc.astype(np.float32).astype(np.float64)
        T_cw = T_cw.astype(np.float32).astype(np.float64)
    V = oracle.Volume(l, mu, prec=prec)
    for d in frames:
        V.integrate(d, K, T_wc, T_cw)
    b = V.blocks()
    loc = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1)
    loc = loc.transpose(2, 1, 0, 3).reshape(512, 3)
    g = b["keys"][:, None, :] * 8 + loc[None]
    p = (g * l).reshape(-1, 3)
    pc = p @ T_cw[:3, :3].T + T_cw[:3, 3]
    u = K[0] * pc[:, 0] / pc[:, 2] + K[2]
    v = K[1] * pc[:, 1] / pc[:, 2] + K[3]
    inside = (pc[:, 2] > 0) & (u > 1) & (u < 64 - 2) & (v > 1) & (v < 48 - 2)
    Ds = np.array(Ds, np.float32).astype(np.float64)  # the frames hold float32 depth
    sdf = Ds[None, :] - pc[:, 2:3]
    # blocks each frame collects (Eq. 1), from a float64 brute force over all pixel segments,
    # with the segment shortened and lengthened by 1e-6 block units to flag boundary cases
    bkey = (g // 8).reshape(-1, 3)
    robust = np.ones(len(p), bool)
    collected = np.zeros((len(p), len(Ds)), bool)
    for k, D in enumerate(Ds):
        sets = []
        for shrink in (1e-6, -1e-6):
            s = set()
            for vv in range(48):
                for uu in range(64):
                    ray = np.array([(uu - K[2]) / K[0], (vv - K[3]) / K[1], 1.0])
                    z0, z1 = max(D - mu, 0.05), D + mu
                    A = (T_wc[:3, :3] @ (ray * z0) + T_wc[:3, 3]) / (8 * l)
                    B = (T_wc[:3, :3] @ (ray * z1) + T_wc[:3, 3]) / (8 * l)
                    dd = (B - A) / np.linalg.norm(B - A)
                    s |= _cells_brute(A + shrink * dd, B - shrink * dd)
            sets.append(s)
        inner, outer = sets
        mem_in = np.array([tuple(b) in inner for b in map(tuple, bkey)])
        mem_out = np.array([tuple(b) in outer for b in map(tuple, bkey)])
        robust &= mem_in == mem_out
        collected[:, k] = mem_in
    seen = (sdf >= -mu) & collected
    # keep voxels whose skip decision is not within rounding of the -mu boundary
    clear = np.all(np.abs(sdf + mu) > 1e-5, axis=1)
    cnt = seen.sum(1)
    mean = np.where(cnt > 0, (np.minimum(sdf, mu) * seen).sum(1) / np.maximum(cnt, 1), 0.0)
    m = inside & clear & robust
    assert m.sum() > 5000
    got_t = b["tsdf"].reshape(-1)[m]
    got_w = b["weight"].reshape(-1)[m]
    np.testing.assert_array_equal(got_w, cnt[m])
    np.testing.assert_allclose(got_t, mean[m], rtol=0, atol=tol)
    # coverage (Eq. 1): every voxel inside the frustum within 0.9 mu of some plane is allocated
    keyset = {tuple(k) for k in b["keys"]}
    zs = np.arange(0.9, 1.1, 0.002)
    for D in Ds:
        for z in zs[np.abs(zs - D) < 0.9 * mu]:
            for (uu, vv) in ((5, 5), (32, 24), (60, 40), (10, 44)):
                xc = np.array([(uu - K[2]) / K[0] * z, (vv - K[3]) / K[1] * z, z])
                pw = T_wc[:3, :3] @ xc + T_wc[:3, 3]
                assert tuple(np.floor(pw / (8 * l)).astype(int)) in keyset


def test_voxels_behind_truncation_are_untouched():
    l, mu = 0.01, 0.04
    frames, K = _plane_frames([1.0])
    V = oracle.Volume(l, mu, prec="f64")
    V.integrate(frames[0], K, np.eye(4), np.eye(4))
    b = V.blocks()
    loc = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1)
    loc = loc.transpose(2, 1, 0, 3).reshape(512, 3)
    z = ((b["keys"][:, None, :] * 8 + loc[None]) * l)[..., 2].reshape(-1)
    w = b["weight"].reshape(-1)
    assert np.all(w[z > 1.0 + mu + 1e-9] == 0)
    assert np.all(b["tsdf"].reshape(-1)[w > 0] <= mu)


def test_sphere_sequence_block_set_float32_equals_float64():
    s = synth.sphere_scene()
    sets = {}
    for prec in ("f32", "f64"):
        V = oracle.Volume.from_config(s.volume, prec=prec)
        for k in range(s.num_frames):
            T = s.pose(k)
            Ti = synth.pose_inverse_f64(T)
            if prec == "f32":
                T, Ti = T.astype(np.float32).astype(np.float64), Ti.astype(np.float32).astype(np.float64)
            V.integrate(s.depth(k), (s.fx, s.fy, s.cx, s.cy), T, Ti)
        sets[prec] = {tuple(k) for k in V.blocks()["keys"]}
    assert len(sets["f32"] ^ sets["f64"]) <= 2
    assert len(sets["f32"]) > 1000
