"""Differentiable path on the GPU against the oracle: dL/dd of the final TSDF and dL/dD of
every leaf depth pixel, for a random linear loss (small room) and for the analytic-SDF loss
of the differentiable workload (sphere orbit, 60 frames, the last 50 depth frames as leaf
tensors).  Decisions (integrated voxels, pixels, branches, topology) are bit-identical on
both sides; the oracle takes the derivatives in float64, the kernels in float32."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import gpu_volume, intrinsics, poses32, sorted_blocks
from tests.meshutil import canonical_triangles

pytestmark = pytest.mark.gpu

LAMBDA_N = 0.1
CENTER = np.array([0.0, 0.0, 0.3])
RADIUS = 0.3


def _key_weights(keys, seed):
    """Per-vertex loss derivatives that depend only on the vertex (its edge key)."""
    k = np.asarray(keys, np.uint64)
    out = []
    for j in range(6):
        x = (k ^ np.uint64(0x9E3779B97F4A7C15 * (j + 1 + 7 * seed) & 0xFFFFFFFFFFFFFFFF)) * np.uint64(0xBF58476D1CE4E5B9)
        x ^= x >> np.uint64(29)
        out.append((x >> np.uint64(11)).astype(np.float64) / float(1 << 53) - 0.5)
    w = np.stack(out, 1)
    return w[:, :3], w[:, 3:]


def _oracle_run(scene, n_const, n_leaf):
    V = oracle.Volume.from_config(scene.volume, prec="f32")
    K = (scene.fx, scene.fy, scene.cx, scene.cy)
    for k in range(n_const + n_leaf):
        if k == n_const:
            V.diff_begin()
        Twc, Tcw = poses32(scene.pose(k))
        V.integrate(scene.depth(k), K, Twc.astype(np.float64), Tcw.astype(np.float64))
    V.update_mesh(full=True, refine=True)
    return V


def _gpu_forward(scene, n_const, n_leaf, torch):
    from paper_1803_03949_b300 import diff_mesh

    g = gpu_volume(scene.volume)
    K = intrinsics(scene)
    for k in range(n_const):
        g.integrate(torch.from_numpy(scene.depth(k)).cuda(), K, *poses32(scene.pose(k)))
    depths = [torch.from_numpy(scene.depth(k)).cuda().requires_grad_(True) for k in range(n_const, n_const + n_leaf)]
    poses = [poses32(scene.pose(k)) for k in range(n_const, n_const + n_leaf)]
    pos, nrm, tris, keys = diff_mesh(g, K, poses, depths, refine=True)
    return g, depths, pos, nrm, keys


def _compare_grad_tsdf(gb, ob, rel):
    g, o = sorted_blocks(gb), sorted_blocks(ob)
    np.testing.assert_array_equal(g["keys"], o["keys"])
    scale = np.abs(o["grad"]).max()
    assert scale > 0
    err = np.abs(g["grad"].astype(np.float64) - o["grad"]).max()
    assert err <= rel * scale, (err, scale)
    return err / scale


def test_linear_loss_gradients_match_oracle_small_room():
    """Through the C ABI directly: begin, recorded integrate calls, full refined mesh,
    dL/dd from the vertices, export, then the depth pass last call first."""
    import torch

    s = synth.small_room_scene(num_frames=8)
    n_const, n_leaf = 3, 5
    V = _oracle_run(s, n_const, n_leaf)
    om = V.mesh()
    A, B = _key_weights(om["vkeys"], 1)
    V.grad_vertices(om["vkeys"], A, B)
    og = dict(keys=V.blocks()["keys"], grad=V.grad_tsdf())
    ogd = V.grad_depth(s.W, s.H)

    g = gpu_volume(s.volume)
    K = intrinsics(s)
    frames = [(torch.from_numpy(s.depth(k)).cuda(), poses32(s.pose(k))) for k in range(n_const + n_leaf)]
    for d, P in frames[:n_const]:
        g.integrate(d, K, *P)
    g.diff_begin(n_leaf)
    for d, P in frames[n_const:]:
        g.integrate(d, K, *P)
    g.update_mesh(full=True, refine=True)
    m = g.download(device=True)
    gk = m["keys"].cpu().numpy().astype(np.uint64)
    np.testing.assert_array_equal(np.sort(gk), om["vkeys"])  # same vertices
    Ag, Bg = _key_weights(gk, 1)
    g.grad_vertices(m["keys"], torch.from_numpy(Ag).float().cuda().contiguous(),
                    torch.from_numpy(Bg).float().cuda().contiguous())
    _compare_grad_tsdf(g.export_grad(), og, 1e-4)
    gd = []
    for f in reversed(range(n_leaf)):
        d, P = frames[n_const + f]
        out = torch.empty_like(d)
        g.grad_depth(f, d, K, *P, out)
        gd.append(out.cpu().numpy())
    g.diff_end()
    g.check()
    gd = np.stack(gd[::-1]).astype(np.float64)
    scale = np.abs(ogd).max()
    assert scale > 0
    err = np.abs(gd - ogd).max()
    assert err <= 2e-4 * scale, (err, scale)
    assert np.count_nonzero(np.abs(ogd) > 1e-3 * scale) > 100


def test_diff_calls_out_of_order_are_refused():
    import torch

    from paper_1803_03949_b300 import VmeshError

    s = synth.small_room_scene(num_frames=3)
    g = gpu_volume(s.volume)
    K = intrinsics(s)
    d = [torch.from_numpy(s.depth(k)).cuda() for k in range(3)]
    g.diff_begin(2)
    g.integrate(d[0], K, *poses32(s.pose(0)))
    g.integrate(d[1], K, *poses32(s.pose(1)))
    with pytest.raises(VmeshError):
        g.integrate(d[2], K, *poses32(s.pose(2)))  # beyond max_frames
    with pytest.raises(VmeshError):
        g.gc()  # recycling while recording
    with pytest.raises(VmeshError):
        g.step(d[2], K, *poses32(s.pose(2)))
    out = torch.empty_like(d[0])
    with pytest.raises(VmeshError):
        g.grad_depth(0, d[0], K, *poses32(s.pose(0)), out)  # the last call comes first
    g.grad_depth(1, d[1], K, *poses32(s.pose(1)), out)
    g.grad_depth(0, d[0], K, *poses32(s.pose(0)), out)
    g.diff_end()
    g.gc()
    g.check()


def _sdf_loss_grads(pos, nrm):
    """The analytic loss of the differentiable workload on float64 host arrays: value and
    dL/dpos, dL/dnrm.  sdf = min(|p - c| - r, p_z) (sphere on the ground plane);
    L = mean sdf^2 + lambda * mean (1 - <n, grad sdf / |grad sdf|>)."""
    p = np.asarray(pos, np.float64)
    n = np.asarray(nrm, np.float64)
    N = len(p)
    r = p - CENTER
    dist = np.linalg.norm(r, axis=1)
    s_sph = dist - RADIUS
    sph = s_sph <= p[:, 2]
    sdf = np.where(sph, s_sph, p[:, 2])
    u = np.where(sph[:, None], r / dist[:, None], np.array([0.0, 0.0, 1.0]))
    dot = np.sum(n * u, 1)
    L = np.mean(sdf ** 2) + LAMBDA_N * np.mean(1.0 - dot)
    gpos = (2.0 / N) * sdf[:, None] * u
    # d<n, u>/dp for the sphere branch: (n - u <n, u>) / |p - c|; the plane's u is constant
    gpos -= (LAMBDA_N / N) * np.where(sph[:, None], (n - u * dot[:, None]) / dist[:, None], 0.0)
    gnrm = -(LAMBDA_N / N) * u
    return L, gpos, gnrm


def _sdf_loss_torch(pos, nrm, torch):
    c = torch.tensor(CENTER, dtype=torch.float32, device=pos.device)
    r = pos - c
    dist = torch.linalg.norm(r, dim=1)
    s_sph = dist - RADIUS
    sph = s_sph <= pos[:, 2]
    sdf = torch.where(sph, s_sph, pos[:, 2])
    up = torch.zeros_like(pos)
    up[:, 2] = 1.0
    u = torch.where(sph[:, None], r / dist[:, None], up)
    return (sdf ** 2).mean() + LAMBDA_N * (1.0 - (nrm * u).sum(1)).mean()


@pytest.fixture(scope="module")
def sphere_workload():
    """Differentiable workload: the sphere orbit extended to 60 frames, frames 0-9 constant,
    frames 10-59 leaf tensors."""
    return synth.sphere_scene(num_frames=60), 10, 50


def test_sdf_loss_gradients_match_oracle_on_sphere_orbit(sphere_workload):
    import torch

    s, n_const, n_leaf = sphere_workload
    V = _oracle_run(s, n_const, n_leaf)
    om = V.mesh()
    L_o, gp, gn = _sdf_loss_grads(om["pos"], om["nrm"])
    V.grad_vertices(om["vkeys"], gp, gn)
    ogd = V.grad_depth(s.W, s.H)

    g, depths, pos, nrm, keys = _gpu_forward(s, n_const, n_leaf, torch)
    loss = _sdf_loss_torch(pos, nrm, torch)
    assert float(loss.detach()) == pytest.approx(L_o, rel=1e-4)
    loss.backward()
    g.check()
    gd = np.stack([d.grad.cpu().numpy() for d in depths]).astype(np.float64)
    scale = np.abs(ogd).max()
    assert scale > 0
    err = np.abs(gd - ogd).max()
    assert err <= 1e-3 * scale, (err, scale)
    assert np.count_nonzero(gd) > 10000


def test_sdf_loss_gradients_match_central_differences(sphere_workload):
    """h = 1e-4 m on random leaf pixels among those with |dL/dD| >= 1% of the largest, the GPU
    forward run twice more (+h, -h); samples whose +-h runs change the mesh's vertices or
    triangles are skipped.  The loss is evaluated in float64 from float32 vertices, and the
    forward is nonlinear in D (t = d0 / (d0 - d1)), so the bar is statistical: median
    relative error below 3 %, 85 % of the samples within 10 %."""
    import torch

    from paper_1803_03949_b300 import diff_mesh

    s, n_const, n_leaf = sphere_workload
    g, depths, pos, nrm, keys = _gpu_forward(s, n_const, n_leaf, torch)
    loss = _sdf_loss_torch(pos, nrm, torch)
    loss.backward()
    g.diff_end()
    gd = np.stack([d.grad.cpu().numpy() for d in depths]).astype(np.float64)
    base = [d.detach().clone() for d in depths]
    K = intrinsics(s)
    poses = [poses32(s.pose(k)) for k in range(n_const, n_const + n_leaf)]
    const = [(torch.from_numpy(s.depth(k)).cuda(), poses32(s.pose(k))) for k in range(n_const)]

    def canon(k, t):
        kk = k.cpu().numpy().astype(np.uint64)
        return np.sort(kk), canonical_triangles(kk[t.cpu().numpy().astype(np.int64)])

    def loss_with(f, v, u, delta):
        vol = gpu_volume(s.volume)
        for d, P in const:
            vol.integrate(d, K, *P)
        ds = [b.clone() for b in base]
        ds[f][v, u] += delta
        with torch.no_grad():
            p, n, t, k = diff_mesh(vol, K, poses, ds, refine=True)
            val = float(_sdf_loss_torch(p.double(), n.double(), torch))
        vol.diff_end()
        mesh = canon(k, t)
        vol.close()
        return val, mesh, float(ds[f][v, u] - base[f][v, u])

    ref = loss_with(0, 0, 0, 0.0)[1]
    cand = np.flatnonzero(np.abs(gd).ravel() >= 1e-2 * np.abs(gd).max())
    rng = np.random.default_rng(17)
    rel = []
    for idx in rng.choice(cand, size=min(60, len(cand)), replace=False):
        f, v, u = np.unravel_index(idx, gd.shape)
        lp, mp, hp = loss_with(f, v, u, 1e-4)
        lm, mm, hm = loss_with(f, v, u, -1e-4)
        if not all(np.array_equal(a, b) for a, b in zip(mp + mm, ref + ref)):
            continue
        fd = (lp - lm) / (hp - hm)
        rel.append(abs(fd - gd[f, v, u]) / abs(gd[f, v, u]))
    rel = np.array(rel)
    assert len(rel) >= 20
    assert np.median(rel) < 0.03, np.sort(rel)
    assert np.mean(rel < 0.1) >= 0.85, np.sort(rel)
