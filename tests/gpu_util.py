"""Runners shared by the GPU tests: the same seeded frames through the oracle and the CUDA path.

Poses are rounded to float32 once (T_cw is inverted in float64 first); both sides receive
those identical float32 values, the oracle as exactly representable doubles.
"""
from __future__ import annotations

import numpy as np

import oracle
import synth
from tests.meshutil import canonical_triangles


def poses32(T_wc):
    T = np.asarray(T_wc, np.float64)
    Ti = synth.pose_inverse_f64(T)
    return T.astype(np.float32), Ti.astype(np.float32)


def gpu_volume(vc, **kw):
    from paper_1803_03949_b300 import Volume

    return Volume.from_config(vc, **kw)


def intrinsics(scene):
    from paper_1803_03949_b300 import Intrinsics

    return Intrinsics(scene.W, scene.H, scene.fx, scene.fy, scene.cx, scene.cy)


def run_frames(scene, frames, gpu=None, orc=None, refine=True, gc=True, mode="calls", separate_refine=False,
               depth_fn=None, after_frame=None):
    """Feed frames to a GPU volume and/or an oracle volume with the same per-frame calls.
    mode: 'calls' (integrate / update / refine / gc), 'step' (vm_step), 'graph' (vm_step + CUDA graph)."""
    import torch

    K = intrinsics(scene) if gpu is not None else None
    for k in frames:
        d = scene.depth(k) if depth_fn is None else depth_fn(k)
        Twc, Tcw = poses32(scene.pose(k))
        if gpu is not None:
            dt = torch.from_numpy(d).cuda()
            if mode == "calls":
                gpu.integrate(dt, K, Twc, Tcw)
                gpu.update_mesh(refine=refine and not separate_refine)
                if refine and separate_refine:
                    gpu.refine_mesh()
                if gc:
                    gpu.gc()
            else:
                gpu.step(dt, K, Twc, Tcw, refine=refine, gc=gc, graph=(mode == "graph"))
        if orc is not None:
            orc.integrate(d, (scene.fx, scene.fy, scene.cx, scene.cy), Twc.astype(np.float64),
                          Tcw.astype(np.float64))
            orc.update_mesh(refine=refine and not separate_refine)
            if refine and separate_refine:
                orc.refine_mesh()
            if gc:
                orc.gc()
        if after_frame is not None:
            after_frame(k)


def sorted_blocks(b):
    keys = np.asarray(b["keys"])
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    return {k: np.asarray(v)[order] for k, v in b.items()}


def compare_blocks(gb, ob, tol=1e-5):
    """Block set bit-exact; TSDF and weight within tol; cube types exact.  Returns stats."""
    g, o = sorted_blocks(gb), sorted_blocks(ob)
    assert g["keys"].shape == o["keys"].shape, (g["keys"].shape, o["keys"].shape)
    np.testing.assert_array_equal(g["keys"], o["keys"])
    dt = np.abs(g["tsdf"].astype(np.float64) - o["tsdf"])
    dw = np.abs(g["weight"].astype(np.float64) - o["weight"])
    assert dt.max(initial=0) <= tol, dt.max()
    assert dw.max(initial=0) <= tol, dw.max()
    np.testing.assert_array_equal(g["code_eff"], o["code_eff"])
    np.testing.assert_array_equal(g["code_prev"], o["code_prev"])
    return dict(blocks=len(g["keys"]), tsdf_max_abs=float(dt.max(initial=0)), weight_max_abs=float(dw.max(initial=0)),
                tsdf_bit_exact=bool(np.array_equal(g["tsdf"].astype(np.float64), o["tsdf"])))


def gpu_mesh_canonical(m):
    keys = np.asarray(m["keys"]).astype(np.uint64)
    tris = np.asarray(m["tris"])
    return keys, canonical_triangles(keys[tris.reshape(-1)].reshape(-1, 3) if len(tris) else np.zeros((0, 3), np.uint64))


def compare_mesh(gm, om, voxel, pos_tol_frac=1e-5, nrm_tol=1e-5):
    """Canonical topology bit-exact; positions within pos_tol_frac * voxel; normals within nrm_tol;
    refcount == degree; no duplicate vertex.  Returns stats."""
    keys, gt = gpu_mesh_canonical(gm)
    assert len(np.unique(keys)) == len(keys), "duplicate vertices"
    ot = canonical_triangles(om["tkeys"])
    assert gt.shape == ot.shape, (gt.shape, ot.shape)
    np.testing.assert_array_equal(gt, ot)
    order = np.argsort(keys)
    np.testing.assert_array_equal(keys[order], om["vkeys"])
    pos = np.asarray(gm["pos"], np.float64)[order]
    nrm = np.asarray(gm["nrm"], np.float64)[order]
    dp = np.abs(pos - om["pos"]).max(initial=0)
    dn = np.abs(nrm - om["nrm"]).max(initial=0)
    assert dp <= pos_tol_frac * voxel, dp
    assert dn <= nrm_tol, dn
    tris = np.asarray(gm["tris"])
    deg = np.bincount(tris.reshape(-1), minlength=len(keys))
    np.testing.assert_array_equal(np.asarray(gm["refcount"]), deg)
    return dict(vertices=len(keys), triangles=len(gt), pos_max_abs=float(dp), nrm_max_abs=float(dn))
