"""TEST INFRASTRUCTURE ONLY: ctypes wrapper of the plain single-threaded CPU oracle.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The product path (``paper_1803_03949_b300``) never does, and the
two share no code.  ``vmesh_oracle.c`` is compiled twice with gcc:

* ``liboracle_f32.so`` (``OR_REAL=float``) -- the parity build: the float32 operation
  order the method's integer decisions (block set, cube types, refinement) are taken in;
* ``liboracle_f64.so`` (``OR_REAL=double``) -- the same steps in float64, for stating the
  float32 error.

Function-level citations are in the C source header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vmesh_oracle.c")
_LIBS = {"f32": os.path.join(_HERE, "liboracle_f32.so"), "f64": os.path.join(_HERE, "liboracle_f64.so")}
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> None:
    """Compile both oracle builds with gcc (no contraction, IEEE arithmetic)."""
    for prec, path in _LIBS.items():
        real = "float" if prec == "f32" else "double"
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            tmp = path + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", *_CFLAGS, "-DOR_REAL=" + real, "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, path)


_loaded: dict = {}


def _lib(prec: str):
    if prec not in _loaded:
        build()
        lib = ctypes.CDLL(_LIBS[prec])
        vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        P = ctypes.POINTER
        lib.or_create.restype = vp
        lib.or_create.argtypes = [d, d, d, d]
        lib.or_destroy.argtypes = [vp]
        lib.or_table_ok.restype = i
        lib.or_mc_table.argtypes = [P(i), P(i)]
        lib.or_dda.restype = i
        lib.or_dda.argtypes = [P(d), P(d), P(i), i]
        lib.or_integrate.argtypes = [vp, P(ctypes.c_float), i, i, P(d), P(d), P(d)]
        lib.or_update_mesh.argtypes = [vp, i, i]
        lib.or_refine_mesh.argtypes = [vp, i]
        lib.or_gc.argtypes = [vp]
        lib.or_refine_code.restype = i
        lib.or_refine_code.argtypes = [i, i, P(d), d]
        lib.or_set_blocks.argtypes = [vp, P(i), i, P(d), P(d)]
        lib.or_num_blocks.argtypes = [vp]
        lib.or_export_blocks.argtypes = [vp, P(i), P(d), P(d), P(ctypes.c_uint8), P(ctypes.c_uint8)]
        lib.or_stats.argtypes = [vp, P(i64)]
        lib.or_mesh_build.restype = i64
        lib.or_mesh_build.argtypes = [vp, P(i64)]
        lib.or_mesh_fetch.argtypes = [vp, P(ctypes.c_uint64), P(d), P(d), P(ctypes.c_uint64)]
        lib.or_diff_begin.argtypes = [vp]
        lib.or_diff_end.argtypes = [vp]
        lib.or_diff_frames.restype = i
        lib.or_diff_frames.argtypes = [vp]
        lib.or_grad_vertices.argtypes = [vp, i64, P(ctypes.c_uint64), P(d), P(d)]
        lib.or_grad_export.argtypes = [vp, P(d)]
        lib.or_grad_depth.argtypes = [vp, i, i, P(d)]
        lib.or_mesh_memory.argtypes = [vp, P(i64)]
        lib.or_set_voxel.restype = i
        lib.or_set_voxel.argtypes = [vp, i, i, i, d]
        _loaded[prec] = lib
    return _loaded[prec]


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def mc_table(prec: str = "f64"):
    """The oracle's marching-cubes table: (ntri[256], tris[256, 5, 3] edge ids, -1 padded)."""
    lib = _lib(prec)
    n = np.zeros(256, np.int32)
    t = np.zeros((256, 5, 3), np.int32)
    lib.or_mc_table(_ptr(n, ctypes.c_int), _ptr(t, ctypes.c_int))
    return n, t


def table_ok(prec: str = "f64") -> bool:
    return bool(_lib(prec).or_table_ok())


def dda(A, B, prec: str = "f64") -> np.ndarray:
    """Block-grid cells visited from A to B (block units), shape (n, 3)."""
    lib = _lib(prec)
    a = np.ascontiguousarray(A, np.float64)
    b = np.ascontiguousarray(B, np.float64)
    n = lib.or_dda(_ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double), None, 0)
    out = np.zeros((n, 3), np.int32)
    lib.or_dda(_ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double), _ptr(out, ctypes.c_int), n)
    return out


def refine_code(raw: int, prev: int, d8, eps: float, prec: str = "f64") -> int:
    """Eqs. 3-5 for one cube."""
    d = np.ascontiguousarray(d8, np.float64)
    return _lib(prec).or_refine_code(int(raw), int(prev), _ptr(d, ctypes.c_double), float(eps))


class Volume:
    """The oracle's volume: same operations as the C-ABI, plain single-threaded C."""

    def __init__(self, voxel_size, trunc, eps_refine=None, w_max=255.0, prec: str = "f32"):
        self.prec = prec
        self._lib = _lib(prec)
        if eps_refine is None:
            eps_refine = 0.2 * voxel_size
        self.voxel_size = voxel_size
        self._h = self._lib.or_create(voxel_size, trunc, eps_refine, w_max)

    @classmethod
    def from_config(cls, vc, prec: str = "f32"):
        return cls(vc.voxel_size, vc.trunc, vc.eps_refine, vc.w_max, prec=prec)

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._lib.or_destroy(h)

    def integrate(self, depth: np.ndarray, intr, T_wc: np.ndarray, T_cw: np.ndarray) -> None:
        """intr = (fx, fy, cx, cy); poses row-major 4x4 (float64; the float32 build rounds them)."""
        d = np.ascontiguousarray(depth, np.float32)
        H, W = d.shape
        k = np.ascontiguousarray(intr, np.float64)
        a = np.ascontiguousarray(T_wc, np.float64).reshape(16)
        b = np.ascontiguousarray(T_cw, np.float64).reshape(16)
        self._lib.or_integrate(self._h, _ptr(d, ctypes.c_float), W, H, _ptr(k, ctypes.c_double),
                               _ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double))

    def update_mesh(self, full: bool = False, refine: bool = False) -> None:
        self._lib.or_update_mesh(self._h, int(full), int(refine))

    def refine_mesh(self, full: bool = False) -> None:
        self._lib.or_refine_mesh(self._h, int(full))

    def gc(self) -> int:
        return self._lib.or_gc(self._h)

    def set_blocks(self, keys: np.ndarray, tsdf: np.ndarray, weight: np.ndarray) -> None:
        k = np.ascontiguousarray(keys, np.int32).reshape(-1, 3)
        t = np.ascontiguousarray(tsdf, np.float64).reshape(-1, 512)
        w = np.ascontiguousarray(weight, np.float64).reshape(-1, 512)
        self._lib.or_set_blocks(self._h, _ptr(k, ctypes.c_int), k.shape[0], _ptr(t, ctypes.c_double),
                                _ptr(w, ctypes.c_double))

    def num_blocks(self) -> int:
        return self._lib.or_num_blocks(self._h)

    def blocks(self):
        """dict(keys (n,3) int32, tsdf/weight (n,512) float64, code_eff/code_prev (n,512) uint8)."""
        n = self.num_blocks()
        keys = np.zeros((n, 3), np.int32)
        tsdf = np.zeros((n, 512), np.float64)
        weight = np.zeros((n, 512), np.float64)
        ce = np.zeros((n, 512), np.uint8)
        cp = np.zeros((n, 512), np.uint8)
        self._lib.or_export_blocks(self._h, _ptr(keys, ctypes.c_int), _ptr(tsdf, ctypes.c_double),
                                   _ptr(weight, ctypes.c_double), _ptr(ce, ctypes.c_uint8),
                                   _ptr(cp, ctypes.c_uint8))
        return dict(keys=keys, tsdf=tsdf, weight=weight, code_eff=ce, code_prev=cp)

    def stats(self):
        out = np.zeros(6, np.int64)
        self._lib.or_stats(self._h, _ptr(out, ctypes.c_int64))
        return dict(cells=int(out[0]), voxels_integrated=int(out[1]), frame_blocks=int(out[2]),
                    update_blocks=int(out[3]), epoch=int(out[4]), truncated=int(out[5]))

    def mesh_memory(self) -> dict:
        """dict(vertices, block_vertices, loose_vertices, triangles) of the current mesh."""
        out = np.zeros(4, np.int64)
        self._lib.or_mesh_memory(self._h, _ptr(out, ctypes.c_int64))
        return dict(vertices=int(out[0]), block_vertices=int(out[1]), loose_vertices=int(out[2]),
                    triangles=int(out[3]))

    # ------------------------------------------------------------ differentiable path
    def diff_begin(self) -> None:
        """Record every integration from now on (and clear dL/dd); no gc until the gradients are taken."""
        self._lib.or_diff_begin(self._h)

    def diff_end(self) -> None:
        self._lib.or_diff_end(self._h)

    def grad_vertices(self, keys, gpos, gnrm) -> None:
        """Add the TSDF gradients of vertices `keys` (edge keys) given dL/dpos, dL/dnrm (n, 3)."""
        k = np.ascontiguousarray(keys, np.uint64)
        a = np.ascontiguousarray(gpos, np.float64).reshape(-1, 3)
        b = np.ascontiguousarray(gnrm, np.float64).reshape(-1, 3)
        self._lib.or_grad_vertices(self._h, k.shape[0], _ptr(k, ctypes.c_uint64), _ptr(a, ctypes.c_double),
                                   _ptr(b, ctypes.c_double))

    def grad_tsdf(self) -> np.ndarray:
        """dL/dd per voxel, (n_blocks, 512), rows in the order of blocks()['keys']."""
        out = np.zeros((self.num_blocks(), 512), np.float64)
        self._lib.or_grad_export(self._h, _ptr(out, ctypes.c_double))
        return out

    def grad_depth(self, W: int, H: int) -> np.ndarray:
        """dL/dD of every recorded frame, (frames, H, W); consumes dL/dd."""
        out = np.zeros((self._lib.or_diff_frames(self._h), H, W), np.float64)
        self._lib.or_grad_depth(self._h, W, H, _ptr(out, ctypes.c_double))
        return out

    def set_voxel(self, g, d: float) -> bool:
        return bool(self._lib.or_set_voxel(self._h, int(g[0]), int(g[1]), int(g[2]), float(d)))

    def mesh(self):
        """dict(vkeys (nv,) uint64 sorted, pos/nrm (nv,3) float64, tkeys (nt,3) uint64)."""
        nt = ctypes.c_int64()
        nv = self._lib.or_mesh_build(self._h, ctypes.byref(nt))
        nt = nt.value
        vkeys = np.zeros(nv, np.uint64)
        pos = np.zeros((nv, 3), np.float64)
        nrm = np.zeros((nv, 3), np.float64)
        tkeys = np.zeros((nt, 3), np.uint64)
        self._lib.or_mesh_fetch(self._h, _ptr(vkeys, ctypes.c_uint64), _ptr(pos, ctypes.c_double),
                                _ptr(nrm, ctypes.c_double), _ptr(tkeys, ctypes.c_uint64))
        return dict(vkeys=vkeys, pos=pos, nrm=nrm, tkeys=tkeys)
