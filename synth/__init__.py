"""Seeded synthetic depth sequences (the inputs shared by the CPU oracle and the CUDA path).

Nothing here computes any part of the meshing method: the module ray-casts analytic
scenes into noisy float32 depth frames and hands out camera poses, plus the exact
scene SDF used by geometric tests.  The scenes stand in for the RGB-D sequences the
paper evaluates on (Sec. VI: ICL-NUIM, TUM, Zhou-Koltun), which are not available;
only their shape is reproduced (640x480 float depth, Kinect-like intrinsics,
handheld trajectories, depth-dependent noise, dropped pixels).

The C source (``synth.c``) is compiled with gcc into ``libsynth.so`` next to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")

SEED_BASE = 180303949  # workload k uses seed SEED_BASE + k


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libsynth.so`` (gcc, OpenMP) if missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i, d, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        P = ctypes.POINTER
        lib.synth_create_sphere.restype = vp
        lib.synth_create_sphere.argtypes = [u64, i, i, i, d, d, d, d, d]
        lib.synth_create_room.restype = vp
        lib.synth_create_room.argtypes = [u64, i, i, i, d, d, d, d, d, d, d, i, d, d]
        lib.synth_create_floor.restype = vp
        lib.synth_create_floor.argtypes = [u64, i, i, i, d, d, d, d, i, d, d, d]
        lib.synth_destroy.argtypes = [vp]
        lib.synth_num_frames.argtypes = [vp]
        lib.synth_num_prims.argtypes = [vp]
        lib.synth_camera.argtypes = [vp, P(i), P(i), P(d)]
        lib.synth_bounds.argtypes = [vp, P(d), P(d)]
        lib.synth_pose.argtypes = [vp, i, P(d)]
        lib.synth_render.argtypes = [vp, i, P(ctypes.c_float)]
        lib.synth_sdf.argtypes = [vp, P(d), i, P(d), P(d)]
        _lib = lib
    return _lib


@dataclass(frozen=True)
class VolumeConfig:
    """Parameters of the volume a workload is fused into (method parameters, no arithmetic)."""

    voxel_size: float  # cube side l, metres
    trunc: float  # truncation distance mu, metres
    hash_buckets: int  # power of two
    max_blocks: int
    max_vertices: int
    max_triangles: int
    eps_refine_frac: float = 0.2  # epsilon of Eq. 5 as a fraction of l
    w_max: float = 255.0
    compact_edges: bool = False  # the compact cube record (one edge-record index per voxel)

    @property
    def eps_refine(self) -> float:
        return self.eps_refine_frac * self.voxel_size


class Scene:
    """A seeded synthetic scene with a camera trajectory; frames render on demand."""

    def __init__(self, handle, lib, name: str, volume: VolumeConfig):
        self._h = handle
        self._lib = lib
        self.name = name
        self.volume = volume
        W, H = ctypes.c_int(), ctypes.c_int()
        intr = (ctypes.c_double * 4)()
        lib.synth_camera(handle, ctypes.byref(W), ctypes.byref(H), intr)
        self.W, self.H = W.value, H.value
        self.fx, self.fy, self.cx, self.cy = list(intr)
        self.num_frames = lib.synth_num_frames(handle)
        self.max_range = None  # depth beyond this (metres) reads as invalid, like a sensor's range

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None and self._lib is not None:
            self._lib.synth_destroy(h)

    @property
    def intrinsics(self):
        return (self.W, self.H, self.fx, self.fy, self.cx, self.cy)

    def bounds(self):
        lo, hi = (ctypes.c_double * 3)(), (ctypes.c_double * 3)()
        self._lib.synth_bounds(self._h, lo, hi)
        return np.array(lo[:]), np.array(hi[:])

    def pose(self, k: int) -> np.ndarray:
        """Camera-to-world pose T_wc of frame k, float64 4x4."""
        T = np.zeros(16, np.float64)
        if self._lib.synth_pose(self._h, int(k), T.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) != 0:
            raise IndexError(k)
        return T.reshape(4, 4)

    def depth(self, k: int) -> np.ndarray:
        """Noisy float32 depth frame k, shape (H, W), 0 = invalid."""
        out = np.zeros((self.H, self.W), np.float32)
        if self._lib.synth_render(self._h, int(k), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))) != 0:
            raise IndexError(k)
        if self.max_range is not None:
            out[out > self.max_range] = 0.0
        return out

    def sdf(self, pts: np.ndarray, with_grad: bool = False):
        """Exact scene SDF (union of primitives) at points (n, 3), optionally its gradient."""
        p = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        n = p.shape[0]
        s = np.zeros(n, np.float64)
        g = np.zeros((n, 3), np.float64) if with_grad else None
        P = ctypes.POINTER(ctypes.c_double)
        self._lib.synth_sdf(self._h, p.ctypes.data_as(P), n, s.ctypes.data_as(P),
                            g.ctypes.data_as(P) if with_grad else None)
        return (s, g) if with_grad else s


def pose_inverse_f64(T_wc: np.ndarray) -> np.ndarray:
    """World-to-camera pose, inverted in float64 ([R^T | -R^T t])."""
    T = np.asarray(T_wc, np.float64).reshape(4, 4)
    R, t = T[:3, :3], T[:3, 3]
    out = np.eye(4)
    out[:3, :3] = R.T
    out[:3, 3] = -R.T @ t
    return out


# ------------------------------------------------------------------ workload recipes

def sphere_scene(num_frames: int = 10, seed: int = SEED_BASE + 1, noise_sigma: float = 0.001) -> Scene:
    """Analytic sphere (r = 0.3 m) on a ground square, 320x240 (fx = fy = 290), orbit at 1.2 m,
    sigma = 1 mm; voxel 1 cm, 8^3 blocks, truncation 4 cm, 2^16 hash buckets."""
    lib = _load()
    h = lib.synth_create_sphere(seed, num_frames, 320, 240, 290.0, 290.0, 160.0, 120.0, noise_sigma)
    vol = VolumeConfig(voxel_size=0.01, trunc=0.04, hash_buckets=1 << 16, max_blocks=1 << 14,
                       max_vertices=1 << 20, max_triangles=1 << 21)
    return Scene(h, lib, "sphere_320x240_l1cm", vol)


def room_scene(num_frames: int = 300, seed: int = SEED_BASE + 2, W: int = 640, H: int = 480) -> Scene:
    """6x4x3 m room with 20 random primitives, 640x480 (fx = fy = 525), smooth random walk,
    noise sigma = 0.0012 z^2 and 2% dropped pixels; voxel 8 mm, truncation 3.2 cm, 2^20 buckets."""
    lib = _load()
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    h = lib.synth_create_room(seed, num_frames, W, H, 525.0, 525.0, cx, cy, 6.0, 4.0, 3.0, 20, 0.0012, 0.02)
    vol = VolumeConfig(voxel_size=0.008, trunc=0.032, hash_buckets=1 << 20, max_blocks=1 << 18,
                       max_vertices=1 << 23, max_triangles=1 << 24)
    return Scene(h, lib, "room_6x4x3_640x480_l8mm", vol)


def floor_scene(num_frames: int = 2000, seed: int = SEED_BASE + 3) -> Scene:
    """20x20x4 m floor of 4x4 rooms with doorways and 8 primitives per room, 640x480, a
    serpentine path through the doorways that covers the floor in `num_frames` frames,
    same noise model with a 4.5 m sensor range (farther depth reads as invalid: at the noise
    model's sigma = 0.0012 z^2 a 10 m reading is off by 12 cm, six truncation widths);
    voxel 5 mm, truncation 2 cm, 2^23 buckets."""
    lib = _load()
    h = lib.synth_create_floor(seed, num_frames, 640, 480, 525.0, 525.0, 319.5, 239.5, 8, 0.0012, 0.02, 8.0)
    vol = VolumeConfig(voxel_size=0.005, trunc=0.02, hash_buckets=1 << 23, max_blocks=1 << 21,
                       max_vertices=1 << 26, max_triangles=1 << 27)
    sc = Scene(h, lib, "floor_20x20x4_640x480_l5mm", vol)
    sc.max_range = 4.5
    return sc


def batch_scenes(num_scenes: int = 32, num_frames: int = 100, seed: int = SEED_BASE + 5,
                 scale_range=(1.0, 3.5), voxel_mm=(5, 10), height: float = 3.0, pool_shift: int = 0) -> list:
    """Independent scenes of uneven sizes for the batched workload: the room recipe with its
    6 x 4 m floor plan scaled by a log-uniform factor in `scale_range` (default [1, 3.5]; height
    3 m, 20 primitives), voxel l drawn from {voxel_mm[0], ..., voxel_mm[1]} mm (default 5-10),
    truncation 4 l, 640 x 480 depth with the room noise model and a 4.5 m sensor range (farther
    depth reads as invalid, as on a structured-light camera); each scene has its own seed and
    trajectory.  Pools: 2^18 blocks at l <= 6 mm, 2^17 at <= 8 mm, else 2^16, times 2^pool_shift."""
    lib = _load()
    rng = np.random.default_rng(seed)
    out = []
    for i in range(num_scenes):
        scale = float(np.exp(rng.uniform(np.log(scale_range[0]), np.log(scale_range[1]))))
        l = int(rng.integers(voxel_mm[0], voxel_mm[1] + 1)) * 1e-3
        sx, sy = 6.0 * scale, 4.0 * scale
        nprims = 20
        h = lib.synth_create_room(seed + 1000 * (i + 1), num_frames, 640, 480, 525.0, 525.0, 319.5, 239.5, sx, sy,
                                  height, nprims, 0.0012, 0.02)
        mb = (1 << 18 if l <= 0.006 else (1 << 17 if l <= 0.008 else 1 << 16)) << pool_shift
        vol = VolumeConfig(voxel_size=l, trunc=4 * l, hash_buckets=4 * mb, max_blocks=mb, max_vertices=64 * mb,
                           max_triangles=128 * mb)
        sc = Scene(h, lib, "room_%.1fx%.1fx%g_640x480_l%dmm" % (sx, sy, height, round(l * 1000)), vol)
        sc.max_range = 4.5
        out.append(sc)
    return out


def small_room_scene(num_frames: int = 8, seed: int = SEED_BASE + 12, W: int = 96, H: int = 72) -> Scene:
    """A small room at reduced resolution: the room recipe at a size the oracle runs in
    well under a second per frame (used for parity cases that span many frames)."""
    lib = _load()
    fx = 525.0 * W / 640.0
    h = lib.synth_create_room(seed, num_frames, W, H, fx, fx, (W - 1) / 2.0, (H - 1) / 2.0, 4.0, 3.0, 2.5,
                              8, 0.0012, 0.02)
    vol = VolumeConfig(voxel_size=0.02, trunc=0.08, hash_buckets=1 << 14, max_blocks=1 << 13,
                       max_vertices=1 << 20, max_triangles=1 << 21)
    return Scene(h, lib, "small_room_%dx%d_l2cm" % (W, H), vol)
