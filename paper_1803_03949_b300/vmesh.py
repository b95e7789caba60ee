"""Python binding of the vmesh C ABI (``include/vmesh.h``): argument marshalling only.

Every step of the per-frame path runs in the CUDA library ``libvmesh.so``; PyTorch only
provides device memory (depth frames, download buffers) and the stream.  There is no
CPU fallback: without the built library, or without a CUDA device, construction fails.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvmesh.so")

VM_FULL, VM_REFINE, VM_GC = 1, 2, 4
VM_PARAM_COMPACT_EDGES = 1
STATUS = {0: "VM_OK", 1: "VM_ERR_INVALID_ARG", 2: "VM_ERR_HASH_FULL", 3: "VM_ERR_POOL_FULL", 4: "VM_ERR_CUDA",
          5: "VM_ERR_OOM"}


class VmeshError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__("%s failed: %s" % (where, STATUS.get(code, code)))
        self.code = code


class vm_params(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_float), ("trunc", ctypes.c_float), ("eps_refine", ctypes.c_float),
                ("w_max", ctypes.c_float), ("hash_buckets", ctypes.c_uint32), ("max_blocks", ctypes.c_uint32),
                ("max_vertices", ctypes.c_uint32), ("max_triangles", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class vm_intrinsics(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class vm_frame_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "frame_blocks", "new_blocks", "update_blocks", "changed_cubes", "live_blocks", "live_vertices",
        "live_triangles", "freed_blocks", "freed_vertices", "created_vertices", "hash_tombstones",
        "block_high_water", "rehashes", "emitted_triangles", "released_triangles", "refreshed_vertices",
        "collected_blocks", "meshed_blocks", "full_pool", "vertex_high_water", "triangle_high_water", "reference_updates")]

POOLS = ["none", "blocks", "vertices", "triangles", "collected_list", "update_list", "dead_vertex_list", "dead_run_list",
         "free_stack", "hash", "edge_records"]


class vm_mesh_memory(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "vertices", "triangles", "block_vertices", "loose_vertices", "blocks", "cube_bytes", "edge_records",
        "bytes_in_use", "bytes_allocated")]


_lib = None

EXPORTS = ["vm_create_volume", "vm_destroy_volume", "vm_set_stream", "vm_integrate_depth", "vm_update_mesh",
           "vm_refine_mesh", "vm_gc", "vm_step", "vm_mesh_counts", "vm_download_mesh", "vm_get_stats",
           "vm_last_error", "vm_num_blocks", "vm_export_blocks", "vm_set_blocks", "vm_enable_timing",
           "vm_kernel_times", "vm_mesh_size_async", "vm_download_mesh_noalloc", "vm_download_mesh_into", "vm_diff_begin",
           "vm_diff_end",
           "vm_grad_vertices", "vm_grad_depth", "vm_export_grad", "vm_batch_create", "vm_batch_destroy",
           "vm_batch_step", "vm_batch_tune", "vm_batch_schedule", "vm_batch_set_schedule", "vm_batch_profile",
           "vm_batch_kernel_ms", "vm_mesh_memory_stats"]


def load_library(path: str = LIB_PATH):
    """Load ``libvmesh.so`` and declare its signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("vmesh CUDA library not built: %s (run paper_1803_03949_b300/build.py)" % path)
    lib = ctypes.CDLL(path)
    vp, i, i64, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
    P = ctypes.POINTER
    F16 = P(f)
    sig = {
        "vm_create_volume": [P(vm_params), vp, P(vp)],
        "vm_destroy_volume": [vp],
        "vm_set_stream": [vp, vp],
        "vm_integrate_depth": [vp, vp, P(vm_intrinsics), F16, F16],
        "vm_update_mesh": [vp, i],
        "vm_refine_mesh": [vp, i],
        "vm_gc": [vp],
        "vm_step": [vp, vp, P(vm_intrinsics), F16, F16, i, i],
        "vm_mesh_counts": [vp, P(i64), P(i64)],
        "vm_download_mesh": [vp, vp, vp, vp, vp, vp, i],
        "vm_get_stats": [vp, P(vm_frame_stats)],
        "vm_last_error": [vp],
        "vm_num_blocks": [vp, P(i64)],
        "vm_export_blocks": [vp, vp, vp, vp, vp, vp],
        "vm_set_blocks": [vp, vp, i64, vp, vp],
        "vm_enable_timing": [vp, i],
        "vm_kernel_times": [vp, P(ctypes.c_char_p), P(ctypes.c_double), P(i64), i, P(i)],
        "vm_mesh_size_async": [vp, vp, i],
        "vm_download_mesh_noalloc": [vp, vp, vp, vp, vp, vp, i64, i64, P(i64), P(i64)],
        "vm_download_mesh_into": [vp, vp, vp, vp, vp, vp, i64, i64, P(i64), P(i64)],
        "vm_diff_begin": [vp, i],
        "vm_diff_end": [vp],
        "vm_grad_vertices": [vp, i64, vp, vp, vp],
        "vm_grad_depth": [vp, i, vp, P(vm_intrinsics), F16, F16, vp],
        "vm_export_grad": [vp, vp, vp],
        "vm_batch_create": [P(vp), i, P(vp)],
        "vm_batch_destroy": [vp],
        "vm_batch_step": [vp, P(vp), P(vm_intrinsics), P(f), P(f), i, i],
        "vm_batch_tune": [vp, i],
        "vm_batch_schedule": [vp, P(i), P(ctypes.c_double)],
        "vm_batch_set_schedule": [vp, P(i)],
        "vm_batch_profile": [vp, i],
        "vm_mesh_memory_stats": [vp, P(vm_mesh_memory)],
        "vm_batch_kernel_ms": [vp, P(ctypes.c_double), P(i)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != 0:
        raise VmeshError(code, where)


def _f16(T) -> ctypes.Array:
    a = np.ascontiguousarray(np.asarray(T, np.float32).reshape(16))
    return (ctypes.c_float * 16)(*a.tolist())


def _contig_cuda(*ts):
    for t in ts:
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("expected contiguous CUDA tensors")


def _ptr(x) -> int:
    """Data pointer of a torch tensor or numpy array (None -> 0)."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


@dataclass
class Intrinsics:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float

    def c(self) -> vm_intrinsics:
        return vm_intrinsics(self.width, self.height, self.fx, self.fy, self.cx, self.cy)


class Volume:
    """A spatially hashed TSDF volume with its incrementally maintained mesh (one GPU)."""

    def __init__(self, voxel_size, trunc, hash_buckets, max_blocks, max_vertices, max_triangles,
                 eps_refine=None, w_max=255.0, stream=None, compact_edges=False):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("vmesh needs a CUDA device; no CPU fallback exists")
        self._lib = load_library()
        if eps_refine is None:
            eps_refine = 0.2 * voxel_size
        self.params = vm_params(voxel_size, trunc, eps_refine, w_max, hash_buckets, max_blocks, max_vertices,
                                max_triangles, VM_PARAM_COMPACT_EDGES if compact_edges else 0)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(self._lib.vm_create_volume(ctypes.byref(self.params), ctypes.c_void_p(self.stream.cuda_stream),
                                          ctypes.byref(h)), "vm_create_volume")
        self._h = h

    @classmethod
    def from_config(cls, vc, **kw):
        kw.setdefault("compact_edges", getattr(vc, "compact_edges", False))
        return cls(vc.voxel_size, vc.trunc, vc.hash_buckets, vc.max_blocks, vc.max_vertices, vc.max_triangles,
                   eps_refine=vc.eps_refine, w_max=vc.w_max, **kw)

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None and h.value:
            self._lib.vm_destroy_volume(h)

    def __del__(self):
        self.close()

    # --------------------------------------------------------------- per-frame path
    def integrate(self, depth, intr: Intrinsics, T_wc, T_cw):
        """depth: float32 tensor (H, W), CUDA or pinned CPU (read across the host link by the
        collection kernel); poses 4x4 (host, rounded to float32)."""
        _check(self._lib.vm_integrate_depth(self._h, ctypes.c_void_p(_ptr(depth)), ctypes.byref(intr.c()),
                                            _f16(T_wc), _f16(T_cw)), "vm_integrate_depth")

    def update_mesh(self, full=False, refine=False):
        _check(self._lib.vm_update_mesh(self._h, (VM_FULL if full else 0) | (VM_REFINE if refine else 0)),
               "vm_update_mesh")

    def refine_mesh(self, full=False):
        _check(self._lib.vm_refine_mesh(self._h, int(bool(full))), "vm_refine_mesh")

    def gc(self):
        _check(self._lib.vm_gc(self._h), "vm_gc")

    def step(self, depth, intr: Intrinsics, T_wc, T_cw, refine=True, gc=True, full=False, graph=False):
        flags = (VM_FULL if full else 0) | (VM_REFINE if refine else 0) | (VM_GC if gc else 0)
        _check(self._lib.vm_step(self._h, ctypes.c_void_p(_ptr(depth)), ctypes.byref(intr.c()), _f16(T_wc),
                                 _f16(T_cw), flags, int(bool(graph))), "vm_step")

    # --------------------------------------------------------------- queries
    def last_error(self) -> int:
        return self._lib.vm_last_error(self._h)

    def check(self):
        code = self.last_error()
        if code != 0:
            pool = self.stats()["full_pool"]
            _check(code, "device status" + (" (%s exhausted)" % POOLS[pool] if 0 < pool < len(POOLS) else ""))

    def stats(self) -> dict:
        s = vm_frame_stats()
        _check(self._lib.vm_get_stats(self._h, ctypes.byref(s)), "vm_get_stats")
        return {n: getattr(s, n) for n, _ in vm_frame_stats._fields_}

    def mesh_memory(self) -> dict:
        """Vertex counts of this mesh against per-block and loose-triangle meshes, and bytes."""
        m = vm_mesh_memory()
        _check(self._lib.vm_mesh_memory_stats(self._h, ctypes.byref(m)), "vm_mesh_memory_stats")
        return {n: getattr(m, n) for n, _ in vm_mesh_memory._fields_}

    def num_blocks(self) -> int:
        n = ctypes.c_int64()
        _check(self._lib.vm_num_blocks(self._h, ctypes.byref(n)), "vm_num_blocks")
        return n.value

    def mesh_size_async(self, dst):
        """Enqueue a copy of (live vertices, live triangles) into dst: a 2-element int32 torch
        tensor, pinned host or CUDA; it holds the values once the stream reaches the copy."""
        import torch

        assert dst.dtype == torch.int32 and dst.numel() >= 2
        _check(self._lib.vm_mesh_size_async(self._h, ctypes.c_void_p(dst.data_ptr()), int(dst.is_cuda)),
               "vm_mesh_size_async")

    def mesh_counts(self):
        nv, nt = ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.vm_mesh_counts(self._h, ctypes.byref(nv), ctypes.byref(nt)), "vm_mesh_counts")
        return nv.value, nt.value

    def download(self, device: bool = False):
        """The live mesh: dict(pos (nv,3) f32, nrm (nv,3) f32, tris (nt,3) i32, keys (nv,) u64,
        refcount (nv,) i32) as numpy arrays (host path) or torch CUDA tensors (device path)."""
        import torch

        if device:
            # buffers sized by the pools' high-water marks (they bound the live counts), then one
            # call that counts, compacts and synchronises once; the outputs are views of the
            # counted length
            st = self.stats()
            cv, ct = max(st["vertex_high_water"], 1), max(st["triangle_high_water"], 1)  # non-empty buffers
            dev = torch.device("cuda")
            pos = torch.empty((cv, 3), dtype=torch.float32, device=dev)
            nrm = torch.empty((cv, 3), dtype=torch.float32, device=dev)
            tris = torch.empty((ct, 3), dtype=torch.int32, device=dev)
            keys = torch.empty((cv,), dtype=torch.int64, device=dev)
            ref = torch.empty((cv,), dtype=torch.int32, device=dev)
            nv, nt = ctypes.c_int64(), ctypes.c_int64()
            _check(self._lib.vm_download_mesh_into(self._h, _ptr(pos), _ptr(nrm), _ptr(tris), _ptr(keys), _ptr(ref),
                                                   cv, ct, ctypes.byref(nv), ctypes.byref(nt)),
                   "vm_download_mesh_into")
            nv, nt = nv.value, nt.value
            return dict(pos=pos[:nv], nrm=nrm[:nv], tris=tris[:nt], keys=keys[:nv], refcount=ref[:nv])
        nv, nt = self.mesh_counts()
        pos = np.empty((nv, 3), np.float32)
        nrm = np.empty((nv, 3), np.float32)
        tris = np.empty((nt, 3), np.int32)
        keys = np.empty((nv,), np.uint64)
        ref = np.empty((nv,), np.int32)
        _check(self._lib.vm_download_mesh(self._h, _ptr(pos), _ptr(nrm), _ptr(tris), _ptr(keys), _ptr(ref), 0),
               "vm_download_mesh")
        return dict(pos=pos, nrm=nrm, tris=tris, keys=keys, refcount=ref)

    def blocks(self) -> dict:
        """Every allocated block: keys (n,3) i32, tsdf/weight (n,512) f32, code_eff/code_prev (n,512) u8."""
        n = self.num_blocks()
        keys = np.empty((n, 3), np.int32)
        tsdf = np.empty((n, 512), np.float32)
        weight = np.empty((n, 512), np.float32)
        ce = np.empty((n, 512), np.uint8)
        cp = np.empty((n, 512), np.uint8)
        _check(self._lib.vm_export_blocks(self._h, _ptr(keys), _ptr(tsdf), _ptr(weight), _ptr(ce), _ptr(cp)),
               "vm_export_blocks")
        return dict(keys=keys, tsdf=tsdf, weight=weight, code_eff=ce, code_prev=cp)

    def set_blocks(self, keys, tsdf, weight):
        k = np.ascontiguousarray(keys, np.int32).reshape(-1, 3)
        t = np.ascontiguousarray(tsdf, np.float32).reshape(-1, 512)
        w = np.ascontiguousarray(weight, np.float32).reshape(-1, 512)
        _check(self._lib.vm_set_blocks(self._h, _ptr(k), k.shape[0], _ptr(t), _ptr(w)), "vm_set_blocks")

    # --------------------------------------------------------------- differentiable path
    def diff_begin(self, max_frames: int):
        """Checkpoint the weights and record the next `max_frames` integrate calls."""
        _check(self._lib.vm_diff_begin(self._h, int(max_frames)), "vm_diff_begin")

    def diff_end(self):
        _check(self._lib.vm_diff_end(self._h), "vm_diff_end")

    def grad_vertices(self, keys, grad_pos, grad_nrm):
        """Add dL/dd from dL/dpos, dL/dnrm: CUDA tensors keys (n,) int64 (edge keys),
        grad_pos, grad_nrm (n, 3) float32."""
        _contig_cuda(keys, grad_pos, grad_nrm)
        _check(self._lib.vm_grad_vertices(self._h, int(keys.shape[0]), _ptr(keys), _ptr(grad_pos), _ptr(grad_nrm)),
               "vm_grad_vertices")

    def grad_depth(self, frame: int, depth, intr: Intrinsics, T_wc, T_cw, out):
        """dL/dD of recorded call `frame` (last first) into `out` (CUDA float32, like depth)."""
        _contig_cuda(depth, out)
        _check(self._lib.vm_grad_depth(self._h, int(frame), _ptr(depth), ctypes.byref(intr.c()), _f16(T_wc),
                                       _f16(T_cw), _ptr(out)), "vm_grad_depth")

    def export_grad(self) -> dict:
        """dL/dd of every allocated block: keys (n,3) i32, grad (n,512) f32."""
        n = self.num_blocks()
        keys = np.empty((n, 3), np.int32)
        grad = np.empty((n, 512), np.float32)
        _check(self._lib.vm_export_grad(self._h, _ptr(keys), _ptr(grad)), "vm_export_grad")
        return dict(keys=keys, grad=grad)

    # --------------------------------------------------------------- timing
    KERNELS = ["k_alloc", "k_integrate", "k_list_all", "k_mesh", "k_gc_vertices", "k_gc_blocks"]

    def enable_timing(self, on=True):
        """on: True (every kernel), False (none) or a list of kernel names to time."""
        if on is True:
            mask = -1
        elif not on:
            mask = 0
        else:
            mask = sum(1 << self.KERNELS.index(k) for k in on)
        _check(self._lib.vm_enable_timing(self._h, mask), "vm_enable_timing")

    def kernel_times(self) -> dict:
        cap = 32
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        cnt = (ctypes.c_int64 * cap)()
        n = ctypes.c_int()
        _check(self._lib.vm_kernel_times(self._h, names, ms, cnt, cap, ctypes.byref(n)), "vm_kernel_times")
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(n.value)}


class Scenes:
    """Independent volumes stepped together: one frame of every scene per tick, five launches
    in total (optionally replayed from one CUDA graph), schedules picked by an autotuner."""

    SLOTS = ["alloc_pixels_per_thread", "integrate_ctas_per_sm", "mesh_ctas_per_sm", "gc_vertices_ctas_per_sm",
             "gc_blocks_ctas_per_sm"]

    def __init__(self, volumes):
        self._lib = load_library()
        self.volumes = list(volumes)
        n = len(self.volumes)
        arr = (ctypes.c_void_p * n)(*[v._h.value for v in self.volumes])
        h = ctypes.c_void_p()
        _check(self._lib.vm_batch_create(arr, n, ctypes.byref(h)), "vm_batch_create")
        self._h = h

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None and h.value:
            self._lib.vm_batch_destroy(h)

    def __del__(self):
        self.close()

    def step_all(self, depths, intrinsics, poses, refine=True, gc=True, graph=True):
        """depths: float32 (H, W) tensors, one per scene, CUDA or pinned CPU; intrinsics:
        Intrinsics per scene; poses: (T_wc, T_cw) per scene (host 4x4, rounded to float32)."""
        n = len(self.volumes)
        assert len(depths) == len(intrinsics) == len(poses) == n
        for d in depths:
            if not d.is_contiguous():
                raise ValueError("expected contiguous depth tensors")
        dp = (ctypes.c_void_p * n)(*[_ptr(d) for d in depths])
        ks = (vm_intrinsics * n)(*[k.c() for k in intrinsics])
        twc = np.ascontiguousarray(np.stack([np.asarray(p[0], np.float32).reshape(16) for p in poses]))
        tcw = np.ascontiguousarray(np.stack([np.asarray(p[1], np.float32).reshape(16) for p in poses]))
        flags = (VM_REFINE if refine else 0) | (VM_GC if gc else 0)
        fp = ctypes.POINTER(ctypes.c_float)
        _check(self._lib.vm_batch_step(self._h, dp, ks, twc.ctypes.data_as(fp), tcw.ctypes.data_as(fp), flags,
                                       int(bool(graph))), "vm_batch_step")

    def tune(self, rounds: int = 2):
        """Autotune on the next 3 * rounds ticks."""
        _check(self._lib.vm_batch_tune(self._h, int(rounds)), "vm_batch_tune")

    def schedule(self) -> dict:
        sc = (ctypes.c_int * 5)()
        ms = (ctypes.c_double * 15)()
        _check(self._lib.vm_batch_schedule(self._h, sc, ms), "vm_batch_schedule")
        return dict(schedule=dict(zip(self.SLOTS, list(sc))),
                    tuned_ms={k: [ms[3 * i + o] for o in range(3)] for i, k in enumerate(self.SLOTS)})

    KERNELS = ["kb_alloc", "kb_integrate", "kb_mesh", "kb_gc_vertices", "kb_gc_blocks"]

    def profile(self, ticks: int):
        """Time each kernel (CUDA events, eager launches) over the next `ticks` steps."""
        _check(self._lib.vm_batch_profile(self._h, int(ticks)), "vm_batch_profile")

    def kernel_ms(self) -> dict:
        ms = (ctypes.c_double * 5)()
        n = ctypes.c_int()
        _check(self._lib.vm_batch_kernel_ms(self._h, ms, ctypes.byref(n)), "vm_batch_kernel_ms")
        return dict(zip(self.KERNELS, list(ms)), ticks=n.value)

    def set_schedule(self, sched):
        sc = (ctypes.c_int * 5)(*[int(x) for x in sched])
        _check(self._lib.vm_batch_set_schedule(self._h, sc), "vm_batch_set_schedule")


def _diff_mesh_function():
    import torch

    class DiffMesh(torch.autograd.Function):
        """Differentiable fusion and meshing: integrates the leaf depth frames (recording
        them), extracts the full mesh (refined when `refine`), and returns vertex positions
        and normals (differentiable), triangles and edge keys.  The backward runs the
        library's gradient kernels: vertices -> TSDF values -> depth pixels, topology fixed."""

        @staticmethod
        def forward(ctx, vol, intr, poses, refine, *depths):
            vol.diff_begin(len(depths))
            for d, (T_wc, T_cw) in zip(depths, poses):
                vol.integrate(d, intr, T_wc, T_cw)
            vol.update_mesh(full=True, refine=refine)
            m = vol.download(device=True)
            ctx.vol, ctx.intr, ctx.poses = vol, intr, poses
            ctx.save_for_backward(m["keys"], *depths)
            ctx.mark_non_differentiable(m["tris"], m["keys"])
            return m["pos"], m["nrm"], m["tris"], m["keys"]

        @staticmethod
        def backward(ctx, g_pos, g_nrm, _g_tris, _g_keys):
            keys, *depths = ctx.saved_tensors
            vol = ctx.vol
            n = keys.shape[0]
            g_pos = torch.zeros((n, 3), dtype=torch.float32, device=keys.device) if g_pos is None else g_pos.contiguous()
            g_nrm = torch.zeros((n, 3), dtype=torch.float32, device=keys.device) if g_nrm is None else g_nrm.contiguous()
            vol.grad_vertices(keys, g_pos, g_nrm)
            grads = [None] * len(depths)
            for k in reversed(range(len(depths))):
                grads[k] = torch.empty_like(depths[k])
                vol.grad_depth(k, depths[k], ctx.intr, *ctx.poses[k], grads[k])
            vol.diff_end()
            return (None, None, None, None, *grads)

    return DiffMesh


_DIFF = None


def diff_mesh(vol: Volume, intr: Intrinsics, poses, depths, refine: bool = True):
    """(pos, nrm, tris, keys) of the mesh after integrating `depths` (CUDA float32 (H, W)
    tensors; gradients flow to those that require them) at `poses` ((T_wc, T_cw) pairs)."""
    global _DIFF
    if _DIFF is None:
        _DIFF = _diff_mesh_function()
    return _DIFF.apply(vol, intr, list(poses), bool(refine), *[d.contiguous() for d in depths])
