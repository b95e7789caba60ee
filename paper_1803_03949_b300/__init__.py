"""vmesh: incremental volumetric meshing on a spatial hash, as hand-written sm_103a CUDA.

Per depth frame: allocate 8^3 voxel blocks in a lossless GPU hash (Sec. V-A, Eq. 1), fuse
the frame into the TSDF (Eq. 2), recompute marching-cubes cube types (Sec. V-B), maintain
edge-owned vertices and triangles (Secs. IV, V-C, V-D), refine cube types by Hamming
distance (Sec. V-F) and recycle dead vertices, triangles and blocks (Sec. V-E).

The C ABI is ``include/vmesh.h``; :mod:`paper_1803_03949_b300.vmesh` is its binding.
"""
from .vmesh import Intrinsics, Scenes, Volume, VmeshError, diff_mesh, load_library  # noqa: F401
