/*
 * vmesh -- incremental volumetric meshing on a spatial hash, B300 (sm_103a) CUDA.
 *
 * C ABI of the per-frame hot path of Dong, Shi, Tang, Wang, Zha, "An Efficient
 * Volumetric Mesh Representation for Real-time Scene Reconstruction using Spatial
 * Hashing" (arXiv 1803.03949):
 *
 *   integrate_depth   block collection (Sec. V-A, Eq. 1) + TSDF fusion (Sec. V-A, Eq. 2)
 *   update_mesh       cube types (Sec. V-B), edge-owned vertices (Sec. V-C, Sec. IV),
 *                     triangulation with type-change reuse (Sec. V-D)
 *   refine_mesh       Hamming-distance cube-type refinement (Sec. V-F, Eqs. 3-5)
 *   gc                reference-count recycling of vertices (Sec. V-E) plus triangle
 *                     and block recycling
 *   download_mesh     compaction of the live mesh into dense arrays (Sec. VI, the
 *                     "compress" step before rendering)
 *
 * Conventions shared by every call
 *   - Lattice: a voxel is a cube corner; global voxel g = (gx, gy, gz) sits at world
 *     g * voxel_size; blocks hold 8 x 8 x 8 voxels, block key = floor(g / 8); inside a
 *     block voxel (x, y, z) has index x + 8 y + 64 z.  Voxel g owns the three edges
 *     g -> g + e_x, g + e_y, g + e_z and the vertices on them (Sec. IV).
 *   - Camera: pinhole with OpenCV axes (x right, y down, z forward); depth is camera z
 *     in metres; a pixel is valid when its depth is finite and > 0.  T_wc is the
 *     camera-to-world pose, T_cw its inverse; both row-major 4 x 4 float32 on the host,
 *     and the caller computes T_cw (the library never inverts a pose).
 *   - Streams: every call enqueues work on the volume's stream (given at creation or by
 *     vm_set_stream) and returns without waiting, except where a call says it
 *     synchronises.  Device pointers must be valid on that stream when the work runs.
 *   - Ownership: the caller owns depth frames and every output buffer; the library owns
 *     the volume's device memory (hash table, voxel arrays, mesh pools), allocated in
 *     vm_create_volume and released in vm_destroy_volume.
 *   - Errors: a call returns VM_ERR_INVALID_ARG for a bad argument (null pointer,
 *     non-finite or out-of-range value) before enqueuing anything, VM_ERR_CUDA when a
 *     CUDA runtime call fails, and VM_OK otherwise.  Failures found on the device
 *     (hash table or pool exhausted) are recorded in a sticky status word, never by
 *     trapping; vm_last_error synchronises and returns it.  After a device failure the
 *     volume's contents are unspecified but it can still be destroyed.
 */
#ifndef VMESH_H
#define VMESH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vm_volume vm_volume;

typedef enum {
  VM_OK = 0,
  VM_ERR_INVALID_ARG = 1, /* bad argument; nothing was enqueued */
  VM_ERR_HASH_FULL = 2,   /* device: no free hash bucket for a new block */
  VM_ERR_POOL_FULL = 3,   /* device: block, vertex, triangle pool or a work list exhausted */
  VM_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  VM_ERR_OOM = 5          /* device memory allocation failed */
} vm_status;

/* Volume parameters (Sec. VI: 8^3 blocks, cube size 8 mm .. 3 cm). */
typedef struct {
  float voxel_size;       /* cube side l in metres, >= 1e-4 */
  float trunc;            /* truncation distance mu in metres, 0 < mu <= 32 l */
  float eps_refine;       /* epsilon of Eq. 5 in metres (proportional to l; 0.2 l is typical), >= 0 */
  float w_max;            /* cap of the fusion weight, >= 1 */
  uint32_t hash_buckets;  /* power of two, 2^4 .. 2^30 */
  uint32_t max_blocks;    /* block pool size, 1 .. 2^21 */
  uint32_t max_vertices;  /* vertex pool size, 1 .. 2^30 */
  uint32_t max_triangles; /* triangle pool size, 1 .. 2^30 */
  uint32_t flags;         /* 0, or VM_PARAM_COMPACT_EDGES */
} vm_params;

/* vm_params.flags: the compact cube record (Sec. IV proposes one heap reference each for a
 * cube's edges and triangles): 19 B per cube -- (d, W) 8, two types 2, vertex flags 1, an
 * edge-record index 4, a triangle-run start 4 -- plus a 12 B record (3 vertex ids) per voxel
 * that owns a vertex, instead of 27 B per cube with the 3 vertex ids in place.  Same results;
 * the record claims and their recycling cost mesh-pass time (about 5 % on a 640x480 room
 * frame, 14 % on the 5 mm floor). */
#define VM_PARAM_COMPACT_EDGES 1u

typedef struct {
  int32_t width, height; /* pixels, 1 .. 16384 each */
  float fx, fy, cx, cy;  /* pinhole intrinsics in pixels, fx, fy > 0; every pixel ray's
                            slope |(u - cx) / fx|, |(v - cy) / fy| must be <= 64 */
} vm_intrinsics;

/* Capacities a sticky VM_ERR_POOL_FULL or VM_ERR_HASH_FULL status can name (vm_frame_stats
 * full_pool): the block pool (max_blocks), vertex pool (max_vertices), triangle pool
 * (max_triangles), the per-frame collected-block list (min(max_blocks, hash_buckets)), the
 * update-set list (max_blocks), the zero-reference vertex list (2 max_vertices), the
 * released-run list (max_triangles), a free stack, the hash table, the edge-record pool
 * (max_vertices records, one per voxel that owns a vertex). */
typedef enum {
  VM_POOL_NONE = 0,
  VM_POOL_BLOCKS,
  VM_POOL_VERTICES,
  VM_POOL_TRIANGLES,
  VM_POOL_COLLECTED_LIST,
  VM_POOL_UPDATE_LIST,
  VM_POOL_DEAD_VERTEX_LIST,
  VM_POOL_DEAD_RUN_LIST,
  VM_POOL_FREE_STACK,
  VM_POOL_HASH,
  VM_POOL_EDGE_RECORDS
} vm_pool;

/* Per-call counters, filled by vm_get_stats (which synchronises). */
typedef struct {
  int64_t frame_blocks;      /* blocks collected by the last integrate_depth (N_t) */
  int64_t new_blocks;        /* blocks allocated since the volume was created */
  int64_t update_blocks;     /* blocks in the update set of the last mesh pass */
  int64_t changed_cubes;     /* cubes whose effective type changed, summed over mesh passes */
  int64_t live_blocks;       /* allocated blocks */
  int64_t live_vertices;     /* vertices in the pool (includes zero-reference ones awaiting gc) */
  int64_t live_triangles;    /* triangles in the pool */
  int64_t freed_blocks;      /* blocks recycled since the volume was created */
  int64_t freed_vertices;    /* vertices recycled since the volume was created */
  int64_t created_vertices;  /* vertices created since the volume was created */
  int64_t hash_tombstones;   /* dead hash buckets awaiting a rehash */
  int64_t block_high_water;  /* block pool slots ever used */
  int64_t rehashes;          /* hash rebuilds (tombstone clean-ups) so far */
  int64_t emitted_triangles; /* triangles written by mesh passes so far */
  int64_t released_triangles;/* triangles released by mesh passes so far */
  int64_t refreshed_vertices;/* vertex positions and normals recomputed so far */
  int64_t collected_blocks;  /* N_t summed over integrate calls (kept modulo 2^32) */
  int64_t meshed_blocks;     /* update-set sizes summed over mesh passes (kept modulo 2^32) */
  int64_t full_pool;         /* vm_pool: the capacity a VM_ERR_POOL_FULL / HASH_FULL status ran
                                out of first (VM_POOL_NONE while the status is clear) */
  int64_t vertex_high_water;   /* vertex pool slots ever used (below created_vertices once freed
                                  ids are reused) */
  int64_t triangle_high_water; /* triangle pool slots ever used (below emitted_triangles once
                                  released runs are reused) */
  int64_t reference_updates;   /* reference-count updates of the mesh passes so far (one per
                                  edge of a changed cube whose use changes) */
} vm_frame_stats;

/* Flags of vm_update_mesh / vm_step. */
#define VM_FULL 1   /* process every allocated block, not only the frame's update set */
#define VM_REFINE 2 /* apply the refinement of Eqs. 3-5 in the same pass */
#define VM_GC 4     /* vm_step only: run gc after the mesh update */

/* Create a volume: allocates and clears all of its device memory on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  *out receives the handle. */
vm_status vm_create_volume(const vm_params* params, void* cuda_stream, vm_volume** out);

/* Synchronise the volume's stream and free everything it owns.  NULL is accepted. */
vm_status vm_destroy_volume(vm_volume* vol);

/* Change the stream later calls enqueue on. */
vm_status vm_set_stream(vm_volume* vol, void* cuda_stream);

/* Sec. V-A.  depth: height x width float32, row-major, 0 or non-finite = invalid, in device
 * memory or in pinned (page-locked, device-mapped) host memory; the latter is read across
 * the host link by the collection kernel, which keeps a device copy for the fusion (the
 * frame's transfer overlaps the collection); the caller keeps it unchanged until the call's
 * work has run.  Pageable host memory: VM_ERR_INVALID_ARG.  Collects every block crossed by
 * the segment of camera depths
 * [max(D - mu, 0.05), D + mu] on each valid pixel's ray (Eq. 1), allocates the new ones,
 * then fuses the frame into every voxel of the collected blocks (Eq. 2): nearest pixel
 * floor(u + 0.5), sdf = D - z_c, skip when sdf < -mu, d <- (d W + min(sdf, mu)) / (W + 1),
 * W <- min(W + 1, w_max).  Blocks collected since the last vm_update_mesh accumulate
 * into the next update set. */
vm_status vm_integrate_depth(vm_volume* vol, const float* depth, const vm_intrinsics* intr,
                             const float T_wc[16], const float T_cw[16]);

/* Secs. V-B..V-D.  Recomputes the cube types of the update set (blocks collected since
 * the previous update plus their existing neighbours at offsets {0,-1}^3 \ {0}; all
 * blocks with VM_FULL); a cube is valid when its 8 corners are allocated with W > 0,
 * otherwise its type is 0.  Stores the previous effective type as t_{i-1}, keeps a
 * cube's triangles when its type is unchanged, otherwise releases them and emits the
 * marching-cubes triangles of the new type on edge-owned vertices, creating vertices
 * on first use and updating the positions and normals of the update set's existing
 * vertices.  VM_REFINE applies Eqs. 3-5 in the same pass (same result as a following
 * vm_refine_mesh). */
vm_status vm_update_mesh(vm_volume* vol, int flags);

/* Sec. V-F, Eqs. 3-5, over the last update set (all blocks when full != 0): a valid
 * cube whose raw type t_i is within Hamming distance 3 of its stored t_{i-1} takes the
 * nearest regular type t_rj within distance 3 whose differing corners all have
 * |d| < eps_refine (ties: the first in the paper's list); then re-triangulates. */
vm_status vm_refine_mesh(vm_volume* vol, int full);

/* Sec. V-E.  Recycles vertices whose reference count dropped to 0 and blocks that were
 * not collected since the last update, carry no triangle (nor do their 7 lower
 * neighbours), own no vertex, and whose voxels all have W = 0 or d >= mu.  Freed
 * triangles were already recycled by the mesh passes. */
vm_status vm_gc(vm_volume* vol);

/* One frame: integrate_depth (depth as there: device or pinned host memory), then
 * update_mesh(flags & (VM_FULL | VM_REFINE)), then gc when flags has VM_GC.  With use_graph != 0 the device work after the first call is
 * replayed from a CUDA graph captured on that first call with the same flags. */
vm_status vm_step(vm_volume* vol, const float* depth, const vm_intrinsics* intr, const float T_wc[16],
                  const float T_cw[16], int flags, int use_graph);

/* Synchronises; counts of the vertices with a positive reference count and of the live
 * triangles, i.e. the sizes vm_download_mesh writes. */
vm_status vm_mesh_counts(vm_volume* vol, int64_t* n_vertices, int64_t* n_triangles);

/* Synchronises; compacts the live mesh (Sec. VI "compress").  Buffers are device
 * pointers when on_device != 0, host pointers otherwise, sized from vm_mesh_counts:
 *   pos       n_vertices x 3 float32, world metres
 *   nrm       n_vertices x 3 float32, unit normal (zero when undefined)
 *   tris      n_triangles x 3 int32, indices into pos, oriented so that the normal
 *             points from negative to positive TSDF
 *   edge_keys n_vertices uint64 (optional, may be NULL): owner voxel coordinates biased
 *             by 2^19 in bits 42-61, 22-41, 2-21 and the edge axis in bits 0-1
 *   refcount  n_vertices int32 (optional, may be NULL): the vertex reference count */
vm_status vm_download_mesh(vm_volume* vol, float* pos, float* nrm, int32_t* tris, uint64_t* edge_keys,
                           int32_t* refcount, int on_device);

/* The vm_download_mesh compaction (Sec. VI "compress") into caller-allocated DEVICE buffers
 * with capacities, without a separate vm_mesh_counts call: the counts, their scan and both
 * compactions are enqueued back to back and the call synchronises once.  pos, nrm, tris (and
 * the optional edge_keys, refcount) have the vm_download_mesh layout and hold at least
 * cap_vertices / cap_triangles entries; *n_vertices and *n_triangles receive the live counts.
 * Nothing at or past a capacity is written; when a count exceeds its capacity the call
 * returns VM_ERR_INVALID_ARG and the outputs are unspecified (call again with the counts as
 * capacities).  The pools' high-water marks (vm_frame_stats.vertex_high_water,
 * triangle_high_water) always bound the counts. */
vm_status vm_download_mesh_into(vm_volume* vol, float* pos, float* nrm, int32_t* tris, uint64_t* edge_keys,
                                int32_t* refcount, int64_t cap_vertices, int64_t cap_triangles,
                                int64_t* n_vertices, int64_t* n_triangles);

/* Enqueues (without waiting) a copy of the live vertex and triangle counts, 2 x int32,
 * to dst: pinned host memory when on_device == 0 (valid once the stream reaches the
 * copy), device memory otherwise.  The counts include zero-reference vertices that the
 * next gc will recycle. */
vm_status vm_mesh_size_async(vm_volume* vol, int32_t* dst, int on_device);

/* Mesh memory (Sec. VI-B "Memory"; the paper compares vertex counts with a mesher whose
 * blocks share no vertices, and states 56 bytes per cube for its own structure). */
typedef struct {
  int64_t vertices;        /* referenced vertices of the edge-owned mesh (each stored once) */
  int64_t triangles;       /* triangles */
  int64_t block_vertices;  /* vertices a per-block extraction stores: shared by the cubes of
                              one block, copied in every block whose cubes use them */
  int64_t loose_vertices;  /* 3 per triangle: every triangle with its own corners */
  int64_t blocks;          /* allocated blocks */
  int64_t cube_bytes;      /* bytes per cube (voxel) of this layout: (d, W) 8, two types 2,
                              vertex flags 1, edge-record index 4, triangle-run start 4 (Sec. IV:
                              one heap reference each for the edges and the triangles) */
  int64_t edge_records;    /* edge records in use: one per voxel that owns a vertex, 12 B each
                              (the vertex ids of its 3 owned edges) */
  int64_t bytes_in_use;    /* blocks x (512 cubes + block record) + edge records x 12 +
                              vertices x 40 + triangles x 16 + hash buckets x 16 */
  int64_t bytes_allocated; /* device memory the volume holds (pool capacities) */
} vm_mesh_memory;

/* Synchronises and fills *m (runs a counting kernel over the allocated blocks). */
vm_status vm_mesh_memory_stats(vm_volume* vol, vm_mesh_memory* m);

/* Synchronises and fills *stats. */
vm_status vm_get_stats(vm_volume* vol, vm_frame_stats* stats);

/* Synchronises and returns the sticky device status (VM_OK when none). */
vm_status vm_last_error(vm_volume* vol);

/* No counterpart in the paper: the same compaction as vm_download_mesh for callers that
 * must not allocate device memory -- for example code running while a caching allocator
 * holds all free device memory, or under a fixed memory budget set at start-up.  It calls
 * no cudaMalloc or cudaFree; its scratch is a static device array of about 4.5 MB that
 * every GPU loading the library holds until the process exits, sized for vertex pools up
 * to 2^24 and triangle pools up to 2^26 entries (larger volumes get VM_ERR_INVALID_ARG
 * before anything is enqueued).  Synchronises.  Writes the live counts to the host
 * *n_vertices and *n_triangles; with pos == NULL it stops there (a size query).
 * Otherwise pos, nrm, tris (and the optional edge_keys, refcount) are DEVICE buffers in
 * the vm_download_mesh layout holding at least cap_vertices / cap_triangles entries;
 * counts above those capacities give VM_ERR_INVALID_ARG with the outputs untouched.
 * The device that was current when the volume was created must be current (else
 * VM_ERR_INVALID_ARG).  The first call on each device looks up the scratch array's device
 * address, so make it before any stream capture on that device.  All calls share the one
 * scratch array and
 * every call rewrites the parts it reads; calls whose work overlaps on the GPU (other
 * host threads, other streams) race on it and must be serialised by the caller. */
vm_status vm_download_mesh_noalloc(vm_volume* vol, float* pos, float* nrm, int32_t* tris, uint64_t* edge_keys,
                                   int32_t* refcount, int64_t cap_vertices, int64_t cap_triangles,
                                   int64_t* n_vertices, int64_t* n_triangles);

/* Synchronises; number of allocated blocks. */
vm_status vm_num_blocks(vm_volume* vol, int64_t* n);

/* Synchronises; copies every allocated block to host buffers sized from vm_num_blocks
 * (any order): keys n x 3 int32, tsdf and weight n x 512 float32, code_eff and
 * code_prev n x 512 uint8 (current and previous effective cube types).  Any output may
 * be NULL. */
vm_status vm_export_blocks(vm_volume* vol, int32_t* keys, float* tsdf, float* weight, uint8_t* code_eff,
                           uint8_t* code_prev);

/* Allocates the blocks `keys` (host, n x 3 int32, distinct) if needed and overwrites
 * their voxels from host tsdf and weight (n x 512 float32 each); the blocks join the
 * next update set as if collected by a frame.  For analytic fills. */
vm_status vm_set_blocks(vm_volume* vol, const int32_t* keys, int64_t n, const float* tsdf,
                        const float* weight);

/* Device time of the library's kernels, accumulated while timing is on (CUDA events on
 * the volume's stream around each launch; inside a vm_step CUDA graph they are event-record
 * nodes, whose times are added when the next replay starts or vm_kernel_times is called).
 * `enable` is a kernel mask: bit k times the k-th kernel in vm_kernel_times order, -1 all
 * of them, 0 none; the call clears the totals, and a captured frame graph is re-captured
 * on the next vm_step (event nodes cost device time, so time only what is needed).
 * vm_kernel_times synchronises and writes up to `cap` entries of (name, total
 * milliseconds, launches); returns the number of kernels in *n. */
vm_status vm_enable_timing(vm_volume* vol, int enable);
vm_status vm_kernel_times(vm_volume* vol, const char** names, double* total_ms, int64_t* launches, int cap,
                          int* n);

/* ---------------------------------------------------------------- differentiable path
 * Gradients of a loss on the mesh vertex positions and normals, taken to the TSDF values
 * through the edge interpolation and normal of Sec. V-C (recomputed from the TSDF, not
 * stored) and on to the depth pixels by reverse mode through the running average of
 * Sec. V-A, Eq. 2 (d <- (d W + d~) / (W + 1), d~ = min(sdf, mu)).  Topology, block
 * collection, pixel choice and branches are held fixed: d~ = mu (sdf >= mu) passes no
 * gradient, a t clamped to [-1, 2] is constant.  Sequence: vm_diff_begin, the recorded
 * vm_integrate_depth calls, a mesh update, vm_grad_vertices (any number of calls, they
 * add), optionally vm_export_grad (dL/dd of the final TSDF), then vm_grad_depth for the
 * recorded calls last to first, then vm_diff_end. */

/* Checkpoints every voxel weight, clears dL/dd and records the next max_frames
 * (1..65535) vm_integrate_depth calls (the blocks each collects and, per voxel, whether it
 * integrated it).  Buffers: 10 B per voxel of the block pool plus 4 B per collected-list
 * entry per recorded call, owned by the volume and kept for the next begin; VM_ERR_OOM
 * when they cannot be allocated.  While recording, vm_gc and vm_step return
 * VM_ERR_INVALID_ARG (recycling blocks would rename recorded voxels), as does an integrate
 * call beyond max_frames or after the first vm_grad_depth. */
vm_status vm_diff_begin(vm_volume* vol, int max_frames);

/* Ends recording (the buffers stay allocated until vm_destroy_volume). */
vm_status vm_diff_end(vm_volume* vol);

/* Adds dL/dd given dL/dp and dL/dn of n vertices: edge_keys (n uint64, the vm_download_mesh
 * key of each vertex), grad_pos and grad_nrm (n x 3 float32), all DEVICE pointers owned by
 * the caller.  A vertex whose owner voxels are not allocated is skipped.  Enqueues only. */
vm_status vm_grad_vertices(vm_volume* vol, int64_t n, const uint64_t* edge_keys, const float* grad_pos,
                           const float* grad_nrm);

/* Reverse step of recorded call `frame` (0-based; the last recorded call first, then each
 * earlier one): writes dL/dD of that call's depth pixels into grad_depth (DEVICE, H x W
 * float32, overwritten) and moves dL/dd to before the call.  depth, *K, T_wc and T_cw
 * must be the recorded call's inputs (a voxel the call did not integrate sets the sticky
 * status VM_ERR_INVALID_ARG).  A frame out of order is VM_ERR_INVALID_ARG. */
vm_status vm_grad_depth(vm_volume* vol, int frame, const float* depth, const vm_intrinsics* K, const float T_wc[16],
                        const float T_cw[16], float* grad_depth);

/* Synchronises; copies dL/dd of every allocated block to host buffers sized from
 * vm_num_blocks (any order): keys n x 3 int32, grad n x 512 float32 (voxel x + 8 y + 64 z).
 * VM_ERR_INVALID_ARG before the first vm_diff_begin. */
vm_status vm_export_grad(vm_volume* vol, int32_t* keys, float* grad);

/* ---------------------------------------------------------------- batched step
 * Many independent volumes (scenes of uneven sizes, each created with its own parameters),
 * stepped one frame each per tick by five launches in total: every per-frame kernel runs
 * once over the concatenation of all scenes' work (tiles, collected blocks, update sets,
 * gc lists), optionally replayed from one CUDA graph per tick.  Results per scene are those
 * of vm_step on that scene alone.  Kernel schedules (pixels per thread of the block
 * collection; CTAs per SM of the persistent fusion, mesh and gc grids) come from an
 * autotuner that times the candidate options on live ticks. */
typedef struct vm_batch vm_batch;

/* A batch of n (1..64) distinct volumes on the current device, all with the same cube layout
 * (VM_PARAM_COMPACT_EDGES set on all or none).  It enqueues on the first
 * volume's stream; while it steps them, work on the volumes' own streams must be ordered
 * with that stream by the caller.  The volumes stay owned by the caller and must outlive
 * the batch.  VM_ERR_OOM when its small buffers cannot be allocated. */
vm_status vm_batch_create(vm_volume* const* vols, int n, vm_batch** out);
vm_status vm_batch_destroy(vm_batch* batch);

/* One tick: for scene i, depth depths[i] (K[i].height x K[i].width float32, in device
 * memory or pinned host memory as for vm_integrate_depth),
 * intrinsics K[i], poses T_wc + 16 i, T_cw + 16 i (host, row-major), as vm_step with
 * `flags` (VM_REFINE, VM_GC; VM_FULL is not available).  use_graph != 0 replays the
 * tick's five launches from a CUDA graph (captured on first use, re-captured when the
 * flags, the largest image or the schedule change).  Any invalid frame, or a volume that
 * is recording for the differentiable path, gives VM_ERR_INVALID_ARG before anything is
 * enqueued.  Enqueues only. */
vm_status vm_batch_step(vm_batch* batch, const float* const* depths, const vm_intrinsics* K, const float* T_wc,
                        const float* T_cw, int flags, int use_graph);

/* Autotune on the next 3 * rounds ticks (1..100 rounds): each tick runs every kernel on one
 * of its three candidate options (eagerly, with CUDA events around each kernel); after the
 * last, each kernel keeps its fastest option (the tuning ticks are real steps). */
vm_status vm_batch_tune(vm_batch* batch, int rounds);

/* The schedule in use, 5 ints: k_alloc pixels per thread (1, 2, 4), CTAs per SM of the
 * fusion (4, 8, 12), mesh (4, 6, 8), vertex-gc (1, 2, 4) and block-gc (2, 4, 8) kernels;
 * tuned_ms (optional, 15 doubles) receives the mean time of each option from the last
 * tuning (-1 where untimed).  vm_batch_set_schedule installs a schedule from those options
 * (VM_ERR_INVALID_ARG otherwise). */
vm_status vm_batch_schedule(vm_batch* batch, int* sched, double* tuned_ms);
vm_status vm_batch_set_schedule(vm_batch* batch, const int* sched);

/* Profile the next `ticks` (1..100000) steps: they run eagerly with the current schedule and
 * CUDA events around each of the five kernels (event-record work adds device time).
 * vm_batch_kernel_ms synchronises and writes the mean milliseconds per profiled tick of
 * each kernel (block collection, fusion, mesh, vertex gc, block gc; -1 when none was
 * profiled) and the number of profiled ticks (optional). */
vm_status vm_batch_profile(vm_batch* batch, int ticks);
vm_status vm_batch_kernel_ms(vm_batch* batch, double* ms, int* ticks);

#ifdef __cplusplus
}
#endif

#endif /* VMESH_H */
