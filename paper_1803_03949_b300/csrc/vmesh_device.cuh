// Device-side layout, constants and helpers of the vmesh CUDA library (sm_103a).
//
// HBM layout of a volume (all arrays owned by the library, cleared at creation):
//   hash      keys u64[B] (packed block key, EMPTY / TOMB), vals i32[B] (block index),
//             stamp u32[B] (integrate call that last collected the bucket's block)
//   blocks    ustamp u32[NB] (mesh epoch in which the block joined the update set),
//             bkey int4[NB] (x, y, z, bucket; bucket < 0 = free), nbr i32[NB][16]
//             (block indices of the neighbours at offsets (o&1, o>>1&1, o>>2&1), o = 1..7,
//             in slots 1..7 and of the neighbours at the negated offsets in slots 9..15;
//             -1 = none), bntri/bnvert i32[NB] (triangles in its cubes / vertices it
//             owns), bnear u8[NB] (some voxel has W > 0 and d < mu), bepoch u32[NB] (epoch
//             it was last collected in), bborn u32[NB] (integrate call that created it)
//   voxels    tw float2[NB*512] (TSDF d, weight W), code_eff/code_prev u8[NB*512],
//             vmask u8[NB*512] (bits 0-2: the owned edge has a vertex), tri_base i32[NB*512],
//             and the vertex ids of the voxel's 3 owned edges (-1 none), either
//             edge_vtx i32[NB*512*3] (wide layout, 27 B per cube) or, with the compact layout
//             (19 B per cube), edge_rec i32[NB*512] (the voxel's edge record, -1 none) into
//             erec i32[NV*3], one record per voxel that owns a vertex, from a pool with its
//             own free stack
//   vertices  vrec float4[2 NV] (per vertex its position, then its normal: one 32-byte sector, so a
//             refresh writes whole sectors), vref i32[NV] (reference count, -1 free),
//             vedge u32[NV] (owning edge id = block*1536 + voxel*3 + axis, below 2^32 for up
//             to 2^21 blocks; NO_EDGE = unattached)
//   triangles tris int4[NT] (three vertex ids, owning cube id; x < 0 = free)
//   free lists block / vertex stacks and five triangle-run stacks (run length 1..5)
//   work lists collected buckets, update set, zero-reference (recycling-candidate) vertices,
//             released triangle runs, plus a control block (counters, status, frame parameters).
#pragma once

#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>
#include <cooperative_groups/scan.h>
#include <cstdint>
#include <cuda_runtime.h>

namespace vmk {

namespace cg = cooperative_groups;

constexpr int BS = 8;       // block side in voxels (Sec. VI: 8^3 in all configurations)
constexpr int BV = 512;     // voxels per block
constexpr int EPB = 1536;   // owned edges per block
constexpr uint32_t NO_EDGE = 0xFFFFFFFFu;  // vedge of a vertex attached to no edge
constexpr uint64_t KEY_EMPTY = ~0ull;
constexpr uint64_t KEY_TOMB = ~0ull - 1ull;
constexpr int KEY_BIAS = 1 << 20;
constexpr int KEY_LIMIT = (1 << 20) - 2;  // |block coordinate| bound
constexpr float Z_NEAR = 0.05f;           // nearest camera depth of a collection segment

enum Status { ST_OK = 0, ST_INVALID = 1, ST_HASH_FULL = 2, ST_POOL_FULL = 3 };

// Counters of the control block (int slots of Ctl::c), one 128-byte line apart: the atomics
// of a mesh pass or a gc pass hit a dozen of them from every CTA, and counters sharing a line
// would queue at one L2 slice.
constexpr int CLINE = 32;
enum Counter {
  C_STATUS = 0 * CLINE,
  C_STATUS_POOL = 1 * CLINE,  // which capacity set the status (PoolCode)
  C_FRAME = 2 * CLINE,  // integrate calls so far + 1 (the host numbers the calls; statistics)
  C_EPOCH = 3 * CLINE,  // mesh epoch, advanced by the first integrate after a mesh update
  C_N_TOUCHED = 4 * CLINE,  // buckets collected by an even-numbered integrate call (touched_count)
  C_N_UPDATE = 5 * CLINE,  // blocks in the update set
  C_N_DEAD = 6 * CLINE,  // zero-reference vertices awaiting gc
  C_N_DEADRUN = 7 * CLINE,  // released triangle runs awaiting gc
  C_N_DEADREC = 8 * CLINE,  // spare edge records of lost record claims, awaiting gc
  C_REC_TOP = 9 * CLINE,
  C_REC_BUMP = 10 * CLINE,
  C_BLK_TOP = 11 * CLINE,
  C_BLK_BUMP = 12 * CLINE,
  C_VTX_TOP = 13 * CLINE,
  C_VTX_BUMP = 14 * CLINE,
  C_RUN_TOP0 = 15 * CLINE,  // free-run stack tops of lengths 1..5, one line apart (run_top)
  C_TRI_BUMP = 20 * CLINE,
  C_LIVE_BLOCKS = 21 * CLINE,
  C_LIVE_VERTS = 22 * CLINE,
  C_LIVE_TRIS = C_LIVE_VERTS + 1,  // beside C_LIVE_VERTS: the mesh size is read as one pair
  C_TOMBS = 23 * CLINE,
  C_REHASH = 24 * CLINE,  // 1 while a hash rebuild is under way
  C_ST_FRAME_BLOCKS = 25 * CLINE,
  C_ST_UPDATE_BLOCKS = 26 * CLINE,
  C_ST_COLLECTED = 27 * CLINE,
  C_ST_MESHED = 28 * CLINE,
  C_ST_NEW_BLOCKS = 29 * CLINE,
  C_ST_CHANGED = 30 * CLINE,
  C_ST_FREED_BLOCKS = 31 * CLINE,
  C_ST_FREED_VERTS = 32 * CLINE,
  C_ST_NEW_VERTS = 33 * CLINE,
  C_ST_REHASHES = 34 * CLINE,
  C_ST_EMITTED = 35 * CLINE,
  C_ST_RELEASED = 36 * CLINE,
  C_ST_REFRESHED = 37 * CLINE,
  C_MESH_NEXT = 38 * CLINE,  // next update-set block a mesh pass hands out (beyond one per CTA)
  C_N_TOUCHED1 = 39 * CLINE,  // buckets collected by an odd-numbered integrate call (touched_count)
  C_ST_REFUPD = 40 * CLINE,  // reference-count updates of the mesh passes
  C_COUNT = 41 * CLINE
};

// Count of the buckets integrate call `frame` collects.  Calls alternate between two counters,
// so that a call can empty the next call's counter at its start while its own is read.
__host__ __device__ constexpr int touched_count(uint32_t frame) { return (frame & 1u) ? C_N_TOUCHED1 : C_N_TOUCHED; }

// Stack top of the free runs of L triangle slots (L = 1..5).
__host__ __device__ constexpr int run_top(int L) { return C_RUN_TOP0 + (L - 1) * CLINE; }


struct FrameParams {
  const float* depth;     // the frame's depth in device memory, read after the collection
  const float* depth_in;  // what the collection reads: depth itself, or mapped pinned host memory
  float* depth_copy;      // null, or where the collection copies depth_in (then depth == depth_copy)
  int W, H;
  float fx, fy, cx, cy;
  float rfx, rfy;  // 1 / fx and 1 / fy, rounded to float (IEEE division on the host)
  float Twc[12];  // rows of [R | t], camera -> world
  float Tcw[12];  // world -> camera
  uint32_t frame;  // number of the integrate call (from 1, consecutive), set by the host
};

struct Ctl {
  int c[C_COUNT];
  FrameParams fp;
};

// Plain-old-data view of a volume passed by value to every kernel.
struct Vol {
  float l, mu, eps, wmax;
  float ibs;  // 1 / (l * 8), the block side's reciprocal rounded to float (IEEE division on the host)
  uint32_t hmask;
  int max_blocks, max_vertices, max_triangles;
  int run_cap[5];
  int list_cap_touched, list_cap_update, list_cap_dead, list_cap_deadrun;

  uint64_t* keys;
  int* vals;
  uint32_t* stamp;
  uint32_t* ustamp;

  int4* bkey;
  int* nbr;
  int* bntri;
  int* bnvert;
  uint8_t* bnear;
  uint32_t* bepoch;
  uint32_t* bborn;

  float2* tw;
  uint8_t* code_eff;
  uint8_t* code_prev;
  uint8_t* vmask;
  int* edge_vtx;  // wide layout: per voxel the vertex ids of its 3 owned edges
  int* edge_rec;  // compact layout: per voxel the index of its edge record, -1 none
  int* erec;      // edge records: 3 vertex ids each (-1 none)
  int* rec_free;  // free stack of edge records
  int* dead_rec;  // spare records of lost claims (recycled by gc)
  int* tri_base;

  float4* vrec;  // vertex v: position vrec[2 v], normal vrec[2 v + 1]
  int* vref;
  uint32_t* vedge;

  int4* tris;

  const uint4* tri_table;  // mesh tables: packed triangles, edge masks, halo pairs (MESH_TABLE_UINT4)

  int* blk_free;
  int* vtx_free;
  int* run_free[5];

  int4* touched;      // blocks collected by this integrate call: {key low, key high, block or -1, bucket}
  int* update;        // update-set blocks
  int* dead;          // zero-reference vertex ids
  int2* deadrun;      // released triangle runs (start, length)

  // differentiable path (null unless allocated): per voxel the integrations since the
  // checkpoint, the checkpoint weight and dL/dd; the blocks each recorded call collected
  // (drec[drec_off[f] .. drec_off[f + 1]) for recorded call f)
  uint16_t* dcnt;
  float* dwck;
  float* dgrad;
  int* drec;
  int* drec_off;

  Ctl* ctl;
};

// ------------------------------------------------------------------ cube tables
// Corners in Bourke order; edge k joins the owner corner EDGE_LO[k] to EDGE_HI[k].
__constant__ int8_t c_corner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                      {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
// owner corner offset and axis of each cube edge
__constant__ int8_t c_edge_owner[12][4] = {{0, 0, 0, 0}, {1, 0, 0, 1}, {0, 1, 0, 0}, {0, 0, 0, 1},
                                           {0, 0, 1, 0}, {1, 0, 1, 1}, {0, 1, 1, 0}, {0, 0, 1, 1},
                                           {0, 0, 0, 2}, {1, 0, 0, 2}, {1, 1, 0, 2}, {0, 1, 0, 2}};
__constant__ uint8_t c_ntri[256];
__constant__ uint8_t c_tri[256][15];
__constant__ uint16_t c_edgemask[256];
// regular cube types of Sec. V-F, in the paper's order
__constant__ uint8_t c_regular[6] = {0xCC, 0x33, 0x99, 0x66, 0xF0, 0x0F};

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ int floordiv8(int g) { return g >> 3; }  // arithmetic shift = floor

__device__ __forceinline__ uint64_t pack_key(int x, int y, int z) {
  return ((uint64_t)(uint32_t)(x + KEY_BIAS) << 42) | ((uint64_t)(uint32_t)(y + KEY_BIAS) << 21) |
         (uint64_t)(uint32_t)(z + KEY_BIAS);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // murmur3 finaliser
  z = (z ^ (z >> 33)) * 0xFF51AFD7ED558CCDull;
  z = (z ^ (z >> 33)) * 0xC4CEB9FE1A85EC53ull;
  return z ^ (z >> 33);
}

// Which capacity ran out (the first one, kept beside the status; values of the C ABI's
// vm_pool enum).
enum PoolCode { P_NONE = 0, P_BLOCKS, P_VERTICES, P_TRIANGLES, P_COLLECTED_LIST, P_UPDATE_LIST, P_DEAD_VERTEX_LIST,
                P_DEAD_RUN_LIST, P_FREE_STACK, P_HASH, P_EDGE_RECORDS };
__device__ __forceinline__ void set_status(const Vol& V, int st, int pool = P_NONE) {
  atomicCAS(&V.ctl->c[C_STATUS], 0, st);
  if (pool != P_NONE) atomicCAS(&V.ctl->c[C_STATUS_POOL], 0, pool);
}
__device__ __forceinline__ int list_pool_code(int c_count) {
  return (c_count == C_N_TOUCHED || c_count == C_N_TOUCHED1)
             ? P_COLLECTED_LIST
             : (c_count == C_N_UPDATE
                    ? P_UPDATE_LIST
                    : (c_count == C_N_DEADREC ? P_EDGE_RECORDS
                                              : (c_count == C_N_DEADRUN ? P_DEAD_RUN_LIST : P_DEAD_VERTEX_LIST)));
}

// Hash lookup: bucket holding `key`, or -1, and its value (loaded with the key, so a hit at
// the first probe costs one round trip).  Linear probing, at most hmask+1 probes.
__device__ __forceinline__ int hash_find(const Vol& V, uint64_t key, int& val) {
  uint32_t s = (uint32_t)mix64(key) & V.hmask;
  val = -1;
  for (uint32_t p = 0; p <= V.hmask; ++p) {
    const uint64_t k = __ldcg(&V.keys[s]);
    const int v = __ldcg(&V.vals[s]);
    if (k == key) {
      val = v;
      return (int)s;
    }
    if (k == KEY_EMPTY) return -1;
    s = (s + 1) & V.hmask;
  }
  return -1;
}

// Block index of block key (x, y, z), or -1.
__device__ __forceinline__ int find_block(const Vol& V, int x, int y, int z) {
  int blk;
  return hash_find(V, pack_key(x, y, z), blk) < 0 ? -1 : blk;
}

// Pop of `stride` consecutive ids per calling lane from a free stack of run starts backed
// by a bump range, aggregated over the lanes that call it together.  Pops and pushes of
// one stack never share a kernel.  The part of a pop the stack cannot supply is added back
// to the top at once, so the top returns to >= 0 when the pops end and no kernel has to
// clamp it.  Returns -1 (and sets POOL_FULL) when the pool is exhausted.
__device__ __forceinline__ int pool_pop(const Vol& V, int* stack, int c_top, int c_bump, int cap, int stride = 1,
                                        int pool = P_VERTICES) {
  cg::coalesced_group g = cg::coalesced_threads();
  int n = (int)g.size(), rank = (int)g.thread_rank();
  int old = 0, bump0 = 0, from_stack = 0;
  if (rank == 0) {
    old = atomicSub(&V.ctl->c[c_top], n);
    from_stack = old <= 0 ? 0 : (old < n ? old : n);
    if (from_stack < n) {
      bump0 = atomicAdd(&V.ctl->c[c_bump], (n - from_stack) * stride);
      atomicAdd(&V.ctl->c[c_top], n - from_stack);
    }
  }
  old = g.shfl(old, 0);
  from_stack = g.shfl(from_stack, 0);
  bump0 = g.shfl(bump0, 0);
  int id;
  if (rank < from_stack) {
    id = __ldcg(&stack[old - 1 - rank]);
  } else {
    long long b = (long long)bump0 + (long long)(rank - from_stack) * stride;
    if (b + stride > cap) {
      set_status(V, ST_POOL_FULL, pool);
      id = -1;
    } else {
      id = (int)b;
    }
  }
  return id;
}

// Push of one id per calling lane, aggregated over the lanes that call it together.
__device__ __forceinline__ void pool_push(const Vol& V, int* stack, int c_top, int cap, int id) {
  cg::coalesced_group g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&V.ctl->c[c_top], (int)g.size());
  base = g.shfl(base, 0) + (int)g.thread_rank();
  if (base < cap) stack[base] = id;
  else set_status(V, ST_POOL_FULL, P_FREE_STACK);
}

// Append to a work list, aggregated over the calling lanes; false (and POOL_FULL) on overflow.
template <typename T>
__device__ __forceinline__ bool list_push(const Vol& V, T* list, int c_count, int cap, T value) {
  cg::coalesced_group g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&V.ctl->c[c_count], (int)g.size());
  base = g.shfl(base, 0) + (int)g.thread_rank();
  if (base < cap) {
    list[base] = value;
    return true;
  }
  set_status(V, ST_POOL_FULL, list_pool_code(c_count));
  return false;
}

// Add `v` to a counter, aggregated over the calling lanes.
__device__ __forceinline__ void counter_add(const Vol& V, int c, int v) {
  cg::coalesced_group g = cg::coalesced_threads();
  int s = cg::reduce(g, v, cg::plus<int>());
  if (g.thread_rank() == 0 && s != 0) atomicAdd(&V.ctl->c[c], s);
}

// Byte-granular atomic OR / AND on a u8 array (through the enclosing 32-bit word).
__device__ __forceinline__ uint8_t atomic_or_u8(uint8_t* p, uint8_t bits) {
  uintptr_t a = reinterpret_cast<uintptr_t>(p);
  unsigned* w = reinterpret_cast<unsigned*>(a & ~uintptr_t(3));
  int sh = (int)(a & 3) * 8;
  return (uint8_t)(atomicOr(w, (unsigned)bits << sh) >> sh);
}
__device__ __forceinline__ uint8_t atomic_and_u8(uint8_t* p, uint8_t bits) {
  uintptr_t a = reinterpret_cast<uintptr_t>(p);
  unsigned* w = reinterpret_cast<unsigned*>(a & ~uintptr_t(3));
  int sh = (int)(a & 3) * 8;
  return (uint8_t)(atomicAnd(w, ~((unsigned)(uint8_t)~bits << sh)) >> sh);
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization
// may start while the previous kernel drains; it waits here (the hardware grid-dependency
// wait, which returns once the previous grid has completed and its memory is visible)
// before reading anything that kernel produced.  Without such a dependency it returns at
// once.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Let the next kernel in the stream be launched early (it still waits for this grid).
__device__ __forceinline__ void allow_dependent_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }


}  // namespace vmk
