// Mesh maintenance: cube types (Sec. V-B), refinement (Sec. V-F, Eqs. 3-5), edge-owned
// vertices (Sec. V-C, Sec. IV), triangulation with type-change reuse (Sec. V-D) and the
// reference counts that drive recycling (Sec. V-E), in one pass over the update set.
//
// One CTA per update-set block (persistent loop), in stages separated by barriers so that
// every stage is wide (one thread per cube, per edge or per changed cube) and no thread
// walks a long chain of dependent memory operations:
//   a. stage the 10^3 voxel halo (the block, local 0..7, plus the +x/+y/+z neighbours'
//      voxels at local 8..9) in shared memory as d, NaN where W = 0, with 16-byte loads;
//      every cube type, and every vertex an edge of these cubes can need, is computed from
//      it.  The block's own cube bytes and run slots are loaded first, the edge slots that
//      carry a vertex (its vertex-flag bytes tell which) with the neighbours' halo voxels;
//      the vertex ids go to shared memory;
//   b. per cube: type (and refinement), previous type; the block's edges that carry a
//      vertex are marked for a refresh; cubes whose effective type changes go to a shared
//      list and take a rank among the block's new runs of their length; the edges their new
//      triangles use are marked for a claim unless the block's own staged slot shows the
//      vertex;
//   c. count the claim and refresh edges per bitmap word (stage d locates the j-th of each
//      from the counts);
//   d. independent work in warp-sized units of one kind, so that the lanes of a warp take
//      one path and the chains of different warps overlap: one pop per run length of all
//      the block's new runs and one reservation of recycling-list slots for the released
//      runs; per claim edge its vertex, created on first use -- the first thread to claim
//      the edge pops an id and publishes it with atomicCAS on the owner's edge slot; a
//      thread that loses the race takes the winner's id and returns its own through the
//      recycling list, so nobody waits and every vertex exists once; per released run the
//      old triangles cleared and the vertices of the edges the cube stops using listed as
//      recycling candidates (their references dropped); per refresh edge the vertex's
//      position and normal from the new TSDF;
//   e. the released runs queued for recycling; per changed cube its new run (from the pop
//      and its rank), its new triangles written, and each of its edges' reference change.
// Reference counts (a vertex's degree, Sec. V-E) move once per edge whose use changes: by
// (triangles of the new type using the edge) - (triangles of the old type using it), with
// reductions nobody waits for; gc recycles exactly the listed candidates whose count is zero
// (its claim CAS(0, -1) skips the others).  On the floor workload that is 2.4x fewer atomics
// than one per triangle corner, and the L2 atomics were the mesh pass's largest cost.
// The paper resolves concurrent vertex creation with an atomic first-claimer lock or with
// grouped serial launches (Sec. V-C); publishing the id with the claim replaces both.
#pragma once

#include "vmesh_device.cuh"

namespace vmk {

enum MeshMode { M_UPDATE = 1, M_REFINE = 2 };

constexpr int MESH_THREADS = 128;
constexpr int HALO = 10;  // local voxel coordinates 0..9 on each axis
constexpr int HALO_N = HALO * HALO * HALO;
constexpr int OWNERS = 9 * 9 * 9;  // owner voxels (local 0..8) of the block's cubes' edges
constexpr int EDGE_SLOTS = OWNERS * 3;
constexpr int EDGE_WORDS = (EDGE_SLOTS + 31) / 32;

// Owner voxel offset and axis of cube edge k (the c_edge_owner table), 5 bits per edge in an
// immediate: bit 0 x offset, bit 1 y offset, bit 2 z offset, bits 3-4 axis.  Edge ids vary
// per thread, and divergent reads of a __constant__ table would serialize across the warp.
constexpr uint64_t EDGE_OWNER_BITS = 0x94e30619a440920ull;
__device__ __forceinline__ int owner_bits(int k) { return (int)((EDGE_OWNER_BITS >> (5 * k)) & 31); }

// Packed triangle table: per cube type, 15 edge ids of 4 bits (triangle t, corner j at bit
// 4 * (3 t + j)) and the triangle count in bits 60..63.
__device__ __forceinline__ int packed_ntri(uint64_t w) { return (int)(w >> 60); }
__device__ __forceinline__ int packed_edge(uint64_t w, int t, int j) { return (int)((w >> (4 * (3 * t + j))) & 15); }

// CTAs per SM, bounded by registers (64) and shared memory (23-25 KB).  Nine (56 registers,
// possible with the default record's 23 KB) measured no faster.
__host__ __device__ constexpr int mesh_ctas_per_sm(bool compact) { return compact ? 8 : 8; }
constexpr int HALO_PAIRS = 244;      // 16-byte pairs of neighbour voxels in the halo (488 voxels)
constexpr int MESH_TABLE_UINT4 = 192;  // 256 packed triangle words, 256 edge masks, 256 pair codes

// The halo's neighbour voxels as pairs adjacent along x (X, X + 1 at halo row Y, Z), packed
// X | Y << 4 | Z << 8: rows y, z < 8 take x = 8..9 from the +x neighbour; the 36 rows with y
// or z at 8..9 take x = 0..9 in five pairs.  Entries past HALO_PAIRS are 0.
__host__ __device__ inline void halo_pairs(uint16_t* out) {
  int i = 0;
  for (int z = 0; z < 8; ++z)
    for (int y = 0; y < 8; ++y) out[i++] = (uint16_t)(8 | y << 4 | z << 8);
  for (int r = 0; r < 36; ++r) {
    const int Y = r < 16 ? 8 + (r & 1) : (r - 16) % 10, Z = r < 16 ? r >> 1 : 8 + (r - 16) / 10;
    for (int s = 0; s < 5; ++s) out[i++] = (uint16_t)(2 * s | Y << 4 | Z << 8);
  }
  for (; i < 256; ++i) out[i] = 0;
}

template <bool CE>
struct __align__(16) MeshSmem {
  float halo[HALO_N];  // d of the voxel, NaN where W = 0 or its block is absent
  alignas(16) uint64_t tri64[256];
  alignas(16) uint16_t emask[256];  // the cube edges each type's triangles use (bit k: edge k)
  alignas(16) uint16_t pairs[256];  // the halo's neighbour voxel pairs (halo_pairs)
  alignas(16) uint64_t euse[256];   // per type, triangles using each cube edge (edge_use)
  int nb[8];
  int dtri;
  int nchg, ndr;               // changed cubes, released runs
  int unext;                   // next free unit of stage d
  int next[2];                 // the CTA's next update-set block (alternating slots)
  int nrun[5];           // new runs per length L = 1..5 (stage b), then their pop (stage d):
  int run_old[5], run_fs[5], run_bump[5];  // stack top seen, entries taken from it, first bump slot
  int dr_base;                             // first recycling-list slot of the released runs
  uint16_t chg_cube[BV];                   // changed cubes of the block
  uint8_t chg_new[BV], chg_old[BV];
  union {
    struct {                  // from stage b2 on:
      uint16_t rrank[BV];     // per changed cube, its rank among the block's new runs of its length
      uint16_t rel[BV];       // changed cubes (list slots) with a released run
    } ch;
    struct {                  // stages a-b: per halo row (y, z), bit x: d < 0, |d| < eps, unusable
      uint32_t neg[HALO * HALO], sml[HALO * HALO], inv[HALO * HALO];
    } rm;
  } u;
  int chg_base[BV];                        // run of the released triangles, -1 none
  unsigned cmark[EDGE_WORDS];  // edges the new triangles use whose vertex may be missing (claims)
  unsigned lmark[EDGE_WORDS];  // the block's own edges that carry a vertex
  unsigned rmark[EDGE_WORDS];  // lmark without cmark: the refreshes
  int ccount[EDGE_WORDS];      // per word, the claim | refresh << 16 bits of the words before it in its row of 32
  int wtot[3];                 // per row of 32 words, its claim | refresh << 16 bits
  alignas(16) int rec[CE ? BV : 4];        // compact layout: the block's edge records (voxel -> record, -1 none)
  int evid[EDGE_SLOTS];                    // vertex id per edge slot (own slots from stage a)
};
// members written or read with 16-byte vector accesses
static_assert(offsetof(MeshSmem<false>, tri64) % 16 == 0 && offsetof(MeshSmem<true>, tri64) % 16 == 0, "tri64");
static_assert(offsetof(MeshSmem<false>, emask) % 16 == 0 && offsetof(MeshSmem<true>, emask) % 16 == 0, "emask");
static_assert(offsetof(MeshSmem<false>, pairs) % 16 == 0 && offsetof(MeshSmem<true>, pairs) % 16 == 0, "pairs");
static_assert(offsetof(MeshSmem<true>, rec) % 16 == 0, "rec");

// Eqs. 3-5: snap a disturbed raw type to the nearest admissible regular type.  `small` has
// bit k set when |d(c_k)| < eps, so a regular type is admissible iff every corner where it
// differs from the raw type is in `small`.
__device__ __forceinline__ int refine_type(int raw, int prev, int small) {
  // an empty or full cube is 4 flips from every regular type: never snapped
  if (raw == 0 || raw == 255 || __popc(raw ^ prev) > 3) return raw;
  int best = -1, bestd = 99;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    // regular types of Sec. V-F in the paper's order: 0xCC 0x33 0x99 0x66 0xF0 0x0F
    const int rj = (int)((0x0FF0669933CCull >> (8 * j)) & 0xFF);
    const int diff = raw ^ rj;
    const int dh = __popc(diff);
    if (dh <= 3 && (diff & ~small) == 0 && dh < bestd) {
      best = rj;
      bestd = dh;
    }
  }
  return best >= 0 ? best : raw;
}

// Bourke corner offsets as bit patterns (folded into shared-memory addresses when k is a
// compile-time constant): corner k is (x, y, z) = (0x66 >> k & 1, 0xCC >> k & 1, 0xF0 >> k & 1).
__device__ __forceinline__ constexpr int corner_x(int k) { return (0x66 >> k) & 1; }
__device__ __forceinline__ constexpr int corner_y(int k) { return (0xCC >> k) & 1; }
__device__ __forceinline__ constexpr int corner_z(int k) { return (0xF0 >> k) & 1; }

// Loads issued where they are written (volatile asm keeps them ahead of the next barrier),
// so they travel while the halo is staged.
__device__ __forceinline__ uint32_t ld_early_u32(const uint8_t* p) {
  uint32_t v;
  asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int4 ld_early_i4(const int* p) {
  int4 v;
  asm volatile("ld.global.cg.v4.s32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ int ld_early_s32(const int* p) {
  int v;
  asm volatile("ld.global.cg.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_early_f4(const float2* p) {
  float4 v;
  asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}

// atomicAdd(p, v) returning the old value when `on`, else no access and 0; predicated rather
// than branched, so that a run of them issues back to back.
__device__ __forceinline__ int atom_add_if(int* p, int v, bool on) {
  int old = 0;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q atom.global.add.s32 %0, [%1], %2;\n\t}"
      : "+r"(old)
      : "l"(p), "r"(v), "r"((unsigned)on)
      : "memory");
  return old;
}

// Halo entry of a voxel (d, W): d, or NaN where W = 0.
__device__ __forceinline__ float halo_value(float d, float w) { return w > 0.0f ? d : __int_as_float(0x7fc00000); }

__device__ __forceinline__ float halo_at(const float* halo, int x, int y, int z) {
  return halo[x + HALO * y + HALO * HALO * z];
}

// Bit j of a 4-bit value to bit 8 j (bit i lands on i + 7 m for the terms m of the product,
// which is a multiple of 8 only for m = i).
__device__ __forceinline__ uint32_t spread4(uint32_t x) { return (x * 0x00204081u) & 0x01010101u; }

// The 8-bit corner masks (Bourke corner order) of 4 cubes consecutive along x, byte j for the
// cube at x0 + j, from 5-bit windows (bits x0 .. x0 + 4) of the masks of the 4 halo rows through
// their corners: w00 row (y, z), w10 (y + 1, z), w01 (y, z + 1), w11 (y + 1, z + 1).  Corners
// 0, 1 are bits (x, x + 1) of row 00; 3, 2 of row 10; 4, 5 of row 01; 7, 6 of row 11.
__device__ __forceinline__ uint32_t cube_bits4(uint32_t w00, uint32_t w10, uint32_t w01, uint32_t w11) {
  return spread4(w00 & 15u) | spread4((w00 >> 1) & 15u) << 1 | spread4((w10 >> 1) & 15u) << 2 |
         spread4(w10 & 15u) << 3 | spread4(w01 & 15u) << 4 | spread4((w01 >> 1) & 15u) << 5 |
         spread4((w11 >> 1) & 15u) << 6 | spread4(w11 & 15u) << 7;
}

// Vertex on the owned edge g -> g + e_a (Sec. V-C) at global voxel (gx, gy, gz), from the
// values d0 = d(g), d1 = d(g + e_a) and, for the two axes b != a, q0[b] = d(g + e_b),
// q1[b] = d(g + e_a + e_b) (NaN where W = 0 or the block is absent): t = d0 / (d0 - d1) (0.5
// when equal), clamped to [-1, 2] so refined cubes extrapolate boundedly; position
// g l + t l e_a; normal = normalised gradient of the owner cube's trilinear interpolant at
// the vertex, component b != a from the corners g+e_b and g+e_a+e_b, 0 when either is
// unusable.  Both mesh passes evaluate vertices through this one function (one operation
// order).
__device__ __forceinline__ void vertex_from_values(float l, int gx, int gy, int gz, int a, float d0, float d1,
                                                   const float* q0, const float* q1, float4* pos, float4* nrm) {
  float t = d0 == d1 ? 0.5f : d0 / (d0 - d1);
  if (t < -1.0f) t = -1.0f;
  if (t > 2.0f) t = 2.0f;
  const int ga = a == 0 ? gx : (a == 1 ? gy : gz);
  const float pa = (float)ga * l + t * l;
  const float p[3] = {a == 0 ? pa : (float)gx * l, a == 1 ? pa : (float)gy * l, a == 2 ? pa : (float)gz * l};
  float n[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (b == a) {
      n[b] = d1 - d0;
      continue;
    }
    n[b] = (!isnan(q0[b]) && !isnan(q1[b])) ? (1.0f - t) * (q0[b] - d0) + t * (q1[b] - d1) : 0.0f;
  }
  const float len = sqrtf((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
  *pos = make_float4(p[0], p[1], p[2], 0.0f);
  if (len > 0.0f) *nrm = make_float4(n[0] / len, n[1] / len, n[2] / len, 0.0f);
  else *nrm = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// The vertex of the owned edge of the voxel at halo coordinates (x, y, z) (0..8) along a,
// from the halo of the block whose key is `key`.
__device__ __forceinline__ void edge_vertex(const float* halo, float l, int4 key, int x, int y, int z, int a,
                                            float4* pos, float4* nrm) {
  const int ax = a == 0, ay = a == 1, az = a == 2;
  const float d0 = halo_at(halo, x, y, z);
  const float d1 = halo_at(halo, x + ax, y + ay, z + az);
  float q0[3], q1[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int bx = b == 0, by = b == 1, bz = b == 2;
    q0[b] = b == a ? 0.0f : halo_at(halo, x + bx, y + by, z + bz);
    q1[b] = b == a ? 0.0f : halo_at(halo, x + ax + bx, y + ay + by, z + az + bz);
  }
  vertex_from_values(l, key.x * BS + x, key.y * BS + y, key.z * BS + z, a, d0, d1, q0, q1, pos, nrm);
}

// Id of the vertex on the edge owned by the voxel at halo coordinates (x, y, z) (0..8) along
// axis a, creating it on first use.  Returns -1 when the vertex pool is exhausted.
// `own`: the voxel is the block's own and its slot, loaded in stage a, held no vertex, so
// the claim starts at once (a vertex another block's pass made since makes the claim fail
// and is taken like any winner's).
// A free vertex carries the reference count -1.  The claimer publishes the popped id with
// atomicCAS and then adds 1, while threads that found the id add their references: the
// additions commute, so the count is exact when the pass ends, and no fence is needed.
// A thread that loses the claim resets its spare id to an unattached zero-reference vertex
// and hands it to gc.
// CE: the compact layout (edge records) rather than three vertex ids per voxel.
template <bool CE>
__device__ __forceinline__ int vertex_of_edge(const Vol& V, const MeshSmem<CE>& S, int x, int y, int z, int a,
                                              bool own, bool& claimed) {
  claimed = false;
  const int ob = S.nb[(x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2)];
  if (ob < 0) return -1;  // cannot happen for a valid cube
  const int ov = (x & 7) + 8 * (y & 7) + 64 * (z & 7);
  const uint32_t e = (uint32_t)ob * EPB + ov * 3 + a;
  const size_t vox = (size_t)ob * BV + ov;
  int* slot;
  if constexpr (CE) {
    // the owner voxel's edge record (claimed like a vertex: first claimer publishes a record
    // from the pool, whose three slots are -1 there; a loser's spare record goes to gc);
    // voxels of the block itself have theirs staged in shared memory
    int rec = own ? S.rec[ov] : __ldcg(&V.edge_rec[vox]);
    if (rec < 0) {
      const int spare = pool_pop(V, V.rec_free, C_REC_TOP, C_REC_BUMP, V.max_vertices, 1, P_EDGE_RECORDS);
      if (spare < 0) return -1;
      rec = atomicCAS(&V.edge_rec[vox], -1, spare);
      if (rec >= 0) list_push(V, V.dead_rec, C_N_DEADREC, V.max_vertices, spare);
      else rec = spare;
    }
    slot = V.erec + (size_t)rec * 3 + a;
  } else {
    slot = V.edge_vtx + (size_t)e;
  }
  if (!own) {
    const int vid = __ldcg(slot);
    if (vid >= 0) return vid;
  }
  const int mine = pool_pop(V, V.vtx_free, C_VTX_TOP, C_VTX_BUMP, V.max_vertices);
  if (mine < 0) return -1;
  const int old = atomicCAS(slot, -1, mine);
  if (old >= 0) {  // another thread claimed the edge first
    V.vref[mine] = 0;
    V.vedge[mine] = NO_EDGE;
    list_push(V, V.dead, C_N_DEAD, V.list_cap_dead, mine);
    return old;
  }
  atomicAdd(&V.vref[mine], 1);  // -1 (free) -> 0, plus the references added by others
  V.vedge[mine] = e;
  atomic_or_u8(V.vmask + vox, (uint8_t)(1 << a));
  atomicAdd(&V.bnvert[ob], 1);
  claimed = true;  // the caller writes its position and normal
  return mine;
}

// Reserve `cnt` consecutive slots of a shared counter for every lane of the (full, converged)
// warp, with one shared atomic per warp; returns this lane's first slot.
__device__ __forceinline__ int warp_reserve(int* counter, int cnt) {
  const int lane = threadIdx.x & 31;
  int x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  int base = 0;
  if (lane == 31 && x > 0) base = atomicAdd(counter, x);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + x - cnt;
}

// Shared-memory slot of the edge owned by the voxel at halo coordinates (x, y, z) along a.
__device__ __forceinline__ int edge_slot(int x, int y, int z, int a) { return ((z * 9 + y) * 9 + x) * 3 + a; }

// Edge slot of the i-th set bit of a shared bitmap (the claim bits: sh = 0, the refresh bits:
// sh = 16): its row of 32 words from the rows' totals, then a binary search of the word among the
// row's prefixes, then the bit within the word.
__device__ __forceinline__ int nth_marked(const unsigned* mark, const int* count, const int* wtot, int sh, int i) {
  const int t0 = (wtot[0] >> sh) & 0xFFFF, t1 = t0 + ((wtot[1] >> sh) & 0xFFFF);
  const int r = (i >= t0) + (i >= t1);
  const int j = i - (r == 0 ? 0 : (r == 1 ? t0 : t1));
  int lo = 32 * r, hi = min(32 * r + 31, EDGE_WORDS - 1);
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (((count[mid] >> sh) & 0xFFFF) <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo * 32 + (int)__fns(mark[lo], 0, j - ((count[lo] >> sh) & 0xFFFF) + 1);
}

// Counters a mesh pass accumulates per CTA.
struct MeshCounts {
  int changed = 0, created = 0, emitted = 0, released = 0, refreshed = 0, dtri = 0, refupd = 0;
};

// Per type, how many of its triangles use each cube edge (3 bits per edge: a fan apex edge is
// used by up to 5).
__device__ __forceinline__ uint64_t edge_use(uint64_t w) {
  uint64_t u = 0;
  for (int q = 0; q < 3 * packed_ntri(w); ++q) u += 1ull << (3 * packed_edge(w, q / 3, q % 3));
  return u;
}
__device__ __forceinline__ int use_of(uint64_t u, int k) { return (int)((u >> (3 * k)) & 7); }

// Vertex id of cube edge k in the old triangles tr (the cube's run under its old type, packed
// triangle word w, nold triangles); -1 if no old triangle uses the edge.
__device__ __forceinline__ int old_vertex(const int4* tr, uint64_t w, int nold, int k) {
  int v = -1;
#pragma unroll
  for (int q = 14; q >= 0; --q) {
    const int t = q / 3, j = q % 3;
    if (t < nold && packed_edge(w, t, j) == k) v = j == 0 ? tr[t].x : (j == 1 ? tr[t].y : tr[t].z);
  }
  return v;
}

// One update-set block `blk` through stages a-e, the calling CTA of MESH_THREADS with its
// shared staging area S (S.tri64 already holds the triangle table).
template <bool CE>
__device__ __forceinline__ void mesh_block(const Vol& V, MeshSmem<CE>& S, int blk, int mode, MeshCounts& cnt) {
  const float eps = V.eps, l = V.l;
  // ---- a. this thread's 4 cubes (c0..c0+3, consecutive along x): their voxels, type,
  //         previous-type and vertex-flag bytes, run slots (and, compact layout, edge
  //         records), all loaded before anything waits; the addresses are valid for a freed
  //         block too
  const int c0 = 4 * threadIdx.x;  // MESH_THREADS * 4 == BV
  const size_t ci0 = (size_t)blk * BV + c0;
  const int nbv = (threadIdx.x >= 1 && threadIdx.x < 8) ? ld_early_s32(&V.nbr[blk * 16 + threadIdx.x]) : blk;
  const float4 h01 = ld_early_f4(V.tw + ci0), h23 = ld_early_f4(V.tw + ci0 + 2);
  const uint32_t eff_w = ld_early_u32(V.code_eff + ci0);
  const uint32_t vm_w = ld_early_u32(V.vmask + ci0);
  const uint32_t prev_w = (mode & M_UPDATE) ? eff_w : ld_early_u32(V.code_prev + ci0);
  const int4 tb4 = ld_early_i4(V.tri_base + ci0);
  const int4 rec4 = CE ? ld_early_i4(V.edge_rec + ci0) : make_int4(-1, -1, -1, -1);  // compact: edge records
  const int4 key = V.bkey[blk];
  if (key.w < 0) return;  // freed since it joined the set (uniform over the CTA)
  if (threadIdx.x < 8) S.nb[threadIdx.x] = nbv;
  if (threadIdx.x == 0) {
    S.dtri = 0;
    S.nchg = 0;
    S.ndr = 0;
    S.unext = 0;
  }
  if (threadIdx.x < 5) S.nrun[threadIdx.x] = 0;
  for (int w = threadIdx.x; w < EDGE_WORDS; w += MESH_THREADS) {
    S.cmark[w] = 0;
    S.lmark[w] = 0;
  }
  for (int w = threadIdx.x; w < 3 * HALO * HALO; w += MESH_THREADS) (&S.u.rm.neg[0])[w] = 0;
  __syncthreads();
  // the neighbours' 488 halo voxels as 244 pairs adjacent along x (16 bytes each)
  float4 qn[2];
  int qx[2], qrow[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int i = threadIdx.x + k * MESH_THREADS;
    qrow[k] = -1;
    qx[k] = 0;
    qn[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < HALO_PAIRS) {
      const int pc = S.pairs[i];
      const int X = pc & 15, Y = (pc >> 4) & 15, Z = pc >> 8;
      const int b = S.nb[(X >> 3) | ((Y >> 3) << 1) | ((Z >> 3) << 2)];
      qx[k] = X;
      qrow[k] = Y + HALO * Z;
      if (b >= 0)
        qn[k] = __ldcg(reinterpret_cast<const float4*>(V.tw + (size_t)b * BV + (X & 7) + 8 * (Y & 7) + 64 * (Z & 7)));
    }
  }
  // the vertex ids of the 4 voxels' edges that carry one (vertex-flag bits), issued with the
  // neighbour halo loads; the other slots hold no vertex
  int ev[12];
  {
    const int rv[4] = {rec4.x, rec4.y, rec4.z, rec4.w};
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const bool live = (vm_w >> (8 * (q / 3) + q % 3)) & 1u;
      if constexpr (CE)
        ev[q] = live && rv[q / 3] >= 0 ? __ldcg(&V.erec[(size_t)rv[q / 3] * 3 + q % 3]) : -1;
      else
        ev[q] = live ? __ldcg(&V.edge_vtx[(ci0 + q / 3) * 3 + q % 3]) : -1;
    }
    if (CE) reinterpret_cast<int4*>(S.rec)[threadIdx.x] = rec4;  // read from stage d on
  }
  const int cx = c0 & 7, cy = (c0 >> 3) & 7, cz = c0 >> 6;
  const int row = cy + HALO * cz;  // the halo row of the thread's 4 voxels
  {
    const float hv[4] = {halo_value(h01.x, h01.y), halo_value(h01.z, h01.w), halo_value(h23.x, h23.y),
                         halo_value(h23.z, h23.w)};
    float* h = S.halo + cx + HALO * row;
    uint32_t ng = 0, sm = 0, iv = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[j] = hv[j];
      ng |= (uint32_t)(hv[j] < 0.0f) << j;
      sm |= (uint32_t)(fabsf(hv[j]) < eps) << j;
      iv |= (uint32_t)isnan(hv[j]) << j;
    }
    if (ng) atomicOr(&S.u.rm.neg[row], ng << cx);
    if (sm) atomicOr(&S.u.rm.sml[row], sm << cx);
    if (iv) atomicOr(&S.u.rm.inv[row], iv << cx);
    // the 4 voxels' 12 edge slots are consecutive in the shared slot array
    int* es = S.evid + edge_slot(cx, cy, cz, 0);
#pragma unroll
    for (int q = 0; q < 12; ++q) es[q] = ev[q];
  }
#pragma unroll
  for (int k = 0; k < 2; ++k)
    if (qrow[k] >= 0) {
      const float a = halo_value(qn[k].x, qn[k].y), b = halo_value(qn[k].z, qn[k].w);
      S.halo[qx[k] + HALO * qrow[k]] = a;
      S.halo[qx[k] + 1 + HALO * qrow[k]] = b;
      const uint32_t ng = (uint32_t)(a < 0.0f) | ((uint32_t)(b < 0.0f) << 1);
      const uint32_t sm = (uint32_t)(fabsf(a) < eps) | ((uint32_t)(fabsf(b) < eps) << 1);
      const uint32_t iv = (uint32_t)isnan(a) | ((uint32_t)isnan(b) << 1);
      if (ng) atomicOr(&S.u.rm.neg[qrow[k]], ng << qx[k]);
      if (sm) atomicOr(&S.u.rm.sml[qrow[k]], sm << qx[k]);
      if (iv) atomicOr(&S.u.rm.inv[qrow[k]], iv << qx[k]);
    }
  __syncthreads();
  // ---- b. cube types, refresh marks, changed-cube list (the type, previous-type and
  //         vertex-flag bytes of the 4 cubes move as 32-bit words)
  {
    if (mode & M_UPDATE) *reinterpret_cast<uint32_t*>(V.code_prev + ci0) = eff_w;
    // edges of the 4 voxels that carry a vertex: 12 consecutive bits of the refresh bitmap
    uint32_t live12 = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) live12 |= ((vm_w >> (8 * j)) & 7u) << (3 * j);
    if (live12) {
      const int es0 = edge_slot(cx, cy, cz, 0), sh = es0 & 31;
      atomicOr(&S.lmark[es0 >> 5], live12 << sh);
      if (sh > 20) atomicOr(&S.lmark[(es0 >> 5) + 1], live12 >> (32 - sh));
    }
    // the 4 cubes' raw types at once from 5-bit windows of the row masks (bit k of a cube's
    // byte is corner k's test: the same decisions as comparing the corners' d one by one); a
    // cube with an unusable corner is invalid, type 0
    const uint32_t raw4 = cube_bits4((S.u.rm.neg[row] >> cx) & 31u, (S.u.rm.neg[row + 1] >> cx) & 31u,
                                     (S.u.rm.neg[row + HALO] >> cx) & 31u, (S.u.rm.neg[row + HALO + 1] >> cx) & 31u);
    const uint32_t i4 = cube_bits4((S.u.rm.inv[row] >> cx) & 31u, (S.u.rm.inv[row + 1] >> cx) & 31u,
                                   (S.u.rm.inv[row + HALO] >> cx) & 31u, (S.u.rm.inv[row + HALO + 1] >> cx) & 31u);
    uint32_t bad = i4 | (i4 >> 4);
    bad |= bad >> 2;
    bad = (bad | (bad >> 1)) & 0x01010101u;
    uint32_t new_w = raw4 & ~(bad * 0xFFu);
    // refinement (Eqs. 3-5) of the valid cubes with a sign change: types 0 and 255 are never
    // snapped
    if (mode & M_REFINE) {
      uint32_t need = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t t = (new_w >> (8 * j)) & 0xFFu;
        need |= (uint32_t)(t != 0u && t != 0xFFu) << j;
      }
      if (need) {
        const uint32_t s4 = cube_bits4((S.u.rm.sml[row] >> cx) & 31u, (S.u.rm.sml[row + 1] >> cx) & 31u,
                                       (S.u.rm.sml[row + HALO] >> cx) & 31u, (S.u.rm.sml[row + HALO + 1] >> cx) & 31u);
#pragma unroll 1
        for (uint32_t m = need; m; m &= m - 1) {
          const int j = __ffs(m) - 1;
          const int e = refine_type((int)((new_w >> (8 * j)) & 0xFFu), (int)((prev_w >> (8 * j)) & 0xFFu),
                                    (int)((s4 >> (8 * j)) & 0xFFu));
          new_w = (new_w & ~(0xFFu << (8 * j))) | ((uint32_t)e << (8 * j));
        }
      }
    }
    if (new_w != eff_w) *reinterpret_cast<uint32_t*>(V.code_eff + ci0) = new_w;
    // the changed cubes into the shared list: one shared atomic per warp
    unsigned chm = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) chm |= (((new_w ^ eff_w) >> (8 * j)) & 0xFFu) ? 1u << j : 0u;
    const int nc = __popc(chm);
    cnt.changed += nc;
    int slot = warp_reserve(&S.nchg, nc);
    while (chm) {
      const int j = __ffs(chm) - 1;
      chm &= chm - 1;
      const int eff_old = (eff_w >> (8 * j)) & 0xFF;
      S.chg_cube[slot] = (uint16_t)(c0 + j);
      S.chg_new[slot] = (uint8_t)((new_w >> (8 * j)) & 0xFF);
      S.chg_old[slot] = (uint8_t)eff_old;
      S.chg_base[slot] = packed_ntri(S.tri64[eff_old]) > 0 ? (j == 0 ? tb4.x : (j == 1 ? tb4.y : (j == 2 ? tb4.z : tb4.w))) : -1;
      ++slot;
    }
  }
  __syncthreads();
  const int nchg = S.nchg;
  // ---- b2. per changed cube (spread over the CTA, wherever the changes cluster): its rank
  //          among the new runs of its length, its released run listed, the edges its new
  //          triangles use marked
  {
    int dtri = 0;
    for (int q = threadIdx.x; q < nchg; q += MESH_THREADS) {
      const int e = S.chg_new[q];
      const int nold = packed_ntri(S.tri64[S.chg_old[q]]), nnew = packed_ntri(S.tri64[e]);
      if (S.chg_base[q] >= 0) S.u.ch.rel[atomicAdd(&S.ndr, 1)] = (uint16_t)q;
      if (nnew > 0) S.u.ch.rrank[q] = (uint16_t)atomicAdd(&S.nrun[nnew - 1], 1);
      dtri += nnew - nold;
    }
    if (dtri) atomicAdd(&S.dtri, dtri);
    // the edges the new triangles use, a (changed cube, cube edge) pair per thread: an existing
    // vertex of the block's own voxels needs nothing more (its slot is staged); a neighbour's
    // edge or a missing vertex needs a claim in stage d
    for (int i = threadIdx.x; i < 12 * nchg; i += MESH_THREADS) {
      const int q = i / 12, k = i - 12 * q;
      if (!((S.emask[S.chg_new[q]] >> k) & 1)) continue;
      const int c = S.chg_cube[q];
      const int ob = owner_bits(k);
      const int ox = (c & 7) + (ob & 1), oy = ((c >> 3) & 7) + ((ob >> 1) & 1), oz = (c >> 6) + ((ob >> 2) & 1);
      const int es = edge_slot(ox, oy, oz, ob >> 3);
      if ((ox | oy | oz) >= 8 || S.evid[es] < 0) atomicOr(&S.cmark[es >> 5], 1u << (es & 31));
    }
  }
  __syncthreads();
  // ---- c. count the claim and refresh edges per bitmap word, a thread per word (warps 0-2, one
  //         row of 32 words each, both counts packed as claim | refresh << 16: a row holds at
  //         most 1024 of each), scanned within the row; stage d locates the j-th of each from
  //         the rows' totals and the prefixes
  static_assert(EDGE_WORDS <= 96 && EDGE_WORDS * 32 < 0x10000, "stage c: three rows, 16-bit counts");
  if (threadIdx.x < 96) {
    const int w = threadIdx.x, lane = w & 31;
    unsigned cm = 0, rm = 0;
    if (w < EDGE_WORDS) {
      cm = S.cmark[w];
      rm = S.lmark[w] & ~cm;
      S.rmark[w] = rm;
    }
    const int c = __popc(cm) | (__popc(rm) << 16);
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (w < EDGE_WORDS) S.ccount[w] = x - c;
    if (lane == 31) S.wtot[w >> 5] = x;
  }
  __syncthreads();
  // ---- d. independent work in units of up to 32 items of one kind, so that the lanes of a
  //         warp take the same path: unit 0 pops the block's new runs of length 1-5 (lanes
  //         0-4) and reserves the released runs' recycling slots (lane 5); then the claims,
  //         the releases (round-trip chains) and the refreshes (arithmetic only), 32 per
  //         unit.  Each warp starts on the unit of its index and takes the next free unit
  //         when it is done, so the chains of different warps overlap
  const int tall = S.wtot[0] + S.wtot[1] + S.wtot[2];
  const int ncand = tall & 0xFFFF, nref = tall >> 16, ndr = S.ndr;
  const int uc = (ncand + 31) >> 5, ur = (ndr + 31) >> 5;
  const int nunits = 1 + uc + ur + ((nref + 31) >> 5);
  const int lane = threadIdx.x & 31;
  for (int u = threadIdx.x >> 5; u < nunits;) {
    int es = -1, vid = -1;
    if (u == 0) {
      if (lane < 5) {
        const int n = S.nrun[lane], L = lane + 1;
        if (n > 0) {  // n runs of L slots: from the free stack, the rest from the bump range
          const int old = atomicSub(&V.ctl->c[run_top(L)], n);
          const int fs = old <= 0 ? 0 : (old < n ? old : n);
          int bump0 = 0;
          if (fs < n) {
            bump0 = atomicAdd(&V.ctl->c[C_TRI_BUMP], (n - fs) * L);
            atomicAdd(&V.ctl->c[run_top(L)], n - fs);  // top back to >= 0 (as pool_pop)
          }
          S.run_old[lane] = old;
          S.run_fs[lane] = fs;
          S.run_bump[lane] = bump0;
        }
      } else if (lane == 5 && ndr > 0) {
        S.dr_base = atomicAdd(&V.ctl->c[C_N_DEADRUN], ndr);
      }
    } else if (u > uc && u <= uc + ur) {
      // the whole warp takes part (lanes past the last released run with nothing to release),
      // so the recycling-list reservation below is one warp-wide scan and one atomic
      const int i = ((u - 1 - uc) << 5) + lane;
      int obase = -1, nold = 0;
      if (i < ndr) {
        const int q = S.u.ch.rel[i];
        obase = S.chg_base[q];
        nold = packed_ntri(S.tri64[S.chg_old[q]]);
      }
      int4 tr[5];
#pragma unroll
      for (int t = 0; t < 5; ++t) tr[t] = t < nold ? __ldcg(&V.tris[obase + t]) : make_int4(-1, -1, -1, -1);
      // the edges the cube stops using: their references dropped, their vertices listed as
      // recycling candidates (one recycling-list reservation for the warp)
      const int q = i < ndr ? S.u.ch.rel[i] : 0;
      const uint64_t wold = i < ndr ? S.tri64[S.chg_old[q]] : 0ull;
      const unsigned cand = i < ndr ? (unsigned)(S.emask[S.chg_old[q]] & ~S.emask[S.chg_new[q]]) : 0u;
      const uint64_t uo = i < ndr ? S.euse[S.chg_old[q]] : 0ull;
      for (int t = 0; t < nold; ++t) V.tris[obase + t] = make_int4(-1, -1, -1, -1);
      const int nz = __popc(cand);
      int incl = nz;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int slot = 0;
      if (lane == 31 && incl > 0) slot = atomicAdd(&V.ctl->c[C_N_DEAD], incl);
      slot = __shfl_sync(0xffffffffu, slot, 31) + incl - nz;
      for (unsigned m = cand; m; m &= m - 1, ++slot) {
        const int k = __ffs(m) - 1;
        const int v = old_vertex(tr, wold, nold, k);  // -1 only after the vertex pool ran out
        if (v >= 0) {
          atomicAdd(&V.vref[v], -use_of(uo, k));
          ++cnt.refupd;
        }
        if (slot < V.list_cap_dead) V.dead[slot] = v;  // gc skips -1
        else set_status(V, ST_POOL_FULL, P_DEAD_VERTEX_LIST);
      }
      cnt.released += nold;
    } else {
      const bool claim = u <= uc;
      const int i = ((claim ? u - 1 : u - 1 - uc - ur) << 5) + lane;
      if (i < (claim ? ncand : nref)) {
        es = nth_marked(claim ? S.cmark : S.rmark, S.ccount, S.wtot, claim ? 0 : 16, i);
        if (claim) {
          const int o = es / 3;
          const int x = o % 9, y = (o / 9) % 9, z = o / 81;
          bool fresh;
          vid = vertex_of_edge<CE>(V, S, x, y, z, es - 3 * o, (x | y | z) < 8, fresh);
          S.evid[es] = vid;
          cnt.created += fresh;
          if (!fresh) es = -1;
        } else {
          vid = S.evid[es];  // an existing vertex of the block: position and normal refreshed
          if (vid < 0) es = -1;
          cnt.refreshed += es >= 0;
        }
      }
    }
    if (es >= 0) {  // a created or refreshed vertex
      const int o = es / 3;
      float4 p, nn;
      edge_vertex(S.halo, l, key, o % 9, (o / 9) % 9, o / 81, es - 3 * o, &p, &nn);
      V.vrec[2 * (size_t)vid] = p;  // position and normal: one 32-byte sector
      V.vrec[2 * (size_t)vid + 1] = nn;
    }
    __syncwarp();
    int next = 0;
    if (lane == 0) next = atomicAdd(&S.unext, 1) + MESH_THREADS / 32;
    u = __shfl_sync(0xffffffffu, next, 0);
  }
  __syncthreads();
  // ---- e. the released runs queued for recycling; per changed cube its new run, the new
  //         triangles and their references
  for (int r = threadIdx.x; r < ndr; r += MESH_THREADS) {
    const int q = S.u.ch.rel[r], slot = S.dr_base + r;
    if (slot < V.list_cap_deadrun) V.deadrun[slot] = make_int2(S.chg_base[q], packed_ntri(S.tri64[S.chg_old[q]]));
    else set_status(V, ST_POOL_FULL, P_DEAD_RUN_LIST);
  }
  for (int q = threadIdx.x; q < nchg; q += MESH_THREADS) {
    const int c = S.chg_cube[q];
    const uint64_t tw64 = S.tri64[S.chg_new[q]];
    const int nt = packed_ntri(tw64);
    // the new run: popped from the free stack (a run start, never negative) or the bump range
    // (none past the pool's end); whether the cube got one is known before the stack entry
    // arrives, so the reference updates below do not wait for it
    int base = -1;
    bool got = false;
    if (nt > 0) {
      const int r = S.u.ch.rrank[q], fs = S.run_fs[nt - 1];
      if (r < fs) {
        base = __ldcg(&V.run_free[nt - 1][S.run_old[nt - 1] - 1 - r]);
        got = true;
      } else {
        const long long b = (long long)S.run_bump[nt - 1] + (long long)(r - fs) * nt;
        if (b + nt > V.max_triangles) set_status(V, ST_POOL_FULL, P_TRIANGLES);
        else base = (int)b;
        got = base >= 0;
      }
    }
    const int ci = blk * BV + c;
    const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
    // the references of the edges the new type uses: (its triangles using the edge, none when
    // its run could not be had) - (the old type's, when it had a run); the edges only the old
    // type used were handled by the release
    {
      const uint64_t un = got ? S.euse[S.chg_new[q]] : 0ull;
      const uint64_t uo = S.chg_base[q] >= 0 ? S.euse[S.chg_old[q]] : 0ull;
#pragma unroll 1
      for (unsigned m = S.emask[S.chg_new[q]]; m; m &= m - 1) {
        const int k = __ffs(m) - 1;
        const int d = use_of(un, k) - use_of(uo, k);
        if (d == 0) continue;
        const int ob = owner_bits(k);
        const int v = S.evid[edge_slot(x + (ob & 1), y + ((ob >> 1) & 1), z + ((ob >> 2) & 1), ob >> 3)];
        if (v < 0) continue;
        atomicAdd(&V.vref[v], d);
        ++cnt.refupd;
      }
    }
    V.tri_base[ci] = base;
    if (base < 0) continue;
    cnt.emitted += nt;
#pragma unroll 1
    for (int t = 0; t < nt; ++t) {
      int vs[3];
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        const int ob = owner_bits(packed_edge(tw64, t, jj));
        vs[jj] = S.evid[edge_slot(x + (ob & 1), y + ((ob >> 1) & 1), z + ((ob >> 2) & 1), ob >> 3)];
      }
      if (vs[0] < 0 || vs[1] < 0 || vs[2] < 0) {  // vertex pool exhausted
        set_status(V, ST_POOL_FULL, P_VERTICES);
        V.tris[base + t] = make_int4(-1, -1, -1, ci);
        continue;
      }
      V.tris[base + t] = make_int4(vs[0], vs[1], vs[2], ci);
    }
  }
  if (threadIdx.x == 0 && S.dtri) {
    atomicAdd(&V.bntri[blk], S.dtri);
    cnt.dtri += S.dtri;
  }
  __syncthreads();
}

// The mesh tables into shared memory (whole CTA; the first barrier of the first block
// orders the copy before any use).
template <bool CE>
__device__ __forceinline__ void mesh_tables(MeshSmem<CE>& S, const uint4* tables) {
  for (int i = threadIdx.x; i < MESH_TABLE_UINT4; i += MESH_THREADS) {
    const uint4 w = tables[i];
    if (i < 128) reinterpret_cast<uint4*>(S.tri64)[i] = w;
    else if (i < 160) reinterpret_cast<uint4*>(S.emask)[i - 128] = w;
    else reinterpret_cast<uint4*>(S.pairs)[i - 160] = w;
  }
  for (int c = threadIdx.x; c < 256; c += MESH_THREADS) S.euse[c] = edge_use(reinterpret_cast<const uint64_t*>(tables)[c]);
}

// Flush a CTA's counters into the volume's statistics.
__device__ __forceinline__ void mesh_flush(const Vol& V, MeshCounts& c) {
  if (c.changed) counter_add(V, C_ST_CHANGED, c.changed);
  if (c.emitted) counter_add(V, C_ST_EMITTED, c.emitted);
  if (c.released) counter_add(V, C_ST_RELEASED, c.released);
  if (c.refreshed) counter_add(V, C_ST_REFRESHED, c.refreshed);
  if (c.refupd) counter_add(V, C_ST_REFUPD, c.refupd);
  if (c.dtri) counter_add(V, C_LIVE_TRIS, c.dtri);
  if (c.created) {
    counter_add(V, C_LIVE_VERTS, c.created);
    counter_add(V, C_ST_NEW_VERTS, c.created);
  }
  c = MeshCounts();
}

// Statistics of a mesh pass over n update-set blocks (one thread, at the start).
__device__ __forceinline__ void mesh_begin(const Vol& V, int n) {
  V.ctl->c[C_ST_UPDATE_BLOCKS] = n;
  reinterpret_cast<unsigned*>(V.ctl->c)[C_ST_MESHED] += (unsigned)n;  // wraps modulo 2^32
}

// Every update-set block, one per CTA iteration.
// mode: M_UPDATE (types from the current TSDF; t_{i-1} := previous effective type; refresh
// the positions and normals of the block's existing vertices), M_REFINE (Eqs. 3-5 with the
// stored t_{i-1}).
template <bool CE>
__global__ void __launch_bounds__(MESH_THREADS, mesh_ctas_per_sm(CE)) k_mesh(Vol V, int mode) {
  __shared__ MeshSmem<CE> S;
  mesh_tables(S, V.tri_table);
  grid_dependency_wait();
  const int n = min(__ldcg(&V.ctl->c[C_N_UPDATE]), V.list_cap_update);
  if (blockIdx.x == 0 && threadIdx.x == 0) mesh_begin(V, n);
  MeshCounts cnt;
  // one block per CTA, then the blocks beyond the grid go to whichever CTA is free first
  // (the cost of a block varies tenfold with its changes)
  for (int i = blockIdx.x, k = 0; i < n; k ^= 1) {
    mesh_block<CE>(V, S, V.update[i], mode, cnt);
    if (threadIdx.x == 0) S.next[k] = (int)gridDim.x + atomicAdd(&V.ctl->c[C_MESH_NEXT], 1);
    __syncthreads();
    i = S.next[k];
  }
  mesh_flush(V, cnt);
  allow_dependent_launch();
}

}  // namespace vmk
