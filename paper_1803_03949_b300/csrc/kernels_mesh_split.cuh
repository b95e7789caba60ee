// Mesh maintenance in two kernels per pass (Secs. IV, V-B..V-F): the same state changes as
// the one-kernel pass of kernels_mesh.cuh (the batched step still uses that one), split
// where the work changes shape.
//
// k_mesh_types streams the update set, one block per CTA iteration (two barriers a block):
//   the 10^3 halo of d (NaN where W = 0) staged in shared memory; per cube the type (Sec. V-B) and, in a refining pass, Eqs. 3-5 (Sec. V-F);
//   the previous / effective type bytes written; every existing vertex on the block's own
//   edges re-evaluated from the new TSDF (Sec. V-C, "otherwise an update"); each cube whose
//   effective type changed and whose old or new type has triangles appended to the pass's
//   changed-cube list (cube id, new and old type): staged in shared memory and reserved in the
//   list once per CTA and flush, since a counter that every warp of the pass hits serialises
//   at its L2 slice.
// k_mesh_cubes takes the changed cubes, one lane each, all of them in flight together:
//   its old triangles released (Sec. V-D: a cube keeps its triangles only while its type is
//   unchanged; reference counts down, zero-reference vertices and the run listed for gc,
//   Sec. V-E); the vertices of its new triangles' edges looked up in the owners' edge slots
//   and created where missing (the first claimer pops an id and publishes it with atomicCAS,
//   Sec. V-C; a loser takes the winner's id and hands its spare to gc); a run of the new
//   triangle count popped and the triangles written with their references.
// Splitting removes the per-block chain of six barrier-separated stages: the streaming half
// has two round trips per block and no atomics on the pools, and the changed cubes (a few per
// cent of the update set's cubes) run their round-trip chains in parallel instead of within
// their block's CTA.
#pragma once

#include "kernels_mesh.cuh"

namespace vmk {

// ------------------------------------------------------------------ pass 1: types
constexpr int MT_THREADS = 128;  // 4 cubes per thread (MT_THREADS * 4 == BV)
constexpr int MT_WARPS = MT_THREADS / 32;
constexpr int MT_CTAS_PER_SM = 10;
constexpr int MT_STAGE = 1024;  // changed-cube records a CTA stages (2 blocks' worth at most)
constexpr int MT_STAGE_BLOCKS = 64;  // blocks whose records a stage holds

// Shared state of the types pass.  The halo (floats, for the vertex refresh) and the row masks
// (for the types) are written only after a block's first barrier, which every thread reaches
// once it has finished the previous block; the neighbour row, the masks and the per-block
// counters are cleared before that barrier and alternate between two slots.
struct __align__(16) TypesSmem {
  float halo[HALO_N];               // d of the voxel, NaN where W = 0 or its block is absent
  alignas(16) uint16_t pairs[256];  // the halo's neighbour voxel pairs (halo_pairs)
  alignas(16) uint8_t ntri[256];    // triangles of each cube type
  int nb[2][8];                     // the block and its upper neighbours
  // per halo row (y, z), bit x: d < 0, |d| < eps, unusable (W = 0 or block absent)
  uint32_t rmask[2][3][HALO * HALO];
  uint32_t rnear[256];              // per raw type, the regular types within 3 flips (refine_near)
  int bdtri[2];                     // the block's triangle-count change
  int nlive[2];                     // the block's own edges that carry a vertex
  int ev[12 * MT_THREADS];          // their vertex ids, per thread and edge (strided)
  uint16_t rlist[EPB];              // the block's live own edges (voxel * 3 + axis)
  // staged changed-cube records: stage-block index << 25 | cube << 16 | old type << 8 | new type
  // (the list record's second word is the low 16 bits: new | old << 8)
  uint32_t rec[MT_STAGE];
  int sblk[MT_STAGE_BLOCKS];        // the staged blocks' indices
  int nrec, nsblk, base;
  int red[3][MT_WARPS];             // end-of-kernel counter sums
};

// Per raw type: the regular types of Sec. V-F within Hamming distance 3, nearest first, ties
// in the paper's order (3 bits each from bit 3, their count in bits 0..2).
__device__ __forceinline__ uint32_t refine_near(int raw) {
  uint32_t out = 0;
  int n = 0;
  for (int dist = 0; dist <= 3; ++dist)
    for (int j = 0; j < 6; ++j) {
      const int rj = (int)((0x0FF0669933CCull >> (8 * j)) & 0xFF);
      if (__popc(raw ^ rj) == dist) out |= (uint32_t)j << (3 + 3 * n++);
    }
  return out | (uint32_t)n;
}

// Eqs. 3-5 as refine_type, with the candidates of `raw` taken from its refine_near entry: the
// first admissible one is the nearest (ties: the paper's order), the same choice.
__device__ __forceinline__ int refine_type_near(int raw, int prev, int small, uint32_t near) {
  if (raw == 0 || raw == 255 || __popc(raw ^ prev) > 3) return raw;
  const int n = (int)(near & 7u);
  for (int i = 0; i < n; ++i) {
    const int j = (int)((near >> (3 + 3 * i)) & 7u);
    const int rj = (int)((0x0FF0669933CCull >> (8 * j)) & 0xFF);
    if (((raw ^ rj) & ~small) == 0) return rj;
  }
  return raw;
}

// The 8-bit cube mask (Bourke corner order) of the cube at x from the masks of the 4 halo
// rows through its corners: (y, z), (y + 1, z), (y, z + 1), (y + 1, z + 1).
__device__ __forceinline__ int cube_bits(uint32_t r00, uint32_t r10, uint32_t r01, uint32_t r11, int x) {
  const uint32_t t00 = (r00 >> x) & 3u, t10 = (r10 >> x) & 3u, t01 = (r01 >> x) & 3u, t11 = (r11 >> x) & 3u;
  // corners 0, 1 at (x, x+1) of row 00; 3, 2 of row 10; 4, 5 of row 01; 7, 6 of row 11
  return (int)(t00 | ((t10 & 1u) << 3) | ((t10 >> 1) << 2) | (t01 << 4) | ((t11 & 1u) << 7) | ((t11 >> 1) << 6));
}

// Copy the CTA's staged records into the pass's list (the whole CTA; one reservation).
__device__ __forceinline__ void flush_records(const Vol& V, TypesSmem& S) {
  const int nrec = S.nrec;
  __syncthreads();  // every thread has read the stage's size
  if (threadIdx.x == 0) S.base = atomicAdd(&V.ctl->c[C_N_CHANGED], nrec);
  __syncthreads();
  const int base = S.base;
  for (int i = threadIdx.x; i < nrec; i += MT_THREADS) {
    const uint32_t r = S.rec[i];
    const int ci = S.sblk[r >> 25] * BV + (int)((r >> 16) & 0x1FF);
    if (base + i < V.list_cap_chg) V.chg[base + i] = make_int2(ci, (int)(r & 0xFFFF));
    else set_status(V, ST_POOL_FULL, P_CHANGED_LIST);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S.nrec = 0;
    S.nsblk = 0;
  }
  __syncthreads();
}

// One update-set block through the types pass (the calling CTA; `buf` alternates per block).
// Accumulates this thread's changed cubes, refreshed vertices and triangle-count change.
template <bool CE>
__device__ __forceinline__ void types_block(const Vol& V, TypesSmem& S, int buf, int blk, int mode, int& changed,
                                            int& refreshed, int& dtri_all) {
  const float eps = V.eps, l = V.l;
  // this thread's 4 cubes (c0..c0+3, consecutive along x): voxels, type, previous-type and
  // vertex-flag bytes (and, compact layout, edge records), loaded before anything waits
  const int c0 = 4 * threadIdx.x;
  const size_t ci0 = (size_t)blk * BV + c0;
  const int nbv = (threadIdx.x >= 1 && threadIdx.x < 8) ? ld_early_s32(&V.nbr[blk * 16 + threadIdx.x]) : blk;
  const float4 h01 = ld_early_f4(V.tw + ci0), h23 = ld_early_f4(V.tw + ci0 + 2);
  const uint32_t eff_w = ld_early_u32(V.code_eff + ci0);
  const uint32_t vm_w = ld_early_u32(V.vmask + ci0);
  const uint32_t prev_w = (mode & M_UPDATE) ? eff_w : ld_early_u32(V.code_prev + ci0);
  const int4 rec4 = CE ? ld_early_i4(V.edge_rec + ci0) : make_int4(-1, -1, -1, -1);
  const int4 key = __ldcg(&V.bkey[blk]);
  if (key.w < 0) return;  // freed since it joined the set (uniform over the CTA)
  float* halo = S.halo;
  int* nb = S.nb[buf];
  uint32_t* rneg = S.rmask[buf][0];
  uint32_t* rsml = S.rmask[buf][1];
  uint32_t* rinv = S.rmask[buf][2];
  if (threadIdx.x < 8) nb[threadIdx.x] = nbv;
  for (int i = threadIdx.x; i < 3 * HALO * HALO; i += MT_THREADS) S.rmask[buf][0][i] = 0u;
  if (threadIdx.x == 0) {
    S.bdtri[buf] = 0;
    S.nlive[buf] = 0;
  }
  __syncthreads();
  // the neighbours' 488 halo voxels as 244 pairs adjacent along x (16 bytes each)
  float4 qn[2];
  int qx[2], qrow[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int i = threadIdx.x + k * MT_THREADS;
    qrow[k] = -1;
    qx[k] = 0;
    qn[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < HALO_PAIRS) {
      const int pc = S.pairs[i];
      const int X = pc & 15, Y = (pc >> 4) & 15, Z = pc >> 8;
      const int b = nb[(X >> 3) | ((Y >> 3) << 1) | ((Z >> 3) << 2)];
      qrow[k] = Y + HALO * Z;
      qx[k] = X;
      if (b >= 0)
        qn[k] = __ldcg(reinterpret_cast<const float4*>(V.tw + (size_t)b * BV + (X & 7) + 8 * (Y & 7) + 64 * (Z & 7)));
    }
  }
  // the vertex ids of the 4 voxels' edges that carry one (vertex-flag bits), issued with the
  // neighbour halo loads
  int ev[12];
  uint32_t live12 = 0;
  {
    const int rv[4] = {rec4.x, rec4.y, rec4.z, rec4.w};
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const bool live = (vm_w >> (8 * (q / 3) + q % 3)) & 1u;
      if constexpr (CE)
        ev[q] = live && rv[q / 3] >= 0 ? __ldcg(&V.erec[(size_t)rv[q / 3] * 3 + q % 3]) : -1;
      else
        ev[q] = live ? __ldcg(&V.edge_vtx[(ci0 + q / 3) * 3 + q % 3]) : -1;
      live12 |= (uint32_t)live << q;
    }
  }
  // the block's edges that carry a vertex, listed for the refresh (spread over the CTA after
  // the next barrier: a thread's own edges would leave the warps' lanes unevenly loaded)
  {
#pragma unroll
    for (int q = 0; q < 12; ++q) S.ev[q * MT_THREADS + threadIdx.x] = ev[q];
    const int nl = __popc(live12);
    if (nl) {
      int pos = atomicAdd(&S.nlive[buf], nl);
      for (uint32_t m = live12; m; m &= m - 1) S.rlist[pos++] = (uint16_t)(3 * c0 + __ffs(m) - 1);
    }
  }
  // the halo and its row masks: this thread's 4 voxels, then its neighbour pairs
  const int cx = c0 & 7, cy = (c0 >> 3) & 7, cz = c0 >> 6;
  const int row = cy + HALO * cz;
  {
    const float hv[4] = {halo_value(h01.x, h01.y), halo_value(h01.z, h01.w), halo_value(h23.x, h23.y),
                         halo_value(h23.z, h23.w)};
    float* h = halo + cx + HALO * row;
    uint32_t ng = 0, sm = 0, iv = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[j] = hv[j];
      ng |= (uint32_t)(hv[j] < 0.0f) << j;
      sm |= (uint32_t)(fabsf(hv[j]) < eps) << j;
      iv |= (uint32_t)isnan(hv[j]) << j;
    }
    if (ng) atomicOr(&rneg[row], ng << cx);
    if (sm) atomicOr(&rsml[row], sm << cx);
    if (iv) atomicOr(&rinv[row], iv << cx);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k)
    if (qrow[k] >= 0) {
      const float a = halo_value(qn[k].x, qn[k].y), b = halo_value(qn[k].z, qn[k].w);
      halo[qx[k] + HALO * qrow[k]] = a;
      halo[qx[k] + 1 + HALO * qrow[k]] = b;
      const uint32_t ng = (uint32_t)(a < 0.0f) | ((uint32_t)(b < 0.0f) << 1);
      const uint32_t sm = (uint32_t)(fabsf(a) < eps) | ((uint32_t)(fabsf(b) < eps) << 1);
      const uint32_t iv = (uint32_t)isnan(a) | ((uint32_t)isnan(b) << 1);
      if (ng) atomicOr(&rneg[qrow[k]], ng << qx[k]);
      if (sm) atomicOr(&rsml[qrow[k]], sm << qx[k]);
      if (iv) atomicOr(&rinv[qrow[k]], iv << qx[k]);
    }
  __syncthreads();
  // cube types from the row masks (the type, previous-type and vertex-flag bytes of the 4
  // cubes move as words): bit k of a mask is corner k's test, the same decisions as comparing
  // the corners' d one by one
  if (mode & M_UPDATE) *reinterpret_cast<uint32_t*>(V.code_prev + ci0) = eff_w;
  uint32_t new_w = eff_w;
  {
    const uint32_t n00 = rneg[row], n10 = rneg[row + 1], n01 = rneg[row + HALO], n11 = rneg[row + HALO + 1];
    const uint32_t s00 = rsml[row], s10 = rsml[row + 1], s01 = rsml[row + HALO], s11 = rsml[row + HALO + 1];
    const uint32_t i00 = rinv[row], i10 = rinv[row + 1], i01 = rinv[row + HALO], i11 = rinv[row + HALO + 1];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int x = cx + j;
      const bool valid = cube_bits(i00, i10, i01, i11, x) == 0;
      const int raw = cube_bits(n00, n10, n01, n11, x);
      const int prev = (prev_w >> (8 * j)) & 0xFF;
      int e = valid ? raw : 0;
      if (valid && (mode & M_REFINE)) e = refine_type_near(raw, prev, cube_bits(s00, s10, s01, s11, x), S.rnear[raw]);
      new_w = (new_w & ~(0xFFu << (8 * j))) | ((uint32_t)e << (8 * j));
    }
  }
  if (new_w != eff_w) *reinterpret_cast<uint32_t*>(V.code_eff + ci0) = new_w;
  // changed cubes with triangles on either side staged for the pass's list
  unsigned chm = 0;
  int dtri = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int o = (eff_w >> (8 * j)) & 0xFF, nw = (new_w >> (8 * j)) & 0xFF;
    if (o != nw) {
      ++changed;
      const int a = S.ntri[o], b = S.ntri[nw];
      dtri += b - a;
      if (a + b > 0) chm |= 1u << j;
    }
  }
  const int nc = __popc(chm);
  const bool any = __syncthreads_or(nc != 0);  // also: every thread has read the masks
  if (any) {
    const int sb = S.nsblk;  // the block's stage index (stage flushed below before it fills)
    if (nc) {
      int slot = atomicAdd(&S.nrec, nc);
      while (chm) {
        const int j = __ffs(chm) - 1;
        chm &= chm - 1;
        const int o = (eff_w >> (8 * j)) & 0xFF, nw = (new_w >> (8 * j)) & 0xFF;
        S.rec[slot++] = (uint32_t)sb << 25 | (uint32_t)(c0 + j) << 16 | (uint32_t)o << 8 | (uint32_t)nw;
      }
    }
    if (dtri) atomicAdd(&S.bdtri[buf], dtri);
  }
  // the block's existing vertices (on its own edges) from the new TSDF, the list's entries
  // spread over the CTA's threads
  refreshed += __popc(live12);
  {
    const int nlive = S.nlive[buf];
#pragma unroll 1
    for (int i = threadIdx.x; i < nlive; i += MT_THREADS) {
      const int e = S.rlist[i];
      const int v = e / 3, a = e - 3 * v;  // voxel of the block, axis
      float4 p, nn;
      edge_vertex(halo, l, key, v & 7, (v >> 3) & 7, v >> 6, a, &p, &nn);
      const int id = S.ev[(3 * (v & 3) + a) * MT_THREADS + (v >> 2)];
      V.vpos[id] = p;
      V.vnrm[id] = nn;
    }
  }
  dtri_all += dtri;
  if (any) {
    __syncthreads();  // the block's records and triangle-count change are staged
    if (threadIdx.x == 0) {
      if (S.bdtri[buf] != 0) atomicAdd(&V.bntri[blk], S.bdtri[buf]);
      S.sblk[S.nsblk] = blk;
      S.nsblk += 1;
    }
    __syncthreads();
    // room for another block's records (and its stage index)?
    if (S.nrec > MT_STAGE - BV || S.nsblk == MT_STAGE_BLOCKS) flush_records(V, S);
  }
}

// Every update-set block, one per CTA iteration (static stride; the next block's index is
// loaded a block ahead).  mode: M_UPDATE (t_{i-1} := previous effective type), M_REFINE
// (Eqs. 3-5 against the stored t_{i-1}).
template <bool CE>
__global__ void __launch_bounds__(MT_THREADS, MT_CTAS_PER_SM) k_mesh_types(Vol V, int mode) {
  __shared__ TypesSmem S;
  for (int i = threadIdx.x; i < 32; i += MT_THREADS) reinterpret_cast<uint4*>(S.pairs)[i] = V.tri_table[160 + i];
  for (int i = threadIdx.x; i < 256; i += MT_THREADS) {
    S.ntri[i] = (uint8_t)packed_ntri(reinterpret_cast<const uint64_t*>(V.tri_table)[i]);
    S.rnear[i] = refine_near(i);
  }
  if (threadIdx.x == 0) {
    S.nrec = 0;
    S.nsblk = 0;
  }
  grid_dependency_wait();
  const int n = min(__ldcg(&V.ctl->c[C_N_UPDATE]), V.list_cap_update);
  if (blockIdx.x == 0 && threadIdx.x == 0) mesh_begin(V, n);
  __syncthreads();  // the tables
  int changed = 0, refreshed = 0, dtri = 0;
  int blk = (int)blockIdx.x < n ? __ldcg(&V.update[blockIdx.x]) : -1;
  for (int i = blockIdx.x, k = 0; i < n; i += gridDim.x, k ^= 1) {
    const int next = i + (int)gridDim.x < n ? __ldcg(&V.update[i + gridDim.x]) : -1;
    types_block<CE>(V, S, k, blk, mode, changed, refreshed, dtri);
    blk = next;
  }
  __syncthreads();  // the last block's records are staged
  if (S.nrec > 0) flush_records(V, S);
  // the statistics, one atomic per CTA and counter
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = __reduce_add_sync(0xffffffffu, changed), r1 = __reduce_add_sync(0xffffffffu, refreshed),
            r2 = __reduce_add_sync(0xffffffffu, dtri);
  if (lane == 0) {
    S.red[0][warp] = r0;
    S.red[1][warp] = r1;
    S.red[2][warp] = r2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    int t = 0;
    for (int w = 0; w < MT_WARPS; ++w) t += S.red[threadIdx.x][w];
    const int c = threadIdx.x == 0 ? C_ST_CHANGED : (threadIdx.x == 1 ? C_ST_REFRESHED : C_LIVE_TRIS);
    if (t) atomicAdd(&V.ctl->c[c], t);
  }
  allow_dependent_launch();
}

// ------------------------------------------------------------------ pass 2: changed cubes
// A CTA takes the list in chunks of MC_THREADS consecutive entries, a lane per changed cube
// (consecutive entries mostly come from one block: they share edges and neighbour rows).  The
// chunk's missing vertices are deduplicated in a shared hash of edge ids, so each is claimed
// once per chunk, and every reservation on a pool or list (vertex ids, runs of each length,
// released-run and recycling-candidate list slots) is made once per chunk from a CTA-wide
// scan: a counter hit by every warp of the pass would serialise at its L2 slice.  A changed
// cube moves each vertex's reference count (its degree) by the change in how many of the cube's
// triangles use that vertex's edge, old type to new type, one reduction per edge whose use
// changes (about 2.4x fewer than one per triangle corner on the floor workload), and nobody
// waits for it; the vertices of the edges the cube stops using are listed as recycling
// candidates, and gc recycles exactly the candidates whose count is zero (its claim CAS(0, -1)
// skips the others).
constexpr int MC_THREADS = 128;
constexpr int MC_WARPS = MC_THREADS / 32;
constexpr int MC_CTAS_PER_SM = 6;
constexpr int MC_HASH = 2048;  // > 12 edges x MC_THREADS: an insert always finds a slot
constexpr int MC_HASH_LOG2 = 11;

// Quantities a chunk reserves, per warp: distinct missing edges (claims), recycling candidates,
// released runs, new runs of length 1..5.
enum ChunkQty { Q_CLAIM = 0, Q_CAND, Q_RUN_REL, Q_RUN1, Q_COUNT = Q_RUN1 + 5 };

struct __align__(16) CubesSmem {
  alignas(16) uint64_t tri64[256];
  alignas(16) uint16_t emask[256];
  alignas(16) uint64_t euse[256];  // per type, 3 bits per cube edge: triangles using the edge
  int sev[12 * MC_THREADS];  // per lane and cube edge: vertex id, -1 not used, <= -3 hash slot tag
  uint32_t hkey[MC_HASH];    // missing edge id + 1 (0 empty)
  int hval[MC_HASH];         // its vertex id once claimed
  uint32_t ulist[12 * MC_THREADS];  // distinct missing edges: hash slot | inserting lane << 16
  int nuniq;
  // per lane: its cube's block's neighbour row (slot 0, unused in the table, holds the block
  // itself), read by the claims
  alignas(16) int4 lr0[MC_THREADS];
  alignas(16) int4 lr1[MC_THREADS];
  int wq[Q_COUNT][MC_WARPS];  // per quantity: warp totals, then their exclusive prefixes
  int base[Q_COUNT];          // the chunk's first slot per quantity (pools: stack top seen)
  int from_stack[Q_COUNT];    // pools: entries the stack supplied; the rest from the bump range
  int bump[Q_COUNT];
  int red[4][MC_WARPS];
};

// Block index of the neighbour at offset o in {0,1}^3 (o = x | y << 1 | z << 2) from the
// block's neighbour-table row r0 (slots 0..3) and r1 (slots 4..7); slot 0 is the block itself.
__device__ __forceinline__ int nb_select(int blk, int4 r0, int4 r1, int o) {
  const int lo = o == 0 ? blk : (o == 1 ? r0.y : (o == 2 ? r0.z : r0.w));
  const int hi = o == 4 ? r1.x : (o == 5 ? r1.y : (o == 6 ? r1.z : r1.w));
  return o < 4 ? lo : hi;
}

// Location of the vertex id of the edge owned by voxel `vox` of block b along axis a.
// Compact layout: its edge record's slot; with `create`, a voxel without a record gets one
// (claimed like a vertex: the first claimer publishes a pooled record, whose slots are all -1
// there; a loser's spare goes to gc).  Null when no record exists (and none was made).
template <bool CE>
__device__ __forceinline__ int* edge_slot_ptr(const Vol& V, int b, int vox, int a, bool create) {
  if constexpr (CE) {
    int rec = __ldcg(&V.edge_rec[(size_t)b * BV + vox]);
    if (rec < 0 && create) {
      const int spare = pool_pop(V, V.rec_free, C_REC_TOP, C_REC_BUMP, V.max_vertices, 1, P_EDGE_RECORDS);
      if (spare < 0) return nullptr;
      rec = atomicCAS(&V.edge_rec[(size_t)b * BV + vox], -1, spare);
      if (rec >= 0) list_push(V, V.dead_rec, C_N_DEADREC, V.max_vertices, spare);
      else rec = spare;
    }
    return rec < 0 ? nullptr : V.erec + (size_t)rec * 3 + a;
  } else {
    return V.edge_vtx + ((size_t)b * BV + vox) * 3 + a;
  }
}

// The d value (NaN where W = 0 or the block is absent) at halo coordinates (X, Y, Z) in 0..9
// of block blk, whose upper neighbours are in r0, r1.
__device__ __forceinline__ float global_halo(const Vol& V, int blk, int4 r0, int4 r1, int X, int Y, int Z) {
  const int b = nb_select(blk, r0, r1, (X >> 3) | ((Y >> 3) << 1) | ((Z >> 3) << 2));
  if (b < 0) return __int_as_float(0x7fc00000);
  const float2 q = __ldcg(&V.tw[(size_t)b * BV + (X & 7) + 8 * (Y & 7) + 64 * (Z & 7)]);
  return halo_value(q.x, q.y);
}

// Edge id of the edge owned by voxel vox of block b along axis a (< 2^32 for 2^21 blocks).
__device__ __forceinline__ uint32_t edge_id(int b, int vox, int a) { return (uint32_t)b * EPB + vox * 3 + a; }

// The chunk's reservations (the whole CTA): per quantity the warps' totals in S.wq become
// exclusive prefixes, and one atomic per quantity (and pool) reserves the chunk's total.
__device__ __forceinline__ void chunk_reserve(const Vol& V, CubesSmem& S) {
  if (threadIdx.x < Q_COUNT) {
    const int q = threadIdx.x;
    int tot = 0;
    if (q == Q_CLAIM) {  // the distinct missing edges, taken by the CTA's threads in turn
      tot = S.nuniq;
    } else {
      for (int w = 0; w < MC_WARPS; ++w) {
        const int c = S.wq[q][w];
        S.wq[q][w] = tot;
        tot += c;
      }
    }
    int base = 0, fs = 0, bump = 0;
    if (tot > 0) {
      if (q == Q_RUN_REL || q == Q_CAND) {
        base = atomicAdd(&V.ctl->c[q == Q_RUN_REL ? C_N_DEADRUN : C_N_DEAD], tot);
      } else {  // a pool: vertex ids, or runs of length L (from the stack, then the bump range)
        const int L = q - Q_RUN1 + 1;
        const int ctop = q == Q_CLAIM ? C_VTX_TOP : run_top(L);
        const int cbump = q == Q_CLAIM ? C_VTX_BUMP : C_TRI_BUMP;
        const int stride = q == Q_CLAIM ? 1 : L;
        base = atomicSub(&V.ctl->c[ctop], tot);
        fs = base <= 0 ? 0 : (base < tot ? base : tot);
        if (fs < tot) {
          bump = atomicAdd(&V.ctl->c[cbump], (tot - fs) * stride);
          atomicAdd(&V.ctl->c[ctop], tot - fs);  // the top back to >= 0 (as pool_pop)
        }
      }
    }
    S.base[q] = base;
    S.from_stack[q] = fs;
    S.bump[q] = bump;
  }
}

// Id number r of the chunk's reservation on a pool (stack entries first, then the bump range
// in steps of `stride`); -1 (and POOL_FULL) when the pool is exhausted.
__device__ __forceinline__ int chunk_pool_id(const Vol& V, const CubesSmem& S, int q, const int* stack, int r,
                                             int stride, int cap, int pool) {
  if (r < S.from_stack[q]) return __ldcg(&stack[S.base[q] - 1 - r]);
  const long long b = (long long)S.bump[q] + (long long)(r - S.from_stack[q]) * stride;
  if (b + stride > cap) {
    set_status(V, ST_POOL_FULL, pool);
    return -1;
  }
  return (int)b;
}

// Exclusive prefix of `cnt` over the lanes that call together and one atomicAdd of their total
// on `counter` (by the first of them); returns this lane's first slot.
__device__ __forceinline__ int group_reserve(int* counter, int cnt) {
  cg::coalesced_group g = cg::coalesced_threads();
  const int incl = cg::inclusive_scan(g, cnt, cg::plus<int>());
  const int tot = g.shfl(incl, (int)g.size() - 1);
  int base = 0;
  if (g.thread_rank() == 0 && tot > 0) base = atomicAdd(counter, tot);
  return g.shfl(base, 0) + incl - cnt;
}

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

// Warp-exclusive prefix of x (full warp) and the warp's total, recorded for quantity q.
__device__ __forceinline__ int warp_prefix(CubesSmem& S, int q, int x) {
  const int lane = threadIdx.x & 31;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) S.wq[q][threadIdx.x >> 5] = incl;
  return incl - x;
}

// One distinct missing edge of a chunk (the i-th; `ent` = hash slot | inserting lane << 16):
// an id from the chunk's reservation published with atomicCAS on the owner's edge slot; the
// winner attaches the vertex and evaluates it from the new TSDF (the owner cube's corners lie in
// the inserting lane's block and its upper neighbours, whose indices are staged, so the voxel
// loads travel with the id's), a loser (another chunk claimed the edge first) takes the
// published id and hands its spare to gc.  The result goes to hval.  Returns whether a vertex
// was created.
template <bool CE>
__device__ __forceinline__ bool claim_edge(const Vol& V, CubesSmem& S, int i, uint32_t ent) {
  const int h = (int)(ent & 0xFFFFu), ln = (int)(ent >> 16);
  const uint32_t e = S.hkey[h] - 1u;
  const int b = (int)(e / EPB), rem = (int)(e - (uint32_t)b * EPB), vox = rem / 3, a = rem - 3 * vox;
  const int4 r0 = S.lr0[ln], r1 = S.lr1[ln];
  const int blk = r0.x;
  const int4 key = __ldcg(&V.bkey[blk]);
  // the owner block's offset from the inserting lane's block, hence the owner voxel's halo
  // coordinates (0..8) in that block's frame
  int o = 0;
#pragma unroll
  for (int k = 7; k >= 1; --k) o = nb_select(blk, r0, r1, k) == b ? k : o;
  const int x = (o & 1) * BS + (vox & 7), y = ((o >> 1) & 1) * BS + ((vox >> 3) & 7), z = ((o >> 2) & 1) * BS + (vox >> 6);
  const int id = chunk_pool_id(V, S, Q_CLAIM, V.vtx_free, i, 1, V.max_vertices, P_VERTICES);
  const int ax = a == 0, ay = a == 1, az = a == 2;
  const float d0 = global_halo(V, blk, r0, r1, x, y, z);
  const float d1 = global_halo(V, blk, r0, r1, x + ax, y + ay, z + az);
  float q0[3], q1[3];
#pragma unroll
  for (int bb = 0; bb < 3; ++bb) {
    const int bx = bb == 0, by = bb == 1, bz = bb == 2;
    q0[bb] = bb == a ? 0.0f : global_halo(V, blk, r0, r1, x + bx, y + by, z + bz);
    q1[bb] = bb == a ? 0.0f : global_halo(V, blk, r0, r1, x + ax + bx, y + ay + by, z + az + bz);
  }
  if (id < 0) {
    S.hval[h] = -1;
    return false;
  }
  int* sp = edge_slot_ptr<CE>(V, b, vox, a, true);
  const int prev = sp ? atomicCAS(sp, -1, id) : -3;
  if (prev != -1) {  // another chunk claimed the edge first (or no edge record could be made)
    S.hval[h] = prev >= 0 ? prev : -1;
    V.vref[id] = 0;
    V.vedge[id] = NO_EDGE;
    list_push(V, V.dead, C_N_DEAD, V.list_cap_dead, id);
    if (prev < -1) set_status(V, ST_POOL_FULL, P_EDGE_RECORDS);
    return false;
  }
  S.hval[h] = id;
  atomicAdd(&V.vref[id], 1);  // -1 (free) -> 0, plus the references added by others
  V.vedge[id] = e;
  atomic_or_u8(V.vmask + (size_t)b * BV + vox, (uint8_t)(1 << a));
  atomicAdd(&V.bnvert[b], 1);
  float4 p, nn;
  vertex_from_values(V.l, key.x * BS + x, key.y * BS + y, key.z * BS + z, a, d0, d1, q0, q1, &p, &nn);
  V.vpos[id] = p;
  V.vnrm[id] = nn;
  return true;
}

// One chunk of the changed-cube list: entries j0 .. j0 + MC_THREADS - 1 (< n), a lane each.
template <bool CE>
__device__ __forceinline__ void cubes_chunk(const Vol& V, CubesSmem& S, int j0, int n, MeshCounts& cnt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* sev = S.sev + threadIdx.x;
  for (int i = threadIdx.x; i < MC_HASH; i += MC_THREADS) S.hkey[i] = 0u;
  if (threadIdx.x == 0) S.nuniq = 0;
  const int j = j0 + threadIdx.x;
  const bool act = j < n;
  const int2 rec = act ? __ldcg(&V.chg[j]) : make_int2(0, 0);
  const int ci = rec.x, nw = rec.y & 0xFF, od = (rec.y >> 8) & 0xFF;
  const int blk = ci >> 9, c = ci & (BV - 1);
  const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
  const uint64_t wnew = S.tri64[nw];
  const int nold = packed_ntri(S.tri64[od]), nnew = packed_ntri(wnew);
  // the old run's start, the block's key and upper neighbours
  const int obase = nold > 0 ? __ldcg(&V.tri_base[ci]) : -1;
  const int4 r0 = act ? __ldcg(reinterpret_cast<const int4*>(V.nbr + (size_t)blk * 16)) : make_int4(-1, -1, -1, -1);
  const int4 r1 = act ? __ldcg(reinterpret_cast<const int4*>(V.nbr + (size_t)blk * 16 + 4)) : make_int4(-1, -1, -1, -1);
  S.lr0[threadIdx.x] = make_int4(blk, r0.y, r0.z, r0.w);
  S.lr1[threadIdx.x] = r1;
  // the vertex ids on the edges the new triangles use (-1 missing)
  const unsigned em = S.emask[nw];
  const bool rel = nold > 0 && obase >= 0;
  {
    int ev[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      ev[k] = -1;
      if ((em >> k) & 1u) {
        const int ob = owner_bits(k);
        const int hx = x + (ob & 1), hy = y + ((ob >> 1) & 1), hz = z + ((ob >> 2) & 1);
        const int b = nb_select(blk, r0, r1, (hx >> 3) | ((hy >> 3) << 1) | ((hz >> 3) << 2));
        const int vox = (hx & 7) + 8 * (hy & 7) + 64 * (hz & 7);
        if (b < 0) {
          ev[k] = -2;  // cannot happen for a valid cube
        } else if constexpr (CE) {
          const int* sp = edge_slot_ptr<true>(V, b, vox, ob >> 3, false);
          ev[k] = sp ? __ldcg(sp) : -1;
        } else {
          ev[k] = __ldcg(&V.edge_vtx[((size_t)b * BV + vox) * 3 + (ob >> 3)]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) sev[k * MC_THREADS] = ev[k];
  }
  // the old triangles; the edges the cube stops using (their vertices are recycling candidates)
  int4 tr[5];
#pragma unroll
  for (int t = 0; t < 5; ++t) tr[t] = rel && t < nold ? __ldcg(&V.tris[obase + t]) : make_int4(-1, -1, -1, -1);
  const uint64_t wold = S.tri64[od];
  const unsigned cand = rel ? (unsigned)(S.emask[od] & ~em) : 0u;
  __syncthreads();  // the hash is empty
  // missing edges into the chunk's hash: the first lane to insert an edge lists it for a claim;
  // every missing edge's slot becomes a tag resolved after the claims
#pragma unroll 1
  for (unsigned m = em; m; m &= m - 1) {
    const int k = __ffs(m) - 1;
    if (sev[k * MC_THREADS] != -1) continue;
    const int ob = owner_bits(k);
    const int hx = x + (ob & 1), hy = y + ((ob >> 1) & 1), hz = z + ((ob >> 2) & 1);
    const int b = nb_select(blk, r0, r1, (hx >> 3) | ((hy >> 3) << 1) | ((hz >> 3) << 2));
    const uint32_t e = edge_id(b, (hx & 7) + 8 * (hy & 7) + 64 * (hz & 7), ob >> 3);
    uint32_t h = (e * 0x9E3779B1u) >> (32 - MC_HASH_LOG2);
    for (int p = 0; p < MC_HASH; ++p) {
      const uint32_t prev = atomicCAS(&S.hkey[h], 0u, e + 1u);
      if (prev == 0u) S.ulist[atomicAdd(&S.nuniq, 1)] = h | ((uint32_t)threadIdx.x << 16);
      if (prev == 0u || prev == e + 1u) break;
      h = (h + 1) & (MC_HASH - 1);
    }
    sev[k * MC_THREADS] = -3 - (int)h;
  }
  // per-warp amounts, then the chunk's reservations
  const int pc = warp_prefix(S, Q_CAND, __popc(cand));
  const unsigned relm = __ballot_sync(0xffffffffu, rel);
  if (lane == 0) S.wq[Q_RUN_REL][warp] = __popc(relm);
  int prun = 0;
#pragma unroll
  for (int L = 1; L <= 5; ++L) {
    const unsigned mL = __ballot_sync(0xffffffffu, act && nnew == L);
    if (lane == 0) S.wq[Q_RUN1 + L - 1][warp] = __popc(mL);
    if (nnew == L) prun = __popc(mL & ((1u << lane) - 1u));
  }
  __syncthreads();
  chunk_reserve(V, S);
  __syncthreads();
  // the old triangles released: cleared, the run and the recycling candidates listed for gc
  if (rel) {
    for (int t = 0; t < nold; ++t) V.tris[obase + t] = make_int4(-1, -1, -1, -1);
    const int rs = S.base[Q_RUN_REL] + S.wq[Q_RUN_REL][warp] + __popc(relm & ((1u << lane) - 1u));
    if (rs < V.list_cap_deadrun) V.deadrun[rs] = make_int2(obase, nold);
    else set_status(V, ST_POOL_FULL, P_DEAD_RUN_LIST);
    int slot = S.base[Q_CAND] + S.wq[Q_CAND][warp] + pc;
    for (unsigned m = cand; m; m &= m - 1, ++slot) {
      const int v = old_vertex(tr, wold, nold, __ffs(m) - 1);
      if (slot < V.list_cap_dead) V.dead[slot] = v;
      else set_status(V, ST_POOL_FULL, P_DEAD_VERTEX_LIST);
    }
    cnt.released += nold;
  }
  // the new run
  int base = -1;
  if (act && nnew > 0) {
    const int q = Q_RUN1 + nnew - 1;
    base = chunk_pool_id(V, S, q, V.run_free[nnew - 1], S.wq[q][warp] + prun, nnew, V.max_triangles, P_TRIANGLES);
  }
  // the chunk's distinct missing edges, claimed by its threads in turn
  const int nu = S.nuniq;
#pragma unroll 1
  for (int i = threadIdx.x; i < nu; i += MC_THREADS) cnt.created += claim_edge<CE>(V, S, i, S.ulist[i]);
  __syncthreads();  // every claim's result is in hval
  // the new triangles and their references
  if (act) {
    V.tri_base[ci] = base;
    if (base >= 0) {
      cnt.emitted += nnew;
#pragma unroll 1
      for (int t = 0; t < nnew; ++t) {
        int vs[3];
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          const int v = sev[packed_edge(wnew, t, jj) * MC_THREADS];
          vs[jj] = v <= -3 ? S.hval[-3 - v] : v;
        }
        if (vs[0] < 0 || vs[1] < 0 || vs[2] < 0) {  // vertex pool exhausted
          set_status(V, ST_POOL_FULL, P_VERTICES);
          V.tris[base + t] = make_int4(-1, -1, -1, ci);
          continue;
        }
        V.tris[base + t] = make_int4(vs[0], vs[1], vs[2], ci);
      }
    }
    // each edge's reference change: (triangles of the new type using it) - (of the old type);
    // a new edge whose vertex could not be made carries no triangle and no reference
    const uint64_t un = S.euse[nw], uo = rel ? S.euse[od] : 0ull;
#pragma unroll 1
    for (unsigned m = (rel ? S.emask[od] : 0u) | (base >= 0 ? em : 0u); m; m &= m - 1) {
      const int k = __ffs(m) - 1;
      const int d = (int)((un >> (3 * k)) & 7) * (base >= 0) - (int)((uo >> (3 * k)) & 7);
      if (d == 0) continue;
      int v;
      if (base >= 0 && ((em >> k) & 1u)) {
        v = sev[k * MC_THREADS];
        v = v <= -3 ? S.hval[-3 - v] : v;
      } else {
        v = old_vertex(tr, wold, nold, k);
      }
      if (v >= 0) atomicAdd(&V.vref[v], d);
    }
  }
  __syncthreads();  // the chunk's shared state is free for the next chunk
}

// Every changed cube of the pass, a lane each, in chunks of MC_THREADS list entries.
template <bool CE>
__global__ void __launch_bounds__(MC_THREADS, MC_CTAS_PER_SM) k_mesh_cubes(Vol V) {
  extern __shared__ __align__(16) unsigned char mc_smem[];
  CubesSmem& S = *reinterpret_cast<CubesSmem*>(mc_smem);
  for (int i = threadIdx.x; i < 160; i += MC_THREADS) {
    const uint4 w = V.tri_table[i];
    if (i < 128) reinterpret_cast<uint4*>(S.tri64)[i] = w;
    else reinterpret_cast<uint4*>(S.emask)[i - 128] = w;
  }
  // per type, how many of its triangles use each cube edge
  for (int c = threadIdx.x; c < 256; c += MC_THREADS) {
    const uint64_t w = reinterpret_cast<const uint64_t*>(V.tri_table)[c];
    uint64_t u = 0;
    for (int q = 0; q < 3 * packed_ntri(w); ++q) u += 1ull << (3 * packed_edge(w, q / 3, q % 3));
    S.euse[c] = u;
  }
  __syncthreads();
  grid_dependency_wait();
  const int n = min(__ldcg(&V.ctl->c[C_N_CHANGED]), V.list_cap_chg);
  MeshCounts cnt;
  for (int j0 = blockIdx.x * MC_THREADS; j0 < n; j0 += gridDim.x * MC_THREADS) cubes_chunk<CE>(V, S, j0, n, cnt);
  // the statistics, one atomic per CTA and counter
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = __reduce_add_sync(0xffffffffu, cnt.emitted), r1 = __reduce_add_sync(0xffffffffu, cnt.released),
            r2 = __reduce_add_sync(0xffffffffu, cnt.created);
  if (lane == 0) {
    S.red[0][warp] = r0;
    S.red[1][warp] = r1;
    S.red[2][warp] = r2;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    const int q = threadIdx.x < 3 ? threadIdx.x : 2;
    int t = 0;
    for (int w = 0; w < MC_WARPS; ++w) t += S.red[q][w];
    const int cc = threadIdx.x == 0 ? C_ST_EMITTED
                                    : (threadIdx.x == 1 ? C_ST_RELEASED : (threadIdx.x == 2 ? C_LIVE_VERTS : C_ST_NEW_VERTS));
    if (t) atomicAdd(&V.ctl->c[cc], t);
  }
  allow_dependent_launch();
}

constexpr size_t MC_SMEM = sizeof(CubesSmem);
static_assert(MC_CTAS_PER_SM * (MC_SMEM + 1024) <= 233472, "k_mesh_cubes: CTAs per SM do not fit the SM's shared memory");

}  // namespace vmk
