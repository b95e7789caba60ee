// Garbage collection (Sec. V-E): vertices whose reference count (= vertex degree)
// dropped to zero are recycled, so are the triangle runs the mesh pass released and the
// blocks that carry no surface any more.
#pragma once

#include "vmesh_device.cuh"

namespace vmk {

// Detach a claimed zero-reference vertex from its edge `e` (NO_EDGE: attached to none).
// Returns whether it was attached.
template <bool CE>
__device__ __forceinline__ bool gc_detach(const Vol& V, uint32_t e) {
  bool detached = false;
  if (e != NO_EDGE) {
    const int ob = (int)(e / EPB), r = (int)(e - (uint32_t)ob * EPB), ov = r / 3, a = r - ov * 3;
    const size_t vox = (size_t)ob * BV + ov;
    if constexpr (CE) {
      const int rec = V.edge_rec[vox];  // exists while the voxel owns a vertex
      if (rec >= 0) V.erec[(size_t)rec * 3 + a] = -1;
      // the thread that clears the voxel's last vertex bit frees its edge record (all -1 now)
      const uint8_t old = atomic_and_u8(V.vmask + vox, (uint8_t)~(1 << a));
      if (((old & 7) & ~(1 << a)) == 0 && rec >= 0) {
        V.edge_rec[vox] = -1;
        pool_push(V, V.rec_free, C_REC_TOP, V.max_vertices, rec);
      }
    } else {
      V.edge_vtx[e] = -1;
      atomic_and_u8(V.vmask + vox, (uint8_t)~(1 << a));
    }
    atomicSub(&V.bnvert[ob], 1);
    detached = true;
  }
  return detached;
}

// atomicCAS(p, cmp, val) returning the old value when `on`, else no access and cmp + 1;
// predicated rather than branched, so that a run of them issues back to back.
__device__ __forceinline__ int atom_cas_if(int* p, int cmp, int val, bool on) {
  int old = cmp + 1;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %4, 0;\n\t@q atom.global.cas.b32 %0, [%1], %2, %3;\n\t}"
      : "+r"(old)
      : "l"(p), "r"(cmp), "r"(val), "r"((unsigned)on)
      : "memory");
  return old;
}

// Inclusive sum over the lanes of a full, converged warp.
template <typename T>
__device__ __forceinline__ T warp_inclusive_sum(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

constexpr int GCV_PER_LIST = 2;  // entries of each list per thread and pass, in flight together
constexpr int GCV_CTAS_PER_SM = 6;
constexpr int GCV_THREADS = 256;
constexpr int GCV_WARPS = GCV_THREADS / 32;

// Free-stack reservations of a whole CTA's pass (both vertex gc kernels): every warp's counts
// of freed vertices and of released runs per length (then their exclusive prefixes over the
// warps), the CTA's first slot on each stack, and its freed count.  The stack tops and the vertex
// counters then take one atomic per CTA instead of one per warp.
struct GcvCta {
  int v[GCV_WARPS];
  int r[GCV_WARPS][5];
  int vbase, rbase[5];
  int freed;
};

// One pass of a full warp over the zero-reference vertex list and the released-run list:
// lane j takes entries b + j + k * stride (k < GCV_PER_LIST) of each.  A listed vertex is
// claimed with CAS(0 -> -1), so a vertex listed twice, or one that regained a reference after
// it was listed, is freed at most once and only when unreferenced; a vertex still attached to
// its edge is detached.  Three round trips for all entries: the list entries; the claims, with
// one free-stack reservation per run length; one free-stack reservation for the freed vertices,
// while the claimed vertices' edges load.  The reservations are the warp's own (sh null) or the
// CTA's (sh: the whole CTA calls the pass together; two barriers).
template <bool CE>
__device__ __forceinline__ void gc_vertices_pass(const Vol& V, int b, int stride, int n, int nr, int& freed,
                                                 GcvCta* sh = nullptr) {
  constexpr int K = GCV_PER_LIST;
  const int lane = threadIdx.x & 31;
  int vid[K];
  int2 run[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = b + lane + k * stride;
    vid[k] = i < n ? __ldcg(&V.dead[i]) : -1;
    run[k] = i < nr ? __ldcg(&V.deadrun[i]) : make_int2(0, 0);
  }
  int old[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int v = vid[k] >= 0 ? vid[k] : 0;
    old[k] = atom_cas_if(V.vref + v, 0, -1, vid[k] >= 0);
  }
  // the edge of each claimed vertex (most listed vertices are still referenced and keep theirs;
  // no gc thread writes it), loaded while the reservations below are made
  uint32_t e[K];
#pragma unroll
  for (int k = 0; k < K; ++k) e[k] = (vid[k] >= 0 && old[k] == 0) ? __ldcg(&V.vedge[vid[k]]) : NO_EDGE;
  // released runs: per length L (8 bits at 8 (L - 1)) this lane's count, its exclusive prefix
  // over the warp, and one free-stack reservation per length (lanes 0..4)
  unsigned long long rc = 0;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (run[k].y >= 1 && run[k].y <= 5) rc += 1ull << (8 * (run[k].y - 1));
  const unsigned long long rinc = warp_inclusive_sum(rc);
  const unsigned long long rtot = __shfl_sync(0xffffffffu, rinc, 31);
  // vertices whose claim succeeded
  unsigned ok = 0;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (vid[k] >= 0 && old[k] == 0) ok |= 1u << k;
  const int nok = __popc(ok);
  const int vinc = warp_inclusive_sum(nok);
  // the first slots of the warp on the vertex stack (vbase) and on each run stack (lanes
  // 0..4: rbase of length lane + 1)
  int vbase = 0, rbase = 0;
  if (sh) {
    const int warp = threadIdx.x >> 5;
    if (lane == 31) sh->v[warp] = vinc;
    if (lane < 5) sh->r[warp][lane] = (int)((rtot >> (8 * lane)) & 0xFF);
    __syncthreads();
    if (threadIdx.x < 6) {  // thread 0: the vertex stack; threads 1..5: run length 1..5
      const int t = threadIdx.x;
      int tot = 0;
      for (int w = 0; w < GCV_WARPS; ++w) {
        int* p = t == 0 ? &sh->v[w] : &sh->r[w][t - 1];
        const int c = *p;
        *p = tot;
        tot += c;
      }
      const int base = tot ? atomicAdd(&V.ctl->c[t == 0 ? C_VTX_TOP : run_top(t)], tot) : 0;
      if (t == 0) sh->vbase = base;
      else sh->rbase[t - 1] = base;
    }
    __syncthreads();
    vbase = sh->vbase + sh->v[warp];
    if (lane < 5) rbase = sh->rbase[lane] + sh->r[warp][lane];
  } else {
    if (lane < 5) {
      const int c = (int)((rtot >> (8 * lane)) & 0xFF);
      if (c) rbase = atomicAdd(&V.ctl->c[run_top(lane + 1)], c);
    }
    if (lane == 31 && vinc > 0) vbase = atomicAdd(&V.ctl->c[C_VTX_TOP], vinc);
    vbase = __shfl_sync(0xffffffffu, vbase, 31);
  }
  vbase += vinc - nok;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if ((ok >> k) & 1u) {
      freed += gc_detach<CE>(V, e[k]);
      if (vbase < V.max_vertices) V.vtx_free[vbase] = vid[k];
      else set_status(V, ST_POOL_FULL, P_FREE_STACK);
      ++vbase;
    }
  // per length, this lane's first slot: the reservation plus the lanes before
  const unsigned long long rex = rinc - rc;
  int rb[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) rb[j] = __shfl_sync(0xffffffffu, rbase, j) + (int)((rex >> (8 * j)) & 0xFF);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int L = run[k].y;
    int slot = -1;
#pragma unroll
    for (int j = 0; j < 5; ++j)
      if (L == j + 1) slot = rb[j]++;
    if (slot < 0) continue;
    if (slot < V.run_cap[L - 1]) V.run_free[L - 1][slot] = run[k].x;
    else set_status(V, ST_POOL_FULL, P_FREE_STACK);
  }
}

// Empty the three lists the vertex gc consumed (one thread; the block gc does it at its
// start, after the vertex gc has ended).
__device__ __forceinline__ void gc_lists_reset(const Vol& V) {
  V.ctl->c[C_N_DEAD] = 0;
  V.ctl->c[C_N_DEADRUN] = 0;
  V.ctl->c[C_N_DEADREC] = 0;
}

// A spare edge record of a lost claim back to its free stack.
__device__ __forceinline__ void gc_record(const Vol& V, int rec) { pool_push(V, V.rec_free, C_REC_TOP, V.max_vertices, rec); }

// Block slot `blk` (one lane) may be freed when it was not collected in the current epoch,
// has no triangles and owns no vertex, and all of its voxels have W = 0 or d >= mu.
// `consumed`: the update set has been meshed since it was collected (else its blocks are
// kept, so that the pending update never lists a recycled block index).  The six records
// are loaded before any is tested (one round trip), lanes reading consecutive slots.
__device__ __forceinline__ bool gc_candidate(const Vol& V, int blk, uint32_t epoch, int consumed) {
  const int4 key = V.bkey[blk];
  const uint32_t be = V.bepoch[blk], us = V.ustamp[blk];
  const int nt = V.bntri[blk], nv = V.bnvert[blk];
  const int nr = V.bnear[blk];
  return (key.w >= 0) & (be != epoch) & (nt == 0) & (nv == 0) & (nr == 0) & (consumed || us != epoch);
}

// Free candidate slot `blk` (the calling warp) unless one of its 7 lower neighbours (whose
// cubes reach into it) has triangles: its bucket becomes a tombstone, its voxels are
// cleared, its neighbours forget it, its index returns to the pool.  Returns (in every lane)
// whether the block was freed.
__device__ __forceinline__ void gc_release_block(const Vol& V, int blk, bool tomb);
__device__ __forceinline__ bool gc_free_block(const Vol& V, int blk, bool tomb = true) {
  const int lane = threadIdx.x & 31;
  bool lower_tri = false;
  if (lane >= 1 && lane < 8) {
    const int nbk = V.nbr[blk * 16 + 8 + lane];
    lower_tri = nbk >= 0 && V.bntri[nbk] != 0;
  }
  if (__any_sync(0xffffffffu, lower_tri)) return false;
  gc_release_block(V, blk, tomb);
  return true;
}

// Free block `blk` (the calling warp; its checks passed): its bucket becomes a tombstone (not
// while the table is being rebuilt: then the block is simply not reinserted), its voxels are
// cleared, its neighbours forget it, its index returns to the pool.
__device__ __forceinline__ void gc_release_block(const Vol& V, int blk, bool tomb = true) {
  const int lane = threadIdx.x & 31;
  const int bucket = V.bkey[blk].w;
  float4* tw = reinterpret_cast<float4*>(V.tw + (size_t)blk * BV);
  for (int j = lane; j < BV / 2; j += 32) tw[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  reinterpret_cast<uint4*>(V.code_eff + (size_t)blk * BV)[lane] = make_uint4(0, 0, 0, 0);
  reinterpret_cast<uint4*>(V.code_prev + (size_t)blk * BV)[lane] = make_uint4(0, 0, 0, 0);
  reinterpret_cast<uint4*>(V.vmask + (size_t)blk * BV)[lane] = make_uint4(0, 0, 0, 0);
  if (lane >= 1 && lane < 16 && lane != 8) {
    // unlink: the neighbour at this slot's offset forgets this block
    const int other = V.nbr[blk * 16 + lane];
    if (other >= 0) V.nbr[other * 16 + (lane ^ 8)] = -1;
  }
  __syncwarp();
  if (lane < 16) V.nbr[blk * 16 + lane] = -1;
  if (lane == 0) {
    if (tomb) {
      V.keys[bucket] = KEY_TOMB;
      V.vals[bucket] = -1;
    }
    V.bkey[blk] = make_int4(0, 0, 0, -1);
    V.bnear[blk] = 0;
    pool_push(V, V.blk_free, C_BLK_TOP, V.max_blocks, blk);
  }
}

__device__ __forceinline__ void gc_flush_blocks(const Vol& V, int& freed, bool tomb = true) {
  if ((threadIdx.x & 31) == 0 && freed) {
    atomicSub(&V.ctl->c[C_LIVE_BLOCKS], freed);
    if (tomb) atomicAdd(&V.ctl->c[C_TOMBS], freed);
    atomicAdd(&V.ctl->c[C_ST_FREED_BLOCKS], freed);
  }
  freed = 0;
}

// Insert live block `blk` (key k) into a table under rebuild: the first empty bucket from its
// home bucket, claimed with atomicCAS (every key is distinct); its index and bucket recorded.
__device__ __forceinline__ void rehash_insert(const Vol& V, int blk, int4 k) {
  const uint64_t key = pack_key(k.x, k.y, k.z);
  uint32_t s = (uint32_t)mix64(key) & V.hmask;
  for (uint32_t p = 0; p <= V.hmask; ++p) {
    const unsigned long long old =
        atomicCAS((unsigned long long*)&V.keys[s], (unsigned long long)KEY_EMPTY, (unsigned long long)key);
    if (old == KEY_EMPTY) {
      V.vals[s] = blk;
      V.bkey[blk].w = (int)s;
      return;
    }
    s = (s + 1) & V.hmask;
  }
  set_status(V, ST_HASH_FULL, P_HASH);
}

// Whether the hash needs a rebuild: live plus dead buckets (the live-block and tombstone
// counts) past half the table.
__device__ __forceinline__ bool gc_rehash_needed(const Vol& V, long long live, long long tomb) {
  return (live + tomb) * 2 > (long long)V.hmask + 1 && tomb > 0;
}

// Zero-reference vertices and released triangle runs (and, CE, spare edge records) back to
// their free stacks.
template <bool CE>
__global__ void __launch_bounds__(GCV_THREADS, GCV_CTAS_PER_SM) k_gc_vertices(Vol V) {
  __shared__ GcvCta sh;
  if (threadIdx.x == 0) sh.freed = 0;
  grid_dependency_wait();
  // the list lengths, and the live-block and tombstone counts the previous block gc left (one
  // round trip for all four)
  const int n = min(__ldcg(&V.ctl->c[C_N_DEAD]), V.list_cap_dead);
  const int nr = min(__ldcg(&V.ctl->c[C_N_DEADRUN]), V.list_cap_deadrun);
  const long long live = __ldcg(&V.ctl->c[C_LIVE_BLOCKS]), tomb = __ldcg(&V.ctl->c[C_TOMBS]);
  int freed = 0;
  const int stride = gridDim.x * blockDim.x, m = max(n, nr);
  // The hash is quiet from here until the block gc that follows: when live plus dead buckets
  // passed half the table, every CTA clears a share of it here and the block gc reinserts the
  // live blocks (the kernel boundary is the grid-wide barrier between the two halves).  All
  // CTAs read the same counts, so they agree on the decision.
  // (the counts change only in the block gc, which resets them after the rebuild)
  const bool rehash = gc_rehash_needed(V, live, tomb);
  if (blockIdx.x == 0 && threadIdx.x == 0) V.ctl->c[C_REHASH] = rehash ? 1 : 0;
  if (rehash)
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s <= V.hmask; s += gridDim.x * blockDim.x) {
      V.keys[s] = KEY_EMPTY;
      V.vals[s] = -1;
      V.stamp[s] = 0;
    }
  // the CTA's passes together (CTA-wide reservations)
  for (int b0 = blockIdx.x * blockDim.x; b0 < m; b0 += stride * GCV_PER_LIST) {
    gc_vertices_pass<CE>(V, b0 + (threadIdx.x & ~31), stride, n, nr, freed, &sh);
    __syncthreads();  // the next pass rewrites sh
  }
  if (CE) {
    const int nrec = min(__ldcg(&V.ctl->c[C_N_DEADREC]), V.max_vertices);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrec; i += gridDim.x * blockDim.x) gc_record(V, V.dead_rec[i]);
  }
  if (freed) atomicAdd(&sh.freed, freed);
  __syncthreads();
  if (threadIdx.x == 0 && sh.freed) {
    atomicAdd(&V.ctl->c[C_LIVE_VERTS], -sh.freed);
    atomicAdd(&V.ctl->c[C_ST_FREED_VERTS], sh.freed);
  }
  allow_dependent_launch();
}

// Block recycling: a lane per pool slot tests it, the warp frees the candidates.  When the vertex
// gc before it cleared the hash for a rebuild, freed blocks leave no tombstone and each warp
// reinserts the live blocks of its slots after its frees.
__global__ void __launch_bounds__(256) k_gc_blocks(Vol V, int consumed) {
  grid_dependency_wait();
  const bool rehash = __ldcg(&V.ctl->c[C_REHASH]) != 0;
  if (rehash && blockIdx.x == 0 && threadIdx.x == 0) {  // no tombstone survives the rebuild
    V.ctl->c[C_TOMBS] = 0;
    V.ctl->c[C_ST_REHASHES] += 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    gc_lists_reset(V);
    if (consumed) V.ctl->c[C_N_UPDATE] = 0;  // the update set (read by nothing here) emptied
  }
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int hw = min(__ldcg(&V.ctl->c[C_BLK_BUMP]), V.max_blocks);
  const uint32_t epoch = (uint32_t)__ldcg(&V.ctl->c[C_EPOCH]);
  const int lane = threadIdx.x & 31;
  int freed = 0;
  for (int base = warp * 32; base < hw; base += nwarps * 32) {
    const int blk = base + lane;
    unsigned m = __ballot_sync(0xffffffffu, blk < hw && gc_candidate(V, blk, epoch, consumed));
    while (m) {
      // four candidates at a time, lanes 8 g + 1..7 testing the lower neighbours of the g-th
      const int g = lane >> 3, o = lane & 7;
      unsigned mg = m;
      for (int j = 0; j < g; ++j) mg &= mg - 1;
      const int cb = mg ? __ffs(mg) - 1 : -1;
      for (int j = 0; j < 4; ++j) m &= m - 1;
      bool lower_tri = false;
      if (cb >= 0 && o >= 1) {
        const int nbk = V.nbr[(base + cb) * 16 + 8 + o];
        lower_tri = nbk >= 0 && V.bntri[nbk] != 0;
      }
      const unsigned kept = __ballot_sync(0xffffffffu, lower_tri);
      for (int gg = 0; gg < 4; ++gg) {
        const int c = __shfl_sync(0xffffffffu, cb, 8 * gg);
        if (c < 0) break;
        if (((kept >> (8 * gg)) & 0xFFu) == 0) {
          gc_release_block(V, base + c, !rehash);
          ++freed;
        }
      }
    }
    __syncwarp();  // lane 0's frees visible to the lane that reads the slot
    if (rehash && blk < hw) {
      const int4 k = V.bkey[blk];
      if (k.w >= 0) rehash_insert(V, blk, k);
    }
  }
  gc_flush_blocks(V, freed, !rehash);
}

}  // namespace vmk
