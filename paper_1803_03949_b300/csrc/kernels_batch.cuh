// Batched step: one frame of each of up to MAX_SCENES independent volumes per launch of
// each per-frame kernel.  Every kernel is the single-volume kernel's per-item body (one
// tile, one collected block, one update-set block, one pool slot...) run over the
// concatenation of all scenes' work, so a tick costs five launches whatever the number of
// scenes, and the GPU is filled by the sum of the scenes' work rather than by one scene.
// Work is handed out so that a CTA (tiles, blocks) or a warp (gc items) never mixes scenes:
// the warp-aggregated appends and counters assume one volume per group of lanes.
#pragma once

#include "kernels_fusion.cuh"
#include "kernels_gc.cuh"
#include "kernels_mesh.cuh"

namespace vmk {

constexpr int MAX_SCENES = 64;

// Launch argument of the batched block collection (replaced before every graph replay).
struct BatchFrames {
  FrameParams fp[MAX_SCENES];
  int advance[MAX_SCENES];  // start a new mesh epoch for this scene (as k_alloc's argument)
};

// Batch control: the last-CTA ticket of the block gc, and the mesh pass's block hand-out
// counter (reset by the fusion's first CTA).
enum BatchDone { BD_MESH = 0, BD_COUNT };

// pre[s] = sum of count(t) over scenes t < s, pre[n] = total (shared memory, whole CTA).
template <typename F>
__device__ __forceinline__ void scene_prefix(int n, int* pre, F count) {
  __shared__ int cnt[MAX_SCENES];
  if (threadIdx.x < n) cnt[threadIdx.x] = count(threadIdx.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int t = 0; t < n; ++t) {
      pre[t] = acc;
      acc += cnt[t];
    }
    pre[n] = acc;
  }
  __syncthreads();
}

// The scene whose range [pre[s], pre[s + 1]) holds global item g (pre ascending, g < pre[n]).
__device__ __forceinline__ int scene_of(const int* pre, int n, int g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Block collection: grid (tiles across, tiles down, scenes); a CTA whose tile lies outside
// its scene's image does nothing; each scene's first CTA starts its epoch.
template <int PPT>
__global__ void __launch_bounds__(ALLOC_TILE_W * ALLOC_TILE_H / PPT)
    kb_alloc(const Vol* __restrict__ vols, int nscenes, const __grid_constant__ BatchFrames bf) {
  __shared__ unsigned long long set[ALLOC_SET];
  const int s = blockIdx.z;
  const Vol& V = vols[s];
  const FrameParams& fp = bf.fp[s];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    V.ctl->fp = fp;  // for the later kernels
    alloc_begin(V, bf.advance[s]);
  }
  if ((int)blockIdx.x * ALLOC_TILE_W < fp.W && (int)blockIdx.y * ALLOC_TILE_H < fp.H)
    alloc_tile<PPT, ALLOC_TILE_W, false>(V, fp, blockIdx.x, blockIdx.y, set);
  allow_dependent_launch();
}

// Fusion: every scene's collected blocks, one per CTA iteration.
__global__ void __launch_bounds__(INTEG_THREADS) kb_integrate(const Vol* __restrict__ vols, int nscenes, int* bdone) {
  grid_dependency_wait();
  __shared__ int pre[MAX_SCENES + 1];
  __shared__ uint32_t sframe[MAX_SCENES], sepoch[MAX_SCENES];
  if (threadIdx.x < nscenes) {
    sframe[threadIdx.x] = __ldcg(&vols[threadIdx.x].ctl->fp.frame);
    sepoch[threadIdx.x] = (uint32_t)__ldcg(&vols[threadIdx.x].ctl->c[C_EPOCH]);
  }
  scene_prefix(nscenes, pre,
               [&](int t) { return min(__ldcg(&vols[t].ctl->c[touched_count(sframe[t])]), vols[t].list_cap_touched); });
  const int total = pre[nscenes];
  if (blockIdx.x == 0) {
    for (int t = threadIdx.x; t < nscenes; t += blockDim.x) integrate_begin(vols[t], pre[t + 1] - pre[t], sframe[t]);
    if (threadIdx.x == 0) bdone[BD_MESH] = 0;
  }
  __shared__ IntegNear N;
  if (threadIdx.x < INTEG_RING) {
    N.any[threadIdx.x] = 0;
    N.done[threadIdx.x] = 0;
  }
  __syncthreads();
  for (int g = blockIdx.x, it = 0; g < total; g += gridDim.x, ++it) {
    const int s = scene_of(pre, nscenes, g);
    const Vol& V = vols[s];
    integrate_block<true>(V, V.ctl->fp, __ldcg(&V.touched[g - pre[s]]), sframe[s], sepoch[s], it, N);
    if ((it & (INTEG_RING - 1)) == INTEG_RING - 1) __syncthreads();
  }
  allow_dependent_launch();
}

// Mesh pass: every scene's update set, one block per CTA iteration.
template <bool CE>
__global__ void __launch_bounds__(MESH_THREADS, mesh_ctas_per_sm(true)) kb_mesh(const Vol* __restrict__ vols, int nscenes, int mode,
                                                           int* bdone) {
  __shared__ MeshSmem<CE> S;
  __shared__ int pre[MAX_SCENES + 1];
  mesh_tables(S, vols[0].tri_table);
  grid_dependency_wait();
  scene_prefix(nscenes, pre, [&](int t) { return min(__ldcg(&vols[t].ctl->c[C_N_UPDATE]), vols[t].list_cap_update); });
  const int total = pre[nscenes];
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < nscenes; t += blockDim.x) mesh_begin(vols[t], pre[t + 1] - pre[t]);
  MeshCounts cnt;
  int cur = -1;
  // one block per CTA, then the rest to whichever CTA is free first
  for (int g = blockIdx.x, k = 0; g < total; k ^= 1) {
    const int s = scene_of(pre, nscenes, g);
    if (s != cur) {
      if (cur >= 0) mesh_flush(vols[cur], cnt);
      cur = s;
    }
    const Vol& V = vols[s];
    mesh_block<CE>(V, S, V.update[g - pre[s]], mode, cnt);
    if (threadIdx.x == 0) S.next[k] = (int)gridDim.x + atomicAdd(&bdone[BD_MESH], 1);
    __syncthreads();
    g = S.next[k];
  }
  if (cur >= 0) mesh_flush(vols[cur], cnt);
  allow_dependent_launch();
}

// Zero-reference vertices and released runs of every scene, in chunks of 512 entries of each
// list (one CTA per chunk, so that the CTA's warps share a scene and its free stacks take one
// reservation per CTA).
template <bool CE>
__global__ void __launch_bounds__(GCV_THREADS) kb_gc_vertices(const Vol* __restrict__ vols, int nscenes) {
  grid_dependency_wait();
  __shared__ int pre_d[MAX_SCENES + 1], pre_e[MAX_SCENES + 1];
  __shared__ GcvCta sh;
  if (threadIdx.x == 0) sh.freed = 0;
  constexpr int CHUNK = GCV_THREADS * GCV_PER_LIST;
  scene_prefix(nscenes, pre_d, [&](int t) {
    const int n = min(__ldcg(&vols[t].ctl->c[C_N_DEAD]), vols[t].list_cap_dead);
    const int nr = min(__ldcg(&vols[t].ctl->c[C_N_DEADRUN]), vols[t].list_cap_deadrun);
    return (max(n, nr) + CHUNK - 1) / CHUNK;
  });
  scene_prefix(nscenes, pre_e,
               [&](int t) { return (min(__ldcg(&vols[t].ctl->c[C_N_DEADREC]), vols[t].max_vertices) + 31) >> 5; });
  // hash rebuilds: a scene whose live plus dead buckets passed half its table (the counts its
  // previous block gc left: every CTA reads the same, nothing changes them in this kernel) has
  // the table cleared by the whole grid here and its live blocks reinserted by the block gc
  __shared__ int rehash[MAX_SCENES];
  if (threadIdx.x < nscenes) {
    const Vol& V = vols[threadIdx.x];
    rehash[threadIdx.x] = gc_rehash_needed(V, __ldcg(&V.ctl->c[C_LIVE_BLOCKS]), __ldcg(&V.ctl->c[C_TOMBS])) ? 1 : 0;
    if (blockIdx.x == 0) V.ctl->c[C_REHASH] = rehash[threadIdx.x];
  }
  __syncthreads();
  for (int t = 0; t < nscenes; ++t)
    if (rehash[t]) {
      const Vol& V = vols[t];
      for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= V.hmask; b += gridDim.x * blockDim.x) {
        V.keys[b] = KEY_EMPTY;
        V.vals[b] = -1;
        V.stamp[b] = 0;
      }
    }
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int u = blockIdx.x; u < pre_d[nscenes]; u += gridDim.x) {
    const int s = scene_of(pre_d, nscenes, u);
    const Vol& V = vols[s];
    const int n = min(__ldcg(&V.ctl->c[C_N_DEAD]), V.list_cap_dead);
    const int nr = min(__ldcg(&V.ctl->c[C_N_DEADRUN]), V.list_cap_deadrun);
    int freed = 0;
    gc_vertices_pass<CE>(V, (u - pre_d[s]) * CHUNK + (threadIdx.x & ~31), GCV_THREADS, n, nr, freed, &sh);
    if (freed) atomicAdd(&sh.freed, freed);
    __syncthreads();
    if (threadIdx.x == 0 && sh.freed) {
      atomicAdd(&V.ctl->c[C_LIVE_VERTS], -sh.freed);
      atomicAdd(&V.ctl->c[C_ST_FREED_VERTS], sh.freed);
      sh.freed = 0;
    }
    __syncthreads();  // the next chunk rewrites sh
  }
  for (int u = warp; CE && u < pre_e[nscenes]; u += nwarps) {
    const int s = scene_of(pre_e, nscenes, u);
    const Vol& V = vols[s];
    const int n = min(__ldcg(&V.ctl->c[C_N_DEADREC]), V.max_vertices);
    const int i = ((u - pre_e[s]) << 5) + lane;
    if (i < n) gc_record(V, V.dead_rec[i]);
  }
  allow_dependent_launch();
}

// Block recycling of every scene: a lane per pool slot in use tests it, the warp frees the
// candidates.  A scene whose table the vertex gc cleared for a rebuild frees without tombstones,
// and each warp reinserts the live blocks of its slots of that scene after its frees.
__global__ void __launch_bounds__(256) kb_gc_blocks(const Vol* __restrict__ vols, int nscenes, int consumed) {
  grid_dependency_wait();
  __shared__ int pre[MAX_SCENES + 1];
  __shared__ uint32_t sepoch[MAX_SCENES];
  __shared__ int rehash[MAX_SCENES];
  if (threadIdx.x < nscenes) {
    const Vol& V = vols[threadIdx.x];
    sepoch[threadIdx.x] = (uint32_t)__ldcg(&V.ctl->c[C_EPOCH]);
    rehash[threadIdx.x] = __ldcg(&V.ctl->c[C_REHASH]);
    if (blockIdx.x == 0) {
      gc_lists_reset(V);
      if (consumed) V.ctl->c[C_N_UPDATE] = 0;  // the update set (read by nothing here) emptied
      if (rehash[threadIdx.x]) {                 // no tombstone survives the rebuild
        V.ctl->c[C_TOMBS] = 0;
        V.ctl->c[C_ST_REHASHES] += 1;
      }
    }
  }
  scene_prefix(nscenes, pre, [&](int t) { return min(__ldcg(&vols[t].ctl->c[C_BLK_BUMP]), vols[t].max_blocks); });
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int total = pre[nscenes];
  for (int base = warp * 32; base < total; base += nwarps * 32) {
    const int g = base + lane;
    int s = 0;
    bool cand = false;
    if (g < total) {
      s = scene_of(pre, nscenes, g);
      cand = gc_candidate(vols[s], g - pre[s], sepoch[s], consumed);
    }
    unsigned m = __ballot_sync(0xffffffffu, cand);
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const int sb = __shfl_sync(0xffffffffu, s, b);
      const bool tomb = !rehash[sb];
      int freed = gc_free_block(vols[sb], base + b - pre[sb], tomb);
      gc_flush_blocks(vols[sb], freed, tomb);
    }
    __syncwarp();  // lane 0's frees visible to the lane that reads the slot
    if (g < total && rehash[s]) {
      const int blk = g - pre[s];
      const int4 k = vols[s].bkey[blk];
      if (k.w >= 0) rehash_insert(vols[s], blk, k);
    }
  }
}

}  // namespace vmk
