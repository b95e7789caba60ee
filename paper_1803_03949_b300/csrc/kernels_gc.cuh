// Garbage collection (Sec. V-E): vertices whose reference count (= vertex degree)
// dropped to zero are recycled, and so are blocks that carry no surface any more.
// Triangles are recycled by the mesh passes as soon as their cube changes type.
#pragma once

#include "vmesh_device.cuh"

namespace vmk {

// Zero-reference vertices: claim with CAS(0 -> -1) so a vertex listed twice, or one that
// regained a reference in a later pass, is freed at most once and only when unreferenced.
__global__ void __launch_bounds__(256) k_gc_vertices(Vol V) {
  const int n = min(__ldcg(&V.ctl->c[C_N_DEAD]), V.list_cap_dead);
  int freed = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int vid = V.dead[i];
    if (atomicCAS(&V.vref[vid], 0, -1) != 0) continue;
    const int e = V.vedge[vid];
    const int ob = e / EPB, r = e - ob * EPB, ov = r / 3, a = r - ov * 3;
    V.edge_vtx[e] = -1;
    atomic_and_u8(V.vmask + (size_t)ob * BV + ov, (uint8_t)~(9 << a));
    atomicSub(&V.bnvert[ob], 1);
    pool_push(V, V.vtx_free, C_VTX_TOP, V.max_vertices, vid);
    ++freed;
  }
  if (freed) {
    atomicSub(&V.ctl->c[C_LIVE_VERTS], freed);
    atomicAdd(&V.ctl->c[C_ST_FREED_VERTS], freed);
  }
  if (last_block(V, C_DONE5)) {
    if (threadIdx.x == 0) {
      V.ctl->c[C_N_DEAD] = 0;
      V.ctl->c[C_DONE5] = 0;
    }
  }
}

// Block recycling, one warp per pool slot.  A block is freed when it was not collected in
// the current epoch, has no triangles and owns no vertex, all of its voxels have W = 0 or
// d >= mu, and none of its 7 lower neighbours (whose cubes reach into it) has triangles.
// Its bucket becomes a tombstone, its voxels are cleared, its index returns to the pool.
// `consumed` says the update set has been meshed since it was collected: then it is
// emptied here; otherwise its blocks are kept so that the pending update never lists a
// recycled (and possibly reallocated) block index.
__global__ void __launch_bounds__(256) k_gc_blocks(Vol V, int consumed) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int hw = min(__ldcg(&V.ctl->c[C_BLK_BUMP]), V.max_blocks);
  const uint32_t epoch = (uint32_t)__ldcg(&V.ctl->c[C_EPOCH]);
  int freed = 0;
  for (int blk = warp; blk < hw; blk += nwarps) {
    const int4 key = V.bkey[blk];
    bool cand = key.w >= 0 && V.bepoch[blk] != epoch && V.bntri[blk] == 0 && V.bnvert[blk] == 0 &&
                V.bnear[blk] == 0 && (consumed || V.ustamp[key.w] != epoch);
    if (!cand) continue;  // warp-uniform
    bool lower_tri = false;
    if (lane >= 1 && lane < 8) {
      int o = lane;
      int nbk = find_block(V, key.x - (o & 1), key.y - ((o >> 1) & 1), key.z - ((o >> 2) & 1));
      lower_tri = nbk >= 0 && V.bntri[nbk] != 0;
    }
    if (__any_sync(0xffffffffu, lower_tri)) continue;
    // free it
    float4* tw = reinterpret_cast<float4*>(V.tw + (size_t)blk * BV);
    for (int j = lane; j < BV / 2; j += 32) tw[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    uint4* ce = reinterpret_cast<uint4*>(V.code_eff + (size_t)blk * BV);
    uint4* cp = reinterpret_cast<uint4*>(V.code_prev + (size_t)blk * BV);
    uint4* vm = reinterpret_cast<uint4*>(V.vmask + (size_t)blk * BV);
    uint4* ch = reinterpret_cast<uint4*>(V.chg + (size_t)blk * BV);
    ce[lane] = make_uint4(0, 0, 0, 0);
    cp[lane] = make_uint4(0, 0, 0, 0);
    vm[lane] = make_uint4(0, 0, 0, 0);
    ch[lane] = make_uint4(0, 0, 0, 0);
    if (lane == 0) {
      V.keys[key.w] = KEY_TOMB;
      V.vals[key.w] = -1;
      V.bkey[blk] = make_int4(0, 0, 0, -1);
      V.bnear[blk] = 0;
      ++freed;
    }
    __syncwarp();
    if (lane == 0) pool_push(V, V.blk_free, C_BLK_TOP, V.max_blocks, blk);
  }
  if (lane == 0 && freed) {
    atomicSub(&V.ctl->c[C_LIVE_BLOCKS], freed);
    atomicAdd(&V.ctl->c[C_TOMBS], freed);
    atomicAdd(&V.ctl->c[C_ST_FREED_BLOCKS], freed);
  }
  if (last_block(V, C_DONE7)) {
    if (threadIdx.x == 0) {
      if (consumed) V.ctl->c[C_N_UPDATE] = 0;
      V.ctl->c[C_DONE7] = 0;
    }
  }
}

// Rebuild the hash without tombstones when live + dead buckets pass half the table:
// check (one thread) -> wipe every bucket -> re-insert every live block from the block
// array (bkey holds its key; the new bucket is written back) -> re-mark the current
// update set so a block is never listed twice.  Each kernel returns at once when no
// rebuild is needed, so the sequence can sit in every gc call (and in a CUDA graph).
__global__ void k_rehash_check(Vol V) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long live = __ldcg(&V.ctl->c[C_LIVE_BLOCKS]), tomb = __ldcg(&V.ctl->c[C_TOMBS]);
    V.ctl->c[C_REHASH] = (live + tomb) * 2 > (long long)V.hmask + 1 && tomb > 0;
  }
}

__global__ void __launch_bounds__(256) k_rehash_wipe(Vol V) {
  if (!__ldcg(&V.ctl->c[C_REHASH])) return;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s <= V.hmask; s += gridDim.x * blockDim.x) {
    V.keys[s] = KEY_EMPTY;
    V.vals[s] = -1;
    V.stamp[s] = 0;
    V.ustamp[s] = 0;
  }
}

__global__ void __launch_bounds__(256) k_rehash_insert(Vol V) {
  if (!__ldcg(&V.ctl->c[C_REHASH])) return;
  const int hw = min(__ldcg(&V.ctl->c[C_BLK_BUMP]), V.max_blocks);
  for (int blk = blockIdx.x * blockDim.x + threadIdx.x; blk < hw; blk += gridDim.x * blockDim.x) {
    int4 k = V.bkey[blk];
    if (k.w < 0) continue;
    uint64_t key = pack_key(k.x, k.y, k.z);
    uint32_t s = (uint32_t)mix64(key) & V.hmask;
    for (uint32_t p = 0; p <= V.hmask; ++p) {
      unsigned long long old = atomicCAS((unsigned long long*)&V.keys[s], (unsigned long long)KEY_EMPTY,
                                         (unsigned long long)key);
      if (old == KEY_EMPTY) break;
      s = (s + 1) & V.hmask;
    }
    V.vals[s] = blk;
    V.bkey[blk].w = (int)s;
  }
}

__global__ void __launch_bounds__(256) k_rehash_mark(Vol V) {
  if (!__ldcg(&V.ctl->c[C_REHASH])) return;
  const int n = min(__ldcg(&V.ctl->c[C_N_UPDATE]), V.list_cap_update);
  const uint32_t epoch = (uint32_t)__ldcg(&V.ctl->c[C_EPOCH]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int4 k = V.bkey[V.update[i]];
    if (k.w >= 0) V.ustamp[k.w] = epoch;
  }
  if (last_block(V, C_DONE6)) {
    if (threadIdx.x == 0) {
      V.ctl->c[C_TOMBS] = 0;
      V.ctl->c[C_REHASH] = 0;
      V.ctl->c[C_ST_REHASHES] += 1;
      V.ctl->c[C_DONE6] = 0;
    }
  }
}

}  // namespace vmk
