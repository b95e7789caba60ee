// Mesh compaction for download (the "compress" step of Sec. VI) and the block
// export / analytic-fill paths used by tests.  None of these run per frame.
#pragma once

#include "kernels_fusion.cuh"
#include "vmesh_device.cuh"

namespace vmk {

constexpr int SCAN_ITEMS = 1024;  // items per CTA (256 threads x 4)

// Per-CTA count of live vertices (refcount > 0) or live triangles (x >= 0), one CTA per
// chunk of the whole pool (the allocation-free download's counting pass).
template <bool TRI>
__global__ void __launch_bounds__(256) k_count_live(Vol V, int* cta_counts) {
  const int n = TRI ? min(__ldcg(&V.ctl->c[C_TRI_BUMP]), V.max_triangles)
                    : min(__ldcg(&V.ctl->c[C_VTX_BUMP]), V.max_vertices);
  const int base = blockIdx.x * SCAN_ITEMS;
  int cnt = 0;
  if (base < n) {
    for (int j = threadIdx.x; j < SCAN_ITEMS && base + j < n; j += 256) {
      bool live = TRI ? V.tris[base + j].x >= 0 : V.vref[base + j] > 0;
      cnt += live;
    }
  }
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  atomicAdd(&s, cnt);
  __syncthreads();
  if (threadIdx.x == 0) cta_counts[blockIdx.x] = s;
}

// Exclusive scan of n counts in place by one CTA of 1024 threads; the total to *total.  Each
// pass covers 16 consecutive counts per thread (their loads in flight together), a serial scan
// of them, then a scan of the threads' totals over the CTA (two barriers per 16384 counts).
__device__ __forceinline__ void scan_in_cta(int* cta_counts, int n, int* total) {
  constexpr int PER = 16, SPAN = PER * 1024;
  __shared__ int warp_sums[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int carry = 0;  // the same in every thread
  for (int base = 0; base < n; base += SPAN) {
    const int i0 = base + threadIdx.x * PER;
    int v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) v[k] = i0 + k < n ? cta_counts[i0 + k] : 0;
    int tsum = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int c = v[k];
      v[k] = tsum;
      tsum += c;
    }
    int x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
      int t = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_sums[lane] = t;
    }
    __syncthreads();
    const int off = carry + (w > 0 ? warp_sums[w - 1] : 0) + x - tsum;
#pragma unroll
    for (int k = 0; k < PER; ++k)
      if (i0 + k < n) cta_counts[i0 + k] = off + v[k];
    carry += warp_sums[31];
    __syncthreads();  // warp_sums is rewritten by the next pass
  }
  if (threadIdx.x == 0) *total = carry;
}

// Phase 2 (one CTA): exclusive scan of the CTA counts in place; total to *total.
__global__ void __launch_bounds__(1024) k_scan_counts(int* cta_counts, int n, int* total) {
  scan_in_cta(cta_counts, n, total);
}

// Pool slots below the vertex (TRI false) or triangle pool's high-water mark, and their
// chunks of SCAN_ITEMS slots: the download's kernels visit no slot above it.
template <bool TRI>
__device__ __forceinline__ int live_slots(const Vol& V) {
  return TRI ? min(__ldcg(&V.ctl->c[C_TRI_BUMP]), V.max_triangles) : min(__ldcg(&V.ctl->c[C_VTX_BUMP]), V.max_vertices);
}
template <bool TRI>
__device__ __forceinline__ int live_chunks(const Vol& V) {
  return (live_slots<TRI>(V) + SCAN_ITEMS - 1) / SCAN_ITEMS;
}

// Download, phase 1: live vertices (refcount > 0) or live triangles (x >= 0) per chunk of
// SCAN_ITEMS slots below the high-water mark (a persistent grid walks the chunks).
template <bool TRI>
__global__ void __launch_bounds__(256) k_chunk_counts(Vol V, int* counts) {
  const int n = live_slots<TRI>(V);
  const int nch = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  for (int ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const int base = ch * SCAN_ITEMS;
    int cnt = 0;
    for (int j = threadIdx.x; j < SCAN_ITEMS && base + j < n; j += 256)
      cnt += TRI ? (V.tris[base + j].x >= 0) : (V.vref[base + j] > 0);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s, cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
      counts[ch] = s;
      s = 0;
    }
    __syncthreads();
  }
}

// Download, phase 2 (one CTA): exclusive scan of the chunk counts below the high-water mark.
template <bool TRI>
__global__ void __launch_bounds__(1024) k_scan_chunks(Vol V, int* counts, int* total) {
  scan_in_cta(counts, live_chunks<TRI>(V), total);
}

__device__ __forceinline__ uint64_t edge_key_of(const Vol& V, uint32_t e) {
  const int ob = (int)(e / EPB), r = (int)(e - (uint32_t)ob * EPB), ov = r / 3, a = r - ov * 3;
  int4 k = V.bkey[ob];
  int gx = k.x * BS + (ov & 7), gy = k.y * BS + ((ov >> 3) & 7), gz = k.z * BS + (ov >> 6);
  return ((uint64_t)(uint32_t)(gx + (1 << 19)) << 42) | ((uint64_t)(uint32_t)(gy + (1 << 19)) << 22) |
         ((uint64_t)(uint32_t)(gz + (1 << 19)) << 2) | (uint64_t)a;
}

// Download, phase 3 (vertices): stable compaction; remap[v] = new index (or -1).  Outputs at or
// past index `cap` are not written.
__global__ void __launch_bounds__(256) k_compact_vertices(Vol V, const int* cta_offsets, int* remap, float* pos,
                                                          float* nrm, uint64_t* keys, int* refcount, int cap) {
  const int n = live_slots<false>(V);
  const int nch = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
  __shared__ int warp_tot[8];
  __shared__ int running;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const int base = ch * SCAN_ITEMS;
    if (threadIdx.x == 0) running = cta_offsets[ch];
    __syncthreads();
    for (int j0 = 0; j0 < SCAN_ITEMS; j0 += 256) {
      int v = base + j0 + threadIdx.x;
      bool live = v < n && V.vref[v] > 0;
      unsigned b = __ballot_sync(0xffffffffu, live);
      if (lane == 0) warp_tot[w] = __popc(b);
      __syncthreads();
      int off = running;
      for (int q = 0; q < w; ++q) off += warp_tot[q];
      off += __popc(b & ((1u << lane) - 1));
      if (v < n) remap[v] = live ? off : -1;
      if (live && off < cap) {
        float4 p = V.vrec[2 * (size_t)v], q4 = V.vrec[2 * (size_t)v + 1];
        pos[3 * (size_t)off] = p.x; pos[3 * (size_t)off + 1] = p.y; pos[3 * (size_t)off + 2] = p.z;
        nrm[3 * (size_t)off] = q4.x; nrm[3 * (size_t)off + 1] = q4.y; nrm[3 * (size_t)off + 2] = q4.z;
        if (keys) keys[off] = edge_key_of(V, V.vedge[v]);
        if (refcount) refcount[off] = V.vref[v];
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 0;
        for (int q = 0; q < 8; ++q) t += warp_tot[q];
        running += t;
      }
      __syncthreads();
    }
  }
}

// Download, phase 3 (triangles): stable compaction with vertex indices remapped.  A chunk's
// 1024 slots are 4 rounds of 256; all four rounds' loads, then all their vertex remaps, are in
// flight together, with one barrier for the warps' counts of every round.  Outputs at or past
// index `cap` are not written.
__global__ void __launch_bounds__(256) k_compact_triangles(Vol V, const int* cta_offsets, const int* remap,
                                                           int* tris_out, int cap) {
  constexpr int R = SCAN_ITEMS / 256;
  const int n = live_slots<true>(V);
  const int nch = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
  __shared__ int warp_tot[R][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1;
  for (int ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const int base = ch * SCAN_ITEMS;
    int4 tr[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int t = base + k * 256 + threadIdx.x;
      tr[k] = t < n ? __ldcs(reinterpret_cast<const int4*>(V.tris) + t) : make_int4(-1, -1, -1, -1);
    }
    unsigned b[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      b[k] = __ballot_sync(0xffffffffu, tr[k].x >= 0);
      if (lane == 0) warp_tot[k][w] = __popc(b[k]);
    }
    const int running = __ldg(cta_offsets + ch);
    __syncthreads();
    int off[R], acc = running;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      int pre = 0, tot = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = warp_tot[k][q];
        pre += q < w ? c : 0;
        tot += c;
      }
      off[k] = acc + pre + __popc(b[k] & lt);
      acc += tot;
    }
    int r[R][3];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const bool live = tr[k].x >= 0;
      r[k][0] = live ? __ldg(remap + tr[k].x) : -1;
      r[k][1] = live && tr[k].y >= 0 ? __ldg(remap + tr[k].y) : -1;
      r[k][2] = live && tr[k].z >= 0 ? __ldg(remap + tr[k].z) : -1;
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (tr[k].x >= 0 && off[k] < cap) {
        int* o = tris_out + 3 * (size_t)off[k];
        o[0] = r[k][0];
        o[1] = r[k][1];
        o[2] = r[k][2];
      }
    __syncthreads();  // warp_tot is rewritten by the next chunk
  }
}

// Export every live block (any order) into dense buffers.
__global__ void __launch_bounds__(256) k_export_blocks(Vol V, int* counter, int* keys, float* tsdf, float* weight,
                                                       uint8_t* ce, uint8_t* cp) {
  const int hw = min(__ldcg(&V.ctl->c[C_BLK_BUMP]), V.max_blocks);
  __shared__ int slot;
  for (int blk = blockIdx.x; blk < hw; blk += gridDim.x) {
    int4 k = V.bkey[blk];
    if (k.w < 0) continue;
    if (threadIdx.x == 0) slot = atomicAdd(counter, 1);
    __syncthreads();
    const int j = slot;
    if (threadIdx.x == 0) {
      keys[3 * j] = k.x; keys[3 * j + 1] = k.y; keys[3 * j + 2] = k.z;
    }
    for (int v = threadIdx.x; v < BV; v += blockDim.x) {
      float2 q = V.tw[(size_t)blk * BV + v];
      tsdf[(size_t)j * BV + v] = q.x;
      weight[(size_t)j * BV + v] = q.y;
      ce[(size_t)j * BV + v] = V.code_eff[(size_t)blk * BV + v];
      cp[(size_t)j * BV + v] = V.code_prev[(size_t)blk * BV + v];
    }
    __syncthreads();
  }
}

// Analytic fill, phase 1: insert the given keys as if collected by a frame.
__global__ void __launch_bounds__(256) k_fill_insert(Vol V, const int* keys, int n, int advance_epoch, uint32_t frame) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    V.ctl->fp.frame = frame;  // the resolve pass that follows reads the call's number there
    alloc_begin(V, advance_epoch);
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int x = keys[3 * j], y = keys[3 * j + 1], z = keys[3 * j + 2];
    if (abs(x) > KEY_LIMIT || abs(y) > KEY_LIMIT || abs(z) > KEY_LIMIT) {
      set_status(V, ST_INVALID);
      continue;
    }
    const uint64_t key = pack_key(x, y, z);
    int blk;
    int s = hash_insert(V, key, x, y, z, frame, blk);
    if (s >= 0) touch_bucket(V, s, key, blk, frame);
  }
}

// Analytic fill, phase 2 (after the collected keys were resolved): copy the voxel values
// and set the near flag.
__global__ void __launch_bounds__(256) k_fill_copy(Vol V, const int* keys, const float* tsdf, const float* weight,
                                                   int n) {
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    int blk = find_block(V, keys[3 * j], keys[3 * j + 1], keys[3 * j + 2]);
    if (blk < 0) continue;
    bool near = false;
    for (int v = threadIdx.x; v < BV; v += blockDim.x) {
      float d = tsdf[(size_t)j * BV + v], w = weight[(size_t)j * BV + v];
      V.tw[(size_t)blk * BV + v] = make_float2(d, w);
      near |= (w > 0.0f && d < V.mu);
    }
    int any = __syncthreads_or(near);
    if (threadIdx.x == 0) V.bnear[blk] = (uint8_t)(any != 0);
  }
}

}  // namespace vmk
