// Mesh memory accounting (Sec. VI-B, "Memory"): the vertex count of the edge-owned mesh
// against what meshes without shared vertices store.  A per-block extraction (each block
// meshed on its own, vertices shared by the cubes of one block only) stores, per block,
// the distinct edges its cubes' triangles use; a mesh of loose triangles stores 3 vertices
// per triangle.
#pragma once

#include "kernels_mesh.cuh"

namespace vmk {

// Sum over allocated blocks of the distinct edges used by the triangles of their cubes'
// effective types, into *out (one CTA per block iteration, edges marked in a bitmap over
// the block's 9^3 edge owners).
__global__ void __launch_bounds__(128) k_block_vertices(Vol V, unsigned long long* out) {
  __shared__ unsigned mark[EDGE_WORDS];
  __shared__ __align__(16) uint64_t tri64[256];  // written as uint4
  for (int i = threadIdx.x; i < 128; i += blockDim.x) reinterpret_cast<uint4*>(tri64)[i] = V.tri_table[i];
  const int hw = min(__ldcg(&V.ctl->c[C_BLK_BUMP]), V.max_blocks);
  for (int blk = blockIdx.x; blk < hw; blk += gridDim.x) {
    if (V.bkey[blk].w < 0) continue;  // uniform over the CTA
    for (int w = threadIdx.x; w < EDGE_WORDS; w += blockDim.x) mark[w] = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < BV; c += blockDim.x) {
      const uint64_t w = tri64[V.code_eff[(size_t)blk * BV + c]];
      const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
      for (int t = 0; t < packed_ntri(w); ++t)
        for (int j = 0; j < 3; ++j) {
          const int ob = owner_bits(packed_edge(w, t, j));
          const int slot = edge_slot(x + (ob & 1), y + ((ob >> 1) & 1), z + ((ob >> 2) & 1), ob >> 3);
          atomicOr(&mark[slot >> 5], 1u << (slot & 31));
        }
    }
    __syncthreads();
    int cnt = 0;
    for (int w = threadIdx.x; w < EDGE_WORDS; w += blockDim.x) cnt += __popc(mark[w]);
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, (unsigned long long)cnt);
    __syncthreads();
  }
}

}  // namespace vmk
