// Differentiable path: gradients of a loss on the mesh vertex positions and normals, taken
// to the TSDF values through the edge interpolation and the normal of Sec. V-C (recomputed
// from the TSDF, nothing stored), and on to the depth pixels by reverse mode through the
// running average of Eq. 2 (d <- (d W + d~) / (W + 1), d~ = min(sdf, mu), sdf = D - z_c).
// Topology, block collection, pixel choice and branches are held fixed.
#pragma once

#include "kernels_fusion.cuh"

namespace vmk {

// Voxel index (block * 512 + local) of global voxel (gx, gy, gz), or -1 when its block is
// not allocated.
__device__ __forceinline__ int voxel_index(const Vol& V, int gx, int gy, int gz) {
  const int blk = find_block(V, gx >> 3, gy >> 3, gz >> 3);  // arithmetic shift: floor(g / 8)
  return blk < 0 ? -1 : blk * BV + (gx & 7) + 8 * (gy & 7) + 64 * (gz & 7);
}

// Checkpoint: the weight of every voxel of the used block slots (the rest of dwck, and
// dcnt, dgrad, were cleared by the host).
__global__ void __launch_bounds__(256) k_diff_checkpoint(Vol V) {
  const int hw = min(__ldcg(&V.ctl->c[C_BLK_BUMP]), V.max_blocks);
  const size_t n = (size_t)hw * BV;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    V.dwck[i] = V.tw[i].y;
}

// After an integrate call: record the blocks it collected as recorded call f and count, per
// voxel, whether the frame integrated it (the frame's parameters are still in the control
// block).  Same per-block layout as the fusion kernel.
__global__ void __launch_bounds__(INTEG_THREADS) k_diff_record(Vol V, int f) {
  const int n = min(__ldcg(&V.ctl->c[C_ST_FRAME_BLOCKS]), V.list_cap_touched);
  const int base = __ldcg(&V.drec_off[f]);
  if (blockIdx.x == 0 && threadIdx.x == 0) V.drec_off[f + 1] = base + n;
  const FrameParams& fp = V.ctl->fp;
  const float mu = V.mu, l = V.l;
  const int v0 = threadIdx.x * 4;
  const int lx = v0 & 7, ly = (v0 >> 3) & 7, lz = v0 >> 6;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int4 t = __ldcg(&V.touched[i]);
    const int blk = t.z >= 0 ? t.z : __ldcg(&V.vals[t.w]);
    if (threadIdx.x == 0) V.drec[base + i] = blk;
    if (blk < 0) continue;
    const int4 key = __ldcg(&V.bkey[blk]);
    const float py = (float)(key.y * BS + ly) * l, pz = (float)(key.z * BS + lz) * l;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float px = (float)(key.x * BS + lx + j) * l;
      int pix;
      float sdf;
      if (project_voxel(fp, mu, px, py, pz, pix, sdf)) V.dcnt[(size_t)blk * BV + v0 + j] += 1;
    }
  }
}

// dL/dd from dL/dp and dL/dn of `n` vertices named by edge key (voxel coordinates biased by
// 2^19 in bits 42.., 22.., 2.., axis in bits 0-1), added into dgrad:
//   p_a = g_a l + t l, t = d0 / (d0 - d1): dt/dd0 = -d1 / (d0 - d1)^2, dt/dd1 = d0 / (d0 - d1)^2
//   (0 where t is clamped to [-1, 2] or d0 = d1);
//   n = m / |m|, m_a = d1 - d0, m_b = (1 - t)(e0_b - d0) + t (e1_b - d1) for b != a when both
//   corners g + e_b, g + e_a + e_b have W > 0 (else m_b = 0):
//   dL/dm = (dL/dn - n (n . dL/dn)) / |m|, 0 when |m| = 0.
__global__ void __launch_bounds__(256) k_grad_vertices(Vol V, int n, const unsigned long long* __restrict__ keys,
                                                       const float* __restrict__ gpos, const float* __restrict__ gnrm) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const unsigned long long key = keys[j];
    const int g[3] = {(int)((key >> 42) & 0xFFFFF) - (1 << 19), (int)((key >> 22) & 0xFFFFF) - (1 << 19),
                      (int)((key >> 2) & 0xFFFFF) - (1 << 19)};
    const int a = (int)(key & 3);
    if (a > 2) continue;
    const int ax = a == 0, ay = a == 1, az = a == 2;
    const int i0 = voxel_index(V, g[0], g[1], g[2]);
    const int i1 = voxel_index(V, g[0] + ax, g[1] + ay, g[2] + az);
    if (i0 < 0 || i1 < 0) continue;
    const float d0 = __ldcg(&V.tw[i0].x), d1 = __ldcg(&V.tw[i1].x);
    float t = d0 == d1 ? 0.5f : d0 / (d0 - d1);
    const bool fixed_t = d0 == d1 || t < -1.0f || t > 2.0f;
    if (t < -1.0f) t = -1.0f;
    if (t > 2.0f) t = 2.0f;
    float dt0 = 0.0f, dt1 = 0.0f;
    if (!fixed_t) {
      const float q = d0 - d1;
      dt0 = -d1 / (q * q);
      dt1 = d0 / (q * q);
    }
    float gt = gpos[3 * j + a] * V.l;
    float m[3], e0[3] = {0.0f, 0.0f, 0.0f}, e1[3] = {0.0f, 0.0f, 0.0f};
    int j0[3] = {-1, -1, -1}, j1[3] = {-1, -1, -1};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b == a) {
        m[b] = d1 - d0;
        continue;
      }
      const int bx = b == 0, by = b == 1, bz = b == 2;
      const int k0 = voxel_index(V, g[0] + bx, g[1] + by, g[2] + bz);
      const int k1 = voxel_index(V, g[0] + ax + bx, g[1] + ay + by, g[2] + az + bz);
      const float2 q0 = k0 >= 0 ? __ldcg(&V.tw[k0]) : make_float2(0.0f, 0.0f);
      const float2 q1 = k1 >= 0 ? __ldcg(&V.tw[k1]) : make_float2(0.0f, 0.0f);
      if (q0.y > 0.0f && q1.y > 0.0f) {
        j0[b] = k0;
        j1[b] = k1;
        e0[b] = q0.x;
        e1[b] = q1.x;
        m[b] = (1.0f - t) * (q0.x - d0) + t * (q1.x - d1);
      } else {
        m[b] = 0.0f;
      }
    }
    float gm[3] = {0.0f, 0.0f, 0.0f};
    const float len = sqrtf((m[0] * m[0] + m[1] * m[1]) + m[2] * m[2]);
    if (len > 0.0f) {
      const float nh[3] = {m[0] / len, m[1] / len, m[2] / len};
      const float dot = nh[0] * gnrm[3 * j] + nh[1] * gnrm[3 * j + 1] + nh[2] * gnrm[3 * j + 2];
#pragma unroll
      for (int i = 0; i < 3; ++i) gm[i] = (gnrm[3 * j + i] - nh[i] * dot) / len;
    }
    float gd0 = -gm[a], gd1 = gm[a];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b == a || j0[b] < 0) continue;
      atomicAdd(&V.dgrad[j0[b]], gm[b] * (1.0f - t));
      atomicAdd(&V.dgrad[j1[b]], gm[b] * t);
      gd0 -= gm[b] * (1.0f - t);
      gd1 -= gm[b] * t;
      gt += gm[b] * ((e1[b] - d1) - (e0[b] - d0));
    }
    gd0 += gt * dt0;
    gd1 += gt * dt1;
    atomicAdd(&V.dgrad[i0], gd0);
    atomicAdd(&V.dgrad[i1], gd1);
  }
}

// Reverse step for recorded call f (calls are taken last to first): for every voxel the
// frame integrated, with W its weight before that integration (the checkpoint weight plus
// the integrations before f, clamped at W_max): dL/dd~ = g / (W + 1) goes to the voxel's
// pixel when d~ = sdf (sdf < mu), and g <- g W / (W + 1).
__global__ void __launch_bounds__(INTEG_THREADS) k_grad_depth(Vol V, int f, const __grid_constant__ FrameParams fp,
                                                              float* __restrict__ gdepth) {
  const int start = __ldcg(&V.drec_off[f]), end = __ldcg(&V.drec_off[f + 1]);
  const float mu = V.mu, l = V.l, wmax = V.wmax;
  const int v0 = threadIdx.x * 4;
  const int lx = v0 & 7, ly = (v0 >> 3) & 7, lz = v0 >> 6;
  for (int i = start + blockIdx.x; i < end; i += gridDim.x) {
    const int blk = __ldcg(&V.drec[i]);
    if (blk < 0) continue;
    const int4 key = __ldcg(&V.bkey[blk]);
    const float py = (float)(key.y * BS + ly) * l, pz = (float)(key.z * BS + lz) * l;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float px = (float)(key.x * BS + lx + j) * l;
      int pix;
      float sdf;
      if (!project_voxel(fp, mu, px, py, pz, pix, sdf)) continue;
      const size_t idx = (size_t)blk * BV + v0 + j;
      if (V.dcnt[idx] == 0) {  // not the recorded frame's inputs
        set_status(V, ST_INVALID);
        continue;
      }
      const int before = (int)V.dcnt[idx] - 1;
      V.dcnt[idx] = (uint16_t)before;
      const float w = fminf(V.dwck[idx] + (float)before, wmax);
      const float g = V.dgrad[idx];
      if (sdf < mu) atomicAdd(gdepth + pix, g / (w + 1.0f));
      V.dgrad[idx] = g * (w / (w + 1.0f));
    }
  }
}

// Export dL/dd of every live block (any order, keys alongside).
__global__ void __launch_bounds__(256) k_export_grad(Vol V, int* counter, int* keys, float* grad) {
  const int hw = min(__ldcg(&V.ctl->c[C_BLK_BUMP]), V.max_blocks);
  __shared__ int slot;
  for (int blk = blockIdx.x; blk < hw; blk += gridDim.x) {
    const int4 k = V.bkey[blk];
    if (k.w < 0) continue;
    if (threadIdx.x == 0) slot = atomicAdd(counter, 1);
    __syncthreads();
    const int j = slot;
    if (threadIdx.x == 0) {
      keys[3 * j] = k.x;
      keys[3 * j + 1] = k.y;
      keys[3 * j + 2] = k.z;
    }
    for (int v = threadIdx.x; v < BV; v += blockDim.x) grad[(size_t)j * BV + v] = V.dgrad[(size_t)blk * BV + v];
    __syncthreads();
  }
}

}  // namespace vmk
