// Block collection (Sec. V-A, Eq. 1) and TSDF fusion (Sec. V-A, Eq. 2) kernels.
//
// Floating-point evaluation order is fixed (the library is built with --fmad=false and
// IEEE division/sqrt), so the collected block set and the fused values are reproducible
// bit for bit by any IEEE float32 implementation that follows the same order.
#pragma once

#include "vmesh_device.cuh"

namespace vmk {

// ------------------------------------------------------------------ block collection
constexpr int ALLOC_TILE_W = 64;     // pixels per tile row (16 threads x 4 pixels)
constexpr int ALLOC_TILE_H = 16;     // tile rows
constexpr int ALLOC_THREADS = 256;
constexpr int ALLOC_SET = 2048;      // CTA-local set of block keys (power of two)
constexpr int DDA_MAX_CELLS = 1 << 16;

// Insert `key` into the global hash; returns its bucket or -1.  A new key takes a block
// from the block pool; its index is published in vals[] for later kernels.
__device__ int hash_insert(const Vol& V, uint64_t key, int bx, int by, int bz) {
  uint32_t s = (uint32_t)mix64(key) & V.hmask;
  for (uint32_t p = 0; p <= V.hmask; ++p) {
    uint64_t k = __ldcg(&V.keys[s]);
    if (k == key) return (int)s;
    if (k == KEY_EMPTY) {
      unsigned long long old = atomicCAS((unsigned long long*)&V.keys[s], (unsigned long long)KEY_EMPTY,
                                         (unsigned long long)key);
      if (old == KEY_EMPTY) {
        int blk;
        int old_top = atomicSub(&V.ctl->c[C_BLK_TOP], 1);
        if (old_top > 0) {
          blk = __ldcg(&V.blk_free[old_top - 1]);
        } else {
          blk = atomicAdd(&V.ctl->c[C_BLK_BUMP], 1);
          if (blk >= V.max_blocks) {
            set_status(V, ST_POOL_FULL);
            blk = -1;
          }
        }
        V.vals[s] = blk;
        if (blk >= 0) {
          V.bkey[blk] = make_int4(bx, by, bz, (int)s);
          atomicAdd(&V.ctl->c[C_LIVE_BLOCKS], 1);
          atomicAdd(&V.ctl->c[C_ST_NEW_BLOCKS], 1);
        }
        return (int)s;
      }
      if (old == key) return (int)s;
    }
    s = (s + 1) & V.hmask;
  }
  set_status(V, ST_HASH_FULL);
  return -1;
}

// Record a collected bucket once per integrate call.
__device__ __forceinline__ void touch_bucket(const Vol& V, int s, uint32_t frame) {
  if (__ldcg(&V.stamp[s]) == frame) return;
  if (atomicExch(&V.stamp[s], frame) != frame) {
    int i = atomicAdd(&V.ctl->c[C_N_TOUCHED], 1);
    if (i < V.list_cap_touched) V.touched[i] = s;
    else set_status(V, ST_POOL_FULL);
  }
}

__device__ __forceinline__ void smem_set_insert(unsigned long long* set, int* overflow, const Vol& V,
                                                uint64_t key, int bx, int by, int bz, uint32_t frame) {
  uint32_t h = (uint32_t)(mix64(key) >> 20) & (ALLOC_SET - 1);
  for (int p = 0; p < 32; ++p) {
    unsigned long long old = atomicCAS(&set[h], (unsigned long long)KEY_EMPTY, (unsigned long long)key);
    if (old == KEY_EMPTY || old == key) return;
    h = (h + 1) & (ALLOC_SET - 1);
  }
  // CTA set saturated: insert directly
  *overflow = 1;
  int s = hash_insert(V, key, bx, by, bz);
  if (s >= 0) touch_bucket(V, s, frame);
}

// Walk the block cells of one pixel's segment (Eq. 1) into the CTA set.
__device__ __forceinline__ void collect_pixel(const Vol& V, const FrameParams& fp, int u, int v, float D,
                                              unsigned long long* set, int* overflow, uint32_t frame) {
  if (!(D > 0.0f) || !isfinite(D)) return;
  float xn = ((float)u - fp.cx) / fp.fx;
  float yn = ((float)v - fp.cy) / fp.fy;
  float z0 = D - V.mu;
  if (z0 < Z_NEAR) z0 = Z_NEAR;
  float z1 = D + V.mu;
  float pa[3] = {xn * z0, yn * z0, z0};
  float pb[3] = {xn * z1, yn * z1, z1};
  float bs = V.l * (float)BS;
  float A[3], B[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float wa = ((fp.Twc[4 * i] * pa[0] + fp.Twc[4 * i + 1] * pa[1]) + fp.Twc[4 * i + 2] * pa[2]) + fp.Twc[4 * i + 3];
    float wb = ((fp.Twc[4 * i] * pb[0] + fp.Twc[4 * i + 1] * pb[1]) + fp.Twc[4 * i + 2] * pb[2]) + fp.Twc[4 * i + 3];
    A[i] = wa / bs;
    B[i] = wb / bs;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (!isfinite(A[i]) || !isfinite(B[i]) || fabsf(A[i]) > (float)KEY_LIMIT || fabsf(B[i]) > (float)KEY_LIMIT) return;
  // 3D DDA over block cells, from floor(A) to floor(B); ties step x before y before z
  int c[3], rem[3], step[3];
  float tmax[3], tdel[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    c[i] = (int)floorf(A[i]);
    int e = (int)floorf(B[i]);
    float dir = B[i] - A[i];
    if (dir > 0.0f) {
      step[i] = 1;
      tdel[i] = 1.0f / dir;
      tmax[i] = (((float)c[i] + 1.0f) - A[i]) / dir;
    } else if (dir < 0.0f) {
      step[i] = -1;
      tdel[i] = 1.0f / (-dir);
      tmax[i] = (A[i] - (float)c[i]) / (-dir);
    } else {
      step[i] = 0;
      tdel[i] = __int_as_float(0x7f800000);
      tmax[i] = __int_as_float(0x7f800000);
    }
    rem[i] = abs(e - c[i]);
  }
  // The walk has rem_x + rem_y + rem_z + 1 cells; the parameter limits checked on the host
  // (voxel >= 0.1 mm, mu <= 32 voxels, |pixel ray slope| <= 64) keep it far below the cap,
  // which only guards against a runaway loop.
  for (int it = 0; it < DDA_MAX_CELLS; ++it) {
    smem_set_insert(set, overflow, V, pack_key(c[0], c[1], c[2]), c[0], c[1], c[2], frame);
    if (rem[0] + rem[1] + rem[2] == 0) break;
    int best = -1;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (rem[i] > 0 && (best < 0 || tmax[i] < tmax[best])) best = i;
    c[best] += step[best];
    tmax[best] += tdel[best];
    rem[best]--;
  }
}

// One CTA per 64 x 16 pixel tile: each thread reads 4 consecutive depths (one float4 when
// the row is 16-byte aligned), walks their segments into a CTA-local key set, then the
// set's unique keys are inserted into the global hash and recorded as collected.
// The last CTA clamps the block free-stack top and, when `advance_epoch`, starts a new
// mesh epoch with an empty update set.
__global__ void __launch_bounds__(ALLOC_THREADS) k_alloc(Vol V, const FrameParams* __restrict__ fpp,
                                                         int advance_epoch) {
  __shared__ unsigned long long set[ALLOC_SET];
  __shared__ int overflow;
  const FrameParams fp = *fpp;
  const uint32_t frame = (uint32_t)__ldcg(&V.ctl->c[C_FRAME]);
  for (int i = threadIdx.x; i < ALLOC_SET; i += blockDim.x) set[i] = KEY_EMPTY;
  if (threadIdx.x == 0) overflow = 0;
  __syncthreads();

  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int u0 = blockIdx.x * ALLOC_TILE_W + tx * 4;
  const int v = blockIdx.y * ALLOC_TILE_H + ty;
  if (v < fp.H && u0 < fp.W) {
    const float* row = fp.depth + (size_t)v * fp.W;
    float d[4];
    if (u0 + 3 < fp.W && ((reinterpret_cast<uintptr_t>(row + u0) & 15) == 0)) {
      float4 q = __ldg(reinterpret_cast<const float4*>(row + u0));
      d[0] = q.x; d[1] = q.y; d[2] = q.z; d[3] = q.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) d[j] = (u0 + j < fp.W) ? __ldg(row + u0 + j) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (u0 + j < fp.W) collect_pixel(V, fp, u0 + j, v, d[j], set, &overflow, frame);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ALLOC_SET; i += blockDim.x) {
    uint64_t key = set[i];
    if (key == KEY_EMPTY) continue;
    int bx = (int)((key >> 42) & 0x1FFFFF) - KEY_BIAS;
    int by = (int)((key >> 21) & 0x1FFFFF) - KEY_BIAS;
    int bz = (int)(key & 0x1FFFFF) - KEY_BIAS;
    int s = hash_insert(V, key, bx, by, bz);
    if (s >= 0) touch_bucket(V, s, frame);
  }
  if (last_block(V, C_DONE0)) {
    if (threadIdx.x == 0) {
      fold_top(V, C_BLK_TOP);
      if (advance_epoch) {
        V.ctl->c[C_EPOCH] += 1;
        V.ctl->c[C_N_UPDATE] = 0;
      }
      V.ctl->c[C_DONE0] = 0;
    }
  }
}

// Collected buckets -> blocks; each collected block and its existing neighbours at
// offsets {0,-1}^3 join the update set once per epoch.  8 lanes per collected bucket.
__global__ void __launch_bounds__(256) k_resolve(Vol V) {
  const int n = __ldcg(&V.ctl->c[C_N_TOUCHED]);
  const uint32_t epoch = (uint32_t)__ldcg(&V.ctl->c[C_EPOCH]);
  const int total = (n < V.list_cap_touched ? n : V.list_cap_touched) * 8;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    int i = t >> 3, o = t & 7;
    int s = V.touched[i];
    int blk = __ldcg(&V.vals[s]);
    if (o == 0) {
      V.touched_blk[i] = blk;
      if (blk >= 0) V.bepoch[blk] = epoch;
    }
    if (blk < 0) continue;
    int4 k = V.bkey[blk];
    int ns = o == 0 ? s : hash_find(V, pack_key(k.x - (o & 1), k.y - ((o >> 1) & 1), k.z - ((o >> 2) & 1)));
    if (ns < 0) continue;
    int nb = __ldcg(&V.vals[ns]);
    if (nb < 0) continue;
    if (__ldcg(&V.ustamp[ns]) == epoch) continue;
    if (atomicExch(&V.ustamp[ns], epoch) != epoch) list_push(V, V.update, C_N_UPDATE, V.list_cap_update, nb);
  }
  if (last_block(V, C_DONE1)) {
    if (threadIdx.x == 0) {
      V.ctl->c[C_ST_FRAME_BLOCKS] = n;
      V.ctl->c[C_DONE1] = 0;
    }
  }
}

// ------------------------------------------------------------------ fusion (Eq. 2)
constexpr int INTEG_THREADS = 128;  // 4 voxels per thread, one block per CTA iteration

// Fuse the frame into every voxel of each collected block.  Voxels stream as float2
// (d, W) pairs, 32 bytes per thread per block; depth is gathered through the read-only
// path.  Also records whether any voxel of the block has W > 0 and d < mu (used by gc).
// The last CTA resets the collected list and advances the frame counter.
__global__ void __launch_bounds__(INTEG_THREADS) k_integrate(Vol V, const FrameParams* __restrict__ fpp) {
  const FrameParams fp = *fpp;
  const int n = min(__ldcg(&V.ctl->c[C_N_TOUCHED]), V.list_cap_touched);
  const float mu = V.mu, l = V.l, wmax = V.wmax;
  const int v0 = threadIdx.x * 4;
  const int lx = v0 & 7, ly = (v0 >> 3) & 7, lz = v0 >> 6;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    int blk = V.touched_blk[i];
    if (blk < 0) continue;
    int4 key = V.bkey[blk];
    float4* p = reinterpret_cast<float4*>(V.tw + (size_t)blk * BV + v0);
    float4 q0 = __ldcs(p), q1 = __ldcs(p + 1);
    float dd[4] = {q0.x, q0.z, q1.x, q1.z};
    float ww[4] = {q0.y, q0.w, q1.y, q1.w};
    bool changed = false;
    const int gy = key.y * BS + ly, gz = key.z * BS + lz;
    const float py = (float)gy * l, pz = (float)gz * l;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float px = (float)(key.x * BS + lx + j) * l;
      float xc = ((fp.Tcw[0] * px + fp.Tcw[1] * py) + fp.Tcw[2] * pz) + fp.Tcw[3];
      float yc = ((fp.Tcw[4] * px + fp.Tcw[5] * py) + fp.Tcw[6] * pz) + fp.Tcw[7];
      float zc = ((fp.Tcw[8] * px + fp.Tcw[9] * py) + fp.Tcw[10] * pz) + fp.Tcw[11];
      if (!(zc > 0.0f)) continue;
      float us = ((fp.fx * xc) / zc + fp.cx) + 0.5f;
      float vs = ((fp.fy * yc) / zc + fp.cy) + 0.5f;
      if (!(us >= 0.0f && us < (float)fp.W && vs >= 0.0f && vs < (float)fp.H)) continue;
      int iu = (int)floorf(us), iv = (int)floorf(vs);
      float D = __ldg(fp.depth + (size_t)iv * fp.W + iu);
      if (!(D > 0.0f) || !isfinite(D)) continue;
      float sdf = D - zc;
      if (sdf < -mu) continue;
      float dt = sdf < mu ? sdf : mu;
      float num = dd[j] * ww[j] + dt;
      float den = ww[j] + 1.0f;
      dd[j] = num / den;
      ww[j] = den < wmax ? den : wmax;
      changed = true;
    }
    if (changed) {
      __stcs(p, make_float4(dd[0], ww[0], dd[1], ww[1]));
      __stcs(p + 1, make_float4(dd[2], ww[2], dd[3], ww[3]));
    }
    bool near = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) near |= (ww[j] > 0.0f && dd[j] < mu);
    int any = __syncthreads_or(near);
    if (threadIdx.x == 0) V.bnear[blk] = (uint8_t)(any != 0);
  }
  if (last_block(V, C_DONE2)) {
    if (threadIdx.x == 0) {
      V.ctl->c[C_N_TOUCHED] = 0;
      V.ctl->c[C_FRAME] += 1;
      V.ctl->c[C_DONE2] = 0;
    }
  }
}

}  // namespace vmk
