// Block collection (Sec. V-A, Eq. 1) and TSDF fusion (Sec. V-A, Eq. 2) kernels.
//
// Floating-point evaluation order is fixed (the library is built with --fmad=false and
// IEEE division/sqrt), so the collected block set and the fused values are reproducible
// bit for bit by any IEEE float32 implementation that follows the same order.
#pragma once

#include "vmesh_device.cuh"

namespace vmk {

// ------------------------------------------------------------------ block collection
constexpr int ALLOC_TILE_W = 64;     // pixels per tile row (batched collection)
constexpr int ALLOC_TILE_W1 = 32;    // pixels per tile row (k_alloc: 600 tiles of a 640 x 480
                                     // frame spread over the SMs more evenly than 300)
constexpr int ALLOC_TILE_H = 16;     // tile rows
constexpr int ALLOC_PPT = 1;         // vertically adjacent pixels per thread (k_alloc; 1 measured
                                     // faster than 2 and 4: the walks of one thread are serial)
constexpr int ALLOC_THREADS = ALLOC_TILE_W1 * ALLOC_TILE_H / ALLOC_PPT;
constexpr int ALLOC_SET_LOG2 = 10;
constexpr int ALLOC_SET = 1 << ALLOC_SET_LOG2;  // CTA-local set of block keys
constexpr int DDA_MAX_CELLS = 1 << 16;

// Insert `key` into the global hash; returns its bucket or -1.  A new key takes a block
// from the block pool (stamped with the creating integrate call); its index is published
// in vals[] for later kernels.  `blk` receives the block index when it is already known
// here, else -1 (a key another thread inserted in the same launch may not have its index
// published yet; readers then take it from vals[] after the launch).
__device__ int hash_insert(const Vol& V, uint64_t key, int bx, int by, int bz, uint32_t frame, int& blk_out) {
  uint32_t s = (uint32_t)mix64(key) & V.hmask;
  blk_out = -1;
  for (uint32_t p = 0; p <= V.hmask; ++p) {
    // the value is loaded with the key (one round trip when the key is found)
    const uint64_t k = __ldcg(&V.keys[s]);
    const int val = __ldcg(&V.vals[s]);
    if (k == key) {
      blk_out = val;
      return (int)s;
    }
    if (k == KEY_EMPTY) {
      unsigned long long old = atomicCAS((unsigned long long*)&V.keys[s], (unsigned long long)KEY_EMPTY,
                                         (unsigned long long)key);
      if (old == KEY_EMPTY) {
        int blk;
        int old_top = atomicSub(&V.ctl->c[C_BLK_TOP], 1);
        if (old_top > 0) {
          blk = __ldcg(&V.blk_free[old_top - 1]);
        } else {
          atomicAdd(&V.ctl->c[C_BLK_TOP], 1);  // the empty stack's top back to >= 0
          blk = atomicAdd(&V.ctl->c[C_BLK_BUMP], 1);
          if (blk >= V.max_blocks) {
            set_status(V, ST_POOL_FULL, P_BLOCKS);
            blk = -1;
          }
        }
        V.vals[s] = blk;
        blk_out = blk;
        if (blk >= 0) {
          V.bkey[blk] = make_int4(bx, by, bz, (int)s);
          V.bborn[blk] = frame;
          atomicAdd(&V.ctl->c[C_LIVE_BLOCKS], 1);
          atomicAdd(&V.ctl->c[C_ST_NEW_BLOCKS], 1);
        }
        return (int)s;
      }
      if (old == key) return (int)s;
    }
    s = (s + 1) & V.hmask;
  }
  set_status(V, ST_HASH_FULL, P_HASH);
  return -1;
}

// Record a collected bucket once per integrate call, as {packed key (low, high word), block
// index or -1, bucket}: the fusion kernel then needs no hash or key lookups of its own.
__device__ __forceinline__ void touch_bucket(const Vol& V, int s, uint64_t key, int blk, uint32_t frame) {
  if (atomicExch(&V.stamp[s], frame) != frame)
    list_push(V, V.touched, touched_count(frame), V.list_cap_touched,
              make_int4((int)(uint32_t)key, (int)(key >> 32), blk, s));
}

// Insert a key of the CTA set into the global hash and record the collection.
__device__ __forceinline__ void alloc_global_insert(const Vol& V, uint64_t key, uint32_t frame) {
  const int bx = (int)((key >> 42) & 0x1FFFFF) - KEY_BIAS;
  const int by = (int)((key >> 21) & 0x1FFFFF) - KEY_BIAS;
  const int bz = (int)(key & 0x1FFFFF) - KEY_BIAS;
  int blk;
  const int s = hash_insert(V, key, bx, by, bz, frame, blk);
  if (s >= 0) touch_bucket(V, s, key, blk, frame);
}

// Per warp of a collection CTA, the set slots whose key one of its threads put in the set
// first: the warp inserts those keys into the global hash once its own pixels are walked, so
// the round trips of a tile's inserts overlap the other warps' walks.
constexpr int ALLOC_WLIST = 64;

// Put `key` in the CTA set; a key new to the set goes on the list `wl` (count `wn`) of the
// calling warp (or, when that list is full, into the hash at once); wl null: no list (the
// caller inserts the set's keys after the walks).
__device__ __forceinline__ void smem_set_insert(unsigned long long* set, uint16_t* wl, int* wn, const Vol& V,
                                                uint64_t key, uint32_t frame) {
  // any spread of the 63 key bits serves here (the set lives for one CTA): fold and multiply
  uint32_t h = (((uint32_t)key ^ (uint32_t)(key >> 21) ^ (uint32_t)(key >> 42)) * 0x9E3779B1u) >> (32 - ALLOC_SET_LOG2);
  for (int p = 0; p < 32; ++p) {
    // a slot changes once (empty -> key), so a plain read that sees the key settles it;
    // most pixels of a tile cross the same few cells, and this keeps them off the atomic
    const unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(&set[h]);
    if (cur == key) return;
    if (cur == KEY_EMPTY) {
      unsigned long long old = atomicCAS(&set[h], (unsigned long long)KEY_EMPTY, (unsigned long long)key);
      if (old == KEY_EMPTY) {
        if (wl) {
          const int pos = atomicAdd(wn, 1);
          if (pos < ALLOC_WLIST) wl[pos] = (uint16_t)h;
          else alloc_global_insert(V, key, frame);
        }
        return;
      }
      if (old == key) return;
    }
    h = (h + 1) & (ALLOC_SET - 1);
  }
  alloc_global_insert(V, key, frame);  // CTA set saturated: insert directly
}

// DDA set-up along one axis: start cell c, remaining steps rem, step direction, the ray
// parameter of the first boundary crossing (tmax) and between crossings (tdel).
__device__ __forceinline__ void dda_axis(float a, float b, int& c, int& rem, int& step, float& tmax, float& tdel) {
  c = (int)floorf(a);
  const int e = (int)floorf(b);
  const float dir = b - a;
  if (dir > 0.0f) {
    step = 1;
    tdel = __frcp_rn(dir);  // the correctly rounded 1 / dir
    tmax = (((float)c + 1.0f) - a) * tdel;
  } else if (dir < 0.0f) {
    step = -1;
    tdel = __frcp_rn(-dir);
    tmax = (a - (float)c) * tdel;
  } else {
    step = 0;
    tdel = __int_as_float(0x7f800000);
    tmax = __int_as_float(0x7f800000);
  }
  rem = abs(e - c);
}

// Walk the block cells of one pixel's segment (Eq. 1) into the CTA set; `last` holds the
// key this thread inserted most recently (neighbouring pixels mostly cross the same cells).
__device__ __forceinline__ void collect_pixel(const Vol& V, const FrameParams& fp, int u, int v, float D,
                                              unsigned long long* set, uint16_t* wl, int* wn, uint32_t frame,
                                              uint64_t& last) {
  if (!(D > 0.0f) || !isfinite(D)) return;
  // divisions as products with the correctly rounded reciprocals of fx, fy and the block side
  // (computed once on the host: the value of 1.0f / x in IEEE arithmetic)
  const float xn = ((float)u - fp.cx) * fp.rfx;
  const float yn = ((float)v - fp.cy) * fp.rfy;
  float z0 = D - V.mu;
  if (z0 < Z_NEAR) z0 = Z_NEAR;
  const float z1 = D + V.mu;
  const float pa0 = xn * z0, pa1 = yn * z0, pa2 = z0;
  const float pb0 = xn * z1, pb1 = yn * z1, pb2 = z1;
  const float ibs = V.ibs;
  float A[3], B[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float wa = ((fp.Twc[4 * i] * pa0 + fp.Twc[4 * i + 1] * pa1) + fp.Twc[4 * i + 2] * pa2) + fp.Twc[4 * i + 3];
    float wb = ((fp.Twc[4 * i] * pb0 + fp.Twc[4 * i + 1] * pb1) + fp.Twc[4 * i + 2] * pb2) + fp.Twc[4 * i + 3];
    A[i] = wa * ibs;
    B[i] = wb * ibs;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (!isfinite(A[i]) || !isfinite(B[i]) || fabsf(A[i]) > (float)KEY_LIMIT || fabsf(B[i]) > (float)KEY_LIMIT) return;
  // 3D DDA over block cells from floor(A) to floor(B): one step at a time along the axis
  // whose next boundary comes first among the axes with steps left (ties x, then y, then z)
  int cx, cy, cz, rx, ry, rz, sx, sy, sz;
  float mx, my, mz, dx, dy, dz;
  dda_axis(A[0], B[0], cx, rx, sx, mx, dx);
  dda_axis(A[1], B[1], cy, ry, sy, my, dy);
  dda_axis(A[2], B[2], cz, rz, sz, mz, dz);
  // The walk has rx + ry + rz + 1 cells; the parameter limits checked on the host
  // (voxel >= 0.1 mm, mu <= 32 voxels, |pixel ray slope| <= 64) keep it far below the cap,
  // which only guards against a runaway loop.
  for (int it = 0; it < DDA_MAX_CELLS; ++it) {
    const uint64_t key = pack_key(cx, cy, cz);
    if (key != last) {
      smem_set_insert(set, wl, wn, V, key, frame);
      last = key;
    }
    if (rx + ry + rz == 0) break;
    int best = rx > 0 ? 0 : -1;
    float bt = mx;
    if (ry > 0 && (best < 0 || my < bt)) { best = 1; bt = my; }
    if (rz > 0 && (best < 0 || mz < bt)) { best = 2; }
    if (best == 0) { cx += sx; mx += dx; --rx; }
    else if (best == 1) { cy += sy; my += dy; --ry; }
    else { cz += sz; mz += dz; --rz; }
  }
}

// One TW x 16 pixel tile (tile column tx, row ty) walked by the calling CTA of
// TW * 16 / PPT threads, PPT vertically adjacent pixels per thread: each pixel's segment goes
// into the CTA-local key set `set`, and each key new to the set is inserted into the global
// hash and recorded as collected: EARLY, by the warp that found it, after its own walks
// (k_alloc); else by the whole CTA after all walks (the batched collection, measured faster
// that way with its larger CTAs).
template <int PPT, int TW, bool EARLY>
__device__ __forceinline__ void alloc_tile(const Vol& V, const FrameParams& fp, int tx, int ty,
                                           unsigned long long* set) {
  constexpr int NW = EARLY ? TW * ALLOC_TILE_H / PPT / 32 : 1;
  __shared__ uint16_t wlist[NW][ALLOC_WLIST];
  __shared__ int wcount[NW];
  const uint32_t frame = fp.frame;
  const int w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < ALLOC_SET; i += blockDim.x) set[i] = KEY_EMPTY;
  if (EARLY && threadIdx.x < NW) wcount[threadIdx.x] = 0;
  const int u = tx * TW + (threadIdx.x & (TW - 1));
  const int v = ty * ALLOC_TILE_H + PPT * (threadIdx.x / TW);
  // the depth pixels: from device memory, or from pinned host memory across the host link (then
  // kept in the device copy the later kernels read)
  float D[PPT];
#pragma unroll
  for (int r = 0; r < PPT; ++r) D[r] = (u < fp.W && v + r < fp.H) ? fp.depth_in[(size_t)(v + r) * fp.W + u] : 0.0f;
  __syncthreads();
  if (fp.depth_copy) {
#pragma unroll
    for (int r = 0; r < PPT; ++r)
      if (u < fp.W && v + r < fp.H) fp.depth_copy[(size_t)(v + r) * fp.W + u] = D[r];
  }
  uint64_t last = KEY_EMPTY;
#pragma unroll
  for (int r = 0; r < PPT; ++r)
    if (u < fp.W && v + r < fp.H)
      collect_pixel(V, fp, u, v + r, D[r], set, EARLY ? wlist[w] : nullptr, EARLY ? &wcount[w] : nullptr, frame, last);
  if (EARLY) {
    __syncwarp();
    const int nw = min(wcount[w], ALLOC_WLIST);
    for (int i = threadIdx.x & 31; i < nw; i += 32) alloc_global_insert(V, set[wlist[w][i]], frame);
  } else {
    __syncthreads();
    for (int i = threadIdx.x; i < ALLOC_SET; i += blockDim.x)
      if (set[i] != KEY_EMPTY) alloc_global_insert(V, set[i], frame);
  }
}

// At the start of a frame's collection (one thread of the first CTA; nothing in the
// collection reads the epoch or the update set): with `advance_epoch`, a new mesh epoch
// with an empty update set.
__device__ __forceinline__ void alloc_begin(const Vol& V, int advance_epoch) {
  if (advance_epoch) {
    V.ctl->c[C_EPOCH] += 1;
    V.ctl->c[C_N_UPDATE] = 0;
  }
}

// One CTA per 32 x 16 pixel tile, a pixel per thread (512 threads; a 640 x 480 frame is 600
// CTAs).  The frame's parameters arrive as a launch argument; the first CTA stores them in the
// control block for the kernels that follow and starts the epoch.  No CTA waits for the
// others: the kernel ends with its last tile.  Registers are bounded for 3 CTAs per SM (40;
// bounding them for 4 spills and measured slower).
__global__ void __launch_bounds__(ALLOC_THREADS, 3) k_alloc(Vol V, const __grid_constant__ FrameParams fp,
                                                         int advance_epoch) {
  __shared__ unsigned long long set[ALLOC_SET];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    V.ctl->fp = fp;  // for the later kernels
    alloc_begin(V, advance_epoch);
  }
  alloc_tile<ALLOC_PPT, ALLOC_TILE_W1, true>(V, fp, blockIdx.x, blockIdx.y, set);
  allow_dependent_launch();
}

// Resolve one collected bucket (lanes t = 0..15 of the resolving warp):
//   - the block and its existing neighbours at offsets {0,-1}^3 join the update set once
//     per epoch (their cubes read corners in the collected block);
//   - a block created by this integrate call links itself into the neighbour table (and
//     its neighbours to it), looking its neighbours up in the hash.
// Old blocks read their lower neighbours from the table.  A new block's table entries may
// race with an old neighbour reading them, but new blocks are collected themselves, so no
// update-set member is lost.
__device__ __forceinline__ void resolve_block(const Vol& V, int blk, int4 key, uint32_t frame, uint32_t epoch, int t) {
  if (t >= 16) return;
  const int o = t & 7;
  const int sgn = t < 8 ? -1 : 1;  // threads 0..7: lower neighbours (and self), 8..15: upper
  // both loads issued together; the table entry is used only for an old block
  const uint32_t born = __ldcg(&V.bborn[blk]);
  const int nb_old = (sgn < 0 && o != 0) ? __ldcg(&V.nbr[blk * 16 + 8 + o]) : -1;
  const bool is_new = born == frame;
  int nb;
  if (o == 0) {
    nb = blk;
  } else if (is_new) {
    nb = find_block(V, key.x + sgn * (o & 1), key.y + sgn * ((o >> 1) & 1), key.z + sgn * ((o >> 2) & 1));
    // table: my slot for this offset, and the neighbour's slot for the opposite offset
    V.nbr[blk * 16 + (sgn > 0 ? o : 8 + o)] = nb;
    if (nb >= 0) V.nbr[nb * 16 + (sgn > 0 ? 8 + o : o)] = blk;
  } else {
    nb = nb_old;
  }
  if (t == 0) V.bepoch[blk] = epoch;
  if (sgn > 0 || nb < 0) return;
  if (atomicExch(&V.ustamp[nb], epoch) != epoch) list_push(V, V.update, C_N_UPDATE, V.list_cap_update, nb);
}

// ------------------------------------------------------------------ fusion (Eq. 2)
// Eq. 2's inputs for the voxel at world point (px, py, pz): false when the frame does not
// integrate it (behind the camera, outside the image, invalid depth, sdf < -mu); else its
// nearest pixel and sdf = D - z_c.  The fusion and its gradient share this definition.
__device__ __forceinline__ bool project_voxel(const FrameParams& fp, float mu, float px, float py, float pz, int& pix,
                                              float& sdf) {
  const float xc = ((fp.Tcw[0] * px + fp.Tcw[1] * py) + fp.Tcw[2] * pz) + fp.Tcw[3];
  const float yc = ((fp.Tcw[4] * px + fp.Tcw[5] * py) + fp.Tcw[6] * pz) + fp.Tcw[7];
  const float zc = ((fp.Tcw[8] * px + fp.Tcw[9] * py) + fp.Tcw[10] * pz) + fp.Tcw[11];
  if (!(zc > 0.0f)) return false;
  const float us = ((fp.fx * xc) / zc + fp.cx) + 0.5f;
  const float vs = ((fp.fy * yc) / zc + fp.cy) + 0.5f;
  if (!(us >= 0.0f && us < (float)fp.W && vs >= 0.0f && vs < (float)fp.H)) return false;
  pix = (int)floorf(vs) * fp.W + (int)floorf(us);
  const float D = __ldg(fp.depth + pix);
  if (!(D > 0.0f) || !isfinite(D)) return false;
  sdf = D - zc;
  return !(sdf < -mu);
}

constexpr int INTEG_THREADS = 128;  // 4 voxels per thread, one block per CTA iteration
constexpr int INTEG_CTAS_PER_SM = 12;  // ~1.8k blocks (a 640 x 480 frame) in one wave

// Per-CTA state of the fusion loop: the near flags of the blocks in flight, OR-ed by their
// warps (a ring; the loop synchronises the CTA once per ring length, so no slot is reused
// while a warp still works on its block).
constexpr int INTEG_RING = 8;
struct IntegNear {
  unsigned any[INTEG_RING];
  int done[INTEG_RING];
};

// One collected block (entry `t` of the collected list, the calling CTA's `it`-th), the CTA of
// INTEG_THREADS: resolve it (update set, neighbour table) in one warp, chosen in turn so that
// the resolutions' round-trip chains of successive blocks run in different warps, then (FUSE)
// fuse the frame into its 512 voxels.  Voxels stream as float2 (d, W) pairs, 32 bytes per
// thread; depth is gathered through the read-only path.  Also records whether any voxel of
// the block has W > 0 and d < mu (used by gc): the block's last warp to finish writes it.
// No barrier: each warp moves on to the CTA's next block as soon as its own part is done.
template <bool FUSE>
__device__ __forceinline__ void integrate_block(const Vol& V, const FrameParams& fp, int4 t, uint32_t frame,
                                                uint32_t epoch, int it, IntegNear& N) {
  const float mu = V.mu, l = V.l, wmax = V.wmax;
  const int v0 = threadIdx.x * 4;
  const int lx = v0 & 7, ly = (v0 >> 3) & 7, lz = v0 >> 6;
  const int lane = threadIdx.x & 31;
  const int blk = t.z >= 0 ? t.z : __ldcg(&V.vals[t.w]);
  if (blk < 0) return;  // uniform over the CTA
  const uint64_t kk = ((uint64_t)(uint32_t)t.y << 32) | (uint32_t)t.x;
  const int4 key = make_int4((int)((kk >> 42) & 0x1FFFFF) - KEY_BIAS, (int)((kk >> 21) & 0x1FFFFF) - KEY_BIAS,
                             (int)(kk & 0x1FFFFF) - KEY_BIAS, t.w);
  if ((threadIdx.x >> 5) == (it & (INTEG_THREADS / 32 - 1))) resolve_block(V, blk, key, frame, epoch, lane);
  if (!FUSE) return;
  float4* p = reinterpret_cast<float4*>(V.tw + (size_t)blk * BV + v0);
  float4 q0 = __ldcg(p), q1 = __ldcg(p + 1);
  float dd[4] = {q0.x, q0.z, q1.x, q1.z};
  float ww[4] = {q0.y, q0.w, q1.y, q1.w};
  bool changed = false;
  const float py = (float)(key.y * BS + ly) * l, pz = (float)(key.z * BS + lz) * l;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float px = (float)(key.x * BS + lx + j) * l;
    int pix;
    float sdf;
    if (!project_voxel(fp, mu, px, py, pz, pix, sdf)) continue;
    const float dt = sdf < mu ? sdf : mu;
    const float num = dd[j] * ww[j] + dt;
    const float den = ww[j] + 1.0f;
    dd[j] = num / den;
    ww[j] = den < wmax ? den : wmax;
    changed = true;
  }
  if (changed) {
    p[0] = make_float4(dd[0], ww[0], dd[1], ww[1]);
    p[1] = make_float4(dd[2], ww[2], dd[3], ww[3]);
  }
  bool near = false;
#pragma unroll
  for (int j = 0; j < 4; ++j) near |= (ww[j] > 0.0f && dd[j] < mu);
  const bool wnear = __any_sync(0xffffffffu, near);
  if (lane == 0) {
    const int slot = it & (INTEG_RING - 1);
    if (wnear) atomicOr(&N.any[slot], 1u);
    __threadfence_block();
    if (atomicAdd(&N.done[slot], 1) == INTEG_THREADS / 32 - 1) {  // the block's last warp
      V.bnear[blk] = (uint8_t)(atomicOr(&N.any[slot], 0u) != 0);
      N.any[slot] = 0;
      N.done[slot] = 0;
    }
  }
}

// The calling CTA's share of the collected list (entries first, first + stride, ...).
template <bool FUSE>
__device__ __forceinline__ void integrate_share(const Vol& V, const FrameParams& fp, int first, int stride, int n,
                                                uint32_t frame, uint32_t epoch) {
  __shared__ IntegNear N;
  if (threadIdx.x < INTEG_RING) {
    N.any[threadIdx.x] = 0;
    N.done[threadIdx.x] = 0;
  }
  __syncthreads();
  for (int i = first, it = 0; i < n; i += stride, ++it) {
    integrate_block<FUSE>(V, fp, __ldcg(&V.touched[i]), frame, epoch, it, N);
    if ((it & (INTEG_RING - 1)) == INTEG_RING - 1) __syncthreads();
  }
}

// At the start of integrate call `frame` over n collected blocks (one thread; nothing in the
// call reads what it writes): statistics, the next call's collected count emptied, the mesh
// pass's block hand-out counter reset for the pass that follows.
__device__ __forceinline__ void integrate_begin(const Vol& V, int n, uint32_t frame) {
  V.ctl->c[C_ST_FRAME_BLOCKS] = n;
  reinterpret_cast<unsigned*>(V.ctl->c)[C_ST_COLLECTED] += (unsigned)n;  // wraps modulo 2^32
  V.ctl->c[touched_count(frame + 1)] = 0;
  V.ctl->c[C_FRAME] = (int)(frame + 1);
  V.ctl->c[C_MESH_NEXT] = 0;
}

// Every collected block, one per CTA iteration (FUSE = false: resolve only, for analytic
// fills).  The call's number and parameters come from the control block (stored by the
// collection).
template <bool FUSE>
__global__ void __launch_bounds__(INTEG_THREADS, INTEG_CTAS_PER_SM) k_integrate(Vol V, const FrameParams* __restrict__ fpp) {
  // the frame's parameters in shared memory: there they cannot alias the voxels the kernel
  // writes, so they are not reloaded from global memory after every block's stores
  __shared__ FrameParams sfp;
  static_assert(sizeof(FrameParams) % 4 == 0 && sizeof(FrameParams) / 4 <= INTEG_THREADS, "FrameParams copy");
  grid_dependency_wait();
  if (threadIdx.x < sizeof(FrameParams) / 4)
    reinterpret_cast<uint32_t*>(&sfp)[threadIdx.x] = __ldcg(reinterpret_cast<const uint32_t*>(fpp) + threadIdx.x);
  __syncthreads();
  const uint32_t frame = sfp.frame;
  const int n = min(__ldcg(&V.ctl->c[touched_count(frame)]), V.list_cap_touched);
  const uint32_t epoch = (uint32_t)__ldcg(&V.ctl->c[C_EPOCH]);
  if (blockIdx.x == 0 && threadIdx.x == 0) integrate_begin(V, n, frame);
  integrate_share<FUSE>(V, sfp, blockIdx.x, gridDim.x, n, frame, epoch);
  allow_dependent_launch();
}

}  // namespace vmk
