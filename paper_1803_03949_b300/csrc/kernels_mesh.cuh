// Mesh maintenance kernels: cube types (Sec. V-B), refinement (Sec. V-F), edge-owned
// vertices (Sec. V-C, Sec. IV), triangulation with type-change reuse (Sec. V-D) and the
// reference counts that drive recycling (Sec. V-E).
//
// One mesh pass is three launches over the update set, with no locks and no waiting:
//   A  k_mesh_types  per block: stage the 9^3 voxel halo (own block plus the +x/+y/+z
//                    neighbours' faces) in shared memory, compute every cube's type,
//                    refine it, refresh the block's existing vertices; for each cube
//                    whose effective type changed, release its old triangles (reference
//                    counts down, run to the free stack) and request the vertices of the
//                    new type's edges from their owner voxels (byte-flag OR, first
//                    requester appends the edge to a list);
//   B  k_vertices    per requested edge: allocate a vertex (aggregated pool pop) and set
//                    its position and normal; only the owner slot is written, so every
//                    vertex exists once (Sec. IV: no duplicate vertices);
//   C  k_triangles   per block: emit the new triangles of changed cubes (aggregated run
//                    pop), count the references, clear the request flags.
// The paper resolves concurrent vertex creation with an atomic first-claimer lock or with
// grouped serial launches (Sec. V-C); owner-computes replaces both here.
#pragma once

#include "vmesh_device.cuh"

namespace vmk {

enum MeshMode { M_UPDATE = 1, M_REFINE = 2 };

constexpr int MESH_THREADS = 256;
constexpr int HALO = 9;  // local voxel coordinates 0..8 on each axis
constexpr int HALO_N = HALO * HALO * HALO;

// Eqs. 3-5: snap a disturbed raw type to the nearest admissible regular type.
__device__ __forceinline__ int refine_type(int raw, int prev, const float* d, float eps) {
  if (__popc(raw ^ prev) > 3) return raw;
  int best = -1, bestd = 99;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    int diff = raw ^ (int)c_regular[j];
    int dh = __popc(diff);
    if (dh > 3) continue;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (((diff >> k) & 1) && !(fabsf(d[k]) < eps)) ok = false;
    if (ok && dh < bestd) {
      best = j;
      bestd = dh;
    }
  }
  return best >= 0 ? (int)c_regular[best] : raw;
}

// Vertex on the owned edge g -> g + e_a (Sec. V-C): t = d0 / (d0 - d1) (0.5 when equal),
// clamped to [-1, 2] so refined cubes extrapolate boundedly; position g l + t l e_a;
// normal = normalised gradient of the owner cube's trilinear interpolant at the vertex,
// component b != a from the corners g+e_b (eb0) and g+e_a+e_b (eb1), 0 if unusable.
__device__ __forceinline__ void edge_vertex(float l, int gx, int gy, int gz, int a, float d0, float d1,
                                            const float* eb0, const float* eb1, const bool* ub, float4* pos,
                                            float4* nrm) {
  float t = d0 == d1 ? 0.5f : d0 / (d0 - d1);
  if (t < -1.0f) t = -1.0f;
  if (t > 2.0f) t = 2.0f;
  float p[3] = {(float)gx * l, (float)gy * l, (float)gz * l};
  int g[3] = {gx, gy, gz};
  p[a] = (float)g[a] * l + t * l;
  float n[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (b == a) n[b] = d1 - d0;
    else n[b] = ub[b] ? (1.0f - t) * (eb0[b] - d0) + t * (eb1[b] - d1) : 0.0f;
  }
  float len = sqrtf((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
  *pos = make_float4(p[0], p[1], p[2], 0.0f);
  if (len > 0.0f) *nrm = make_float4(n[0] / len, n[1] / len, n[2] / len, 0.0f);
  else *nrm = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// Triangle-run free stacks (run length L = 1..5), aggregated over lanes with the same L.
__device__ __forceinline__ void run_push(const Vol& V, int L, int base) {
  cg::coalesced_group g0 = cg::coalesced_threads();
  cg::coalesced_group g = cg::labeled_partition(g0, L);
  int slot = 0;
  if (g.thread_rank() == 0) slot = atomicAdd(&V.ctl->c[C_RUN_TOP0 + L - 1], (int)g.size());
  slot = g.shfl(slot, 0) + (int)g.thread_rank();
  if (slot < V.run_cap[L - 1]) V.run_free[L - 1][slot] = base;
  else set_status(V, ST_POOL_FULL);
}

__device__ __forceinline__ int run_pop(const Vol& V, int L) {
  cg::coalesced_group g0 = cg::coalesced_threads();
  cg::coalesced_group g = cg::labeled_partition(g0, L);
  int n = (int)g.size(), rank = (int)g.thread_rank();
  int old = 0, from_stack = 0, bump0 = 0;
  if (rank == 0) {
    old = atomicSub(&V.ctl->c[C_RUN_TOP0 + L - 1], n);
    from_stack = old <= 0 ? 0 : (old < n ? old : n);
    if (from_stack < n) bump0 = atomicAdd(&V.ctl->c[C_TRI_BUMP], (n - from_stack) * L);
  }
  old = g.shfl(old, 0);
  from_stack = g.shfl(from_stack, 0);
  bump0 = g.shfl(bump0, 0);
  if (rank < from_stack) return __ldcg(&V.run_free[L - 1][old - 1 - rank]);
  long long b = (long long)bump0 + (long long)(rank - from_stack) * L;
  if (b + L > V.max_triangles) {
    set_status(V, ST_POOL_FULL);
    return -1;
  }
  return (int)b;
}

// Neighbour blocks at offsets (o & 1, o >> 1 & 1, o >> 2 & 1) of block `blk` (o = 0: itself).
__device__ __forceinline__ void load_neighbours(const Vol& V, int blk, int4 key, int* nb) {
  if (threadIdx.x < 8) {
    int o = threadIdx.x;
    nb[o] = o == 0 ? blk : find_block(V, key.x + (o & 1), key.y + ((o >> 1) & 1), key.z + ((o >> 2) & 1));
  }
}

// Pass A.  mode: M_UPDATE (types from the current TSDF; t_{i-1} := previous effective
// type; refresh existing vertices), M_REFINE (apply Eqs. 3-5 with the stored t_{i-1}).
__global__ void __launch_bounds__(MESH_THREADS) k_mesh_types(Vol V, int mode) {
  __shared__ float2 halo[HALO_N];
  __shared__ int nb[8];
  __shared__ int s_dtri;
  const int n = min(__ldcg(&V.ctl->c[C_N_UPDATE]), V.list_cap_update);
  const float eps = V.eps, l = V.l;
  int changed_local = 0;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int blk = V.update[i];
    const int4 key = V.bkey[blk];
    if (key.w < 0) continue;  // freed since it joined the set
    load_neighbours(V, blk, key, nb);
    if (threadIdx.x == 0) s_dtri = 0;
    __syncthreads();
    for (int h = threadIdx.x; h < HALO_N; h += MESH_THREADS) {
      int x = h % HALO, y = (h / HALO) % HALO, z = h / (HALO * HALO);
      int b = nb[(x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2)];
      halo[h] = b >= 0 ? __ldcg(&V.tw[(size_t)b * BV + (x & 7) + 8 * (y & 7) + 64 * (z & 7)]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    int dtri = 0;
    for (int c = threadIdx.x; c < BV; c += MESH_THREADS) {
      const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
      const size_t ci = (size_t)blk * BV + c;
      float d[8];
      bool valid = true;
      int raw = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float2 hv = halo[(x + c_corner[k][0]) + HALO * (y + c_corner[k][1]) + HALO * HALO * (z + c_corner[k][2])];
        d[k] = hv.x;
        valid &= hv.y > 0.0f;
        raw |= (hv.x < 0.0f) << k;
      }
      const int eff_old = V.code_eff[ci];
      int prev;
      if (mode & M_UPDATE) {
        prev = eff_old;
        V.code_prev[ci] = (uint8_t)eff_old;
      } else {
        prev = V.code_prev[ci];
      }
      int e = valid ? raw : 0;
      if (valid && (mode & M_REFINE)) e = refine_type(raw, prev, d, eps);
      if (e != eff_old) {
        ++changed_local;
        const int nold = c_ntri[eff_old];
        const int base = nold > 0 ? V.tri_base[ci] : -1;
        if (base >= 0) {
          for (int t = 0; t < nold; ++t) {
            int4 tr = V.tris[base + t];
            int vs[3] = {tr.x, tr.y, tr.z};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              if (vs[j] < 0) continue;
              if (atomicSub(&V.vref[vs[j]], 1) == 1) list_push(V, V.dead, C_N_DEAD, V.list_cap_dead, vs[j]);
            }
            V.tris[base + t] = make_int4(-1, -1, -1, -1);
          }
          run_push(V, nold, base);
        }
        const unsigned em = c_edgemask[e];
        for (int k = 0; k < 12; ++k) {
          if (!((em >> k) & 1)) continue;
          int ox = x + c_edge_owner[k][0], oy = y + c_edge_owner[k][1], oz = z + c_edge_owner[k][2];
          int a = c_edge_owner[k][3];
          int ob = nb[(ox >> 3) | ((oy >> 3) << 1) | ((oz >> 3) << 2)];
          if (ob < 0) continue;  // cannot happen for a valid cube
          int ov = (ox & 7) + 8 * (oy & 7) + 64 * (oz & 7);
          uint8_t* fm = V.vmask + (size_t)ob * BV + ov;
          if ((__ldcg(fm) >> a) & 1) continue;  // vertex exists
          uint8_t old = atomic_or_u8(fm, (uint8_t)(8 << a));
          if (!((old >> a) & 1) && !((old >> (3 + a)) & 1))
            list_push(V, V.newedge, C_N_NEWEDGE, V.list_cap_newedge, ob * EPB + ov * 3 + a);
        }
        V.tri_base[ci] = -1;
        V.chg[ci] = c_ntri[e] > 0 ? 1 : 0;
        V.code_eff[ci] = (uint8_t)e;
        dtri += (int)c_ntri[e] - nold;
      }
      if (mode & M_UPDATE) {
        // refresh the vertices this voxel owns (existing before this pass) from the new TSDF
        const uint8_t vm = __ldcg(V.vmask + ci);
        const int live = vm & ~(vm >> 3) & 7;
        if (live) {
          const float2 h0 = halo[x + HALO * y + HALO * HALO * z];
          const int gx = key.x * BS + x, gy = key.y * BS + y, gz = key.z * BS + z;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (!((live >> a) & 1)) continue;
            const int vid = V.edge_vtx[ci * 3 + a];
            if (vid < 0) continue;
            int oa[3] = {a == 0, a == 1, a == 2};
            float2 h1 = halo[(x + oa[0]) + HALO * (y + oa[1]) + HALO * HALO * (z + oa[2])];
            float eb0[3] = {0, 0, 0}, eb1[3] = {0, 0, 0};
            bool ub[3] = {false, false, false};
#pragma unroll
            for (int b = 0; b < 3; ++b) {
              if (b == a) continue;
              int ob3[3] = {b == 0, b == 1, b == 2};
              float2 q0 = halo[(x + ob3[0]) + HALO * (y + ob3[1]) + HALO * HALO * (z + ob3[2])];
              float2 q1 = halo[(x + oa[0] + ob3[0]) + HALO * (y + oa[1] + ob3[1]) + HALO * HALO * (z + oa[2] + ob3[2])];
              eb0[b] = q0.x;
              eb1[b] = q1.x;
              ub[b] = q0.y > 0.0f && q1.y > 0.0f;
            }
            float4 p, nn;
            edge_vertex(l, gx, gy, gz, a, h0.x, h1.x, eb0, eb1, ub, &p, &nn);
            V.vpos[vid] = p;
            V.vnrm[vid] = nn;
          }
        }
      }
    }
    if (dtri) atomicAdd(&s_dtri, dtri);
    __syncthreads();
    if (threadIdx.x == 0 && s_dtri) {
      atomicAdd(&V.bntri[blk], s_dtri);
      atomicAdd(&V.ctl->c[C_LIVE_TRIS], s_dtri);
    }
    __syncthreads();
  }
  if (changed_local) atomicAdd(&V.ctl->c[C_ST_CHANGED], changed_local);
}

// Value of local voxel (x, y, z) in 0..8 relative to block `ob` (key `k`); nbc caches the
// 8 neighbour block indices (-2 = not looked up).  Returns false when unusable (W == 0).
__device__ __forceinline__ bool voxel_rel(const Vol& V, int ob, int4 k, int* nbc, int x, int y, int z, float* d) {
  int o = (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2);
  if (nbc[o] == -2) nbc[o] = o == 0 ? ob : find_block(V, k.x + (o & 1), k.y + ((o >> 1) & 1), k.z + ((o >> 2) & 1));
  int b = nbc[o];
  if (b < 0) return false;
  float2 v = __ldcg(&V.tw[(size_t)b * BV + (x & 7) + 8 * (y & 7) + 64 * (z & 7)]);
  *d = v.x;
  return v.y > 0.0f;
}

// Pass B: one thread per requested edge creates its vertex.  The last CTA clamps the
// vertex free-stack top.
__global__ void __launch_bounds__(256) k_vertices(Vol V) {
  const int n = min(__ldcg(&V.ctl->c[C_N_NEWEDGE]), V.list_cap_newedge);
  int created = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e = V.newedge[i];
    const int ob = e / EPB, r = e - ob * EPB, ov = r / 3, a = r - ov * 3;
    const int4 k = V.bkey[ob];
    const int x = ov & 7, y = (ov >> 3) & 7, z = ov >> 6;
    int nbc[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) nbc[o] = -2;
    int oa[3] = {a == 0, a == 1, a == 2};
    float d0 = 0.f, d1 = 0.f;
    voxel_rel(V, ob, k, nbc, x, y, z, &d0);
    voxel_rel(V, ob, k, nbc, x + oa[0], y + oa[1], z + oa[2], &d1);
    float eb0[3] = {0, 0, 0}, eb1[3] = {0, 0, 0};
    bool ub[3] = {false, false, false};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b == a) continue;
      int o3[3] = {b == 0, b == 1, b == 2};
      bool u0 = voxel_rel(V, ob, k, nbc, x + o3[0], y + o3[1], z + o3[2], &eb0[b]);
      bool u1 = voxel_rel(V, ob, k, nbc, x + oa[0] + o3[0], y + oa[1] + o3[1], z + oa[2] + o3[2], &eb1[b]);
      ub[b] = u0 && u1;
    }
    float4 p, nn;
    edge_vertex(V.l, k.x * BS + x, k.y * BS + y, k.z * BS + z, a, d0, d1, eb0, eb1, ub, &p, &nn);
    const int vid = pool_pop(V, V.vtx_free, C_VTX_TOP, C_VTX_BUMP, V.max_vertices);
    if (vid < 0) continue;
    V.vpos[vid] = p;
    V.vnrm[vid] = nn;
    V.vref[vid] = 0;
    V.vedge[vid] = e;
    V.edge_vtx[e] = vid;
    __threadfence();
    atomic_or_u8(V.vmask + (size_t)ob * BV + ov, (uint8_t)(1 << a));
    atomicAdd(&V.bnvert[ob], 1);
    ++created;
  }
  if (created) {
    atomicAdd(&V.ctl->c[C_LIVE_VERTS], created);
    atomicAdd(&V.ctl->c[C_ST_NEW_VERTS], created);
  }
  if (last_block(V, C_DONE3)) {
    if (threadIdx.x == 0) {
      fold_top(V, C_VTX_TOP);
      V.ctl->c[C_DONE3] = 0;
    }
  }
}

// Pass C: emit the triangles of every changed cube of the update set and count their
// vertex references; then clear this pass's vertex-request flags.  The last CTA clamps
// the triangle-run stacks and empties the request list.
__global__ void __launch_bounds__(MESH_THREADS) k_triangles(Vol V) {
  __shared__ int nb[8];
  const int n = min(__ldcg(&V.ctl->c[C_N_UPDATE]), V.list_cap_update);
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int blk = V.update[i];
    const int4 key = V.bkey[blk];
    if (key.w < 0) continue;
    load_neighbours(V, blk, key, nb);
    __syncthreads();
    for (int c = threadIdx.x; c < BV; c += MESH_THREADS) {
      const size_t ci = (size_t)blk * BV + c;
      if (!V.chg[ci]) continue;
      const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
      const int e = V.code_eff[ci];
      const int nt = c_ntri[e];
      int base = -1;
      for (int L = 1; L <= 5; ++L)
        if (nt == L) base = run_pop(V, L);
      V.chg[ci] = 0;
      if (base < 0) continue;
      for (int t = 0; t < nt; ++t) {
        int vs[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          int k = c_tri[e][3 * t + j];
          int ox = x + c_edge_owner[k][0], oy = y + c_edge_owner[k][1], oz = z + c_edge_owner[k][2];
          int ob = nb[(ox >> 3) | ((oy >> 3) << 1) | ((oz >> 3) << 2)];
          int ov = (ox & 7) + 8 * (oy & 7) + 64 * (oz & 7);
          vs[j] = ob < 0 ? -1 : __ldcg(&V.edge_vtx[((size_t)ob * BV + ov) * 3 + c_edge_owner[k][3]]);
        }
        if (vs[0] < 0 || vs[1] < 0 || vs[2] < 0) {  // a vertex could not be created (pool full)
          set_status(V, ST_POOL_FULL);
          V.tris[base + t] = make_int4(-1, -1, -1, (int)ci);
          continue;
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) atomicAdd(&V.vref[vs[j]], 1);
        V.tris[base + t] = make_int4(vs[0], vs[1], vs[2], (int)ci);
      }
      V.tri_base[ci] = base;
    }
    __syncthreads();
  }
  // clear the request flags of this pass
  const int nr = min(__ldcg(&V.ctl->c[C_N_NEWEDGE]), V.list_cap_newedge);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
    const int e = V.newedge[i];
    const int ob = e / EPB, r = e - ob * EPB, ov = r / 3, a = r - ov * 3;
    atomic_and_u8(V.vmask + (size_t)ob * BV + ov, (uint8_t)~(8 << a));
  }
  if (last_block(V, C_DONE4)) {
    if (threadIdx.x == 0) {
#pragma unroll
      for (int L = 0; L < 5; ++L) fold_top(V, C_RUN_TOP0 + L);
      V.ctl->c[C_N_NEWEDGE] = 0;
      V.ctl->c[C_ST_UPDATE_BLOCKS] = n;
      V.ctl->c[C_DONE4] = 0;
    }
  }
}

}  // namespace vmk
