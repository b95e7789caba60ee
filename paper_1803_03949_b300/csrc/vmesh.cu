// C ABI of the vmesh library (declared in include/vmesh.h): volume lifetime, the
// per-frame calls, CUDA-graph replay of a whole frame, per-kernel timing and the
// download / export paths.  All device work is the kernels in this directory.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <climits>
#include <vector>

#include "vmesh.h"
#include "kernels_batch.cuh"
#include "kernels_diff.cuh"
#include "kernels_fusion.cuh"
#include "kernels_gc.cuh"
#include "kernels_io.cuh"
#include "kernels_memory.cuh"
#include "kernels_mesh.cuh"
#include "mc_table.h"
#include "vmesh_device.cuh"

using namespace vmk;

namespace {

enum KernelId { K_ALLOC = 0, K_INTEGRATE, K_LIST_ALL, K_MESH, K_GC_VERTICES, K_GC_BLOCKS, K_COUNT_ };
const char* kKernelNames[K_COUNT_] = {"k_alloc", "k_integrate", "k_list_all", "k_mesh", "k_gc_vertices", "k_gc_blocks"};

// Every allocated block joins the update set (full extraction).
__global__ void __launch_bounds__(256) k_list_all(Vol V) {
  const int hw = min(__ldcg(&V.ctl->c[C_BLK_BUMP]), V.max_blocks);
  const uint32_t epoch = (uint32_t)__ldcg(&V.ctl->c[C_EPOCH]);
  for (int blk = blockIdx.x * blockDim.x + threadIdx.x; blk < hw; blk += gridDim.x * blockDim.x) {
    int4 k = V.bkey[blk];
    if (k.w < 0) continue;
    V.ustamp[blk] = epoch;
    list_push(V, V.update, C_N_UPDATE, V.list_cap_update, blk);
  }
}

struct TimingRec {
  int kernel;
  cudaEvent_t a, b;
};

}  // namespace

struct vm_volume {
  vm_params p;
  Vol V;
  cudaStream_t stream = nullptr;      // the caller's stream: every call enqueues here
  cudaStream_t cur = nullptr;         // stream launches go to (the capture stream while capturing)
  cudaStream_t cap_stream = nullptr;  // owned non-blocking stream for graph capture
  int device = 0;                     // the device current when the volume was created
  int num_sms = 148;
  bool advance_pending = false;
  uint32_t frame = 1;  // number of the next integrate call (consecutive: the collected-count
                       // counters alternate with its parity)
  std::vector<void*> allocs;
  size_t bytes_allocated = 0;  // device memory held through allocs
  float* depth_buf = nullptr;  // device copy of a depth frame passed in pinned host memory
  size_t depth_cap = 0;        // its capacity in floats
  // download scratch: per-chunk counts (then offsets) of live vertices and triangles, the two
  // totals, the vertex remap table
  int* cta_counts = nullptr;
  int* cta_counts_t = nullptr;
  int* scan_total = nullptr;
  int* remap = nullptr;
  int cta_cap = 0;
  // timing
  unsigned timing_mask = 0;  // kernels (bit = KernelId) timed with events
  bool capturing = false;
  std::vector<TimingRec> recs;
  std::vector<TimingRec> graph_recs;  // event-record nodes of the captured frame graph
  bool graph_pending = false;         // a replay's node timings not yet collected
  std::vector<cudaEvent_t> event_pool;
  double tot_ms[K_COUNT_] = {0};
  long long launches[K_COUNT_] = {0};
  // differentiable path: recording state and its buffers (owned here, freed in free_all)
  bool diff_on = false;     // integrate calls are being recorded
  int diff_max = 0;         // recorded calls the buffers hold
  int diff_frames = 0;      // recorded calls so far
  int grad_next = -1;       // next recorded call vm_grad_depth takes (-1: gradients not started)
  int diff_rec_cap = 0;     // ints in V.drec
  std::vector<void*> diff_allocs;
  // graph replay of vm_step; the frame's parameters reach the graph as k_alloc's launch
  // arguments, replaced in alloc_node before every replay
  cudaGraph_t graph = nullptr;
  cudaGraphNode_t alloc_node = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_flags = -1;
  int graph_W = -1, graph_H = -1;
};

namespace {

vm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? VM_OK : VM_ERR_CUDA; }

cudaEvent_t get_event(vm_volume* v) {
  if (!v->event_pool.empty()) {
    cudaEvent_t e = v->event_pool.back();
    v->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch helper: records a pair of events around the launch while timing is on.  During
// graph capture the records become event-record nodes of the graph (their timings are
// collected after each replay).
template <typename F>
vm_status launch(vm_volume* v, int kid, F&& f) {
  cudaEvent_t a = nullptr, b = nullptr;
  const bool timed = (v->timing_mask >> kid) & 1;
  if (timed) {
    a = get_event(v);
    b = get_event(v);
    if (v->capturing) cudaEventRecordWithFlags(a, v->cur, cudaEventRecordExternal);
    else cudaEventRecord(a, v->cur);
  }
  (void)cudaGetLastError();  // drop a stale non-sticky error so it is not blamed on this launch
  f();
  cudaError_t e = cudaGetLastError();
  if (timed) {
    if (v->capturing) {
      cudaEventRecordWithFlags(b, v->cur, cudaEventRecordExternal);
      v->graph_recs.push_back({kid, a, b});
    } else {
      cudaEventRecord(b, v->cur);
      v->recs.push_back({kid, a, b});
    }
  }
  return cuda_status(e);
}

// Add the timings of the last graph replay (waits for it).
void collect_graph_timing(vm_volume* v) {
  if (!v->graph_pending) return;
  v->graph_pending = false;
  for (auto& r : v->graph_recs) {
    float ms = 0;
    cudaEventSynchronize(r.b);
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      v->tot_ms[r.kernel] += ms;
      v->launches[r.kernel] += 1;
    }
  }
}

template <typename T>
bool dalloc(vm_volume* v, T** p, size_t count, int fill_byte) {
  void* q = nullptr;
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = sizeof(T);
  if (cudaMalloc(&q, bytes) != cudaSuccess) return false;
  v->allocs.push_back(q);
  v->bytes_allocated += bytes;
  if (cudaMemsetAsync(q, fill_byte, bytes, v->cur) != cudaSuccess) return false;
  *p = static_cast<T*>(q);
  return true;
}

bool finite_all(const float* a, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

bool make_frame(const vm_intrinsics* K, const float* Twc, const float* Tcw, const float* depth, FrameParams* fp) {
  if (!K || !Twc || !Tcw || !depth) return false;
  if (K->width < 1 || K->height < 1 || K->width > 16384 || K->height > 16384) return false;
  if (!(K->fx > 0) || !(K->fy > 0) || !std::isfinite(K->fx) || !std::isfinite(K->fy) || !std::isfinite(K->cx) ||
      !std::isfinite(K->cy))
    return false;
  if (!finite_all(Twc, 16) || !finite_all(Tcw, 16)) return false;
  // bound the slope of every pixel ray (a field of view below ~178 degrees)
  const double sx = std::fmax(std::fabs((double)K->cx), std::fabs(K->width - 1 - (double)K->cx)) / K->fx;
  const double sy = std::fmax(std::fabs((double)K->cy), std::fabs(K->height - 1 - (double)K->cy)) / K->fy;
  if (!(sx <= 64.0) || !(sy <= 64.0)) return false;
  fp->depth = depth;
  fp->depth_in = depth;
  fp->depth_copy = nullptr;
  fp->W = K->width;
  fp->H = K->height;
  fp->fx = K->fx;
  fp->fy = K->fy;
  fp->cx = K->cx;
  fp->cy = K->cy;
  fp->rfx = 1.0f / K->fx;
  fp->rfy = 1.0f / K->fy;
  for (int i = 0; i < 12; ++i) {
    fp->Twc[i] = Twc[i];
    fp->Tcw[i] = Tcw[i];
  }
  return true;
}

int grid_for(vm_volume* v, int per_sm) { return v->num_sms * per_sm; }

// A depth frame in device memory is read where it is.  One in pinned host memory (mapped into
// the device's address space) is read by the collection kernel across the host link, and that
// kernel keeps a device copy for the kernels after it: the frame's transfer overlaps the
// collection instead of preceding it.  Pageable host memory is refused.
vm_status prepare_depth(vm_volume* v, FrameParams* fp) {
  cudaPointerAttributes a = {};
  if (cudaPointerGetAttributes(&a, fp->depth_in) != cudaSuccess) {
    (void)cudaGetLastError();
    return VM_ERR_INVALID_ARG;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return VM_OK;
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return VM_ERR_INVALID_ARG;
  const size_t n = (size_t)fp->W * fp->H;
  if (n > v->depth_cap) {
    if (v->depth_buf) {  // frames already enqueued (on any stream) may still read the old copy
      if (cudaDeviceSynchronize() != cudaSuccess) return VM_ERR_CUDA;
      cudaFree(v->depth_buf);
      v->depth_buf = nullptr;
      v->depth_cap = 0;
    }
    if (cudaMalloc(&v->depth_buf, n * sizeof(float)) != cudaSuccess) {
      (void)cudaGetLastError();
      v->depth_buf = nullptr;
      return VM_ERR_OOM;
    }
    v->depth_cap = n;
  }
  fp->depth_in = static_cast<const float*>(a.devicePointer);
  fp->depth_copy = v->depth_buf;
  fp->depth = v->depth_buf;
  return VM_OK;
}

// Launch with programmatic stream serialization: the kernel may be scheduled while the
// previous kernel in the stream drains; it waits for that kernel's results in-kernel.
template <typename... Params, typename... Args>
void launch_dependent(void (*kernel)(Params...), int grid, int block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---- enqueue helpers (no validation)
dim3 alloc_grid(const FrameParams& fp) {
  return dim3((fp.W + ALLOC_TILE_W1 - 1) / ALLOC_TILE_W1, (fp.H + ALLOC_TILE_H - 1) / ALLOC_TILE_H);
}

vm_status enqueue_integrate(vm_volume* v, const FrameParams& fp) {
  Ctl* ctl = v->V.ctl;
  const int adv = v->advance_pending ? 1 : 0;
  vm_status st = launch(v, K_ALLOC, [&] { k_alloc<<<alloc_grid(fp), ALLOC_THREADS, 0, v->cur>>>(v->V, fp, adv); });
  if (st) return st;
  st = launch(v, K_INTEGRATE, [&] {
    launch_dependent(k_integrate<true>, grid_for(v, INTEG_CTAS_PER_SM), INTEG_THREADS, 0, v->cur, v->V, (const FrameParams*)&ctl->fp);
  });
  v->advance_pending = false;
  return st;
}

vm_status enqueue_list_all(vm_volume* v) {
  cudaError_t e = cudaMemsetAsync(&v->V.ctl->c[C_N_UPDATE], 0, sizeof(int), v->cur);
  if (e != cudaSuccess) return VM_ERR_CUDA;
  return launch(v, K_LIST_ALL, [&] { k_list_all<<<grid_for(v, 4), 256, 0, v->cur>>>(v->V); });
}

// after_integrate: the pass directly follows an integrate call, whose first CTA resets the
// pass's block hand-out counter; otherwise it is reset here.
vm_status enqueue_mesh_pass(vm_volume* v, int mode, bool after_integrate) {
  const bool ce = (v->p.flags & VM_PARAM_COMPACT_EDGES) != 0;
  if (!after_integrate && cudaMemsetAsync(&v->V.ctl->c[C_MESH_NEXT], 0, sizeof(int), v->cur) != cudaSuccess)
    return VM_ERR_CUDA;
  return launch(v, K_MESH, [&] {
    launch_dependent(ce ? k_mesh<true> : k_mesh<false>, grid_for(v, mesh_ctas_per_sm(ce)), MESH_THREADS, 0, v->cur,
                     v->V, mode);
  });
}

vm_status enqueue_update(vm_volume* v, int flags, bool after_integrate) {
  vm_status st = VM_OK;
  if (flags & VM_FULL) st = enqueue_list_all(v);
  if (st) return st;
  st = enqueue_mesh_pass(v, M_UPDATE | ((flags & VM_REFINE) ? M_REFINE : 0), after_integrate && !(flags & VM_FULL));
  v->advance_pending = true;
  return st;
}

vm_status enqueue_gc(vm_volume* v) {
  const bool ce = (v->p.flags & VM_PARAM_COMPACT_EDGES) != 0;
  vm_status st = launch(v, K_GC_VERTICES, [&] {
    launch_dependent(ce ? k_gc_vertices<true> : k_gc_vertices<false>, grid_for(v, GCV_CTAS_PER_SM), GCV_THREADS, 0, v->cur, v->V);
  });
  if (st) return st;
  const int consumed = v->advance_pending ? 1 : 0;
  return launch(v, K_GC_BLOCKS,
                [&] { launch_dependent(k_gc_blocks, grid_for(v, 2), 256, 0, v->cur, v->V, consumed); });
}

vm_status sync_status(vm_volume* v) {
  if (cudaStreamSynchronize(v->stream) != cudaSuccess) return VM_ERR_CUDA;
  return VM_OK;
}

int read_counter(vm_volume* v, int c) {
  int x = 0;
  cudaMemcpy(&x, &v->V.ctl->c[c], sizeof(int), cudaMemcpyDeviceToHost);
  return x;
}

// The kernel node of `g` that launches `func`, or null.
cudaGraphNode_t find_kernel_node(cudaGraph_t g, void* func) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return nullptr;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return nullptr;
  for (cudaGraphNode_t node : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(node, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    if (cudaGraphKernelNodeGetParams(node, &kp) == cudaSuccess && kp.func == func) return node;
  }
  return nullptr;
}

void drop_graph(vm_volume* v) {
  if (v->graph_exec) {
    cudaStreamSynchronize(v->stream);
    cudaGraphExecDestroy(v->graph_exec);
  }
  if (v->graph) cudaGraphDestroy(v->graph);
  v->graph = nullptr;
  v->alloc_node = nullptr;
  v->graph_exec = nullptr;
  v->graph_flags = -1;
  v->graph_pending = false;
  for (auto& r : v->graph_recs) {
    v->event_pool.push_back(r.a);
    v->event_pool.push_back(r.b);
  }
  v->graph_recs.clear();
}

void free_all(vm_volume* v) {
  drop_graph(v);
  for (auto& r : v->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : v->event_pool) cudaEventDestroy(e);
  for (void* p : v->allocs) cudaFree(p);
  v->allocs.clear();
  if (v->depth_buf) cudaFree(v->depth_buf);
  v->depth_buf = nullptr;
  v->depth_cap = 0;
  for (void* p : v->diff_allocs) cudaFree(p);
  v->diff_allocs.clear();
  if (v->cap_stream) cudaStreamDestroy(v->cap_stream);
  v->cap_stream = nullptr;
}

// Enqueue the counts of the live vertices and triangles below their pools' high-water marks:
// per-chunk offsets in cta_counts / cta_counts_t, the totals in scan_total[0] / [1].
vm_status enqueue_live_counts(vm_volume* v) {
  const int grid = grid_for(v, 8);
  k_chunk_counts<false><<<grid, 256, 0, v->stream>>>(v->V, v->cta_counts);
  k_scan_chunks<false><<<1, 1024, 0, v->stream>>>(v->V, v->cta_counts, v->scan_total);
  k_chunk_counts<true><<<grid, 256, 0, v->stream>>>(v->V, v->cta_counts_t);
  k_scan_chunks<true><<<1, 1024, 0, v->stream>>>(v->V, v->cta_counts_t, v->scan_total + 1);
  return cudaGetLastError() == cudaSuccess ? VM_OK : VM_ERR_CUDA;
}

// The live counts on the host (one synchronisation).
vm_status live_counts(vm_volume* v, int* nv, int* nt) {
  vm_status st = enqueue_live_counts(v);
  if (st) return st;
  int tot[2] = {0, 0};
  if (cudaMemcpyAsync(tot, v->scan_total, sizeof(tot), cudaMemcpyDeviceToHost, v->stream) != cudaSuccess)
    return VM_ERR_CUDA;
  if ((st = sync_status(v))) return st;
  *nv = tot[0];
  *nt = tot[1];
  return VM_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

vm_status vm_create_volume(const vm_params* p, void* cuda_stream, vm_volume** out) {
  if (!p || !out) return VM_ERR_INVALID_ARG;
  *out = nullptr;
  const uint32_t hb = p->hash_buckets;
  if (!(p->voxel_size >= 1e-4f) || !std::isfinite(p->voxel_size) || !(p->trunc > 0) ||
      !(p->trunc <= 32.0f * p->voxel_size) || !(p->eps_refine >= 0) || !std::isfinite(p->eps_refine) ||
      !(p->w_max >= 1) || !std::isfinite(p->w_max) || hb < 16 || hb > (1u << 30) || (hb & (hb - 1)) ||
      p->max_blocks < 1 || p->max_blocks > (1u << 21) || p->max_vertices < 1 || p->max_vertices > (1u << 30) ||
      p->max_triangles < 1 || p->max_triangles > (1u << 30) || (p->flags & ~VM_PARAM_COMPACT_EDGES))
    return VM_ERR_INVALID_ARG;
  static vmk_host::McTable table;
  static bool table_built = false;
  if (!table_built) {
    vmk_host::build_mc_table(table);
    table_built = true;
  }
  if (!table.ok) return VM_ERR_INVALID_ARG;

  vm_volume* v = new vm_volume();
  v->p = *p;
  v->stream = static_cast<cudaStream_t>(cuda_stream);
  v->cur = v->stream;
  int dev = 0;
  cudaGetDevice(&dev);
  v->device = dev;
  cudaDeviceGetAttribute(&v->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (v->num_sms <= 0) v->num_sms = 148;
  // the mesh kernel keeps ~32 KB of shared memory per CTA: ask for the largest carveout
  cudaFuncSetAttribute(k_mesh<false>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_mesh<true>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(kb_mesh<false>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(kb_mesh<true>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  (void)cudaGetLastError();
  if (cudaMemcpyToSymbol(c_ntri, table.ntri, sizeof(table.ntri)) != cudaSuccess ||
      cudaMemcpyToSymbol(c_tri, table.tri, sizeof(table.tri)) != cudaSuccess ||
      cudaMemcpyToSymbol(c_edgemask, table.edgemask, sizeof(table.edgemask)) != cudaSuccess) {
    delete v;
    return VM_ERR_CUDA;
  }

  Vol& V = v->V;
  V.l = p->voxel_size;
  V.ibs = 1.0f / (V.l * (float)BS);
  V.mu = p->trunc;
  V.eps = p->eps_refine;
  V.wmax = p->w_max;
  V.hmask = hb - 1;
  V.max_blocks = (int)p->max_blocks;
  V.max_vertices = (int)p->max_vertices;
  V.max_triangles = (int)p->max_triangles;
  for (int L = 1; L <= 5; ++L) V.run_cap[L - 1] = (int)(p->max_triangles / L) + 1;
  V.list_cap_touched = (int)(p->max_blocks < hb ? p->max_blocks : hb);
  V.list_cap_update = (int)p->max_blocks;
  V.list_cap_dead = (int)((2ull * p->max_vertices) < (1ull << 31) - 1 ? 2ull * p->max_vertices : (1ull << 31) - 1);
  V.list_cap_deadrun = (int)p->max_triangles;
  const size_t NB = p->max_blocks, NV = p->max_vertices, NT = p->max_triangles;
  const bool compact = (p->flags & VM_PARAM_COMPACT_EDGES) != 0;
  bool ok = dalloc(v, &V.keys, hb, 0xFF) && dalloc(v, &V.vals, hb, 0xFF) && dalloc(v, &V.stamp, hb, 0) &&
            dalloc(v, &V.ustamp, NB, 0) && dalloc(v, &V.bkey, NB, 0xFF) && dalloc(v, &V.nbr, NB * 16, 0xFF) &&
            dalloc(v, &V.bntri, NB, 0) && dalloc(v, &V.bnvert, NB, 0) && dalloc(v, &V.bnear, NB, 0) &&
            dalloc(v, &V.bepoch, NB, 0) && dalloc(v, &V.bborn, NB, 0) && dalloc(v, &V.tw, NB * BV, 0) &&
            dalloc(v, &V.code_eff, NB * BV, 0) && dalloc(v, &V.code_prev, NB * BV, 0) &&
            dalloc(v, &V.vmask, NB * BV, 0) &&
            (compact ? dalloc(v, &V.edge_rec, NB * BV, 0xFF) && dalloc(v, &V.erec, NV * 3, 0xFF) &&
                           dalloc(v, &V.rec_free, NV, 0) && dalloc(v, &V.dead_rec, NV, 0)
                     : dalloc(v, &V.edge_vtx, NB * BV * 3, 0xFF)) &&
            dalloc(v, &V.tri_base, NB * BV, 0xFF) && dalloc(v, &V.vrec, 2 * (size_t)NV, 0) &&
            dalloc(v, &V.vref, NV, 0xFF) && dalloc(v, &V.vedge, NV, 0xFF) && dalloc(v, &V.tris, NT, 0xFF) &&
            dalloc(v, &V.blk_free, NB, 0) && dalloc(v, &V.vtx_free, NV, 0) &&
            dalloc(v, &V.touched, (size_t)V.list_cap_touched, 0) && dalloc(v, &V.update, NB, 0) &&
            dalloc(v, &V.dead, (size_t)V.list_cap_dead, 0) && dalloc(v, &V.deadrun, (size_t)V.list_cap_deadrun, 0) &&
            dalloc(v, &V.ctl, 1, 0);
  for (int L = 0; L < 5 && ok; ++L) ok = dalloc(v, &V.run_free[L], (size_t)V.run_cap[L], 0);
  uint4* tt = nullptr;
  if (ok) ok = dalloc(v, &tt, MESH_TABLE_UINT4, 0);
  if (ok) {
    // the mesh pass's tables, copied to shared memory by every CTA:
    // packed triangles: 15 edge ids of 4 bits (triangle t, corner j at bit 4 (3 t + j)), the
    // count in bits 60..63; the edge mask of each type; the halo's neighbour voxel pairs
    struct {
      uint64_t packed[256];
      uint16_t emask[256];
      uint16_t pairs[256];
    } tab = {};
    for (int c = 0; c < 256; ++c) {
      uint64_t w = (uint64_t)table.ntri[c] << 60;
      for (int i = 0; i < 3 * table.ntri[c]; ++i) w |= (uint64_t)(table.tri[c][i] & 15) << (4 * i);
      tab.packed[c] = w;
      tab.emask[c] = table.edgemask[c];
    }
    halo_pairs(tab.pairs);
    static_assert(sizeof(tab) == MESH_TABLE_UINT4 * sizeof(uint4), "mesh table layout");
    ok = cudaMemcpyAsync(tt, &tab, sizeof(tab), cudaMemcpyHostToDevice, v->stream) == cudaSuccess &&
         cudaStreamSynchronize(v->stream) == cudaSuccess;
    V.tri_table = tt;
  }
  if (!ok) {
    free_all(v);
    delete v;
    return VM_ERR_OOM;
  }
  int init[C_EPOCH + 1] = {};
  init[C_FRAME] = 1;
  init[C_EPOCH] = 1;
  if (cudaMemcpyAsync(V.ctl->c, init, sizeof(init), cudaMemcpyHostToDevice, v->stream) != cudaSuccess ||
      cudaStreamSynchronize(v->stream) != cudaSuccess) {
    free_all(v);
    delete v;
    return VM_ERR_CUDA;
  }
  *out = v;
  return VM_OK;
}

vm_status vm_destroy_volume(vm_volume* v) {
  if (!v) return VM_OK;
  cudaStreamSynchronize(v->stream);
  free_all(v);
  delete v;
  return VM_OK;
}

vm_status vm_set_stream(vm_volume* v, void* s) {
  if (!v) return VM_ERR_INVALID_ARG;
  drop_graph(v);
  v->stream = static_cast<cudaStream_t>(s);
  v->cur = v->stream;
  return VM_OK;
}

vm_status vm_integrate_depth(vm_volume* v, const float* depth, const vm_intrinsics* K, const float Twc[16],
                             const float Tcw[16]) {
  if (!v) return VM_ERR_INVALID_ARG;
  FrameParams fp;
  if (!make_frame(K, Twc, Tcw, depth, &fp)) return VM_ERR_INVALID_ARG;
  if (v->diff_on && (v->diff_frames >= v->diff_max || v->grad_next >= 0)) return VM_ERR_INVALID_ARG;
  fp.frame = v->frame;
  vm_status st = prepare_depth(v, &fp);
  if (st) return st;
  st = enqueue_integrate(v, fp);
  if (st) return st;
  ++v->frame;
  if (!v->diff_on) return st;
  (void)cudaGetLastError();
  k_diff_record<<<grid_for(v, INTEG_CTAS_PER_SM), INTEG_THREADS, 0, v->stream>>>(v->V, v->diff_frames);
  ++v->diff_frames;
  return cuda_status(cudaGetLastError());
}

vm_status vm_update_mesh(vm_volume* v, int flags) {
  if (!v || (flags & ~(VM_FULL | VM_REFINE))) return VM_ERR_INVALID_ARG;
  return enqueue_update(v, flags, false);
}

vm_status vm_refine_mesh(vm_volume* v, int full) {
  if (!v) return VM_ERR_INVALID_ARG;
  vm_status st = VM_OK;
  if (full) st = enqueue_list_all(v);
  if (st) return st;
  return enqueue_mesh_pass(v, M_REFINE, false);
}

vm_status vm_gc(vm_volume* v) {
  if (!v || v->diff_on) return VM_ERR_INVALID_ARG;  // recycling would rename recorded voxels
  return enqueue_gc(v);
}

vm_status vm_step(vm_volume* v, const float* depth, const vm_intrinsics* K, const float Twc[16], const float Tcw[16],
                  int flags, int use_graph) {
  if (!v || (flags & ~(VM_FULL | VM_REFINE | VM_GC)) || v->diff_on) return VM_ERR_INVALID_ARG;
  FrameParams fp;
  if (!make_frame(K, Twc, Tcw, depth, &fp)) return VM_ERR_INVALID_ARG;
  fp.frame = v->frame;
  if (const vm_status ps = prepare_depth(v, &fp)) return ps;
  auto body = [&]() -> vm_status {
    vm_status s = enqueue_integrate(v, fp);
    if (s) return s;
    s = enqueue_update(v, flags & (VM_FULL | VM_REFINE), true);
    if (s) return s;
    if (flags & VM_GC) s = enqueue_gc(v);
    return s;
  };
  // A frame graph is captured with the epoch advancing at its start, i.e. for frames that
  // follow a mesh update; other frames run as plain launches.
  if (!use_graph || !v->advance_pending) {
    const vm_status s = body();
    if (!s) ++v->frame;
    return s;
  }
  if (!v->graph_exec || v->graph_flags != flags || v->graph_W != fp.W || v->graph_H != fp.H) {
    drop_graph(v);
    // Capture on an owned stream (the legacy NULL stream cannot be captured); the graph is
    // then launched on the caller's stream.
    if (!v->cap_stream && cudaStreamCreateWithFlags(&v->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      v->cap_stream = nullptr;
      return VM_ERR_CUDA;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(v->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      (void)cudaGetLastError();
      return VM_ERR_CUDA;
    }
    v->capturing = true;
    v->cur = v->cap_stream;
    vm_status s = body();
    cudaError_t e = cudaStreamEndCapture(v->cap_stream, &g);
    v->capturing = false;
    v->cur = v->stream;
    if (s) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return VM_ERR_CUDA;
    }
    v->graph = g;
    v->alloc_node = find_kernel_node(g, reinterpret_cast<void*>(k_alloc));
    e = v->alloc_node ? cudaGraphInstantiate(&v->graph_exec, g, 0) : cudaErrorInvalidValue;
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      v->graph_exec = nullptr;
      drop_graph(v);
      return VM_ERR_CUDA;
    }
    v->graph_flags = flags;
    v->graph_W = fp.W;
    v->graph_H = fp.H;
  }
  v->advance_pending = true;
  collect_graph_timing(v);  // a previous replay's node events are about to be re-recorded
  // this frame's parameters become k_alloc's arguments (the captured graph advances the
  // epoch at its start, so advance_epoch is 1)
  int adv = 1;
  void* args[3] = {&v->V, &fp, &adv};
  cudaKernelNodeParams kp = {};
  kp.func = reinterpret_cast<void*>(k_alloc);
  kp.gridDim = alloc_grid(fp);
  kp.blockDim = dim3(ALLOC_THREADS);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  cudaError_t e = cudaGraphExecKernelNodeSetParams(v->graph_exec, v->alloc_node, &kp);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return VM_ERR_CUDA;
  }
  e = cudaGraphLaunch(v->graph_exec, v->stream);
  v->graph_pending = v->timing_mask && !v->graph_recs.empty();
  if (e == cudaSuccess) ++v->frame;
  return cuda_status(e);
}

vm_status vm_last_error(vm_volume* v) {
  if (!v) return VM_ERR_INVALID_ARG;
  if (sync_status(v)) return VM_ERR_CUDA;
  int st = read_counter(v, C_STATUS);
  return (vm_status)st;
}

static vm_status ensure_scan_scratch(vm_volume* v) {
  if (v->remap) return VM_OK;
  const int items = v->p.max_vertices > v->p.max_triangles ? v->p.max_vertices : v->p.max_triangles;
  v->cta_cap = (items + SCAN_ITEMS - 1) / SCAN_ITEMS + 1;
  if (!dalloc(v, &v->cta_counts, (size_t)v->cta_cap, 0) || !dalloc(v, &v->cta_counts_t, (size_t)v->cta_cap, 0) ||
      !dalloc(v, &v->scan_total, 2, 0) ||
      !dalloc(v, &v->remap, v->p.max_vertices, 0xFF))
    return VM_ERR_OOM;
  return VM_OK;
}

vm_status vm_mesh_counts(vm_volume* v, int64_t* nv, int64_t* nt) {
  if (!v || !nv || !nt) return VM_ERR_INVALID_ARG;
  vm_status st = ensure_scan_scratch(v);
  if (st) return st;
  int a = 0, b = 0;
  if ((st = live_counts(v, &a, &b))) return st;
  *nv = a;
  *nt = b;
  return VM_OK;
}

vm_status vm_mesh_memory_stats(vm_volume* v, vm_mesh_memory* m) {
  if (!v || !m) return VM_ERR_INVALID_ARG;
  int64_t nv = 0, nt = 0;
  vm_status st = vm_mesh_counts(v, &nv, &nt);
  if (st) return st;
  unsigned long long* d = nullptr;
  unsigned long long bv = 0;
  (void)cudaGetLastError();
  bool ok = cudaMalloc(&d, sizeof(*d)) == cudaSuccess && cudaMemsetAsync(d, 0, sizeof(*d), v->stream) == cudaSuccess;
  if (ok) {
    k_block_vertices<<<grid_for(v, 8), 128, 0, v->stream>>>(v->V, d);
    ok = cudaGetLastError() == cudaSuccess &&
         cudaMemcpyAsync(&bv, d, sizeof(bv), cudaMemcpyDeviceToHost, v->stream) == cudaSuccess &&
         cudaStreamSynchronize(v->stream) == cudaSuccess;
  }
  cudaFree(d);
  if (!ok) {
    (void)cudaGetLastError();
    return VM_ERR_CUDA;
  }
  const int64_t blocks = read_counter(v, C_LIVE_BLOCKS);
  const bool ce = (v->p.flags & VM_PARAM_COMPACT_EDGES) != 0;
  const int64_t records =
      !ce ? 0
          : std::max<int64_t>(0, (int64_t)std::min(read_counter(v, C_REC_BUMP), (int)v->p.max_vertices) -
                                     std::max(read_counter(v, C_REC_TOP), 0));
  // per voxel (cube): (d, W) 8, current and previous type 2, vertex flags 1, then either the
  // vertex ids of its 3 owned edges 12 or (compact) an edge-record index 4 with a 12 B record
  // per voxel that owns a vertex; triangle-run start 4
  const int64_t cube = 8 + 2 + 1 + (ce ? 4 : 12) + 4;
  // per block: key + bucket 16, neighbour table 64, triangle/vertex counts 8, near flag 1,
  // three stamps 12; per vertex: position 16, normal 16, reference count 4, owning edge 4;
  // per triangle: 16; per hash bucket: key 8, block index 4, stamp 4
  const int64_t per_block = 16 + 64 + 8 + 1 + 12, per_vertex = 40, per_tri = 16, per_bucket = 16;
  m->vertices = nv;
  m->triangles = nt;
  m->block_vertices = (int64_t)bv;
  m->loose_vertices = 3 * nt;
  m->blocks = blocks;
  m->cube_bytes = cube;
  m->edge_records = records;
  m->bytes_in_use = blocks * (BV * cube + per_block) + records * 12 + nv * per_vertex + nt * per_tri +
                    (int64_t)(v->V.hmask + 1) * per_bucket;
  m->bytes_allocated = (int64_t)v->bytes_allocated;
  return VM_OK;
}

vm_status vm_download_mesh(vm_volume* v, float* pos, float* nrm, int32_t* tris, uint64_t* keys, int32_t* refcount,
                           int on_device) {
  if (!v || !pos || !nrm || !tris) return VM_ERR_INVALID_ARG;
  vm_status st = ensure_scan_scratch(v);
  if (st) return st;
  const int grid = grid_for(v, 8);
  if (on_device) {  // counts, offsets and both compactions in stream order; one synchronisation
    if ((st = enqueue_live_counts(v))) return st;
    k_compact_vertices<<<grid, 256, 0, v->stream>>>(v->V, v->cta_counts, v->remap, pos, nrm, keys, refcount, INT_MAX);
    k_compact_triangles<<<grid, 256, 0, v->stream>>>(v->V, v->cta_counts_t, v->remap, tris, INT_MAX);
    if (cudaGetLastError() != cudaSuccess) return VM_ERR_CUDA;
    return sync_status(v);
  }
  // host buffers: the counts first (device staging buffers of those sizes), then the same
  int nv = 0, nt = 0;
  if ((st = live_counts(v, &nv, &nt))) return st;
  std::vector<void*> tmp;
  auto tmp_alloc = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes ? bytes : 4) != cudaSuccess) return nullptr;
    tmp.push_back(q);
    return q;
  };
  auto cleanup = [&]() {
    for (void* q : tmp) cudaFree(q);
  };
  float* dpos = (float*)tmp_alloc((size_t)nv * 12);
  float* dnrm = (float*)tmp_alloc((size_t)nv * 12);
  uint64_t* dkeys = keys ? (uint64_t*)tmp_alloc((size_t)nv * 8) : nullptr;
  int32_t* dref = refcount ? (int32_t*)tmp_alloc((size_t)nv * 4) : nullptr;
  int32_t* dtris = (int32_t*)tmp_alloc((size_t)nt * 12);
  if (!dpos || !dnrm || (keys && !dkeys) || (refcount && !dref) || !dtris) {
    (void)cudaGetLastError();
    cleanup();
    return VM_ERR_OOM;
  }
  k_compact_vertices<<<grid, 256, 0, v->stream>>>(v->V, v->cta_counts, v->remap, dpos, dnrm, dkeys, dref, nv);
  k_compact_triangles<<<grid, 256, 0, v->stream>>>(v->V, v->cta_counts_t, v->remap, dtris, nt);
  bool ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(v->stream) == cudaSuccess;
  ok = ok && cudaMemcpy(pos, dpos, (size_t)nv * 12, cudaMemcpyDeviceToHost) == cudaSuccess &&
       cudaMemcpy(nrm, dnrm, (size_t)nv * 12, cudaMemcpyDeviceToHost) == cudaSuccess &&
       cudaMemcpy(tris, dtris, (size_t)nt * 12, cudaMemcpyDeviceToHost) == cudaSuccess &&
       (!keys || cudaMemcpy(keys, dkeys, (size_t)nv * 8, cudaMemcpyDeviceToHost) == cudaSuccess) &&
       (!refcount || cudaMemcpy(refcount, dref, (size_t)nv * 4, cudaMemcpyDeviceToHost) == cudaSuccess);
  cleanup();
  return ok ? VM_OK : VM_ERR_CUDA;
}

vm_status vm_download_mesh_into(vm_volume* v, float* pos, float* nrm, int32_t* tris, uint64_t* keys,
                                int32_t* refcount, int64_t cap_v, int64_t cap_t, int64_t* nv, int64_t* nt) {
  if (!v || !pos || !nrm || !tris || !nv || !nt || cap_v < 0 || cap_t < 0) return VM_ERR_INVALID_ARG;
  vm_status st = ensure_scan_scratch(v);
  if (st) return st;
  const int grid = grid_for(v, 8);
  const int cv = (int)std::min<int64_t>(cap_v, INT_MAX), ct = (int)std::min<int64_t>(cap_t, INT_MAX);
  int tot[2] = {0, 0};
  if ((st = enqueue_live_counts(v))) return st;
  k_compact_vertices<<<grid, 256, 0, v->stream>>>(v->V, v->cta_counts, v->remap, pos, nrm, keys, refcount, cv);
  k_compact_triangles<<<grid, 256, 0, v->stream>>>(v->V, v->cta_counts_t, v->remap, tris, ct);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(tot, v->scan_total, sizeof(tot), cudaMemcpyDeviceToHost, v->stream) != cudaSuccess)
    return VM_ERR_CUDA;
  if ((st = sync_status(v))) return st;
  *nv = tot[0];
  *nt = tot[1];
  return (tot[0] > cap_v || tot[1] > cap_t) ? VM_ERR_INVALID_ARG : VM_OK;
}

vm_status vm_mesh_size_async(vm_volume* v, int32_t* dst, int on_device) {
  if (!v || !dst) return VM_ERR_INVALID_ARG;
  // live vertices and live triangles are adjacent counters
  static_assert(C_LIVE_TRIS == C_LIVE_VERTS + 1, "counter layout");
  return cuda_status(cudaMemcpyAsync(dst, &v->V.ctl->c[C_LIVE_VERTS], 2 * sizeof(int32_t),
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, v->stream));
}

vm_status vm_get_stats(vm_volume* v, vm_frame_stats* s) {
  if (!v || !s) return VM_ERR_INVALID_ARG;
  if (sync_status(v)) return VM_ERR_CUDA;
  int c[C_COUNT];
  if (cudaMemcpy(c, v->V.ctl->c, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return VM_ERR_CUDA;
  s->frame_blocks = c[C_ST_FRAME_BLOCKS];
  s->new_blocks = c[C_ST_NEW_BLOCKS];
  s->update_blocks = c[C_ST_UPDATE_BLOCKS];
  s->changed_cubes = c[C_ST_CHANGED];
  s->live_blocks = c[C_LIVE_BLOCKS];
  s->live_vertices = c[C_LIVE_VERTS];
  s->live_triangles = c[C_LIVE_TRIS];
  s->freed_blocks = c[C_ST_FREED_BLOCKS];
  s->freed_vertices = c[C_ST_FREED_VERTS];
  s->created_vertices = c[C_ST_NEW_VERTS];
  s->hash_tombstones = c[C_TOMBS];
  s->block_high_water = c[C_BLK_BUMP] < (int)v->p.max_blocks ? c[C_BLK_BUMP] : (int)v->p.max_blocks;
  s->rehashes = c[C_ST_REHASHES];
  s->emitted_triangles = c[C_ST_EMITTED];
  s->released_triangles = c[C_ST_RELEASED];
  s->refreshed_vertices = c[C_ST_REFRESHED];
  s->collected_blocks = (uint32_t)c[C_ST_COLLECTED];
  s->meshed_blocks = (uint32_t)c[C_ST_MESHED];
  s->full_pool = c[C_STATUS_POOL];
  s->vertex_high_water = c[C_VTX_BUMP] < (int)v->p.max_vertices ? c[C_VTX_BUMP] : (int)v->p.max_vertices;
  s->triangle_high_water = c[C_TRI_BUMP] < (int)v->p.max_triangles ? c[C_TRI_BUMP] : (int)v->p.max_triangles;
  s->reference_updates = (uint32_t)c[C_ST_REFUPD];
  return VM_OK;
}

vm_status vm_num_blocks(vm_volume* v, int64_t* n) {
  if (!v || !n) return VM_ERR_INVALID_ARG;
  if (sync_status(v)) return VM_ERR_CUDA;
  *n = read_counter(v, C_LIVE_BLOCKS);
  return VM_OK;
}

vm_status vm_export_blocks(vm_volume* v, int32_t* keys, float* tsdf, float* weight, uint8_t* ce, uint8_t* cp) {
  if (!v) return VM_ERR_INVALID_ARG;
  if (sync_status(v)) return VM_ERR_CUDA;
  const int n = read_counter(v, C_LIVE_BLOCKS);
  void *dk = nullptr, *dt = nullptr, *dw = nullptr, *dce = nullptr, *dcp = nullptr, *cnt = nullptr;
  const size_t nn = n > 0 ? (size_t)n : 1;
  bool ok = cudaMalloc(&dk, nn * 12) == cudaSuccess && cudaMalloc(&dt, nn * BV * 4) == cudaSuccess &&
            cudaMalloc(&dw, nn * BV * 4) == cudaSuccess && cudaMalloc(&dce, nn * BV) == cudaSuccess &&
            cudaMalloc(&dcp, nn * BV) == cudaSuccess && cudaMalloc(&cnt, 4) == cudaSuccess;
  if (ok) {
    cudaMemsetAsync(cnt, 0, 4, v->stream);
    k_export_blocks<<<grid_for(v, 8), 256, 0, v->stream>>>(v->V, (int*)cnt, (int*)dk, (float*)dt, (float*)dw,
                                                           (uint8_t*)dce, (uint8_t*)dcp);
    ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(v->stream) == cudaSuccess;
    if (ok && n > 0) {
      ok = (!keys || cudaMemcpy(keys, dk, (size_t)n * 12, cudaMemcpyDeviceToHost) == cudaSuccess) &&
           (!tsdf || cudaMemcpy(tsdf, dt, (size_t)n * BV * 4, cudaMemcpyDeviceToHost) == cudaSuccess) &&
           (!weight || cudaMemcpy(weight, dw, (size_t)n * BV * 4, cudaMemcpyDeviceToHost) == cudaSuccess) &&
           (!ce || cudaMemcpy(ce, dce, (size_t)n * BV, cudaMemcpyDeviceToHost) == cudaSuccess) &&
           (!cp || cudaMemcpy(cp, dcp, (size_t)n * BV, cudaMemcpyDeviceToHost) == cudaSuccess);
    }
  }
  cudaFree(dk);
  cudaFree(dt);
  cudaFree(dw);
  cudaFree(dce);
  cudaFree(dcp);
  cudaFree(cnt);
  return ok ? VM_OK : VM_ERR_CUDA;
}

// ---- differentiable path
vm_status vm_diff_begin(vm_volume* v, int max_frames) {
  if (!v || max_frames < 1 || max_frames > 65535) return VM_ERR_INVALID_ARG;
  const size_t nvox = (size_t)v->p.max_blocks * BV;
  const size_t rec = (size_t)max_frames * (size_t)v->V.list_cap_touched;
  if (!v->V.dgrad || (size_t)v->diff_rec_cap < rec) {
    if (sync_status(v)) return VM_ERR_CUDA;
    for (void* p : v->diff_allocs) cudaFree(p);
    v->diff_allocs.clear();
    v->V.dcnt = nullptr;
    v->V.dwck = v->V.dgrad = nullptr;
    v->V.drec = v->V.drec_off = nullptr;
    v->diff_rec_cap = 0;
    void *a = nullptr, *b = nullptr, *c = nullptr, *d = nullptr, *e = nullptr;
    const bool ok = cudaMalloc(&a, nvox * sizeof(uint16_t)) == cudaSuccess &&
                    cudaMalloc(&b, nvox * sizeof(float)) == cudaSuccess &&
                    cudaMalloc(&c, nvox * sizeof(float)) == cudaSuccess &&
                    cudaMalloc(&d, rec * sizeof(int)) == cudaSuccess &&
                    cudaMalloc(&e, (size_t)(max_frames + 1) * sizeof(int)) == cudaSuccess;
    for (void* p : {a, b, c, d, e})
      if (p) v->diff_allocs.push_back(p);
    if (!ok) {
      (void)cudaGetLastError();
      for (void* p : v->diff_allocs) cudaFree(p);
      v->diff_allocs.clear();
      return VM_ERR_OOM;
    }
    v->V.dcnt = static_cast<uint16_t*>(a);
    v->V.dwck = static_cast<float*>(b);
    v->V.dgrad = static_cast<float*>(c);
    v->V.drec = static_cast<int*>(d);
    v->V.drec_off = static_cast<int*>(e);
    v->diff_rec_cap = (int)(rec < (size_t)INT32_MAX ? rec : (size_t)INT32_MAX);
  }
  drop_graph(v);  // frame graphs captured the volume view without the record buffers
  (void)cudaGetLastError();
  cudaMemsetAsync(v->V.dcnt, 0, nvox * sizeof(uint16_t), v->stream);
  cudaMemsetAsync(v->V.dwck, 0, nvox * sizeof(float), v->stream);
  cudaMemsetAsync(v->V.dgrad, 0, nvox * sizeof(float), v->stream);
  cudaMemsetAsync(v->V.drec_off, 0, sizeof(int), v->stream);
  k_diff_checkpoint<<<grid_for(v, 8), 256, 0, v->stream>>>(v->V);
  v->diff_on = true;
  v->diff_max = max_frames;
  v->diff_frames = 0;
  v->grad_next = -1;
  return cuda_status(cudaGetLastError());
}

vm_status vm_diff_end(vm_volume* v) {
  if (!v) return VM_ERR_INVALID_ARG;
  v->diff_on = false;
  v->grad_next = -1;
  return VM_OK;
}

vm_status vm_grad_vertices(vm_volume* v, int64_t n, const uint64_t* edge_keys, const float* grad_pos,
                           const float* grad_nrm) {
  if (!v || !v->diff_on || n < 0 || n > INT32_MAX || (n > 0 && (!edge_keys || !grad_pos || !grad_nrm)))
    return VM_ERR_INVALID_ARG;
  if (n == 0) return VM_OK;
  (void)cudaGetLastError();
  k_grad_vertices<<<grid_for(v, 8), 256, 0, v->stream>>>(v->V, (int)n,
                                                          reinterpret_cast<const unsigned long long*>(edge_keys),
                                                          grad_pos, grad_nrm);
  return cuda_status(cudaGetLastError());
}

vm_status vm_grad_depth(vm_volume* v, int frame, const float* depth, const vm_intrinsics* K, const float Twc[16],
                        const float Tcw[16], float* grad_depth) {
  if (!v || !v->diff_on || !grad_depth) return VM_ERR_INVALID_ARG;
  const int expect = v->grad_next >= 0 ? v->grad_next : v->diff_frames - 1;
  if (frame != expect || frame < 0) return VM_ERR_INVALID_ARG;
  FrameParams fp;
  if (!make_frame(K, Twc, Tcw, depth, &fp)) return VM_ERR_INVALID_ARG;
  (void)cudaGetLastError();
  if (cudaMemsetAsync(grad_depth, 0, (size_t)fp.W * fp.H * sizeof(float), v->stream) != cudaSuccess)
    return VM_ERR_CUDA;
  k_grad_depth<<<grid_for(v, INTEG_CTAS_PER_SM), INTEG_THREADS, 0, v->stream>>>(v->V, frame, fp, grad_depth);
  v->grad_next = frame - 1;
  return cuda_status(cudaGetLastError());
}

vm_status vm_export_grad(vm_volume* v, int32_t* keys, float* grad) {
  if (!v || !v->V.dgrad || !keys || !grad) return VM_ERR_INVALID_ARG;
  if (sync_status(v)) return VM_ERR_CUDA;
  const int n = read_counter(v, C_LIVE_BLOCKS);
  void *dk = nullptr, *dg = nullptr, *cnt = nullptr;
  const size_t nn = n > 0 ? (size_t)n : 1;
  bool ok = cudaMalloc(&dk, nn * 12) == cudaSuccess && cudaMalloc(&dg, nn * BV * 4) == cudaSuccess &&
            cudaMalloc(&cnt, 4) == cudaSuccess;
  if (ok) {
    cudaMemsetAsync(cnt, 0, 4, v->stream);
    k_export_grad<<<grid_for(v, 8), 256, 0, v->stream>>>(v->V, (int*)cnt, (int*)dk, (float*)dg);
    ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(v->stream) == cudaSuccess;
    if (ok && n > 0)
      ok = cudaMemcpy(keys, dk, (size_t)n * 12, cudaMemcpyDeviceToHost) == cudaSuccess &&
           cudaMemcpy(grad, dg, (size_t)n * BV * 4, cudaMemcpyDeviceToHost) == cudaSuccess;
  }
  (void)cudaGetLastError();
  cudaFree(dk);
  cudaFree(dg);
  cudaFree(cnt);
  return ok ? VM_OK : VM_ERR_CUDA;
}

vm_status vm_set_blocks(vm_volume* v, const int32_t* keys, int64_t n, const float* tsdf, const float* weight) {
  if (!v || n < 0 || (n > 0 && (!keys || !tsdf || !weight)) || n > (int64_t)v->p.max_blocks)
    return VM_ERR_INVALID_ARG;
  if (n == 0) return VM_OK;
  void *dk = nullptr, *dt = nullptr, *dw = nullptr;
  bool ok = cudaMalloc(&dk, (size_t)n * 12) == cudaSuccess && cudaMalloc(&dt, (size_t)n * BV * 4) == cudaSuccess &&
            cudaMalloc(&dw, (size_t)n * BV * 4) == cudaSuccess;
  if (ok) {
    ok = cudaMemcpyAsync(dk, keys, (size_t)n * 12, cudaMemcpyHostToDevice, v->stream) == cudaSuccess &&
         cudaMemcpyAsync(dt, tsdf, (size_t)n * BV * 4, cudaMemcpyHostToDevice, v->stream) == cudaSuccess &&
         cudaMemcpyAsync(dw, weight, (size_t)n * BV * 4, cudaMemcpyHostToDevice, v->stream) == cudaSuccess;
  }
  if (ok) {
    const int adv = v->advance_pending ? 1 : 0;
    k_fill_insert<<<grid_for(v, 2), 256, 0, v->stream>>>(v->V, (const int*)dk, (int)n, adv, v->frame);
    k_integrate<false><<<grid_for(v, INTEG_CTAS_PER_SM), INTEG_THREADS, 0, v->stream>>>(v->V, &v->V.ctl->fp);
    k_fill_copy<<<grid_for(v, 4), 256, 0, v->stream>>>(v->V, (const int*)dk, (const float*)dt, (const float*)dw,
                                                       (int)n);
    ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(v->stream) == cudaSuccess;
    v->advance_pending = false;
    ++v->frame;
  }
  cudaFree(dk);
  cudaFree(dt);
  cudaFree(dw);
  return ok ? VM_OK : VM_ERR_CUDA;
}

vm_status vm_enable_timing(vm_volume* v, int enable) {
  if (!v) return VM_ERR_INVALID_ARG;
  cudaStreamSynchronize(v->stream);
  const unsigned mask = (unsigned)enable & ((1u << K_COUNT_) - 1);
  if (mask != v->timing_mask) drop_graph(v);  // re-capture with the new event nodes
  v->graph_pending = false;
  for (auto& r : v->recs) {
    v->event_pool.push_back(r.a);
    v->event_pool.push_back(r.b);
  }
  v->recs.clear();
  for (int k = 0; k < K_COUNT_; ++k) {
    v->tot_ms[k] = 0;
    v->launches[k] = 0;
  }
  v->timing_mask = mask;
  return VM_OK;
}

vm_status vm_kernel_times(vm_volume* v, const char** names, double* total_ms, int64_t* launches, int cap, int* n) {
  if (!v || !n) return VM_ERR_INVALID_ARG;
  if (sync_status(v)) return VM_ERR_CUDA;
  collect_graph_timing(v);
  for (auto& r : v->recs) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      v->tot_ms[r.kernel] += ms;
      v->launches[r.kernel] += 1;
    }
    v->event_pool.push_back(r.a);
    v->event_pool.push_back(r.b);
  }
  v->recs.clear();
  *n = K_COUNT_;
  for (int k = 0; k < K_COUNT_ && k < cap; ++k) {
    if (names) names[k] = kKernelNames[k];
    if (total_ms) total_ms[k] = v->tot_ms[k];
    if (launches) launches[k] = v->launches[k];
  }
  return VM_OK;
}

}  // extern "C"

// ====================================================================== allocation-free download
// vm_download_mesh keeps its scan scratch (per-chunk counts and a vertex remap table) in
// device memory the library allocates on first use, and stages host outputs through
// temporary allocations.  Some callers cannot allow that: code running while a
// caching allocator owns all free device memory, inside a memory budget that forbids
// growth after start-up, or on a path that must never touch the allocator.  For them
// vm_download_mesh_noalloc does the same compaction with its scratch in the static array
// below (a liveness bitmask and per-32-slot prefix instead of a full remap table).  Every
// GPU that loads the library holds this array until the process exits.
namespace {
constexpr int NA_MAX_VERTICES = 1 << 24;   // vertex-pool size the static scratch covers
constexpr int NA_MAX_TRIANGLES = 1 << 26;  // triangle-pool size the static scratch covers
constexpr int NA_WORDS = NA_MAX_VERTICES / 32;
constexpr int NA_VCHUNKS = NA_MAX_VERTICES / SCAN_ITEMS;
constexpr int NA_TCHUNKS = NA_MAX_TRIANGLES / SCAN_ITEMS;
constexpr size_t NA_INTS = 2 * (size_t)NA_WORDS + NA_VCHUNKS + NA_TCHUNKS + 64;  // ~4.5 MB
constexpr int NA_MAX_DEVICES = 64;
// Device address of na_scratch per device, filled on the first call with that device current.
// Concurrent first calls from several host threads store the same address, so a plain atomic
// store suffices.
std::atomic<int*> na_scratch_addr[NA_MAX_DEVICES];
}  // namespace

static __device__ __align__(256) int na_scratch[NA_INTS];

namespace {

// Liveness bitmask of the vertex pool (one word per 32 slots) and the live count of every
// 1024-slot chunk.  Every word and count of the launched range is rewritten each call.
__global__ void __launch_bounds__(256) k_na_vertex_words(Vol V, unsigned* mask, int* chunk_counts) {
  const int n = min(__ldcg(&V.ctl->c[C_VTX_BUMP]), V.max_vertices);
  const int base = blockIdx.x * SCAN_ITEMS;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  int cnt = 0;
  for (int j0 = 0; j0 < SCAN_ITEMS; j0 += 256) {
    const int v = base + j0 + threadIdx.x;
    const bool live = v < n && V.vref[v] > 0;
    const unsigned b = __ballot_sync(0xffffffffu, live);
    if (lane == 0) mask[(base + j0) / 32 + w] = b;
    cnt += live;
  }
  atomicAdd(&s, cnt);
  __syncthreads();
  if (threadIdx.x == 0) chunk_counts[blockIdx.x] = s;
}

// New index of vertex slot v from the bitmask and per-word prefix (-1 when not live).
__device__ __forceinline__ int na_remap(const unsigned* mask, const int* wprefix, int v) {
  if (v < 0) return -1;
  const unsigned m = mask[v >> 5];
  const unsigned bit = 1u << (v & 31);
  return (m & bit) ? wprefix[v >> 5] + __popc(m & (bit - 1u)) : -1;
}

// Per-word prefixes of the chunk (from its scanned offset), then the stable compaction.
__global__ void __launch_bounds__(256) k_na_vertex_compact(Vol V, const unsigned* mask, const int* chunk_off,
                                                           int* wprefix, float* pos, float* nrm, uint64_t* keys,
                                                           int* refcount) {
  const int n = min(__ldcg(&V.ctl->c[C_VTX_BUMP]), V.max_vertices);
  const int base = blockIdx.x * SCAN_ITEMS;
  const int word0 = base / 32;
  if (threadIdx.x < 32) {
    const int c = __popc(mask[word0 + threadIdx.x]);
    int x = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if ((int)threadIdx.x >= o) x += y;
    }
    wprefix[word0 + threadIdx.x] = chunk_off[blockIdx.x] + x - c;
  }
  __syncthreads();
  for (int j0 = 0; j0 < SCAN_ITEMS; j0 += 256) {
    const int v = base + j0 + threadIdx.x;
    if (v >= n) break;
    const int off = na_remap(mask, wprefix, v);
    if (off < 0) continue;
    const float4 p = V.vrec[2 * (size_t)v], q = V.vrec[2 * (size_t)v + 1];
    pos[3 * (size_t)off] = p.x; pos[3 * (size_t)off + 1] = p.y; pos[3 * (size_t)off + 2] = p.z;
    nrm[3 * (size_t)off] = q.x; nrm[3 * (size_t)off + 1] = q.y; nrm[3 * (size_t)off + 2] = q.z;
    if (keys) keys[off] = edge_key_of(V, V.vedge[v]);
    if (refcount) refcount[off] = V.vref[v];
  }
}

// Stable compaction of the live triangles with vertex indices remapped from the bitmask.
__global__ void __launch_bounds__(256) k_na_compact_triangles(Vol V, const int* chunk_off, const unsigned* mask,
                                                              const int* wprefix, int* tris_out) {
  const int n = min(__ldcg(&V.ctl->c[C_TRI_BUMP]), V.max_triangles);
  const int base = blockIdx.x * SCAN_ITEMS;
  if (base >= n) return;
  __shared__ int warp_tot[8];
  __shared__ int running;
  if (threadIdx.x == 0) running = chunk_off[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j0 = 0; j0 < SCAN_ITEMS; j0 += 256) {
    const int t = base + j0 + threadIdx.x;
    const int4 tr = t < n ? V.tris[t] : make_int4(-1, -1, -1, -1);
    const bool live = tr.x >= 0;
    const unsigned b = __ballot_sync(0xffffffffu, live);
    if (lane == 0) warp_tot[w] = __popc(b);
    __syncthreads();
    int off = running;
    for (int q = 0; q < w; ++q) off += warp_tot[q];
    off += __popc(b & ((1u << lane) - 1));
    if (live) {
      tris_out[3 * (size_t)off] = na_remap(mask, wprefix, tr.x);
      tris_out[3 * (size_t)off + 1] = na_remap(mask, wprefix, tr.y);
      tris_out[3 * (size_t)off + 2] = na_remap(mask, wprefix, tr.z);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int s = 0;
      for (int q = 0; q < 8; ++q) s += warp_tot[q];
      running += s;
    }
    __syncthreads();
  }
}

}  // namespace

extern "C" vm_status vm_download_mesh_noalloc(vm_volume* v, float* pos, float* nrm, int32_t* tris,
                                              uint64_t* edge_keys, int32_t* refcount, int64_t cap_vertices,
                                              int64_t cap_triangles, int64_t* n_vertices, int64_t* n_triangles) {
  if (!v || !n_vertices || !n_triangles || cap_vertices < 0 || cap_triangles < 0) return VM_ERR_INVALID_ARG;
  if (v->p.max_vertices > (uint32_t)NA_MAX_VERTICES || v->p.max_triangles > (uint32_t)NA_MAX_TRIANGLES)
    return VM_ERR_INVALID_ARG;  // pools larger than the static scratch covers
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return VM_ERR_CUDA;
  }
  // the scratch array used is the one of the volume's device, which must be current
  if (dev != v->device || dev < 0 || dev >= NA_MAX_DEVICES) return VM_ERR_INVALID_ARG;
  // First call on this device: look up the device address of the static scratch array.
  int* scratch = na_scratch_addr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, na_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return VM_ERR_CUDA;
    }
    scratch = static_cast<int*>(p);
    na_scratch_addr[dev].store(scratch, std::memory_order_release);
  }
  unsigned* mask = reinterpret_cast<unsigned*>(scratch);
  int* wprefix = scratch + NA_WORDS;
  int* vchunk = wprefix + NA_WORDS;
  int* tchunk = vchunk + NA_VCHUNKS;
  int* totals = tchunk + NA_TCHUNKS;
  const int nvc = ((int)v->p.max_vertices + SCAN_ITEMS - 1) / SCAN_ITEMS;
  const int ntc = ((int)v->p.max_triangles + SCAN_ITEMS - 1) / SCAN_ITEMS;
  cudaStream_t s = v->stream;
  (void)cudaGetLastError();
  k_na_vertex_words<<<nvc, 256, 0, s>>>(v->V, mask, vchunk);
  k_scan_counts<<<1, 1024, 0, s>>>(vchunk, nvc, totals);
  k_count_live<true><<<ntc, 256, 0, s>>>(v->V, tchunk);
  k_scan_counts<<<1, 1024, 0, s>>>(tchunk, ntc, totals + 1);
  int tot[2] = {0, 0};
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(tot, totals, sizeof(tot), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return VM_ERR_CUDA;
  *n_vertices = tot[0];
  *n_triangles = tot[1];
  if (!pos) return VM_OK;  // size query
  if (!nrm || !tris || tot[0] > cap_vertices || tot[1] > cap_triangles) return VM_ERR_INVALID_ARG;
  k_na_vertex_compact<<<nvc, 256, 0, s>>>(v->V, mask, vchunk, wprefix, pos, nrm, edge_keys, refcount);
  k_na_compact_triangles<<<ntc, 256, 0, s>>>(v->V, tchunk, mask, wprefix, tris);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return VM_ERR_CUDA;
  return VM_OK;
}

// ====================================================================== batched step
namespace {

// Schedule options the autotuner picks from, per kernel (index = schedule slot):
//   0 k_alloc pixels per thread (CTA of 1024 / ppt threads per 64 x 16 tile), 1-4 CTAs per SM
//   of the fusion, mesh, vertex-gc and block-gc kernels (persistent grids).
constexpr int SCHED_SLOTS = 5;
constexpr int SCHED_OPTS = 3;
const int kSchedOptions[SCHED_SLOTS][SCHED_OPTS] = {{1, 2, 4}, {4, 8, 12}, {4, 6, 8}, {1, 2, 4}, {2, 4, 8}};
const int kSchedDefault[SCHED_SLOTS] = {2, 12, 8, 2, 8};

struct TuneRec {
  int opt;
  cudaEvent_t ev[SCHED_SLOTS + 1];
};

}  // namespace

struct vm_batch {
  std::vector<vm_volume*> vols;
  int n = 0;
  bool compact = false;  // every volume of a batch has the same cube layout
  Vol* d_vols = nullptr;
  int* d_done = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int num_sms = 148;
  int sched[SCHED_SLOTS];
  // graph of one tick; the frame table reaches it as kb_alloc's launch argument
  cudaGraph_t graph = nullptr;
  cudaGraphNode_t alloc_node = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_flags = -1, graph_tx = -1, graph_ty = -1;
  // autotuning: ticks still to time, the timed ticks, per-option totals
  int tune_left = 0;
  std::vector<TuneRec> tune_recs;
  double tune_ms[SCHED_SLOTS][SCHED_OPTS] = {};
  int tune_cnt[SCHED_SLOTS][SCHED_OPTS] = {};
  // profiling: ticks still to time with the current schedule, their records, totals
  int prof_left = 0;
  std::vector<TuneRec> prof_recs;
  double prof_ms[SCHED_SLOTS] = {};
  int prof_cnt = 0;
  BatchFrames* frames = nullptr;  // host staging of the launch argument (8.5 KB)
};

namespace {

void batch_drop_graph(vm_batch* b) {
  if (b->exec) {
    cudaStreamSynchronize(b->stream);
    cudaGraphExecDestroy(b->exec);
  }
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->alloc_node = nullptr;
  b->graph_flags = -1;
}

void* batch_alloc_kernel(int ppt) {
  switch (ppt) {
    case 1: return reinterpret_cast<void*>(kb_alloc<1>);
    case 4: return reinterpret_cast<void*>(kb_alloc<4>);
    default: return reinterpret_cast<void*>(kb_alloc<2>);
  }
}

// Enqueue one tick's five launches with schedule `sc`; with `rec`, event pairs around each.
vm_status batch_enqueue(vm_batch* b, cudaStream_t st, const int* sc, int flags, int tx, int ty, TuneRec* rec) {
  const int mode = M_UPDATE | ((flags & VM_REFINE) ? M_REFINE : 0);
  (void)cudaGetLastError();
  if (rec) cudaEventRecord(rec->ev[0], st);
  const dim3 grid(tx, ty, b->n);
  const int threads = ALLOC_TILE_W * ALLOC_TILE_H / sc[0];
  switch (sc[0]) {
    case 1: kb_alloc<1><<<grid, threads, 0, st>>>(b->d_vols, b->n, *b->frames); break;
    case 4: kb_alloc<4><<<grid, threads, 0, st>>>(b->d_vols, b->n, *b->frames); break;
    default: kb_alloc<2><<<grid, threads, 0, st>>>(b->d_vols, b->n, *b->frames); break;
  }
  if (rec) cudaEventRecord(rec->ev[1], st);
  launch_dependent(kb_integrate, b->num_sms * sc[1], INTEG_THREADS, 0, st, (const Vol*)b->d_vols, b->n, b->d_done);
  if (rec) cudaEventRecord(rec->ev[2], st);
  launch_dependent(b->compact ? kb_mesh<true> : kb_mesh<false>, b->num_sms * sc[2], MESH_THREADS, 0, st,
                   (const Vol*)b->d_vols, b->n, mode, b->d_done);
  if (rec) cudaEventRecord(rec->ev[3], st);
  if (flags & VM_GC) {
    launch_dependent(b->compact ? kb_gc_vertices<true> : kb_gc_vertices<false>, b->num_sms * sc[3], 256, 0, st,
                     (const Vol*)b->d_vols, b->n);
    if (rec) cudaEventRecord(rec->ev[4], st);
    launch_dependent(kb_gc_blocks, b->num_sms * sc[4], 256, 0, st, (const Vol*)b->d_vols, b->n, 1);
  } else if (rec) {
    cudaEventRecord(rec->ev[4], st);
  }
  if (rec) cudaEventRecord(rec->ev[5], st);
  return cuda_status(cudaGetLastError());
}

// Fold the timed ticks into the per-option totals and pick each kernel's fastest option.
vm_status batch_finish_tuning(vm_batch* b) {
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return VM_ERR_CUDA;
  for (auto& r : b->tune_recs) {
    for (int k = 0; k < SCHED_SLOTS; ++k) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, r.ev[k], r.ev[k + 1]) == cudaSuccess) {
        b->tune_ms[k][r.opt] += ms;
        b->tune_cnt[k][r.opt] += 1;
      }
    }
    for (auto e : r.ev) cudaEventDestroy(e);
  }
  b->tune_recs.clear();
  for (int k = 0; k < SCHED_SLOTS; ++k) {
    int best = -1;
    double best_ms = 0;
    for (int o = 0; o < SCHED_OPTS; ++o) {
      if (!b->tune_cnt[k][o]) continue;
      const double m = b->tune_ms[k][o] / b->tune_cnt[k][o];
      if (best < 0 || m < best_ms) best = o, best_ms = m;
    }
    if (best >= 0) b->sched[k] = kSchedOptions[k][best];
  }
  batch_drop_graph(b);
  return VM_OK;
}

}  // namespace

extern "C" {

vm_status vm_batch_create(vm_volume* const* vols, int n, vm_batch** out) {
  if (!vols || !out || n < 1 || n > MAX_SCENES) return VM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!vols[i]) return VM_ERR_INVALID_ARG;
    if ((vols[i]->p.flags ^ vols[0]->p.flags) & VM_PARAM_COMPACT_EDGES) return VM_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (vols[j] == vols[i]) return VM_ERR_INVALID_ARG;
  }
  vm_batch* b = new vm_batch();
  b->vols.assign(vols, vols + n);
  b->n = n;
  b->compact = (vols[0]->p.flags & VM_PARAM_COMPACT_EDGES) != 0;
  b->stream = vols[0]->stream;
  b->num_sms = vols[0]->num_sms;
  for (int k = 0; k < SCHED_SLOTS; ++k) b->sched[k] = kSchedDefault[k];
  std::vector<Vol> host(n);
  for (int i = 0; i < n; ++i) host[i] = vols[i]->V;
  (void)cudaGetLastError();
  bool ok = cudaMalloc(&b->d_vols, sizeof(Vol) * n) == cudaSuccess &&
            cudaMalloc(&b->d_done, sizeof(int) * BD_COUNT) == cudaSuccess &&
            cudaMallocHost(&b->frames, sizeof(BatchFrames)) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(b->d_vols, host.data(), sizeof(Vol) * n, cudaMemcpyHostToDevice, b->stream) == cudaSuccess &&
       cudaMemsetAsync(b->d_done, 0, sizeof(int) * BD_COUNT, b->stream) == cudaSuccess &&
       cudaStreamSynchronize(b->stream) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();
    cudaFree(b->d_vols);
    cudaFree(b->d_done);
    if (b->frames) cudaFreeHost(b->frames);
    delete b;
    return VM_ERR_OOM;
  }
  memset(b->frames, 0, sizeof(BatchFrames));
  *out = b;
  return VM_OK;
}

vm_status vm_batch_destroy(vm_batch* b) {
  if (!b) return VM_ERR_INVALID_ARG;
  cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  for (auto& r : b->tune_recs)
    for (auto e : r.ev) cudaEventDestroy(e);
  for (auto& r : b->prof_recs)
    for (auto e : r.ev) cudaEventDestroy(e);
  cudaFree(b->d_vols);
  cudaFree(b->d_done);
  cudaFreeHost(b->frames);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
  return VM_OK;
}

vm_status vm_batch_step(vm_batch* b, const float* const* depths, const vm_intrinsics* K, const float* T_wc,
                        const float* T_cw, int flags, int use_graph) {
  if (!b || !depths || !K || !T_wc || !T_cw || (flags & ~(VM_REFINE | VM_GC))) return VM_ERR_INVALID_ARG;
  int tx = 1, ty = 1;
  BatchFrames& bf = *b->frames;
  for (int i = 0; i < b->n; ++i) {
    if (b->vols[i]->diff_on) return VM_ERR_INVALID_ARG;
    if (!make_frame(&K[i], T_wc + 16 * i, T_cw + 16 * i, depths[i], &bf.fp[i])) return VM_ERR_INVALID_ARG;
    bf.fp[i].frame = b->vols[i]->frame;
    if (const vm_status ps = prepare_depth(b->vols[i], &bf.fp[i])) return ps;
    tx = std::max(tx, (bf.fp[i].W + ALLOC_TILE_W - 1) / ALLOC_TILE_W);
    ty = std::max(ty, (bf.fp[i].H + ALLOC_TILE_H - 1) / ALLOC_TILE_H);
  }
  for (int i = 0; i < b->n; ++i) bf.advance[i] = b->vols[i]->advance_pending ? 1 : 0;
  vm_status st = VM_OK;
  if (b->tune_left > 0) {
    // autotuning tick: eager launches, every kernel on its option (tick index mod 3)
    TuneRec r;
    r.opt = (int)(b->tune_recs.size() % SCHED_OPTS);
    for (auto& e : r.ev) cudaEventCreate(&e);
    int sc[SCHED_SLOTS];
    for (int k = 0; k < SCHED_SLOTS; ++k) sc[k] = kSchedOptions[k][r.opt];
    st = batch_enqueue(b, b->stream, sc, flags, tx, ty, &r);
    b->tune_recs.push_back(r);
    if (--b->tune_left == 0 && !st) st = batch_finish_tuning(b);
  } else if (b->prof_left > 0) {
    TuneRec r;
    r.opt = -1;
    for (auto& e : r.ev) cudaEventCreate(&e);
    st = batch_enqueue(b, b->stream, b->sched, flags, tx, ty, &r);
    b->prof_recs.push_back(r);
    --b->prof_left;
  } else if (!use_graph) {
    st = batch_enqueue(b, b->stream, b->sched, flags, tx, ty, nullptr);
  } else {
    if (!b->exec || b->graph_flags != flags || b->graph_tx != tx || b->graph_ty != ty) {
      batch_drop_graph(b);
      if (!b->cap_stream && cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        b->cap_stream = nullptr;
        return VM_ERR_CUDA;
      }
      if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        (void)cudaGetLastError();
        return VM_ERR_CUDA;
      }
      vm_status s = batch_enqueue(b, b->cap_stream, b->sched, flags, tx, ty, nullptr);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
      if (s || e != cudaSuccess) {
        (void)cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return s ? s : VM_ERR_CUDA;
      }
      b->graph = g;
      b->alloc_node = find_kernel_node(g, batch_alloc_kernel(b->sched[0]));
      e = b->alloc_node ? cudaGraphInstantiate(&b->exec, g, 0) : cudaErrorInvalidValue;
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        b->exec = nullptr;
        batch_drop_graph(b);
        return VM_ERR_CUDA;
      }
      b->graph_flags = flags;
      b->graph_tx = tx;
      b->graph_ty = ty;
    }
    const Vol* dv = b->d_vols;
    int n = b->n;
    void* args[3] = {&dv, &n, b->frames};
    cudaKernelNodeParams kp = {};
    kp.func = batch_alloc_kernel(b->sched[0]);
    kp.gridDim = dim3(tx, ty, b->n);
    kp.blockDim = dim3(ALLOC_TILE_W * ALLOC_TILE_H / b->sched[0]);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    cudaError_t e = cudaGraphExecKernelNodeSetParams(b->exec, b->alloc_node, &kp);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) (void)cudaGetLastError();
    st = cuda_status(e);
  }
  if (!st)
    for (auto* v : b->vols) {
      v->advance_pending = true;
      ++v->frame;
    }
  return st;
}

vm_status vm_batch_tune(vm_batch* b, int rounds) {
  if (!b || rounds < 1 || rounds > 100) return VM_ERR_INVALID_ARG;
  for (auto& r : b->tune_recs)
    for (auto e : r.ev) cudaEventDestroy(e);
  b->tune_recs.clear();
  memset(b->tune_ms, 0, sizeof(b->tune_ms));
  memset(b->tune_cnt, 0, sizeof(b->tune_cnt));
  b->tune_left = rounds * SCHED_OPTS;
  return VM_OK;
}

vm_status vm_batch_schedule(vm_batch* b, int* sched, double* tuned_ms) {
  if (!b || !sched) return VM_ERR_INVALID_ARG;
  for (int k = 0; k < SCHED_SLOTS; ++k) sched[k] = b->sched[k];
  if (tuned_ms)
    for (int k = 0; k < SCHED_SLOTS; ++k)
      for (int o = 0; o < SCHED_OPTS; ++o)
        tuned_ms[k * SCHED_OPTS + o] = b->tune_cnt[k][o] ? b->tune_ms[k][o] / b->tune_cnt[k][o] : -1.0;
  return VM_OK;
}

vm_status vm_batch_profile(vm_batch* b, int ticks) {
  if (!b || ticks < 1 || ticks > 100000) return VM_ERR_INVALID_ARG;
  for (auto& r : b->prof_recs)
    for (auto e : r.ev) cudaEventDestroy(e);
  b->prof_recs.clear();
  memset(b->prof_ms, 0, sizeof(b->prof_ms));
  b->prof_cnt = 0;
  b->prof_left = ticks;
  return VM_OK;
}

vm_status vm_batch_kernel_ms(vm_batch* b, double* ms, int* ticks) {
  if (!b || !ms) return VM_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return VM_ERR_CUDA;
  for (auto& r : b->prof_recs) {
    for (int k = 0; k < SCHED_SLOTS; ++k) {
      float t = 0;
      if (cudaEventElapsedTime(&t, r.ev[k], r.ev[k + 1]) == cudaSuccess) b->prof_ms[k] += t;
    }
    ++b->prof_cnt;
    for (auto e : r.ev) cudaEventDestroy(e);
  }
  b->prof_recs.clear();
  for (int k = 0; k < SCHED_SLOTS; ++k) ms[k] = b->prof_cnt ? b->prof_ms[k] / b->prof_cnt : -1.0;
  if (ticks) *ticks = b->prof_cnt;
  return VM_OK;
}

vm_status vm_batch_set_schedule(vm_batch* b, const int* sched) {
  if (!b || !sched) return VM_ERR_INVALID_ARG;
  for (int k = 0; k < SCHED_SLOTS; ++k) {
    bool ok = false;
    for (int o = 0; o < SCHED_OPTS; ++o) ok |= sched[k] == kSchedOptions[k][o];
    if (!ok) return VM_ERR_INVALID_ARG;
  }
  for (int k = 0; k < SCHED_SLOTS; ++k) b->sched[k] = sched[k];
  batch_drop_graph(b);
  return VM_OK;
}

}  // extern "C"
