// C ABI of libdawn (declared in include/dawn.h): graph ingest and
// validation, solver workspace, launches of the persistent GOVM kernel, the
// backward pass, status and counters.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>

#include "dawn_common.cuh"

using dawn::DeviceCtl;
using dawn::GovmParams;

struct dawn_graph_s {
  int32_t n = 0;
  int64_t m = 0;
  int wtype = 0;
  int device = 0;
  int sms = 0;
  int64_t l2_bytes = 0;  // the device's L2 size
  int32_t *row_ptr = nullptr;
  int32_t *col = nullptr;   // staging copy of the columns (freed after interleaving)
  uint32_t *w = nullptr;    // staging copy of host weights (freed after creation; dawn_set_weights
                            // allocates it again on its first host-memory call)
  uint2 *cw = nullptr;      // (column, weight bits) per edge: the array the solver streams
  int32_t *src = nullptr;
  unsigned long long *trace = nullptr;
  int32_t trace_cap = 0;
  // solver workspace for up to ws_k instances
  int32_t ws_k = 0;
  unsigned long long *state = nullptr;
  uint32_t *bitmap = nullptr;
  uint4 *queue = nullptr;
  int32_t *tiles = nullptr;
  unsigned long long *tails = nullptr;
  int64_t words = 0, tiles_cap = 0;
  DeviceCtl *ctl = nullptr;
  unsigned *vflags = nullptr;  // validation flags [0], max weight [1], max out-degree [2]
  int32_t max_deg = 0;         // largest out-degree (read back at creation)
  // backward scratch (one allocation, made by the first dawn_sssp_backward):
  // bw_edges | inner | rem | par | acc; the first three are cleared per call
  // by one memset
  unsigned char *bw_base = nullptr;
  unsigned long long *bw_edges = nullptr;  // [4] tree edges expected, handled; blocks finished; unused
  int32_t *bw_cnt = nullptr;      // [3n] has-children flags, children still to arrive, tree parents
  float *bw_acc = nullptr;        // [n] subtree sums of dL/ddist
  // options
  int64_t max_steps = 0;
  unsigned long long wait_limit_ns = 4000000000ull;
  int grid_blocks = 0;
  int ctas_per_sm = 0;  // kernel build (0 = default)
  int batch = 0;        // instances per msssp launch (0 = automatic)
  int small_path = 0;   // DAWN_OPT_SMALL_PATH
  int test_stall = 0;
  int64_t fail_alloc = 0;  // test hook: the fail_alloc-th next workspace allocation fails
  int gsvm = 0;
  int frontier = 0;     // DAWN_OPT_FRONTIER
  int skip_remarked = 1;  // DAWN_OPT_SKIP_REMARKED
  int occupancy[2] = {0, 0};  // co-resident CTAs per SM of the 4- and 5-CTA builds (cached)
  int last_k = 0;
  cudaStream_t last_stream = nullptr;
};

namespace {

enum : unsigned { kBadRowPtr = 1u, kBadCol = 2u, kBadWeight = 4u };

__global__ void validate_kernel(const int32_t *row_ptr, const int32_t *col, const uint32_t *w, int32_t n, int64_t m,
                                int wtype, unsigned *flags) {
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsize = (long long)gridDim.x * blockDim.x;
  unsigned bad = 0, wmax = 0, dmax = 0;
  for (long long v = gtid; v <= n; v += gsize) {
    const int32_t r = row_ptr[v];
    if (v == 0 && r != 0) bad |= kBadRowPtr;
    if (v == n && (int64_t)r != m) bad |= kBadRowPtr;
    if (v < n) {
      const int32_t r1 = row_ptr[v + 1];
      if (r1 < r) bad |= kBadRowPtr;
      else dmax = max(dmax, (unsigned)(r1 - r));
    }
  }
  for (long long e = gtid; e < m; e += gsize) {
    if (col) {
      const int32_t c = col[e];
      if (c < 0 || c >= n) bad |= kBadCol;
    }
    const uint32_t x = w[e];
    if (wtype == DAWN_W_F32) {
      const float f = __uint_as_float(x);
      if (!(f >= 0.0f) || isinf(f)) bad |= kBadWeight;  // NaN fails f >= 0
    } else if (wtype == DAWN_W_I32) {
      const int32_t y = (int32_t)x;
      wmax = max(wmax, y < 0 ? (uint32_t)(-(int64_t)y) : (uint32_t)y);  // |w|
    } else {
      wmax = max(wmax, x);
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, d);
    wmax = max(wmax, __shfl_xor_sync(0xFFFFFFFFu, wmax, d));
    dmax = max(dmax, __shfl_xor_sync(0xFFFFFFFFu, dmax, d));
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(flags, bad);
    if (wmax) atomicMax(flags + 1, wmax);
    if (dmax) atomicMax(flags + 2, dmax);
  }
}

// src[e] = tail of edge e (one warp per row).
__global__ void edge_tail_kernel(const int32_t *row_ptr, int32_t n, int32_t *src) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (long long u = warp; u < n; u += nwarps) {
    const int32_t b = row_ptr[u], e = row_ptr[u + 1];
    for (int32_t i = b + lane; i < e; i += 32) src[i] = (int32_t)u;
  }
}

// cw[e] = (col[e], w[e]); with col == null only the weight half is rewritten.
__global__ void interleave_kernel(const int32_t *col, const uint32_t *w, int64_t m, uint2 *cw) {
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsize = (long long)gridDim.x * blockDim.x;
  for (long long e = gtid; e < m; e += gsize) {
    if (col) cw[e] = make_uint2((uint32_t)col[e], w[e]);
    else cw[e].y = w[e];
  }
}

// New weights (dawn_set_weights) in one pass: each weight is checked as at
// creation (float32: finite and >= 0; the largest |w| is kept for the
// overflow bound of integer types) and written into the weight half of the
// interleaved (column, weight) array.
__global__ void weights_kernel(const uint32_t *w, int64_t m, int wtype, uint2 *cw, unsigned *flags) {
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsize = (long long)gridDim.x * blockDim.x;
  unsigned bad = 0, wmax = 0;
  for (long long e = gtid; e < m; e += gsize) {
    const uint32_t x = w[e];
    if (wtype == DAWN_W_F32) {
      const float f = __uint_as_float(x);
      if (!(f >= 0.0f) || isinf(f)) bad |= kBadWeight;  // NaN fails f >= 0
    } else if (wtype == DAWN_W_I32) {
      const int32_t y = (int32_t)x;
      wmax = max(wmax, y < 0 ? (uint32_t)(-(int64_t)y) : (uint32_t)y);  // |w|
    } else {
      wmax = max(wmax, x);
    }
    cw[e].y = x;
  }
  for (int d = 16; d > 0; d >>= 1) {
    bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, d);
    wmax = max(wmax, __shfl_xor_sync(0xFFFFFFFFu, wmax, d));
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(flags, bad);
    if (wmax) atomicMax(flags + 1, wmax);
  }
}

// Backward of dist w.r.t. the weights along the parent tree, children before
// parents: acc[v] starts at dL/ddist[v]; once every tree child of v has added
// its acc, acc[v] is the sum of dL/ddist over v's subtree, grad_w of v's
// parent edge is set to it and it is added to the parent.  A thread starts at
// each leaf and walks up, going through a parent only as the last of its
// children to arrive, so every tree edge is handled once (O(n) work, no
// barrier).  Edges off the tree keep grad_w = 0.  A parent array with a cycle
// leaves the cycle's edges unhandled, which the final check reports.

__device__ __forceinline__ int atom_add_acq_rel_s32(int *p, int v) {
  int o;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(o) : "l"(p), "r"(v) : "memory");
  return o;
}

// acc = dL/ddist; par[v] = tree parent of v (or -1); rem[u] = number of tree
// children of u and inner[u] = 1 when there is one (both start at zero);
// edges[0] = tree edges; grad_w = 0 (the walk writes the tree edges after
// this kernel).
__global__ void bw_count_kernel(const int32_t *parent_edge, const float *grad_dist, const int32_t *src, int32_t n,
                                int64_t m, float *acc, int32_t *inner, int32_t *rem, int32_t *par,
                                unsigned long long *edges, float *grad_w, DeviceCtl *ctl) {
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsize = (long long)gridDim.x * blockDim.x;
  for (long long e = gtid; e < m; e += gsize) grad_w[e] = 0.0f;
  unsigned long long mine = 0;
  for (long long v = gtid; v < n; v += gsize) {
    acc[v] = grad_dist[v];
    const int32_t e = parent_edge[v];
    par[v] = -1;
    if (e < 0) continue;
    if ((int64_t)e >= m) {
      atomicCAS(&ctl->status, 0, (int)DAWN_ERR_INVALID);
      continue;
    }
    const int32_t u = src[e];
    par[v] = u;
    inner[u] = 1;  // a plain store: every child writes the same value
    atomicAdd(rem + u, 1);
    ++mine;
  }
  for (int d = 16; d > 0; d >>= 1) mine += __shfl_xor_sync(0xFFFFFFFFu, mine, d);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(edges, mine);
}

// The walks; the last block to finish checks that every tree edge was
// handled once (otherwise the parent array had a cycle).
__global__ void bw_walk_kernel(const int32_t *parent_edge, const int32_t *par, int32_t n, float *acc,
                               const int32_t *inner, int32_t *rem, float *grad_w, unsigned long long *edges,
                               DeviceCtl *ctl) {
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsize = (long long)gridDim.x * blockDim.x;
  unsigned long long mine = 0;
  for (long long v = gtid; v < n; v += gsize) {
    if (inner[v] != 0) continue;  // walks start at leaves only
    int32_t x = (int32_t)v;
    for (int32_t hop = 0; hop < n; ++hop) {  // a tree path has fewer than n edges
      const int32_t u = par[x];            // -1: a root, or an edge index the count rejected
      const int32_t e = parent_edge[x];
      const float sum = __ldcg(acc + x);  // complete: every child of x has added to it
      if (u < 0) break;
      grad_w[e] = sum;
      ++mine;
      atomicAdd(acc + u, sum);
      // release: the add above is visible to the sibling that arrives last;
      // acquire: as the last, every sibling's add is visible below
      if (atom_add_acq_rel_s32(rem + u, -1) != 1) break;
      x = u;
    }
  }
  for (int d = 16; d > 0; d >>= 1) mine += __shfl_xor_sync(0xFFFFFFFFu, mine, d);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(edges + 1, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long done = atomicAdd(edges + 2, 1ull);
    if (done == gridDim.x - 1) {  // last block: all walks have finished
      __threadfence();
      if (__ldcg(edges) != __ldcg(edges + 1)) atomicCAS(&ctl->status, 0, (int)DAWN_ERR_INVALID);
    }
  }
}

int cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return DAWN_ERR_OOM;
  }
  return DAWN_ERR_CUDA;
}

// Device memory of every handle comes from one stream-ordered memory pool
// per device that the library owns (cudaMallocFromPoolAsync /
// cudaFreeAsync).  Freed blocks stay in the pool and serve the next
// allocation without a new mapping, and neither call synchronises the
// device, so a serving loop that builds the next graph while the current
// one's solves run, then destroys the old handle, leaves no idle gap on the
// GPU.  Reuse across streams happens only once a free has completed in its
// stream's order (no hidden cross-stream dependencies).  Freed memory stays
// in the pool until dawn_trim_memory: growing a pool maps new memory, which
// can stall solves running at the same time, so a loop that creates and
// destroys graphs reaches a steady state with no mapping at all.
struct DevicePool {
  cudaMemPool_t pool = nullptr;
};
constexpr int kPoolDevices = 64;
std::mutex g_pool_mutex;
DevicePool g_pools[kPoolDevices];

cudaMemPool_t device_pool(int device) {
  if (device < 0 || device >= kPoolDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  DevicePool &d = g_pools[device];
  if (!d.pool) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;  // keep freed memory for reuse until dawn_trim_memory
    int off = 0;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &off) != cudaSuccess) {
      cudaGetLastError();
      cudaMemPoolDestroy(pool);
      return nullptr;
    }
    d.pool = pool;
  }
  return d.pool;
}

// Stream-ordered allocation on `stream` from the device's pool: usable by
// work on `stream` at once, and by any stream once `stream` has passed this
// point.  Refused during stream capture (the workspace must exist before a
// capture starts: dawn_reserve).
template <typename T>
int dalloc(int device, T **p, size_t count, cudaStream_t stream) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return DAWN_ERR_CUDA;
  }
  cudaMemPool_t pool = device_pool(device);
  if (!pool) return DAWN_ERR_CUDA;
  void *q = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&q, count * sizeof(T), pool, stream);
  if (e != cudaSuccess) return cuda_fail(e);
  if ((uintptr_t)q % 16 != 0) {  // every kernel here assumes at least 16-byte alignment
    cudaFreeAsync(q, stream);
    return DAWN_ERR_CUDA;
  }
  *p = (T *)q;
  return DAWN_OK;
}

// Stream-ordered free: the block returns to the pool once `stream` reaches
// this point, so every use of it must be ordered before that on `stream`.
void dfree(void *p, cudaStream_t stream) {
  if (p) cudaFreeAsync(p, stream);
}

// Allocation of a handle's workspace (solver, backward, trace), with the
// DAWN_OPT_TEST_FAIL_ALLOC hook: a host-side stand-in for an out-of-memory
// device, so the OOM paths are tested without exhausting a shared GPU.
template <typename T>
int halloc(dawn_graph g, T **p, size_t count, cudaStream_t stream) {
  if (g->fail_alloc > 0 && --g->fail_alloc == 0) {
    *p = nullptr;
    return DAWN_ERR_OOM;
  }
  return dalloc(g->device, p, count, stream);
}

void free_workspace(dawn_graph g, cudaStream_t stream) {
  dfree(g->state, stream);
  dfree(g->bitmap, stream);
  dfree(g->queue, stream);
  dfree(g->tiles, stream);
  dfree(g->tails, stream);
  g->state = nullptr;
  g->bitmap = nullptr;
  g->queue = nullptr;
  g->tiles = nullptr;
  g->tails = nullptr;
  g->ws_k = 0;
}

// Largest number of instances one launch may hold: the per-block instance
// prefix, the int32 tile numbering and a device-memory budget.
int32_t max_chunk(dawn_graph g) {
  const int64_t tiles_cap = g->m / dawn::kTile + 2;
  int64_t by_tiles = (int64_t)0x7FFFFFFF / tiles_cap;
  const int64_t per_inst = (int64_t)g->n * (8 + 16) + 8 * ((g->n + 31) / 32) + 4 * tiles_cap + 16;
  size_t free_b = 0, total_b = 0;
  int64_t budget = (int64_t)48 << 30;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) budget = std::min<int64_t>(budget, (int64_t)(free_b / 2));
  int64_t by_mem = std::max<int64_t>(1, budget / std::max<int64_t>(per_inst, 1));
  return (int32_t)std::max<int64_t>(1, std::min<int64_t>({(int64_t)dawn::kMaxInstancesPerLaunch, by_tiles, by_mem}));
}

// Grows the solver workspace to k instances, allocating on `stream`.  The
// old workspace is freed on `stream` after the handle's previous stream has
// drained (one stream at a time per handle, but possibly a different one).
int ensure_workspace(dawn_graph g, int32_t k, cudaStream_t stream) {
  if (g->ws_k >= k) return DAWN_OK;
  if (g->ws_k > 0 && g->last_stream != stream && cudaStreamSynchronize(g->last_stream) != cudaSuccess)
    return DAWN_ERR_CUDA;
  free_workspace(g, stream);
  g->words = (g->n + 31) / 32;
  g->tiles_cap = g->m / dawn::kTile + 2;
  const size_t kn = (size_t)k * g->n;
  int rc;
  if ((rc = halloc(g, &g->state, kn, stream)) || (rc = halloc(g, &g->bitmap, (size_t)2 * k * g->words, stream)) ||
      (rc = halloc(g, &g->queue, kn, stream)) || (rc = halloc(g, &g->tiles, (size_t)k * g->tiles_cap, stream)) ||
      (rc = halloc(g, &g->tails, (size_t)2 * k, stream))) {
    free_workspace(g, stream);
    return rc;
  }
  g->ws_k = k;
  return DAWN_OK;
}

int kernel_ctas(dawn_graph g) { return g->ctas_per_sm == 4 ? 4 : 5; }

int occupancy(dawn_graph g, int ctas) {
  int &c = g->occupancy[ctas == 4 ? 0 : 1];
  if (c == 0) c = std::max(1, dawn::govm_max_blocks_per_sm(g->wtype, ctas));
  return c;
}

int grid_for(dawn_graph g, int32_t k) {
  const int cap = occupancy(g, kernel_ctas(g)) * g->sms;
  if (g->grid_blocks > 0) return std::min(g->grid_blocks, cap);
  // small problems get a small grid: barriers are cheaper with fewer blocks
  const int64_t work = (int64_t)k * std::max<int64_t>(g->m, g->n);
  const int64_t want = (work + 16383) / 16384;
  return (int)std::max<int64_t>(1, std::min<int64_t>(cap, want));
}

// Largest n * max|w| the weight type allows; 0 = no bound.
uint32_t weight_limit(int wtype) {
  // uint32: every candidate dist(u) + w is at most n * max(w) (shortest paths
  // are simple); it must stay below the unreachable sentinel.
  if (wtype == DAWN_W_U32) return 0xFFFFFFFFu;
  // int32: every simple-path sum and candidate lies in [-n max|w|, n max|w|],
  // which must stay inside int32 and below the unreachable sentinel INT32_MAX
  if (wtype == DAWN_W_I32) return 0x7FFFFFFFu;
  return 0;
}

// The small-graph kernel's compact form (32-bit keys, 16-bit frontier ids)
// serves calls that want no parents on graphs of non-negative weights with
// at most 65,536 vertices.
bool small_compact(dawn_graph g, bool parents) {
  return !parents && g->wtype != DAWN_W_I32 && g->n <= 65536;
}

// The small-graph kernel's mode for this handle and call: 0 = not used,
// 1 = with the solver state in shared memory, 2 = with the CSR there too.
int small_mode(dawn_graph g, bool compact) {
  if (g->small_path == DAWN_SMALL_NEVER || g->gsvm || g->test_stall || g->trace) return 0;
  const size_t limit = dawn::small_smem_limit();
  if (dawn::small_layout(g->n, g->m, true, compact).total <= limit) return 2;
  if (g->small_path == DAWN_SMALL_WHEN_STATE_FITS && dawn::small_layout(g->n, g->m, false, compact).total <= limit)
    return 1;
  return 0;
}

// Direct steps (the frontier read from the bitmap, one barrier per step) or
// queue steps (the frontier compacted into a queue of 128-edge tiles).
// Direct steps serve single-instance launches (dawn_sssp, dawn_sssp_roots).
int direct_steps(dawn_graph g, int32_t k) {
  if (k != 1 || g->gsvm || g->frontier == DAWN_FRONTIER_QUEUE) return 0;
  return g->frontier == DAWN_FRONTIER_BITMAP || g->max_deg <= dawn::kDirectMaxDegree;
}

// One persistent launch.  `accumulate` (later launches of one batched call)
// keeps the status and the counters of the earlier launches: only the
// barrier word and the per-step change flags start again from zero.
int run_solve(dawn_graph g, const int32_t *seeds, int32_t nseeds, int32_t source, int32_t k, int roots_mode,
              void *dist, int32_t *parent, int32_t *parent_edge, cudaStream_t stream, bool accumulate = false) {
  const bool compact = small_compact(g, parent || parent_edge);
  const int small = small_mode(g, compact);
  int rc = small ? DAWN_OK : ensure_workspace(g, k, stream);  // the small kernel keeps its state on-chip
  if (rc) return rc;
  GovmParams p = {};
  p.row_ptr = g->row_ptr;
  p.cw = g->cw;
  p.src = g->src;
  p.n = g->n;
  p.m = g->m;
  p.k = k;
  p.roots_mode = roots_mode;
  p.seeds = seeds;
  p.nseeds = nseeds;
  p.source = source;
  p.state = g->state;
  p.bitmap = g->bitmap;
  p.queue = g->queue;
  p.tiles = g->tiles;
  p.tails = g->tails;
  p.words = g->words;
  p.tiles_cap = g->tiles_cap;
  p.dist = dist;
  p.parent = parent;
  p.parent_edge = parent_edge;
  p.ctl = g->ctl;
  p.max_steps = g->max_steps > 0 ? g->max_steps : g->n;
  p.wait_limit_ns = g->wait_limit_ns;
  p.test_stall = g->test_stall;
  p.gsvm = g->gsvm;
  p.direct = direct_steps(g, k);
  p.skip_remarked = g->skip_remarked && !g->gsvm;  // Algorithm 1's bitmap holds every reached vertex
  p.trace = g->trace;
  p.trace_cap = g->trace_cap;
  p.vflags = g->vflags;
  p.vlimit = weight_limit(g->wtype);
  cudaError_t e;
  if (accumulate) {
    e = cudaMemsetAsync(&g->ctl->bar, 0, sizeof(g->ctl->bar), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->ctl->changed, 0, sizeof(g->ctl->changed), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->ctl->marks, 0, sizeof(g->ctl->marks), stream);
  } else {
    e = cudaMemsetAsync(g->ctl, 0, sizeof(DeviceCtl), stream);
  }
  if (e == cudaSuccess && g->trace)
    e = cudaMemsetAsync(g->trace, 0, (size_t)g->trace_cap * 4 * sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = small ? dawn::launch_govm_small(p, g->wtype, roots_mode ? 1 : k, small == 2, compact, stream)
            : dawn::launch_govm(p, g->wtype, kernel_ctas(g), grid_for(g, k), stream);
  if (e != cudaSuccess) return cuda_fail(e);
  g->last_stream = stream;
  return DAWN_OK;
}

int set_device(dawn_graph g) {
  return cudaSetDevice(g->device) == cudaSuccess ? DAWN_OK : DAWN_ERR_CUDA;
}

int copy_in(void *dst, const void *src, size_t bytes, int on_device, cudaStream_t stream) {
  if (bytes == 0) return DAWN_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  stream);
  return e == cudaSuccess ? DAWN_OK : cuda_fail(e);
}

// Validates the device copy of the graph; synchronous.
// Runs the validation kernel; with `wait` the verdict is read back and
// returned, otherwise only the next solve sees it (through GovmParams).
int validate(dawn_graph g, cudaStream_t stream, bool wait = true) {
  cudaError_t e = cudaMemsetAsync(g->vflags, 0, 4 * sizeof(unsigned), stream);
  if (e != cudaSuccess) return cuda_fail(e);
  const int64_t work = std::max<int64_t>(g->m, (int64_t)g->n + 1);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)g->sms * 8));
  validate_kernel<<<blocks, 256, 0, stream>>>(g->row_ptr, g->col, g->w, g->n, g->m, g->wtype,
                                               g->vflags);
  unsigned h[3] = {0, 0, 0};
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  if (!wait) return DAWN_OK;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, g->vflags, sizeof(h), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e);
  if (h[0]) return DAWN_ERR_INVALID;
  g->max_deg = (int32_t)std::min<unsigned>(h[2], 0x7FFFFFFFu);
  const uint32_t lim = weight_limit(g->wtype);
  if (lim && (uint64_t)g->n * (uint64_t)h[1] >= lim) return DAWN_ERR_INVALID;
  return DAWN_OK;
}

// Frees every device buffer of the handle on `stream` (which the handle's
// work has been ordered on or has finished), waits until the frees have
// completed (so a later dawn_trim_memory can return the memory) and deletes
// the handle.
void release(dawn_graph g, cudaStream_t stream) {
  free_workspace(g, stream);
  dfree(g->row_ptr, stream);
  dfree(g->col, stream);
  dfree(g->w, stream);
  dfree(g->cw, stream);
  dfree(g->trace, stream);
  dfree(g->src, stream);
  dfree(g->ctl, stream);
  dfree(g->vflags, stream);
  dfree(g->bw_base, stream);
  delete g;
  cudaStreamSynchronize(stream);
}

}  // namespace

namespace dawn {
int launch_limits(dawn_graph g, LaunchLimits *out) {
  if (!g || !out) return DAWN_ERR_INVALID;
  if (set_device(g)) return DAWN_ERR_CUDA;
  out->sms = g->sms;
  out->occupancy4 = occupancy(g, 4);
  out->occupancy5 = occupancy(g, 5);
  out->max_batch = max_chunk(g);
  out->ctas_per_sm = g->ctas_per_sm;
  out->grid_blocks = g->grid_blocks;
  out->batch = g->batch;
  out->small_path = g->small_path;
  out->frontier = g->frontier;
  out->auto_frontier = g->max_deg <= dawn::kDirectMaxDegree ? DAWN_FRONTIER_BITMAP : DAWN_FRONTIER_QUEUE;
  // the tuner times its candidates without parent outputs
  out->small_state_fits =
      dawn::small_layout(g->n, g->m, false, small_compact(g, false)).total <= dawn::small_smem_limit();
  return DAWN_OK;
}
}  // namespace dawn

extern "C" {

const char *dawn_status_string(int code) {
  switch (code) {
    case DAWN_OK: return "DAWN_OK";
    case DAWN_ERR_INVALID: return "DAWN_ERR_INVALID: invalid argument or graph";
    case DAWN_ERR_OOM: return "DAWN_ERR_OOM: device allocation failed";
    case DAWN_ERR_CUDA: return "DAWN_ERR_CUDA: CUDA runtime error";
    case DAWN_ERR_NOT_CONVERGED: return "DAWN_ERR_NOT_CONVERGED: step cap reached";
    case DAWN_ERR_TIMEOUT: return "DAWN_ERR_TIMEOUT: bounded in-kernel wait ran out";
    case DAWN_ERR_BOUNDS: return "DAWN_ERR_BOUNDS: internal capacity check failed";
    default: return "unknown dawn status";
  }
}

int dawn_create_graph(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col_idx, const void *weights,
                      int wtype, int inputs_on_device, void *stream, dawn_graph *out) {
  if (!out) return DAWN_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || m < 0 || m > 0x7FFFFFFF || !row_ptr || (m > 0 && (!col_idx || !weights)) ||
      (wtype != DAWN_W_U32 && wtype != DAWN_W_F32 && wtype != DAWN_W_I32))
    return DAWN_ERR_INVALID;
  dawn_graph g = new (std::nothrow) dawn_graph_s();
  if (!g) return DAWN_ERR_OOM;
  g->n = n;
  g->m = m;
  g->wtype = wtype;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = DAWN_OK;
  int l2 = 0;
  if (cudaGetDevice(&g->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device) != cudaSuccess) {
    delete g;
    return DAWN_ERR_CUDA;
  }
  g->l2_bytes = l2;
  if (g->device >= kPoolDevices) {
    delete g;
    return DAWN_ERR_CUDA;
  }
  const int dev = g->device;
  if ((rc = dalloc(dev, &g->row_ptr, (size_t)n + 1, s)) || (rc = dalloc(dev, &g->col, (size_t)m, s)) ||
      (rc = dalloc(dev, &g->w, (size_t)m, s)) || (rc = dalloc(dev, &g->cw, (size_t)m, s)) ||
      (rc = dalloc(dev, &g->src, (size_t)m, s)) || (rc = dalloc(dev, &g->ctl, 1, s)) ||
      (rc = dalloc(dev, &g->vflags, 4, s)) ||
      (rc = copy_in(g->row_ptr, row_ptr, ((size_t)n + 1) * 4, inputs_on_device, s)) ||
      (rc = copy_in(g->col, col_idx, (size_t)m * 4, inputs_on_device, s)) ||
      (rc = copy_in(g->w, weights, (size_t)m * 4, inputs_on_device, s)) || (rc = validate(g, s))) {
    release(g, s);
    return rc;
  }
  if (cudaMemsetAsync(g->ctl, 0, sizeof(DeviceCtl), s) != cudaSuccess) {
    release(g, s);
    return DAWN_ERR_CUDA;
  }
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n * 32 + 255) / 256, (int64_t)g->sms * 16));
  edge_tail_kernel<<<blocks, 256, 0, s>>>(g->row_ptr, n, g->src);
  const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)g->sms * 16));
  interleave_kernel<<<eb, 256, 0, s>>>(g->col, g->w, m, g->cw);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    release(g, s);
    return DAWN_ERR_CUDA;
  }
  dfree(g->col, s);  // columns and weights now live in cw
  dfree(g->w, s);
  g->col = nullptr;
  g->w = nullptr;
  g->last_stream = s;
  *out = g;
  return DAWN_OK;
}

int dawn_set_weights(dawn_graph g, const void *weights, int flags, void *stream) {
  if (!g || (g->m > 0 && !weights) || (flags & ~(DAWN_WEIGHTS_ON_DEVICE | DAWN_WEIGHTS_DEFER_CHECK)))
    return DAWN_ERR_INVALID;
  if (set_device(g)) return DAWN_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t *src = (const uint32_t *)weights;
  int rc;
  if (!(flags & DAWN_WEIGHTS_ON_DEVICE) && g->m > 0) {  // host weights go through a device staging copy
    if (!g->w && (rc = halloc(g, &g->w, (size_t)g->m, s))) return rc;
    if ((rc = copy_in(g->w, weights, (size_t)g->m * 4, 0, s))) return rc;
    src = g->w;
  }
  g->last_stream = s;
  cudaError_t e = cudaMemsetAsync(g->vflags, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (g->m > 0) {
    const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((g->m + 255) / 256, (int64_t)g->sms * 16));
    weights_kernel<<<eb, 256, 0, s>>>(src, g->m, g->wtype, g->cw, g->vflags);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  }
  if (flags & DAWN_WEIGHTS_DEFER_CHECK) return DAWN_OK;  // the next solve reads the verdict itself
  unsigned h[2] = {0, 0};
  e = cudaMemcpyAsync(h, g->vflags, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (h[0]) return DAWN_ERR_INVALID;
  const uint32_t lim = weight_limit(g->wtype);
  if (lim && (uint64_t)g->n * (uint64_t)h[1] >= lim) return DAWN_ERR_INVALID;
  return DAWN_OK;
}

int dawn_reserve(dawn_graph g, int32_t k) {
  if (!g || k < 1) return DAWN_ERR_INVALID;
  if (set_device(g)) return DAWN_ERR_CUDA;
  // allocated in the order of the handle's stream, then made usable on any
  int rc = ensure_workspace(g, std::min(k, max_chunk(g)), g->last_stream);
  if (rc == DAWN_OK && cudaStreamSynchronize(g->last_stream) != cudaSuccess) rc = DAWN_ERR_CUDA;
  return rc;
}

int dawn_sssp(dawn_graph g, int32_t source, void *dist, int32_t *parent, int32_t *parent_edge, void *stream) {
  if (!g || !dist || source < 0 || source >= g->n) return DAWN_ERR_INVALID;
  if (set_device(g)) return DAWN_ERR_CUDA;
  g->last_k = 1;
  return run_solve(g, nullptr, 1, source, 1, 0, dist, parent, parent_edge, (cudaStream_t)stream);
}

int dawn_msssp(dawn_graph g, const int32_t *sources, int32_t k, void *dist, int32_t *parent, void *stream) {
  if (!g || !sources || !dist || k < 1) return DAWN_ERR_INVALID;
  if (set_device(g)) return DAWN_ERR_CUDA;
  int32_t chunk = g->batch > 0 ? std::min({k, g->batch, max_chunk(g)})
                               : std::min(k, g->ws_k > 0 ? std::max(g->ws_k, std::min(k, max_chunk(g)))
                                                         : max_chunk(g));
  // Automatic batch on a graph where fewer than 32 instances' packed states
  // fit L2 together: as many instances per launch as fit (at least 4), so
  // that their state gathers stay L2 hits (R-MAT s20 16 and s22 4 per launch:
  // 1.32x and 1.39x faster than the largest batch).  With smaller states the
  // largest batch is fastest (R-MAT s18: 512 per launch, 64 fit L2).
  const int64_t state = 8 * (int64_t)g->n;
  if (g->batch <= 0 && g->l2_bytes > 0 && state * 32 > g->l2_bytes)
    chunk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(chunk, std::max<int64_t>(4, g->l2_bytes / state)));
  g->last_k = k;
  for (int32_t b = 0; b < k; b += chunk) {
    const int32_t kk = std::min(chunk, k - b);
    const size_t off = (size_t)b * g->n;
    int rc = run_solve(g, sources + b, kk, 0, kk, 0, (uint32_t *)dist + off, parent ? parent + off : nullptr,
                       nullptr, (cudaStream_t)stream, b > 0);
    if (rc) return rc;
  }
  return DAWN_OK;
}

int dawn_sssp_roots(dawn_graph g, const int32_t *roots, int32_t k, void *dist, int32_t *parent, int32_t *parent_edge,
                    void *stream) {
  if (!g || !roots || !dist || k < 1) return DAWN_ERR_INVALID;
  if (set_device(g)) return DAWN_ERR_CUDA;
  g->last_k = 1;
  return run_solve(g, roots, k, 0, 1, 1, dist, parent, parent_edge, (cudaStream_t)stream);
}

int dawn_sssp_backward(dawn_graph g, const int32_t *parent_edge, const float *grad_dist, float *grad_w, void *stream) {
  if (!g || !parent_edge || !grad_dist || (g->m > 0 && !grad_w)) return DAWN_ERR_INVALID;
  if (g->wtype != DAWN_W_F32) return DAWN_ERR_INVALID;
  if (set_device(g)) return DAWN_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)g->n;
  if (!g->bw_base) {
    int rc = halloc(g, &g->bw_base, 32 + 16 * n, s);
    if (rc) return rc;
    g->bw_edges = (unsigned long long *)g->bw_base;
    g->bw_cnt = (int32_t *)(g->bw_base + 32);  // inner [n], rem [n], par [n]
    g->bw_acc = (float *)(g->bw_base + 32 + 12 * n);
  }
  // status word, then the edge counters and the inner / rem flags in one memset
  cudaError_t e = cudaMemsetAsync(g->ctl, 0, sizeof(DeviceCtl), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->bw_base, 0, 32 + 8 * n, s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (g->m > 0) {
    const int64_t work = std::max<int64_t>(g->m, g->n);
    const int cb = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)g->sms * 8));
    bw_count_kernel<<<cb, 256, 0, s>>>(parent_edge, grad_dist, g->src, g->n, g->m, g->bw_acc, g->bw_cnt,
                                       g->bw_cnt + g->n, g->bw_cnt + 2 * (size_t)g->n, g->bw_edges, grad_w,
                                       g->ctl);
    const int vb = (int)std::max<int64_t>(1, std::min<int64_t>((g->n + 255) / 256, (int64_t)g->sms * 8));
    bw_walk_kernel<<<vb, 256, 0, s>>>(parent_edge, g->bw_cnt + 2 * (size_t)g->n, g->n, g->bw_acc, g->bw_cnt,
                                      g->bw_cnt + g->n, grad_w, g->bw_edges, g->ctl);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  g->last_stream = s;
  return DAWN_OK;
}

int dawn_status(dawn_graph g, int sync) {
  if (!g) return DAWN_ERR_INVALID;
  if (set_device(g)) return DAWN_ERR_CUDA;
  if (sync && cudaStreamSynchronize(g->last_stream) != cudaSuccess) return DAWN_ERR_CUDA;
  int st = 0;
  if (cudaMemcpy(&st, &g->ctl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DAWN_ERR_CUDA;
  return st;
}

int dawn_get_stats(dawn_graph g, dawn_stats *out) {
  if (!g || !out) return DAWN_ERR_INVALID;
  if (set_device(g)) return DAWN_ERR_CUDA;
  if (cudaStreamSynchronize(g->last_stream) != cudaSuccess) return DAWN_ERR_CUDA;
  DeviceCtl h;
  if (cudaMemcpy(&h, g->ctl, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return DAWN_ERR_CUDA;
  out->steps = (int64_t)h.steps;
  out->frontier_sum = (int64_t)h.frontier_sum;
  out->edges_scanned = (int64_t)h.edges_scanned;
  out->updates = (int64_t)h.updates;
  out->edges_skipped = (int64_t)h.edges_skipped;
  out->instances = g->last_k;
  return DAWN_OK;
}

int dawn_set_option(dawn_graph g, int option, int64_t value) {
  if (!g) return DAWN_ERR_INVALID;
  switch (option) {
    case DAWN_OPT_MAX_STEPS: g->max_steps = value; return DAWN_OK;
    case DAWN_OPT_WAIT_LIMIT_NS:
      if (value <= 0) return DAWN_ERR_INVALID;
      g->wait_limit_ns = (unsigned long long)value;
      return DAWN_OK;
    case DAWN_OPT_GRID_BLOCKS:
      if (value < 0) return DAWN_ERR_INVALID;
      g->grid_blocks = (int)value;
      return DAWN_OK;
    case DAWN_OPT_CTAS_PER_SM:
      if (value != 0 && value != 4 && value != 5) return DAWN_ERR_INVALID;
      g->ctas_per_sm = (int)value;
      return DAWN_OK;
    case DAWN_OPT_BATCH:
      if (value < 0 || value > 0x7FFFFFFF) return DAWN_ERR_INVALID;
      g->batch = (int)value;
      return DAWN_OK;
    case DAWN_OPT_SMALL_PATH:
      if (value < 0 || value > DAWN_SMALL_WHEN_STATE_FITS) return DAWN_ERR_INVALID;
      g->small_path = (int)value;
      return DAWN_OK;
    case DAWN_OPT_TEST_STALL: g->test_stall = value != 0; return DAWN_OK;
    case DAWN_OPT_TEST_FAIL_ALLOC:
      if (value < 0) return DAWN_ERR_INVALID;
      g->fail_alloc = value;
      return DAWN_OK;
    case DAWN_OPT_GSVM: g->gsvm = value != 0; return DAWN_OK;
    case DAWN_OPT_SKIP_REMARKED: g->skip_remarked = value != 0; return DAWN_OK;
    case DAWN_OPT_FRONTIER:
      if (value < DAWN_FRONTIER_AUTO || value > DAWN_FRONTIER_BITMAP) return DAWN_ERR_INVALID;
      g->frontier = (int)value;
      return DAWN_OK;
    case DAWN_OPT_TRACE_STEPS: {
      if (value < 0 || value > (1 << 24)) return DAWN_ERR_INVALID;
      if (set_device(g)) return DAWN_ERR_CUDA;
      cudaStream_t s = g->last_stream;
      if (cudaStreamSynchronize(s) != cudaSuccess) return DAWN_ERR_CUDA;
      dfree(g->trace, s);
      g->trace = nullptr;
      g->trace_cap = 0;
      if (value == 0) return DAWN_OK;
      int rc = halloc(g, &g->trace, (size_t)value * 4, s);
      if (rc) return rc;
      if (cudaMemsetAsync(g->trace, 0, (size_t)value * 4 * sizeof(unsigned long long), s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return DAWN_ERR_CUDA;
      g->trace_cap = (int32_t)value;
      return DAWN_OK;
    }
    default: return DAWN_ERR_INVALID;
  }
}

int dawn_get_trace(dawn_graph g, int64_t *out, int32_t cap) {
  if (!g || !out || cap < 0) return -DAWN_ERR_INVALID;
  if (!g->trace) return 0;
  if (set_device(g)) return -DAWN_ERR_CUDA;
  if (cudaStreamSynchronize(g->last_stream) != cudaSuccess) return -DAWN_ERR_CUDA;
  const int32_t rows = std::min(cap, g->trace_cap);
  if (rows == 0) return 0;
  if (cudaMemcpy(out, g->trace, (size_t)rows * 4 * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return -DAWN_ERR_CUDA;
  int32_t used = 0;
  while (used < rows && out[4 * used] != 0) {
    const bool last = out[4 * used + 3] == 1;
    ++used;
    if (last) break;
  }
  return used;
}

int dawn_graph_info(dawn_graph g, int32_t *n, int64_t *m, int *wtype) {
  if (!g) return DAWN_ERR_INVALID;
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (wtype) *wtype = g->wtype;
  return DAWN_OK;
}

void dawn_destroy(dawn_graph g) {
  if (!g) return;
  cudaSetDevice(g->device);
  cudaStreamSynchronize(g->last_stream);  // the handle's work has finished: its memory can go back
  release(g, g->last_stream);
}

int dawn_trim_memory(void) {
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DAWN_ERR_CUDA;
  int rc = DAWN_OK;
  for (int d = 0; d < kPoolDevices; ++d) {
    if (!g_pools[d].pool) continue;
    if (cudaSetDevice(d) != cudaSuccess || cudaMemPoolTrimTo(g_pools[d].pool, 0) != cudaSuccess) {
      cudaGetLastError();
      rc = DAWN_ERR_CUDA;
    }
  }
  if (cudaSetDevice(dev) != cudaSuccess) rc = DAWN_ERR_CUDA;
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free single-source solve.
//
// Some callers cannot allocate device memory while they run: code that
// executes inside a memory budget fixed up front, real-time or embedded
// hosts that forbid allocator calls after start-up, and callers that must not
// trigger the implicit synchronisation of cudaMalloc / cudaFree.  For them,
// dawn_sssp_noalloc runs the same GOVM kernel with its whole per-solve
// workspace carved out of one fixed-size array in device global memory that
// is part of this library (every GPU that loads the library holds it until
// the process exits).
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name only stands in for the symbol; the address comes from
// cudaGetSymbolAddress, looked up once per device (on the first call).
int noalloc_scratch(int device, unsigned char **out) {
  if (device < 0 || device >= kMaxDevices) return DAWN_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return DAWN_ERR_CUDA;
    }
    g_noalloc_ptr[device] = ptr;
  }
  *out = (unsigned char *)g_noalloc_ptr[device];
  return DAWN_OK;
}

}  // namespace

extern "C" int dawn_sssp_noalloc(dawn_graph g, int32_t source, void *dist, int32_t *parent, int32_t *parent_edge,
                                 int32_t *status_out, void *stream) {
  if (!g || !dist || source < 0 || source >= g->n) return DAWN_ERR_INVALID;
  if (set_device(g)) return DAWN_ERR_CUDA;
  // workspace layout inside the fixed array (each piece 256-byte aligned)
  const int64_t words = (g->n + 31) / 32;
  const int64_t tiles_cap = g->m / dawn::kTile + 2;
  size_t used = 0;
  auto take = [&used](size_t bytes) {
    const size_t at = used;
    used = (used + bytes + 255) & ~(size_t)255;
    return at;
  };
  const size_t o_ctl = take(sizeof(DeviceCtl));
  const size_t o_tails = take(2 * sizeof(unsigned long long));
  const size_t o_state = take((size_t)g->n * sizeof(unsigned long long));
  const size_t o_bitmap = take((size_t)2 * words * sizeof(uint32_t));
  const size_t o_queue = take((size_t)g->n * sizeof(uint4));
  const size_t o_tiles = take((size_t)tiles_cap * sizeof(int32_t));
  if (used > kNoAllocScratchBytes) return DAWN_ERR_INVALID;  // graph too large for the fixed scratch
  unsigned char *base = nullptr;
  int rc = noalloc_scratch(g->device, &base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceCtl *ctl = (DeviceCtl *)(base + o_ctl);
  GovmParams p = {};
  p.row_ptr = g->row_ptr;
  p.cw = g->cw;
  p.src = g->src;
  p.n = g->n;
  p.m = g->m;
  p.k = 1;
  p.roots_mode = 0;
  p.seeds = nullptr;
  p.nseeds = 1;
  p.source = source;
  p.state = (unsigned long long *)(base + o_state);
  p.bitmap = (uint32_t *)(base + o_bitmap);
  p.queue = (uint4 *)(base + o_queue);
  p.tiles = (int32_t *)(base + o_tiles);
  p.tails = (unsigned long long *)(base + o_tails);
  p.words = words;
  p.tiles_cap = tiles_cap;
  p.dist = dist;
  p.parent = parent;
  p.parent_edge = parent_edge;
  p.ctl = ctl;
  p.max_steps = g->max_steps > 0 ? g->max_steps : g->n;
  p.wait_limit_ns = g->wait_limit_ns;
  p.test_stall = g->test_stall;
  p.gsvm = g->gsvm;
  p.direct = direct_steps(g, 1);
  p.skip_remarked = g->skip_remarked && !g->gsvm;
  p.trace = g->trace;  // allocated when the option was set, not here
  p.trace_cap = g->trace_cap;
  p.vflags = g->vflags;
  p.vlimit = weight_limit(g->wtype);
  // the control block (barrier counters, status) must start at zero; the
  // kernel itself resets everything else it reads
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(DeviceCtl), s);
  if (e == cudaSuccess && g->trace)
    e = cudaMemsetAsync(g->trace, 0, (size_t)g->trace_cap * 4 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = dawn::launch_govm(p, g->wtype, kernel_ctas(g), grid_for(g, 1), s);
  // the handle's own control block receives this solve's status and
  // counters, so dawn_status / dawn_get_stats report it like any other solve
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->ctl, ctl, sizeof(DeviceCtl), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && status_out)
    e = cudaMemcpyAsync(status_out, &ctl->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e);
  g->last_k = 1;
  g->last_stream = s;  // dawn_status(g, 1), dawn_get_stats and dawn_destroy wait on it
  return DAWN_OK;
}
