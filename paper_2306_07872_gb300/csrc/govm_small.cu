// Small-graph GOVM kernel (weighted DAWN, arxiv 2306.07872, Section 3.4,
// Algorithm 2) for sm_103a.
//
// One thread block solves one instance with the packed state alpha, the
// bitmap beta and the frontier delta in shared memory, and the CSR too when
// it fits.  A step then ends with block barriers instead of device-wide ones,
// and every access except the initial CSR copy stays on-chip.  Blocks of
// different instances never wait on one another, so a batch of small
// instances runs as an ordinary (non-cooperative) launch of one block each.
//   relax  a group of `group` threads (a power of two near the average
//          degree) per frontier vertex, its threads over the vertex's
//          out-edges (two per thread and round when the CSR is read from
//          L2); the vertex's distance is read in place (Algorithm 2); a candidate
//          that beats alpha[t] updates it with a packed 64-bit atomicMin in
//          shared memory, and marks beta[t] when that atomic strictly lowered
//          the distance;
//   build  beta is compacted into delta (vertices with an out-edge, read
//          from a bitmap built once per block, so the build touches shared
//          memory only) by a block-wide prefix sum and cleared.
// The same (distance, lowest parent edge) fixpoint as the persistent kernel
// results: both are exact minima of the packed keys.
// Compact form, for solves that want no parents on graphs with non-negative
// weights and at most 65,536 vertices: alpha holds the 32-bit distance keys
// alone and delta 16-bit vertex ids, half the shared memory, so that two
// instances fit on an SM (each block's barrier waits overlap the other's
// work).  The distances are the same minima; with non-negative weights no
// candidate can beat a source's zero key, so the source guard needs no parent
// field to tell a source apart.
#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>

#include "dawn_common.cuh"
#include "dawn_keys.cuh"

namespace dawn {

__host__ __device__ static inline size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ SmallLayout small_layout(int32_t n, int64_t m, bool csr, bool compact) {
  SmallLayout L{};
  L.state = 0;
  L.bitmap = L.state + round16((compact ? 4 : 8) * (size_t)n);
  L.front = L.bitmap + round16(4 * (size_t)((n + 31) / 32));
  L.scan = L.front + round16((compact ? 2 : 4) * (size_t)n);
  L.hasout = L.scan + round16(4 * (size_t)(2 * kSmallWarps + 2));
  L.row_ptr = L.hasout + round16(4 * (size_t)((n + 31) / 32));
  L.cw = L.row_ptr + (csr ? round16(4 * ((size_t)n + 1)) : 0);
  L.total = L.cw + (csr ? round16(8 * (size_t)m) : 0);
  return L;
}

namespace {

constexpr unsigned kFullMask = 0xFFFFFFFFu;

// Block-wide exclusive prefix of x; *total receives the sum.  Every thread
// of the block must call it; sc holds 2 * kSmallWarps + 2 ints.
__device__ __forceinline__ int32_t block_prefix(int32_t x, int32_t *sc, int32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t o = __shfl_up_sync(kFullMask, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) sc[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int32_t v = lane < kSmallWarps ? sc[lane] : 0;
    int32_t vi = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t o = __shfl_up_sync(kFullMask, vi, d);
      if (lane >= d) vi += o;
    }
    if (lane < kSmallWarps) sc[kSmallWarps + lane] = vi - v;  // exclusive warp offsets
    if (lane == 31) sc[2 * kSmallWarps] = vi;                 // block total
  }
  __syncthreads();
  const int32_t r = sc[kSmallWarps + warp] + incl - x;
  *total = sc[2 * kSmallWarps];
  __syncthreads();  // sc is reused by the next call
  return r;
}

// delta <- beta restricted to vertices with an out-edge; beta <- {}.  Returns
// the new frontier size (block-uniform) and adds the marked vertices to
// *marks (a thread-local partial sum).  `ho` is the bitmap of vertices with
// an out-edge, built once per block, so the build reads shared memory only.
// Each thread owns a contiguous range of bitmap words, so the frontier lists
// its vertices in increasing order.
template <typename FrontT>
__device__ int32_t small_build(int32_t n, const uint32_t *ho, uint32_t *bm, FrontT *front, int32_t *sc,
                               unsigned long long *marks) {
  const int32_t words = (n + 31) / 32;
  const int32_t per = (words + (int32_t)blockDim.x - 1) / (int32_t)blockDim.x;
  const int32_t w0 = min((int32_t)threadIdx.x * per, words), w1 = min(w0 + per, words);
  int32_t mine = 0;
  for (int32_t w = w0; w < w1; ++w) {
    const uint32_t b = bm[w];
    *marks += __popc(b);
    mine += __popc(b & ho[w]);
  }
  int32_t total = 0;
  int32_t at = block_prefix(mine, sc, &total);
  for (int32_t w = w0; w < w1; ++w) {
    uint32_t b = bm[w] & ho[w];
    bm[w] = 0u;  // only this thread reads its words
    while (b) {
      front[at++] = (FrontT)(w * 32 + __ffs(b) - 1);
      b &= b - 1;
    }
  }
  __syncthreads();
  return total;
}

template <int WT, bool COMPACT>
__global__ void __launch_bounds__(kSmallThreads, COMPACT ? 2 : 1) govm_small_kernel(GovmParams p, int32_t csr_in_smem,
                                                                                   int32_t group) {
  extern __shared__ __align__(16) unsigned char smem[];
  using FrontT = typename std::conditional<COMPACT, uint16_t, int32_t>::type;
  const SmallLayout L = small_layout(p.n, p.m, csr_in_smem != 0, COMPACT);
  unsigned long long *st = reinterpret_cast<unsigned long long *>(smem + L.state);  // packed form
  uint32_t *sk = reinterpret_cast<uint32_t *>(smem + L.state);                      // compact form: keys
  uint32_t *bm = reinterpret_cast<uint32_t *>(smem + L.bitmap);
  uint32_t *ho = reinterpret_cast<uint32_t *>(smem + L.hasout);
  FrontT *front = reinterpret_cast<FrontT *>(smem + L.front);
  int32_t *sc = reinterpret_cast<int32_t *>(smem + L.scan);
  const int tid = threadIdx.x, lane = tid & 31;
  const int32_t n = p.n, inst = blockIdx.x;
  const int32_t gid = tid / group, glane = tid % group, ngroups = kSmallThreads / group;
  DeviceCtl *ctl = p.ctl;
  const unsigned long long kInfState = ((unsigned long long)Key<WT>::inf << 32) | kNoEdge;
  const unsigned long long kSourceState = ((unsigned long long)Key<WT>::zero << 32) | kNoEdge;

  // Weights refused by validation (possibly deferred): no solve, no output.
  if (p.vflags) {
    const unsigned bad = __ldcg(p.vflags), wmax = __ldcg(p.vflags + 1);
    if (bad || (p.vlimit && (unsigned long long)n * wmax >= p.vlimit)) {
      if (tid == 0) atomicCAS(&ctl->status, 0, (int)DAWN_ERR_INVALID);
      return;  // uniform for the block
    }
  }

  // 1. alpha = +inf, beta = {}; the CSR into shared memory when it fits.
  for (int32_t v = tid; v < n; v += blockDim.x) {
    if (COMPACT) sk[v] = Key<WT>::inf;
    else st[v] = kInfState;
  }
  for (int32_t w = tid; w < (n + 31) / 32; w += blockDim.x) {
    bm[w] = 0u;
    ho[w] = 0u;
  }
  const int32_t *rp = p.row_ptr;
  const uint2 *cw = p.cw;
  if (csr_in_smem) {
    int32_t *srp = reinterpret_cast<int32_t *>(smem + L.row_ptr);
    uint2 *scw = reinterpret_cast<uint2 *>(smem + L.cw);
    for (int32_t v = tid; v <= n; v += blockDim.x) srp[v] = __ldg(p.row_ptr + v);
    for (int64_t e = tid; e < p.m; e += blockDim.x) scw[e] = __ldg(p.cw + e);
    rp = srp;
    cw = scw;
  }
  __syncthreads();
  // vertices with an out-edge (the build keeps only those in delta)
  for (int32_t v = tid; v < n; v += blockDim.x)
    if (rp[v + 1] > rp[v]) atomicOr(ho + (v >> 5), 1u << (v & 31));

  // 2. Seeds: alpha[s] = 0, s enters beta.
  const int32_t nseeds = p.roots_mode ? p.nseeds : 1;
  for (int32_t i = tid; i < nseeds; i += blockDim.x) {
    const int32_t s = p.seeds ? p.seeds[p.roots_mode ? i : inst] : p.source;
    if (s < 0 || s >= n) {
      atomicCAS(&ctl->status, 0, (int)DAWN_ERR_INVALID);
      continue;
    }
    if (COMPACT) sk[s] = Key<WT>::zero;
    else st[s] = kSourceState;
    atomicOr(bm + (s >> 5), 1u << (s & 31));
  }
  __syncthreads();
  unsigned long long fsum = 0, esum = 0, seeded = 0, updates = 0;
  int32_t count = small_build(n, ho, bm, front, sc, &seeded);

  // 3. GOVM steps.
  long long step = 0;
  for (;; ++step) {
    if (count == 0) break;
    if (step >= p.max_steps) {
      if (tid == 0) atomicCAS(&ctl->status, 0, (int)DAWN_ERR_NOT_CONVERGED);
      break;
    }
    fsum += (unsigned long long)count;
    for (int32_t fi = gid; fi < count; fi += ngroups) {
      const int32_t u = front[fi];
      // alpha[u] in place, as Algorithm 2 reads it
      const uint32_t du = COMPACT ? sk[u] : (uint32_t)(st[u] >> 32);
      const int32_t b = rp[u], e = rp[u + 1];
      if (glane == 0) esum += (unsigned long long)(e - b);
      auto relax = [&](uint2 c, int32_t x) {
        const uint32_t t = c.x;
        const uint32_t ckey = Key<WT>::add(du, c.y);
        if (COMPACT) {  // keys alone: a source's zero key is never beaten (weights >= 0)
          if (ckey < sk[t]) {
            const uint32_t old = atomicMin(sk + t, ckey);
            if (ckey < old) atomicOr(bm + (t >> 5), 1u << (t & 31));
          }
        } else {
          const unsigned long long cand = ((unsigned long long)ckey << 32) | (uint32_t)x;
          const unsigned long long cur = st[t];
          if (cand < cur && cur != kSourceState) {  // the source guard: never relax into a source
            const unsigned long long old = atomicMin(st + t, cand);
            if (ckey < (uint32_t)(old >> 32)) atomicOr(bm + (t >> 5), 1u << (t & 31));
          }
        }
      };
      if (csr_in_smem) {
        for (int32_t x = b + glane; x < e; x += group) relax(cw[x], x);
      } else {  // edges from L2: two per lane and round, both loads issued before either is used
        for (int32_t x = b + glane; x < e; x += 2 * group) {
          const int32_t x1 = x + group;
          const uint2 c0 = cw[x];
          const uint2 c1 = x1 < e ? cw[x1] : make_uint2(0u, 0u);
          relax(c0, x);
          if (x1 < e) relax(c1, x1);
        }
      }
    }
    __syncthreads();
    count = small_build(n, ho, bm, front, sc, &updates);
  }

  // 4. Outputs.
  uint32_t *dist = reinterpret_cast<uint32_t *>(p.dist) + (size_t)inst * n;
  int32_t *par = p.parent ? p.parent + (size_t)inst * n : nullptr;
  int32_t *pe = p.parent_edge ? p.parent_edge + (size_t)inst * n : nullptr;
  for (int32_t v = tid; v < n; v += blockDim.x) {
    if (COMPACT) {  // no parent output in this form
      dist[v] = Key<WT>::out(sk[v]);
      continue;
    }
    const unsigned long long s = st[v];
    const uint32_t key = (uint32_t)(s >> 32), e = (uint32_t)s;
    const bool unreachable = key == Key<WT>::inf;
    dist[v] = Key<WT>::out(key);
    if (par) par[v] = unreachable ? -1 : (e == kNoEdge ? v : __ldg(p.src + e));
    if (pe) pe[v] = (unreachable || e == kNoEdge) ? -1 : (int32_t)e;
  }

  // counters: frontier sizes and their out-edges per step, path updates
  for (int d = 16; d > 0; d >>= 1) updates += __shfl_xor_sync(kFullMask, updates, d);
  for (int d = 16; d > 0; d >>= 1) esum += __shfl_xor_sync(kFullMask, esum, d);
  if (lane == 0 && updates) atomicAdd(&ctl->updates, updates);
  if (lane == 0 && esum) atomicAdd(&ctl->edges_scanned, esum);
  if (tid == 0) {
    atomicAdd(&ctl->frontier_sum, fsum);
    atomicMax(&ctl->steps, (unsigned long long)step);
  }
}

using SmallFn = void (*)(GovmParams, int32_t, int32_t);

// The compact form exists for the non-negative weight types only.
SmallFn small_for(int wtype, bool compact) {
  if (wtype == DAWN_W_F32) return compact ? govm_small_kernel<DAWN_W_F32, true> : govm_small_kernel<DAWN_W_F32, false>;
  if (wtype == DAWN_W_I32) return govm_small_kernel<DAWN_W_I32, false>;
  return compact ? govm_small_kernel<DAWN_W_U32, true> : govm_small_kernel<DAWN_W_U32, false>;
}

}  // namespace

size_t small_smem_limit() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return (size_t)v;
}

cudaError_t launch_govm_small(const GovmParams &p, int wtype, int32_t blocks, bool csr_in_smem, bool compact,
                              cudaStream_t stream) {
  static std::atomic<unsigned long long> done{0};  // kernels opted in to the large shared memory, per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  const size_t limit = small_smem_limit();
  if (!(done.load() & bit)) {
    for (int w : {DAWN_W_U32, DAWN_W_F32, DAWN_W_I32})
      for (bool c : {false, true}) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(small_for(w, c), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
        // the compact form wants two blocks' worth of shared memory per SM
        if (e == cudaSuccess && c)
          e = cudaFuncSetAttribute(small_for(w, c), cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared);
      }
    if (e != cudaSuccess) return e;
    done.fetch_or(bit);
  }
  compact = compact && wtype != DAWN_W_I32 && p.n <= 65536 && !p.parent && !p.parent_edge;
  const size_t bytes = small_layout(p.n, p.m, csr_in_smem, compact).total;
  // threads per frontier vertex: the average out-degree rounded up to a power of two, 2..32
  int32_t group = 2;
  while (group < 32 && (int64_t)group * p.n < p.m) group <<= 1;
  small_for(wtype, compact)<<<(unsigned)blocks, kSmallThreads, bytes, stream>>>(p, csr_in_smem ? 1 : 0, group);
  return cudaGetLastError();
}

}  // namespace dawn
