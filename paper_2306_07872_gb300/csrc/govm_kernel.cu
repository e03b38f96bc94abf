// Persistent GOVM kernel (weighted DAWN, arxiv 2306.07872, Section 3.4,
// Algorithm 2) for sm_103a.
//
// One cooperative launch runs a whole solve:
//   1. alpha = +inf (packed state), beta = {} (bitmap);
//   2. seeds: alpha[s] = 0 and s enters beta (every instance's source, or
//      all roots);
//   3. GOVM steps, in one of two forms (a template parameter):
//      queue steps: build delta from beta, then per step
//      relax   every warp takes 128-edge tiles of the frontier's virtual edge
//              list (the concatenated out-edges of all frontier vertices, so
//              work is balanced by edges, not vertices), relaxes each edge
//              with one 64-bit packed atomicMin (distance and parent edge
//              together) and marks beta for every candidate that beats the
//              distance it read; both are fire-and-forget reductions, so no
//              warp waits for an atomic's result;
//      build   beta is consumed in chunks of up to 32 words and compacted
//              into delta (one entry per marked vertex with an out-edge), one
//              warp atomicAdd per 128 vertices reserving entries and edge
//              offsets together;
//      each phase ends with a device-wide barrier (bounded wait); the loop
//      stops when delta is empty (no path changed) or at the step cap;
//      bitmap steps (single-instance solves on graphs of short rows): the
//      previous step's marks are the frontier; each warp expands the marked
//      vertices of its bitmap words directly (same edge phase) and marks a
//      second bitmap; one barrier per step; the loop stops after a step that
//      lowered no distance;
//   4. unpack dist / parent / parent_edge.
// No host round trip happens between steps.
#include <cuda_runtime.h>

#include <atomic>

#include "dawn_common.cuh"
#include "dawn_keys.cuh"

namespace dawn {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int *p) { return *(volatile const int *)p; }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int32_t kMark = 0x100;  // above every entry index of a tile (at most kTile)
static_assert(kTile < kMark && kEdgesPerLane <= 4, "entry indices of a tile fit 8 bits, four per register");

struct WarpTile {
  uint32_t ebase[kTile + 1];  // per entry: CSR index of its edge at virtual offset 0 (mod 2^32)
  uint32_t dkey[kTile + 1];   // per entry: current distance key of its vertex
  uint32_t vert[kTile + 1];   // per entry: its vertex (the tail of its edges)
  int32_t own[kTile];         // owning entry (relative index) of every virtual edge
};

struct BlockShared {
  int32_t tprefix[kMaxInstancesPerLaunch + 1];
  unsigned long long scan[kWarpsPerBlock];
  int32_t flag;
  int32_t any_mark;               // direct steps: some warp of the block made a strict improvement
  uint32_t pool[kWarpsPerBlock];  // direct steps: marked vertices in each warp's words of the round
  unsigned long long trace_sum[2];  // direct steps of a traced solve: the block's frontier and edges this step
  unsigned long long bar_target;  // arrivals that end the next device-wide barrier (thread 0)
  WarpTile wt[kWarpsPerBlock];
};

constexpr unsigned long long kBarError = 1ull << 63;

__device__ __noinline__ void set_status(DeviceCtl *ctl, int code) {
  atomicCAS(&ctl->status, 0, code);
  atomicOr(&ctl->bar, kBarError);
}

__device__ __forceinline__ unsigned long long atom_add_acq_rel_u64(unsigned long long *p, unsigned long long v) {
  unsigned long long o;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(o) : "l"(p), "l"(v) : "memory");
  return o;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Device-wide barrier with a bounded wait on a monotonic arrival counter:
// barrier number b ends when the counter reaches b * gridDim.x, so no block
// resets it or publishes a generation (one atomic per block and one poll per
// waiter are all the barrier costs).  The arrival is an acquire-release add
// (it publishes the block's writes, ordered before it by the block barrier);
// waiters acquire the counter.  Any error sets bit 63 of the counter as well
// as the status word, which releases every waiter at once.  Returns false
// (uniformly for the block) on an error or when the wait ran out.
__device__ bool grid_barrier(DeviceCtl *ctl, unsigned long long limit_ns, int32_t *s_flag, unsigned long long *s_target) {
  if (gridDim.x == 1) {  // one block: the block barrier already orders its memory operations
    __syncthreads();
    if (threadIdx.x == 0) *s_flag = ld_volatile_i32(&ctl->status) == 0;
    __syncthreads();
    return *s_flag != 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long target = *s_target + gridDim.x;
    *s_target = target;
    unsigned long long v = atom_add_acq_rel_u64(&ctl->bar, 1ull) + 1ull;
    if (!(v & kBarError) && v < target) {
      const unsigned long long t0 = global_ns();
      unsigned ns = 16;
      do {
        __nanosleep(ns);
        if (ns < 128) ns <<= 1;
        v = ld_acquire_u64(&ctl->bar);
        if (!(v & kBarError) && v < target && global_ns() - t0 > limit_ns) {
          set_status(ctl, DAWN_ERR_TIMEOUT);
          v = kBarError;
        }
      } while (!(v & kBarError) && v < target);
    }
    *s_flag = !(v & kBarError);
  }
  __syncthreads();
  return *s_flag != 0;
}

// Block-wide exclusive scan of one 64-bit value per thread; `total` receives
// the block sum.  Must be reached by every thread of the block.
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long x, unsigned long long &total,
                                                              BlockShared &sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    unsigned long long o = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) sh.scan[warp] = incl;
  __syncthreads();
  unsigned long long before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kWarpsPerBlock; ++w) {
    const unsigned long long s = sh.scan[w];
    if (w < warp) before += s;
    all += s;
  }
  __syncthreads();
  total = all;
  return before + incl - x;
}

// Exclusive prefix over instances of the number of tiles of each current
// frontier (tiles = ceil(edges / kTile)).  Returns the total.
__device__ int32_t scan_tiles(const unsigned long long *tails_cur, int32_t k, BlockShared &sh) {
  const int tid = threadIdx.x;
  if (k == 1) {  // one instance: no prefix needed
    const uint32_t e = (uint32_t)(__ldcg(tails_cur) >> 32);
    const int32_t t = (int32_t)((e + kTile - 1) / kTile);
    // every thread stores the same two values before reading them; the
    // device-wide barrier that ended the previous phase already ordered the
    // previous step's readers before these stores
    sh.tprefix[0] = 0;
    sh.tprefix[1] = t;
    return t;
  }
  constexpr int kPer = kMaxInstancesPerLaunch / kBlockThreads;
  int32_t vals[kPer];
  int32_t sum = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = tid * kPer + q;
    int32_t t = 0;
    if (i < k) {
      const uint32_t e = (uint32_t)(__ldcg(tails_cur + i) >> 32);
      t = (int32_t)((e + kTile - 1) / kTile);
    }
    vals[q] = t;
    sum += t;
  }
  unsigned long long total = 0;
  int32_t base = (int32_t)block_excl_scan((unsigned long long)sum, total, sh);
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = tid * kPer + q;
    if (i < k) sh.tprefix[i] = base;
    base += vals[q];
  }
  if (tid == 0) sh.tprefix[k] = (int32_t)total;
  __syncthreads();
  return sh.tprefix[k];
}

// Largest i with tprefix[i] <= g (skips instances with no tiles).
__device__ __forceinline__ int32_t find_instance(const int32_t *tprefix, int32_t k, int32_t g) {
  int32_t lo = 0, hi = k;
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (tprefix[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Inclusive max-scan over a tile's own[] marks: afterwards own[s] is the
// entry owning virtual edge x0 + s.  `first` (kMark | j) stands for the
// entry that owns the tile's first edge when no entry starts there.
__device__ __forceinline__ void owner_scan(WarpTile &wt, int32_t first) {
  const int lane = threadIdx.x & 31;
  int32_t vals[kEdgesPerLane];
  int32_t run = first;
#pragma unroll
  for (int q2 = 0; q2 < kEdgesPerLane; ++q2) {
    run = max(run, wt.own[lane * kEdgesPerLane + q2]);
    vals[q2] = run;
  }
  int32_t incl = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t o = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl = max(incl, o);
  }
  int32_t excl = __shfl_up_sync(kFull, incl, 1);
  if (lane == 0) excl = first;
  __syncwarp();
#pragma unroll
  for (int q2 = 0; q2 < kEdgesPerLane; ++q2) wt.own[lane * kEdgesPerLane + q2] = max(vals[q2], excl) & (kMark - 1);
}

// Width in words of the bitmap chunks a warp takes in the build and in a
// direct step: 32 words (1024 vertices), or narrower when the bitmaps of all
// instances hold fewer chunks than half the warps (a small graph, one
// block), so that more warps share the work.
__device__ __forceinline__ int64_t chunk_words(const GovmParams &p, int64_t nwarps) {
  if ((p.words * p.k + 31) / 32 * 2 < nwarps)
    return max((int64_t)1, min((int64_t)32, (p.words * p.k + nwarps - 1) / nwarps));
  return 32;
}

// Build delta (queue + tile table + tails_next) from beta (the bitmap) for
// every instance; consumes (clears) the bitmap.  Work is split into chunks
// of up to 32 words (1024 vertices) handed to warps round-robin; a warp ranks the marked
// vertices of its chunk with a popcount scan and expands them in rounds of
// 128 (four consecutive ranks per lane), so all row_ptr reads of a round are
// in flight together and no block-wide synchronisation is needed.  One
// atomicAdd per round reserves the entries and their edge offsets.  The tile
// starts of a row spanning more than two tiles are written by the whole warp
// (one such row per lane and round; hub rows hold thousands of tiles).
constexpr int kBuildPerLane = 4;

__device__ void build_frontier(const GovmParams &p, unsigned long long *tails_next, WarpTile &wt,
                               unsigned long long &marked) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t cwd = chunk_words(p, nwarps);
  const int64_t cpi = (p.words + cwd - 1) / cwd;  // chunks per instance
  const int64_t chunks = cpi * p.k;
  uint32_t *wbits = wt.ebase;  // the relax tile buffers are free during the build
  uint32_t *wstart = wt.dkey;
  for (int64_t ch = gwarp; ch < chunks; ch += nwarps) {
    const int32_t inst = (int32_t)(ch / cpi);
    const int64_t w0 = (ch - (int64_t)inst * cpi) * cwd;
    uint32_t *bm = p.bitmap + (size_t)inst * p.words;
    uint32_t bits = 0;
    if (lane < cwd && w0 + lane < p.words) {
      bits = __ldcg(bm + w0 + lane);
      if (bits && !p.gsvm) bm[w0 + lane] = 0u;  // Algorithm 1 keeps every reached vertex
    }
    const uint32_t pc = __popc(bits);
    marked += pc;
    uint32_t incl = pc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += o;
    }
    const uint32_t T = __shfl_sync(kFull, incl, 31);
    if (T == 0) continue;  // warp-uniform
    __syncwarp();
    wbits[lane] = bits;
    wstart[lane] = incl - pc;
    __syncwarp();
    uint4 *q = p.queue + (size_t)inst * p.n;
    int32_t *tl = p.tiles + (size_t)inst * p.tiles_cap;
    for (uint32_t r0 = 0; r0 < T; r0 += 32 * kBuildPerLane) {  // warp-uniform
      const uint32_t lo = r0 + lane * kBuildPerLane;
      const uint32_t hi = min(lo + kBuildPerLane, T);
      int32_t v[kBuildPerLane];
#pragma unroll
      for (int i = 0; i < kBuildPerLane; ++i) v[i] = -1;
      if (lo < hi) {
        int32_t a = 0, b = 32;  // word holding rank lo: largest w with wstart[w] <= lo
        while (b - a > 1) {
          const int32_t mid = (a + b) >> 1;
          if (wstart[mid] <= lo) a = mid; else b = mid;
        }
        int32_t w = a;
        uint32_t m = wbits[w];
        for (uint32_t skip = lo - wstart[w]; skip > 0; --skip) m &= m - 1;
#pragma unroll
        for (int i = 0; i < kBuildPerLane; ++i) {
          if (lo + i < hi) {
            while (m == 0 && w + 1 < 32) m = wbits[++w];
            if (m == 0) {  // cannot happen: every rank below T has a marked bit
              set_status(p.ctl, DAWN_ERR_BOUNDS);
              break;
            }
            v[i] = (int32_t)((w0 + w) * 32 + __ffs(m) - 1);
            m &= m - 1;
          }
        }
      }
      uint32_t rs[kBuildPerLane], d[kBuildPerLane];
#pragma unroll
      for (int i = 0; i < kBuildPerLane; ++i) {
        rs[i] = v[i] >= 0 ? (uint32_t)__ldg(p.row_ptr + v[i]) : 0u;
        d[i] = v[i] >= 0 ? (uint32_t)__ldg(p.row_ptr + v[i] + 1) : 0u;
      }
      uint32_t cnt = 0, degsum = 0;
#pragma unroll
      for (int i = 0; i < kBuildPerLane; ++i) {
        d[i] -= rs[i];
        cnt += d[i] > 0;
        degsum += d[i];
      }
      const unsigned long long mine = ((unsigned long long)degsum << 32) | cnt;
      unsigned long long pre = mine;
#pragma unroll
      for (int s2 = 1; s2 < 32; s2 <<= 1) {
        const unsigned long long o = __shfl_up_sync(kFull, pre, s2);
        if (lane >= s2) pre += o;
      }
      const unsigned long long total = __shfl_sync(kFull, pre, 31);
      if (total == 0) continue;  // warp-uniform
      unsigned long long base = 0;
      if (lane == 31) base = atomicAdd(tails_next + inst, total);
      base = __shfl_sync(kFull, base, 31);
      const unsigned long long pos = base + pre - mine;
      uint32_t idx = (uint32_t)pos;
      uint32_t off = (uint32_t)(pos >> 32);
      uint32_t lb0 = 0, lb1 = 0, lidx = 0;  // this lane's first long entry, written by the warp
#pragma unroll
      for (int i = 0; i < kBuildPerLane; ++i) {
        if (d[i] == 0) continue;
        if (idx >= (uint32_t)p.n) {  // cannot happen: each vertex has one bit
          set_status(p.ctl, DAWN_ERR_BOUNDS);
          break;
        }
        q[idx] = make_uint4(rs[i], off, rs[i] - off, (uint32_t)v[i]);
        const uint32_t tb0 = (off + kTile - 1) / kTile;
        uint32_t tb1 = (off + d[i] + kTile - 1) / kTile;
        if (tb1 > (uint32_t)p.tiles_cap) {
          set_status(p.ctl, DAWN_ERR_BOUNDS);
          tb1 = max(tb0, (uint32_t)p.tiles_cap);
        }
        if (tb1 - tb0 > 2 && lb1 == 0) {
          lb0 = tb0;
          lb1 = tb1;
          lidx = idx;
        } else {
          for (uint32_t tb = tb0; tb < tb1; ++tb) tl[tb] = (int32_t)idx;
        }
        ++idx;
        off += d[i];
      }
      unsigned bal = __ballot_sync(kFull, lb1 != 0);
      while (bal) {
        const int src = __ffs(bal) - 1;
        bal &= bal - 1;
        const uint32_t b0 = __shfl_sync(kFull, lb0, src);
        const uint32_t b1 = __shfl_sync(kFull, lb1, src);
        const int32_t ix = (int32_t)__shfl_sync(kFull, lidx, src);
        for (uint32_t tb = b0 + lane; tb < b1; tb += 32) tl[tb] = ix;
      }
    }
  }
}

// Edge phase of one kTile-edge tile of a laid-out edge list: lane handles
// virtual edges x0 + 32 r + lane (r < kEdgesPerLane) below xend.  wt.own[s]
// is the entry owning virtual edge x0 + s (unless jone >= 0: then entry jone
// owns them all), wt.ebase[j] the CSR index of entry j's virtual offset 0
// (mod 2^32) and wt.dkey[j] the distance key of entry j's vertex, which
// fill_keys() writes after the loads are issued (so that in-place key reads
// still in flight overlap the edge loads).  Every load of the phase is
// issued before any result is used, so a lane's requests are in flight
// together.  Returns the lanes' strict-improvement masks (bit r: round r
// lowered a distance).
template <int WT, typename FillKeys>
__device__ __forceinline__ unsigned relax_edges(const GovmParams &p, WarpTile &wt, unsigned long long *st,
                                                uint32_t *bm, uint32_t x0, uint32_t xend, int32_t jone,
                                                FillKeys fill_keys) {
  const int lane = threadIdx.x & 31;
  const unsigned long long kSourceState = ((unsigned long long)Key<WT>::zero << 32) | kNoEdge;  // no parent edge
  uint32_t eidx[kEdgesPerLane];
  unsigned valid = 0, jpack = 0;  // jpack: each round's owning entry (8 bits each), reused for the keys
  bool bad = false;
  uint2 cw[kEdgesPerLane];
  if (jone >= 0) {
    // One row owns the tile, so its edges are contiguous from e0: each lane
    // loads two 16-byte (column, weight) pairs from the even-aligned start
    // (half the load instructions of one pair per edge); when the start is
    // odd, lane 0's first slot (the edge before the row's part) takes the
    // tile's last edge instead.
    const uint32_t e0 = x0 + wt.ebase[jone];
    const uint32_t cnt = xend - x0;
    const uint32_t ea = e0 & ~1u;
    const uint32_t mm = (uint32_t)p.m;
    jpack = (uint32_t)jone * 0x01010101u;
    if (lane == 0 && (uint64_t)e0 + cnt > mm) bad = true;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t ep = ea + 2u * (uint32_t)(h * 32 + lane);
      const bool in0 = ep >= e0 && ep < e0 + cnt && ep < mm;
      const bool in1 = ep + 1 >= e0 && ep + 1 < e0 + cnt && ep + 1 < mm;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (in1) {
        v = __ldcs(reinterpret_cast<const uint4 *>(p.cw + ep));
      } else if (in0) {
        const uint2 t = __ldcs(p.cw + ep);
        v.x = t.x;
        v.y = t.y;
      }
      cw[2 * h] = make_uint2(v.x, v.y);
      cw[2 * h + 1] = make_uint2(v.z, v.w);
      eidx[2 * h] = ep;
      eidx[2 * h + 1] = ep + 1;
      valid |= (in0 ? 1u : 0u) << (2 * h);
      valid |= (in1 ? 1u : 0u) << (2 * h + 1);
    }
    if (lane == 0 && (e0 & 1u) && cnt == (uint32_t)kTile && ea + kTile < mm) {
      cw[0] = __ldcs(p.cw + ea + kTile);
      eidx[0] = ea + kTile;
      valid |= 1u;
    }
  } else {  // rows laid end to end: lane takes edges x0 + 32 r + lane, each owned by wt.own[]
#pragma unroll
    for (int r = 0; r < kEdgesPerLane; ++r) {
      const uint32_t x = x0 + r * 32 + lane;
      eidx[r] = 0;
      if (x < xend) {
        const int32_t j = wt.own[r * 32 + lane];
        jpack |= (uint32_t)j << (8 * r);
        const uint32_t e = x + wt.ebase[j];
        if (e < (uint32_t)p.m) {
          valid |= 1u << r;
          eidx[r] = e;
        } else {
          bad = true;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kEdgesPerLane; ++r)
      cw[r] = (valid & (1u << r)) ? __ldcs(p.cw + eidx[r]) : make_uint2(0u, 0u);
  }
  if (bad) set_status(p.ctl, DAWN_ERR_BOUNDS);
  unsigned long long curst[kEdgesPerLane];
#pragma unroll
  for (int r = 0; r < kEdgesPerLane; ++r)
    curst[r] = (valid & (1u << r)) ? ld_relaxed_u64(st + cw[r].x) : 0ull;
  fill_keys();
  __syncwarp();
  // Relax.  A candidate that beats the distance read marks beta (the thread
  // whose atomicMin strictly lowers a distance always read a larger value, so
  // every strict improvement is marked); equal-distance candidates with a
  // lower edge index only update the parent.  The low half of a candidate is
  // its edge when the call wants parent_edge, else the edge's tail: CSR edge
  // indices grow with the tail, so for equal keys both select the same parent
  // vertex (distances and marks do not depend on the low half), and the
  // output unpack then reads the parent without a gather of the edge's tail.
  uint32_t ckey[kEdgesPerLane];
  unsigned need = 0;
#pragma unroll
  for (int r = 0; r < kEdgesPerLane; ++r) {
    const uint32_t j = (jpack >> (8 * r)) & 0xFFu;
    ckey[r] = Key<WT>::add(wt.dkey[j], cw[r].y);
    if (p.parent_edge == nullptr) eidx[r] = wt.vert[j];
    const unsigned long long cand = ((unsigned long long)ckey[r] << 32) | eidx[r];
    if ((valid & (1u << r)) && cand < curst[r] && curst[r] != kSourceState) need |= 1u << r;
  }
  // Both atomics are fire-and-forget reductions: nothing waits for them.
  unsigned strict = 0;
#pragma unroll
  for (int r = 0; r < kEdgesPerLane; ++r) {
    if (need & (1u << r)) {
      const uint32_t t = cw[r].x;
      if (ckey[r] < (uint32_t)(curst[r] >> 32)) {
        atomicOr(bm + (t >> 5), 1u << (t & 31));
        strict |= 1u << r;
      }
      atomicMin(st + t, ((unsigned long long)ckey[r] << 32) | eidx[r]);
    }
  }
  return strict;
}

// Relax the out-edges in virtual-edge tile t of instance inst's frontier.
template <int WT>
__device__ __forceinline__ void relax_tile(const GovmParams &p, WarpTile &wt, int32_t inst, int32_t t,
                                           unsigned long long tail_cur, int32_t tiles_i, unsigned *changed) {
  const int lane = threadIdx.x & 31;
  const uint32_t E = (uint32_t)(tail_cur >> 32);
  const int32_t c = (int32_t)(uint32_t)tail_cur;
  const uint32_t x0 = (uint32_t)t * kTile;
  const uint32_t xend = min(x0 + (uint32_t)kTile, E);
  const int32_t *tiles = p.tiles + (size_t)inst * p.tiles_cap;
  const uint4 *q = p.queue + (size_t)inst * p.n;
  uint32_t *bm = p.bitmap + (size_t)inst * p.words;
  unsigned long long *st = p.state + (size_t)inst * p.n;

  __syncwarp();  // the previous tile of this warp has finished with wt
  const int32_t ia = __ldcg(tiles + t);
  const int32_t ib = (t + 1 < tiles_i) ? __ldcg(tiles + t + 1) : c - 1;
  const int32_t nent = ib - ia + 1;
  // a tile overlaps at most kTile + 1 entries (every entry has an out-edge)
  if (ia < 0 || ib >= c || nent < 1 || nent > kTile + 1) {
    if (lane == 0) set_status(p.ctl, DAWN_ERR_BOUNDS);
    return;
  }
  // A tile inside one long row needs no owner search (hub rows of skewed
  // degree distributions are mostly such tiles).
  const bool one = nent == 1;
  // Entries lane and lane + 32 are loaded together.  Each entry's distance
  // key alpha[v] is read in place, as Algorithm 2 does (improvements made
  // earlier in this step are used at once); those reads are consumed only
  // after the edge loads below have been issued.  An entry's start marks
  // own[] with kMark | j: every value left there by an earlier tile is below
  // kMark, so the marks need no clearing.
  const int32_t j0 = lane, j1 = lane + 32;
  uint4 e0 = make_uint4(0u, 0u, 0u, 0u), e1 = e0;
  if (j0 < nent) e0 = __ldcg(q + ia + j0);
  if (j1 < nent) e1 = __ldcg(q + ia + j1);
  unsigned long long f0 = ~0ull, f1 = ~0ull;
  if (j0 < nent) {
    wt.ebase[j0] = e0.z;
    wt.vert[j0] = e0.w;
    if (j0 > 0 && e0.y >= x0 && e0.y < x0 + (uint32_t)kTile) wt.own[e0.y - x0] = kMark | j0;
    f0 = ld_relaxed_u64(st + e0.w);
  }
  if (j1 < nent) {
    wt.ebase[j1] = e1.z;
    wt.vert[j1] = e1.w;
    if (e1.y >= x0 && e1.y < x0 + (uint32_t)kTile) wt.own[e1.y - x0] = kMark | j1;
    f1 = ld_relaxed_u64(st + e1.w);
  }
  for (int32_t j = lane + 64; j < nent; j += 32) {  // tiles of many short rows
    const uint4 en = __ldcg(q + ia + j);
    wt.ebase[j] = en.z;
    wt.vert[j] = en.w;
    wt.dkey[j] = (uint32_t)(ld_relaxed_u64(st + en.w) >> 32);
    if (en.y >= x0 && en.y < x0 + (uint32_t)kTile) wt.own[en.y - x0] = kMark | j;
  }
  __syncwarp();
  // Inclusive max-scan of entry starts: own[s] = entry owning edge x0 + s.
  if (!one) owner_scan(wt, kMark);
  __syncwarp();
  const unsigned strict = relax_edges<WT>(p, wt, st, bm, x0, xend, one ? 0 : -1, [&] {
    if (j0 < nent) wt.dkey[j0] = (uint32_t)(f0 >> 32);
    if (j1 < nent) wt.dkey[j1] = (uint32_t)(f1 >> 32);
  });
  // Algorithm 1's "ptr": some path changed in this step
  if (changed && __any_sync(kFull, strict != 0) && lane == 0) atomicOr(changed, 1u);
}

// One direct GOVM step, for single-instance solves on graphs whose rows are
// all short (the host picks this form): the frontier delta is read straight
// from `bm`, the bitmap of the previous step's marks, so no queue or tile
// table is built and the step ends with a single device-wide barrier.  Warp
// g owns bitmap words g, g + W, g + 2W, ... (W = warps in the grid), 32 at a
// time, one per lane: spreading each warp's words over the whole bitmap
// keeps warps evenly loaded even where the frontier is spatially dense (a
// grid's wavefront).  Each warp clears its words; the marked vertices of all
// the block's words are ranked together (a block barrier), and every warp of
// the block expands up to 32 of them at a time (a round's ranks split evenly
// over the warps), one per lane, so a warp whose words hold many marks does
// not expand them alone: each lane reads its vertex's
// row bounds and, in place, its distance key; the 32 rows' out-edges are laid
// end to end and relaxed in kTile-edge tiles with the same edge phase as
// relax_tile.  Must be reached by every thread of the block.  Marks go to
// `bn`.  With p.skip_remarked, a vertex whose bit
// in `bn` is already set (its distance dropped again earlier in this step)
// is not expanded now: it is in the next frontier and is expanded there with
// a key no larger.  Counters: `marked` (the vertices consumed), `front`
// (those with an out-edge), `edges` (their out-edges) and `skipped` (the
// out-edges of the vertices not expanded).  `first_bits` is the lane's word
// of the first round, which the caller loads before its stop test.  Returns
// whether this warp made any strict improvement (a mark in bn).
template <int WT>
__device__ bool direct_step(const GovmParams &p, uint32_t *bm, uint32_t *bn, uint32_t first_bits, BlockShared &sh,
                            unsigned long long &marked, unsigned long long &front, unsigned long long &edges,
                            unsigned long long &skipped) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpTile &wt = sh.wt[warp];
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t bwarp0 = (int64_t)blockIdx.x * kWarpsPerBlock;  // the block's first warp in the grid
  // wt.ebase / wt.dkey hold the round's 32 entries in [0, 32); the warp's
  // words' bits and rank starts live above them, where the block's other
  // warps read them too
  uint32_t *wbits = wt.ebase + 64;
  uint32_t *wstart = wt.dkey + 64;
  unsigned long long *st = p.state;
  unsigned strict_any = 0;
  for (int64_t r = 0; bwarp0 + r < p.words; r += 32 * nwarps) {  // block-uniform
    const int64_t base = bwarp0 + warp + r;             // this warp's first word of the round
    const int64_t w = base + (int64_t)lane * nwarps;  // this lane's word
    uint32_t bits = 0;
    if (w < p.words) {
      bits = r == 0 ? first_bits : __ldcg(bm + w);  // the first round's word was loaded by the caller
      if (bits) bm[w] = 0u;  // consumed: this bitmap receives the marks of the next step
    }
    const uint32_t pc = __popc(bits);
    marked += pc;
    uint32_t incl = pc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += o;
    }
    wbits[lane] = bits;
    wstart[lane] = incl - pc;
    if (lane == 31) sh.pool[warp] = incl;
    __syncthreads();
    // The block's marked vertices are ranked across its warps (warp s's
    // words first, then warp s + 1's), and every warp expands 32 of them per
    // round: a warp whose words hold many marks no longer expands them alone.
    uint32_t cnt = lane < kWarpsPerBlock ? sh.pool[lane] : 0u;
    uint32_t sincl = cnt;
#pragma unroll
    for (int d = 1; d < kWarpsPerBlock; d <<= 1) {
      const uint32_t o = __shfl_up_sync(kFull, sincl, d);
      if (lane >= d) sincl += o;
    }
    const uint32_t sstart = sincl - cnt;  // lanes below kWarpsPerBlock: warp `lane`'s first rank
    const uint32_t T = __shfl_sync(kFull, sincl, kWarpsPerBlock - 1);
    for (uint32_t r0 = 0; r0 < T; r0 += kBlockThreads) {  // block-uniform
      // the round's ranks split evenly over the warps, consecutive ranks per
      // warp (a round of fewer than 256 ranks still keeps every warp busy)
      const uint32_t per = (min(T - r0, (uint32_t)kBlockThreads) + kWarpsPerBlock - 1) / kWarpsPerBlock;
      const uint32_t rank = r0 + (uint32_t)warp * per + lane;
      int32_t owner = 0;  // warp whose words hold this rank: the largest with a start at or below it
#pragma unroll
      for (int q = 1; q < kWarpsPerBlock; ++q)
        if (__shfl_sync(kFull, sstart, q) <= rank) owner = q;
      const uint32_t orank = rank - __shfl_sync(kFull, sstart, owner);
      int32_t v = -1;
      if (lane < (int)per && rank < T) {
        const uint32_t *obits = sh.wt[owner].ebase + 64;
        const uint32_t *ostart = sh.wt[owner].dkey + 64;
        int32_t a = 0, b = 32;  // lane whose word holds this rank: largest a with ostart[a] <= orank
        while (b - a > 1) {
          const int32_t mid = (a + b) >> 1;
          if (ostart[mid] <= orank) a = mid; else b = mid;
        }
        uint32_t m = obits[a];
        for (uint32_t skip = orank - ostart[a]; skip > 0; --skip) m &= m - 1;
        if (m == 0) {  // cannot happen: every rank below T has a marked bit
          set_status(p.ctl, DAWN_ERR_BOUNDS);
        } else {
          v = (int32_t)((bwarp0 + owner + r + (int64_t)a * nwarps) * 32 + __ffs(m) - 1);
        }
      }
      uint32_t rs = 0, deg = 0;
      unsigned long long f = ~0ull;
      bool again = false;
      if (v >= 0 && v < p.n) {
        rs = (uint32_t)__ldg(p.row_ptr + v);
        deg = (uint32_t)__ldg(p.row_ptr + v + 1) - rs;
        f = ld_relaxed_u64(st + v);  // alpha[v] in place, as Algorithm 2 reads it
        // a vertex marked again in this step is in the next frontier and is
        // expanded there with a key no larger: not now
        if (p.skip_remarked) again = (__ldcg(bn + (v >> 5)) >> (v & 31)) & 1u;
      }
      front += deg > 0;
      edges += deg;
      if (again) {
        skipped += deg;
        deg = 0;
      }
      uint32_t off = deg;  // exclusive prefix of the degrees: lane's first virtual edge
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(kFull, off, d);
        if (lane >= d) off += o;
      }
      const uint32_t D = __shfl_sync(kFull, off, 31);
      off -= deg;
      if (D == 0) continue;  // warp-uniform
      __syncwarp();
      wt.ebase[lane] = rs - off;
      wt.dkey[lane] = (uint32_t)(f >> 32);
      wt.vert[lane] = (uint32_t)v;
      __syncwarp();
      for (uint32_t x0 = 0; x0 < D; x0 += kTile) {  // warp-uniform
        const uint32_t xend = min(x0 + (uint32_t)kTile, D);
        // entry owning edge x0: the last lane with an out-edge starting at or
        // before it; entries starting inside the tile mark own[]
        const unsigned before = __ballot_sync(kFull, deg > 0 && off <= x0);
        const bool starts = deg > 0 && off > x0 && off < xend;
        const bool one = __ballot_sync(kFull, starts) == 0;
        if (!one) {
          __syncwarp();  // the previous tile's readers of own[] are done
          if (starts) wt.own[off - x0] = kMark | lane;
          __syncwarp();
          owner_scan(wt, kMark | (31 - __clz(before)));
          __syncwarp();
        }
        const unsigned strict =
            relax_edges<WT>(p, wt, st, bn, x0, xend, one ? 31 - __clz(before) : -1, [] {});
        strict_any |= __any_sync(kFull, strict != 0);
      }
    }
    __syncthreads();  // every warp is done with the round's words before the next round rewrites them
  }
  return strict_any != 0;
}

// MINB = CTAs per SM the build targets: 5 caps a thread at 48 registers
// (40 resident warps per SM, the most latency hiding), 4 at 64 (more loads in
// flight per warp).  Both spill a few dozen bytes, mostly in the frontier
// build (ptxas -v).  Which is faster depends on the graph; dawn_autotune picks.
// DIRECT selects the step form (p.direct): direct steps (the frontier read
// from the bitmap, one barrier per step) or queue steps (relax tiles, then
// build).  Each form is its own instantiation, so neither pays the other's
// registers.  A call without a parent_edge output packs each state's parent
// as the edge's tail instead of the edge (relax_edges), so the output unpack
// needs no gather of the tail; that choice is a run-time flag, not a further
// instantiation, because the instantiated form measured slower.
template <int WT, int MINB, bool DIRECT>
__global__ void __launch_bounds__(kBlockThreads, MINB) govm_kernel(GovmParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockShared &sh = *reinterpret_cast<BlockShared *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
  const long long gsize = (long long)gridDim.x * blockDim.x;
  DeviceCtl *ctl = p.ctl;
  const unsigned long long kInfState = ((unsigned long long)Key<WT>::inf << 32) | kNoEdge;
  const unsigned long long kSourceState = ((unsigned long long)Key<WT>::zero << 32) | kNoEdge;
  unsigned long long updates = 0;  // vertices entering beta, summed over steps
  unsigned long long skipped = 0;  // direct steps: frontier out-edges not relaxed (their vertex was marked again)
  unsigned long long seeded = 0;   // the seeds' own marks (not path updates)
  if (tid == 0) {
    sh.bar_target = 0;
    sh.any_mark = 0;
    sh.trace_sum[0] = sh.trace_sum[1] = 0;
  }
  for (int s = lane; s < kTile; s += 32) sh.wt[warp].own[s] = 0;
  __syncwarp();
  long long step = 0;
  bool quiescent = false;

  // Test hook: one thread waits on a flag that nothing sets; the bounded
  // wait runs out and every block leaves through the barrier's error path.
  if (p.test_stall && blockIdx.x == 0 && tid == 0) {
    const unsigned long long t0 = global_ns();
    while (ld_volatile_i32(&ctl->stall_flag) == 0) {
      if (global_ns() - t0 > p.wait_limit_ns) {
        set_status(ctl, DAWN_ERR_TIMEOUT);
        break;
      }
      __nanosleep(1000);
    }
  }

  // Weights refused by validation (possibly deferred, see dawn_set_weights)
  // stop the solve before its first barrier, with no output written.
  if (p.vflags && blockIdx.x == 0 && tid == 0) {
    const unsigned bad = __ldcg(p.vflags), wmax = __ldcg(p.vflags + 1);
    if (bad || (p.vlimit && (unsigned long long)p.n * wmax >= p.vlimit)) set_status(ctl, DAWN_ERR_INVALID);
  }

  // 1. alpha = +inf, beta = {} (direct steps keep two bitmaps: this step's
  // frontier and the next one's marks).
  for (long long i = gtid; i < (long long)p.k * p.n; i += gsize) p.state[i] = kInfState;
  for (long long i = gtid; i < (DIRECT ? 2LL : 1LL) * p.k * p.words; i += gsize) p.bitmap[i] = 0u;
  for (long long i = gtid; i < 2LL * p.k; i += gsize) p.tails[i] = 0ull;
  if (!grid_barrier(ctl, p.wait_limit_ns, &sh.flag, &sh.bar_target)) goto finish;

  // 2. Seeds: alpha[s] = 0, s enters beta.
  for (long long i = gtid; i < (p.roots_mode ? (long long)p.nseeds : (long long)p.k); i += gsize) {
    const int32_t s = p.seeds ? p.seeds[i] : p.source;
    if (s < 0 || s >= p.n) {
      set_status(ctl, DAWN_ERR_INVALID);
      continue;
    }
    const int32_t inst = p.roots_mode ? 0 : (int32_t)i;
    p.state[(size_t)inst * p.n + s] = kSourceState;
    atomicOr(p.bitmap + (size_t)inst * p.words + (s >> 5), 1u << (s & 31));
  }
  if (!grid_barrier(ctl, p.wait_limit_ns, &sh.flag, &sh.bar_target)) goto finish;

  // 3. GOVM steps.
  if (DIRECT) {  // one barrier per step; the frontier stays a bitmap
    unsigned long long front = 0, edges = 0;
    for (;; ++step) {
      // this lane's first frontier word, loaded before the stop test so that
      // the two round trips overlap
      uint32_t *bm_cur = p.bitmap + (size_t)(step & 1) * p.words;
      const long long w0 = (gtid >> 5) + (long long)lane * (gsize >> 5);
      const uint32_t first_bits = w0 < p.words ? __ldcg(bm_cur + w0) : 0u;
      // stop after a step that lowered no distance (its marks would be the
      // next frontier)
      if (step > 0 && ld_volatile_i32((const int *)&ctl->marks[(step - 1) % 3]) == 0) {
        quiescent = true;
        break;
      }
      if (step >= p.max_steps) {
        if (gtid == 0) set_status(ctl, DAWN_ERR_NOT_CONVERGED);
        quiescent = true;
        break;
      }
      if (blockIdx.x == 0 && tid == 0) {
        if (p.trace && step < p.trace_cap) {
          unsigned long long *tr = p.trace + 4 * step;
          tr[0] = global_ns();
          tr[1] = __ldcg(&ctl->frontier_sum);  // cumulative before this step
          tr[2] = __ldcg(&ctl->edges_scanned);
          tr[3] = 0;
        }
        ctl->marks[(step + 1) % 3] = 0u;  // set in step + 1, read two steps from now
      }
      const unsigned long long f0 = front, e0 = edges;
      const bool any = direct_step<WT>(p, bm_cur, p.bitmap + (size_t)((step + 1) & 1) * p.words, first_bits, sh,
                                       step == 0 ? seeded : updates, front, edges, skipped);
      if (any && lane == 0) sh.any_mark = 1;
      if (p.trace) {  // traced solves keep the cumulative counters current per step
        unsigned long long df = front - f0, de = edges - e0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          df += __shfl_down_sync(kFull, df, d);
          de += __shfl_down_sync(kFull, de, d);
        }
        if (lane == 0 && df) atomicAdd(&sh.trace_sum[0], df);
        if (lane == 0 && de) atomicAdd(&sh.trace_sum[1], de);
      }
      __syncthreads();
      if (tid == 0 && sh.any_mark) {  // one flag write per block; the barrier's release publishes it
        atomicOr(&ctl->marks[step % 3], 1u);
        sh.any_mark = 0;
      }
      if (tid == 0 && p.trace) {  // one counter update per block
        if (sh.trace_sum[0]) atomicAdd(&ctl->frontier_sum, sh.trace_sum[0]);
        if (sh.trace_sum[1]) atomicAdd(&ctl->edges_scanned, sh.trace_sum[1]);
        sh.trace_sum[0] = sh.trace_sum[1] = 0;
      }
      if (!grid_barrier(ctl, p.wait_limit_ns, &sh.flag, &sh.bar_target)) break;
    }
    if (!p.trace) {
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        front += __shfl_down_sync(kFull, front, d);
        edges += __shfl_down_sync(kFull, edges, d);
      }
      if (lane == 0 && front) atomicAdd(&ctl->frontier_sum, front);
      if (lane == 0 && edges) atomicAdd(&ctl->edges_scanned, edges);
    }
  } else {
  build_frontier(p, p.tails, sh.wt[warp], seeded);
  if (!grid_barrier(ctl, p.wait_limit_ns, &sh.flag, &sh.bar_target)) goto finish;
  for (;; ++step) {
    unsigned long long *tails_cur = p.tails + (size_t)(step & 1) * p.k;
    unsigned long long *tails_next = p.tails + (size_t)((step + 1) & 1) * p.k;
    const int32_t total_tiles = scan_tiles(tails_cur, p.k, sh);
    if (total_tiles == 0) {
      quiescent = true;
      break;
    }
    // Algorithm 1 stops after a step in which no path changed (its frontier,
    // every reached vertex, never empties)
    if (p.gsvm && step > 0 && ld_volatile_i32((const int *)&ctl->changed[(step - 1) % 3]) == 0) {
      quiescent = true;
      break;
    }
    if (step >= p.max_steps) {
      if (gtid == 0) set_status(ctl, DAWN_ERR_NOT_CONVERGED);
      quiescent = true;
      break;
    }
    if (blockIdx.x == 0) {
      if (tid == 0 && p.trace && step < p.trace_cap) {
        unsigned long long *tr = p.trace + 4 * step;
        tr[0] = global_ns();
        tr[1] = __ldcg(&ctl->frontier_sum);  // cumulative before this step
        tr[2] = __ldcg(&ctl->edges_scanned);
        tr[3] = 0;
      }
      __syncthreads();
      unsigned long long fs = 0, es = 0;
      for (int32_t i = tid; i < p.k; i += blockDim.x) {
        const unsigned long long tl = __ldcg(tails_cur + i);
        fs += (uint32_t)tl;
        es += tl >> 32;
        tails_next[i] = 0ull;  // last read in the previous step; filled by this step's build
      }
      if (fs) atomicAdd(&ctl->frontier_sum, fs);
      if (es) atomicAdd(&ctl->edges_scanned, es);
      if (tid == 0) ctl->changed[(step + 1) % 3] = 0u;  // read two steps from now
    }
    // relax
    const int32_t gw = blockIdx.x * kWarpsPerBlock + warp;
    const int32_t nw = gridDim.x * kWarpsPerBlock;
    for (int32_t g = gw; g < total_tiles; g += nw) {
      const int32_t inst = find_instance(sh.tprefix, p.k, g);
      relax_tile<WT>(p, sh.wt[warp], inst, g - sh.tprefix[inst], __ldcg(tails_cur + inst),
                      sh.tprefix[inst + 1] - sh.tprefix[inst], p.gsvm ? &ctl->changed[step % 3] : nullptr);
    }
    if (!grid_barrier(ctl, p.wait_limit_ns, &sh.flag, &sh.bar_target)) break;
    // build the next frontier
    build_frontier(p, tails_next, sh.wt[warp], updates);
    if (!grid_barrier(ctl, p.wait_limit_ns, &sh.flag, &sh.bar_target)) break;
  }
  }

  if (quiescent && blockIdx.x == 0 && tid == 0 && p.trace && step < p.trace_cap) {
    unsigned long long *tr = p.trace + 4 * step;
    tr[0] = global_ns();
    tr[1] = __ldcg(&ctl->frontier_sum);
    tr[2] = __ldcg(&ctl->edges_scanned);
    tr[3] = 1;  // final row
  }

  // 4. Outputs (only from a quiescent state: every block left the loop at the
  // same step, after a completed barrier).
  // State and outputs share the [k][n] layout, so one flat index covers all
  // instances; each thread handles four elements per round with all their
  // loads (the parent's tail gather included) in flight together.
  if (quiescent) {
    constexpr int kU = 4;
    const long long total = (long long)p.k * p.n;
    uint32_t *dist = (uint32_t *)p.dist;
    for (long long base = gtid; base < total; base += kU * gsize) {
      unsigned long long s[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long idx = base + u * gsize;
        s[u] = idx < total ? __ldcg(p.state + idx) : 0ull;
      }
      int32_t pv[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long idx = base + u * gsize;
        const uint32_t key = (uint32_t)(s[u] >> 32), e = (uint32_t)s[u];
        pv[u] = -1;
        if (p.parent && idx < total && key != Key<WT>::inf)
          pv[u] = e == kNoEdge ? (int32_t)(idx % p.n) : p.parent_edge == nullptr ? (int32_t)e : __ldg(p.src + e);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long idx = base + u * gsize;
        if (idx >= total) break;
        const uint32_t key = (uint32_t)(s[u] >> 32), e = (uint32_t)s[u];
        dist[idx] = Key<WT>::out(key);
        if (p.parent) p.parent[idx] = pv[u];
        if (p.parent_edge) p.parent_edge[idx] = (key == Key<WT>::inf || e == kNoEdge) ? -1 : (int32_t)e;
      }
    }
  }

finish:
  // counters
  {
    unsigned long long u = updates;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) u += __shfl_down_sync(kFull, u, d);
    if (lane == 0 && u) atomicAdd(&ctl->updates, u);
    unsigned long long sk = skipped;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sk += __shfl_down_sync(kFull, sk, d);
    if (lane == 0 && sk) atomicAdd(&ctl->edges_skipped, sk);
    if (gtid == 0) atomicMax(&ctl->steps, (unsigned long long)step);  // batched calls: the longest launch
  }
}

// The block's shared memory is dynamic; the opt-in to sizes above 48 KB is
// set once per kernel and device, so that kTile may grow without a change here.
using GovmFn = void (*)(GovmParams);

template <int MINB, bool DIRECT>
GovmFn kernel_for_wtype(int wtype) {
  if (wtype == DAWN_W_F32) return govm_kernel<DAWN_W_F32, MINB, DIRECT>;
  if (wtype == DAWN_W_I32) return govm_kernel<DAWN_W_I32, MINB, DIRECT>;
  return govm_kernel<DAWN_W_U32, MINB, DIRECT>;
}

GovmFn kernel_for(int wtype, int ctas_per_sm, bool direct) {
  if (direct) return ctas_per_sm == 4 ? kernel_for_wtype<4, true>(wtype) : kernel_for_wtype<5, true>(wtype);
  return ctas_per_sm == 4 ? kernel_for_wtype<4, false>(wtype) : kernel_for_wtype<5, false>(wtype);
}

cudaError_t prepare_kernels() {
  // function attributes are per device: remember which devices are done
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return cudaSuccess;
  for (int wtype : {DAWN_W_U32, DAWN_W_F32, DAWN_W_I32})
    for (int c : {4, 5})
      for (bool direct : {false, true})
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(kernel_for(wtype, c, direct), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(BlockShared));
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

}  // namespace

cudaError_t launch_govm(const GovmParams &p, int wtype, int ctas_per_sm, int grid_blocks, cudaStream_t stream) {
  cudaError_t e = prepare_kernels();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid_blocks);
  cfg.blockDim = dim3(kBlockThreads);
  cfg.dynamicSmemBytes = sizeof(BlockShared);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel_for(wtype, ctas_per_sm, p.direct != 0), p);
}

int govm_max_blocks_per_sm(int wtype, int ctas_per_sm) {
  int nb = 0;
  if (prepare_kernels() != cudaSuccess) return 0;
  // both step forms share the launch bounds, so the queue form stands for both
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_for(wtype, ctas_per_sm, false),
                                                                      kBlockThreads, sizeof(BlockShared));
  return e == cudaSuccess ? nb : 0;
}

}  // namespace dawn
