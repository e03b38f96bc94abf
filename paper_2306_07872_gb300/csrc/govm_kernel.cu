// Persistent GOVM kernel (weighted DAWN, arxiv 2306.07872, Section 3.4,
// Algorithm 2) for sm_103a.
//
// One cooperative launch runs a whole solve:
//   1. fill alpha with +inf (packed state), clear both frontier bitmaps;
//   2. seed the frontier (the source of every instance, or all roots);
//   3. GOVM steps until the frontier is empty:
//        every warp takes 256-edge tiles of the frontier's virtual edge list
//        (the concatenated out-edges of all frontier vertices, balanced by
//        edges rather than vertices), relaxes each edge with a 64-bit packed
//        atomicMin (distance and parent edge together), marks strictly
//        improved vertices in the next bitmap (beta) and appends first-time
//        marks to the next queue with one warp-aggregated atomicAdd that
//        yields both the entry index and the entry's edge offset;
//        a device-wide barrier (bounded wait) ends the step;
//   4. unpack dist / parent / parent_edge.
// No host round trip happens between steps.
#include <cuda_runtime.h>

#include "dawn_common.cuh"

namespace dawn {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int *p) { return *(volatile const int *)p; }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Distance keys: uint32 distances are their own key; non-negative float32
// distances are keyed by their bit pattern (monotone for x >= 0).
template <bool F32>
struct Key;
template <>
struct Key<false> {
  static constexpr uint32_t inf = kInfKeyU32;
  static __device__ __forceinline__ uint32_t add(uint32_t d, uint32_t w) { return d + w; }
};
template <>
struct Key<true> {
  static constexpr uint32_t inf = kInfKeyF32;
  static __device__ __forceinline__ uint32_t add(uint32_t d, uint32_t w) {
    return __float_as_uint(__fadd_rn(__uint_as_float(d), __uint_as_float(w)));
  }
};

constexpr int kStage = 2 * kTile;  // staged entries per warp (flushed above kStage - kTile)

struct WarpTile {
  int32_t rs[kTile + 1];     // CSR row start of each entry of the tile
  uint32_t off[kTile + 1];   // virtual offset of each entry's first edge
  uint32_t dkey[kTile + 1];  // distance key of each entry's vertex (read at expansion time)
  int32_t own[kTile];        // owning entry (relative index) of every virtual edge
  int32_t bv[kStage];        // staged next-frontier vertices
  uint32_t bd[kStage];       // and their out-degrees
};

struct BlockShared {
  int32_t tprefix[kMaxInstancesPerLaunch + 1];
  int32_t warp_sums[kWarpsPerBlock];
  int32_t flag;
  WarpTile wt[kWarpsPerBlock];
};

// Device-wide barrier with a bounded wait.  Returns false (uniformly for the
// block) when the status word reports an error or the wait ran out.
__device__ bool grid_barrier(DeviceCtl *ctl, unsigned long long limit_ns, int32_t *s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned gen = ld_acquire_u32(&ctl->bar_gen);
    __threadfence();
    unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      st_release_u32(&ctl->bar_gen, gen + 1);
    } else {
      unsigned long long t0 = global_ns();
      unsigned ns = 16;
      while (ld_acquire_u32(&ctl->bar_gen) == gen) {
        if (ld_volatile_i32(&ctl->status) != 0) break;
        if (global_ns() - t0 > limit_ns) {
          atomicCAS(&ctl->status, 0, (int)DAWN_ERR_TIMEOUT);
          break;
        }
        __nanosleep(ns);
        if (ns < 128) ns <<= 1;
      }
    }
    __threadfence();
    *s_flag = ld_volatile_i32(&ctl->status) == 0;
  }
  __syncthreads();
  return *s_flag != 0;
}

__device__ __forceinline__ void set_status(DeviceCtl *ctl, int code) { atomicCAS(&ctl->status, 0, code); }

// Exclusive prefix over instances of the number of tiles of each current
// frontier (tiles = ceil(edges / kTile)).  Returns the total.
__device__ int32_t scan_tiles(const unsigned long long *tails_cur, int32_t k, BlockShared &sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kPer = kMaxInstancesPerLaunch / kBlockThreads;
  int32_t vals[kPer];
  int32_t sum = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    int i = tid * kPer + q;
    int32_t t = 0;
    if (i < k) {
      uint32_t e = (uint32_t)(__ldcg(tails_cur + i) >> 32);
      t = (int32_t)((e + kTile - 1) / kTile);
    }
    vals[q] = t;
    sum += t;
  }
  int32_t incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int32_t o = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) sh.warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int32_t x = lane < kWarpsPerBlock ? sh.warp_sums[lane] : 0;
    int32_t xi = x;
#pragma unroll
    for (int d = 1; d < kWarpsPerBlock; d <<= 1) {
      int32_t o = __shfl_up_sync(kFull, xi, d);
      if (lane >= d) xi += o;
    }
    if (lane < kWarpsPerBlock) sh.warp_sums[lane] = xi - x;  // exclusive
    if (lane == kWarpsPerBlock - 1) sh.tprefix[k] = xi;      // total (k <= kMaxInstancesPerLaunch)
  }
  __syncthreads();
  int32_t base = sh.warp_sums[warp] + incl - sum;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    int i = tid * kPer + q;
    if (i < k) sh.tprefix[i] = base;
    base += vals[q];
  }
  __syncthreads();
  return sh.tprefix[k];
}

// Largest i with tprefix[i] <= g.
__device__ __forceinline__ int32_t find_instance(const int32_t *tprefix, int32_t k, int32_t g) {
  int32_t lo = 0, hi = k;
  while (hi - lo > 1) {
    int32_t mid = (lo + hi) >> 1;
    if (tprefix[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Next-frontier entries found by a warp are staged in its shared-memory
// buffer (vertex, out-degree) and appended to the instance's queue in bulk:
// one atomicAdd on the packed tail (count | degree-sum << 32) per flush
// reserves a block of entries and the matching block of virtual edges, so the
// queue order equals the offset order.  Staging across tiles keeps the number
// of atomics on the (single, hot) tail word low.

// Stage the lanes' pending entries (bit r of mask: vertex tgt[r], out-degree
// dg[r]); `count` is the warp-uniform number of staged entries.
__device__ __forceinline__ void stage_entries(WarpTile &wt, int &count, unsigned mask,
                                              const int32_t (&tgt)[kEdgesPerLane],
                                              const uint32_t (&dg)[kEdgesPerLane]) {
  const int lane = threadIdx.x & 31;
  const int mine = __popc(mask);
  int incl = mine;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int o = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += o;
  }
  int pos = count + incl - mine;
#pragma unroll
  for (int r = 0; r < kEdgesPerLane; ++r) {
    if (mask & (1u << r)) {
      wt.bv[pos] = tgt[r];
      wt.bd[pos] = dg[r];
      ++pos;
    }
  }
  count += __shfl_sync(kFull, incl, 31);
  __syncwarp();
}

// Append the staged entries to instance inst's queue `nxt` and record, in the
// next frontier's tile table, which entry owns the first edge of each tile.
__device__ void flush_entries(const GovmParams &p, WarpTile &wt, int &count, int32_t inst, int nxt,
                              unsigned long long *tails_next) {
  const int lane = threadIdx.x & 31;
  if (count == 0) return;
  unsigned long long degsum = 0;
  for (int i = lane; i < count; i += 32) degsum += wt.bd[i];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) degsum += __shfl_xor_sync(kFull, degsum, d);
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(tails_next + inst, (degsum << 32) | (unsigned long long)count);
  base = __shfl_sync(kFull, base, 0);
  const uint32_t idx0 = (uint32_t)base;
  uint32_t run = (uint32_t)(base >> 32);
  int2 *q = (nxt ? p.queue1 : p.queue0) + (size_t)inst * p.n;
  int32_t *tl = (nxt ? p.tiles1 : p.tiles0) + (size_t)inst * p.tiles_cap;
  for (int b = 0; b < count; b += 32) {
    const int i = b + lane;
    const uint32_t d = i < count ? wt.bd[i] : 0u;
    uint32_t incl = d;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      uint32_t o = __shfl_up_sync(kFull, incl, s);
      if (lane >= s) incl += o;
    }
    if (i < count) {
      const uint32_t idx = idx0 + (uint32_t)i;
      const uint32_t off = run + incl - d;
      if (idx >= (uint32_t)p.n) {  // cannot happen: the bitmap admits a vertex once per step
        set_status(p.ctl, DAWN_ERR_BOUNDS);
      } else {
        q[idx] = make_int2(wt.bv[i], (int32_t)off);
        const uint32_t end = off + d;
        for (uint32_t tb = (off + kTile - 1) / kTile; tb * (uint32_t)kTile < end; ++tb) {
          if (tb >= (uint32_t)p.tiles_cap) {
            set_status(p.ctl, DAWN_ERR_BOUNDS);
            break;
          }
          tl[tb] = (int32_t)idx;
        }
      }
    }
    run += __shfl_sync(kFull, incl, 31);
  }
  count = 0;
  __syncwarp();
}

// Relax the out-edges in virtual-edge tile t of instance inst's frontier.
template <bool F32>
__device__ __forceinline__ void process_tile(const GovmParams &p, WarpTile &wt, int32_t inst, int32_t t,
                                             unsigned long long tail_cur, int32_t tiles_i, int cur,
                                             int &staged, unsigned long long &updates) {
  const int lane = threadIdx.x & 31;
  const uint32_t E = (uint32_t)(tail_cur >> 32);
  const int32_t c = (int32_t)(uint32_t)tail_cur;
  const uint32_t x0 = (uint32_t)t * kTile;
  const uint32_t xend = min(x0 + (uint32_t)kTile, E);
  const int32_t *tiles = (cur ? p.tiles1 : p.tiles0) + (size_t)inst * p.tiles_cap;
  const int2 *q = (cur ? p.queue1 : p.queue0) + (size_t)inst * p.n;
  uint32_t *bm_cur = (cur ? p.bitmap1 : p.bitmap0) + (size_t)inst * p.words;
  uint32_t *bm_next = (cur ? p.bitmap0 : p.bitmap1) + (size_t)inst * p.words;
  unsigned long long *st = p.state + (size_t)inst * p.n;
  const unsigned long long kSourceState = (unsigned long long)kNoEdge;  // key 0, no parent edge

  __syncwarp();  // the previous tile of this warp has finished with wt
  const int32_t ia = __ldcg(tiles + t);
  const int32_t ib = (t + 1 < tiles_i) ? __ldcg(tiles + t + 1) : c - 1;
  const int32_t nent = ib - ia + 1;
  // a tile overlaps at most kTile + 1 entries (every entry has an out-edge)
  if (ia < 0 || ib >= c || nent < 1 || nent > kTile + 1) {
    if (lane == 0) set_status(p.ctl, DAWN_ERR_BOUNDS);
    return;
  }

  // Load the entries overlapping the tile; clear the current-bitmap words of
  // entries that start here (every entry starts in exactly one tile, so the
  // whole current bitmap is zero when the step ends).
  for (int s = lane; s < kTile; s += 32) wt.own[s] = 0;
  __syncwarp();
  for (int32_t j = lane; j < nent; j += 32) {
    int2 en = __ldcg(q + ia + j);
    uint32_t off = (uint32_t)en.y;
    int32_t v = en.x;
    wt.rs[j] = __ldg(p.row_ptr + v);
    wt.off[j] = off;
    wt.dkey[j] = (uint32_t)(ld_relaxed_u64(st + v) >> 32);
    if (off >= x0 && off < x0 + (uint32_t)kTile) {
      bm_cur[v >> 5] = 0u;
      if (j > 0) wt.own[off - x0] = j;
    }
  }
  __syncwarp();
  // Inclusive max-scan of entry starts: own[s] = entry owning edge x0 + s.
  {
    int32_t vals[kEdgesPerLane];
    int32_t run = 0;
#pragma unroll
    for (int q2 = 0; q2 < kEdgesPerLane; ++q2) {
      run = max(run, wt.own[lane * kEdgesPerLane + q2]);
      vals[q2] = run;
    }
    int32_t incl = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int32_t o = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl = max(incl, o);
    }
    int32_t excl = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) excl = 0;
    __syncwarp();
#pragma unroll
    for (int q2 = 0; q2 < kEdgesPerLane; ++q2) wt.own[lane * kEdgesPerLane + q2] = max(vals[q2], excl);
  }
  __syncwarp();

  // Edge phase: lane handles edges x0 + 32 r + lane, r = 0..7 (coalesced rounds).
  int32_t tgt[kEdgesPerLane];
  uint32_t ckey[kEdgesPerLane];
  uint32_t eidx[kEdgesPerLane];
  unsigned valid = 0;
#pragma unroll
  for (int r = 0; r < kEdgesPerLane; ++r) {
    const int slot = r * 32 + lane;
    const uint32_t x = x0 + slot;
    tgt[r] = 0;
    ckey[r] = 0;
    eidx[r] = 0;
    if (x < xend) {
      const int32_t j = wt.own[slot];
      const uint32_t e = (uint32_t)wt.rs[j] + (x - wt.off[j]);
      if (e >= (uint32_t)p.m) {
        set_status(p.ctl, DAWN_ERR_BOUNDS);
        continue;
      }
      valid |= 1u << r;
      eidx[r] = e;
      const uint2 cw = __ldcs(p.cw + e);
      tgt[r] = (int32_t)cw.x;
      ckey[r] = Key<F32>::add(wt.dkey[j], cw.y);
    }
  }
  unsigned long long curst[kEdgesPerLane];
#pragma unroll
  for (int r = 0; r < kEdgesPerLane; ++r)
    curst[r] = (valid & (1u << r)) ? ld_relaxed_u64(st + tgt[r]) : 0ull;
  // Relax: packed atomicMin where the candidate beats the current state.
  unsigned need = 0;
  unsigned long long old[kEdgesPerLane];
  int32_t rp0[kEdgesPerLane], rp1[kEdgesPerLane];
#pragma unroll
  for (int r = 0; r < kEdgesPerLane; ++r) {
    const unsigned long long cand = ((unsigned long long)ckey[r] << 32) | eidx[r];
    old[r] = 0;
    rp0[r] = rp1[r] = 0;
    if ((valid & (1u << r)) && cand < curst[r] && curst[r] != kSourceState) {
      need |= 1u << r;
      rp0[r] = __ldg(p.row_ptr + tgt[r]);
      rp1[r] = __ldg(p.row_ptr + tgt[r] + 1);
      old[r] = atomicMin(st + tgt[r], cand);
    }
  }
  // Strict improvements enter beta (first setter appends to the next queue).
  unsigned mark = 0;
  uint32_t obits[kEdgesPerLane], dg[kEdgesPerLane];
#pragma unroll
  for (int r = 0; r < kEdgesPerLane; ++r) {
    obits[r] = 0;
    dg[r] = 0;
    if ((need & (1u << r)) && (uint32_t)(old[r] >> 32) > ckey[r]) {
      ++updates;
      dg[r] = (uint32_t)(rp1[r] - rp0[r]);
      if (dg[r] > 0) {
        mark |= 1u << r;
        obits[r] = atomicOr(bm_next + (tgt[r] >> 5), 1u << (tgt[r] & 31));
      }
    }
  }
  unsigned mask = 0;
#pragma unroll
  for (int r = 0; r < kEdgesPerLane; ++r)
    if ((mark & (1u << r)) && !(obits[r] & (1u << (tgt[r] & 31)))) mask |= 1u << r;
  stage_entries(wt, staged, mask, tgt, dg);
}

template <bool F32>
__global__ void __launch_bounds__(kBlockThreads) govm_kernel(GovmParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockShared &sh = *reinterpret_cast<BlockShared *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
  const long long gsize = (long long)gridDim.x * blockDim.x;
  DeviceCtl *ctl = p.ctl;
  const unsigned long long kInfState = ((unsigned long long)Key<F32>::inf << 32) | kNoEdge;
  const unsigned long long kSourceState = (unsigned long long)kNoEdge;
  unsigned long long updates = 0;
  long long step = 0;
  bool quiescent = false;

  // Test hook: one thread waits on a flag that nothing sets; the bounded
  // wait runs out and every block leaves through the barrier's error path.
  if (p.test_stall && blockIdx.x == 0 && tid == 0) {
    unsigned long long t0 = global_ns();
    while (ld_volatile_i32(&ctl->stall_flag) == 0) {
      if (global_ns() - t0 > p.wait_limit_ns) {
        set_status(ctl, DAWN_ERR_TIMEOUT);
        break;
      }
      __nanosleep(1000);
    }
  }

  // 1. alpha = +inf, empty frontiers.
  for (int32_t i = 0; i < p.k; ++i) {
    unsigned long long *st = p.state + (size_t)i * p.n;
    for (long long v = gtid; v < p.n; v += gsize) st[v] = kInfState;
  }
  for (long long i = gtid; i < (long long)p.k * p.words; i += gsize) {
    p.bitmap0[i] = 0u;
    p.bitmap1[i] = 0u;
  }
  for (long long i = gtid; i < 3LL * p.k; i += gsize) p.tails[i] = 0ull;
  if (!grid_barrier(ctl, p.wait_limit_ns, &sh.flag)) goto finish;

  // 2. Seeds: alpha[s] = 0, delta = {s}.
  if (!p.roots_mode) {
    for (long long i = gtid; i < p.k; i += gsize) {
      const int32_t s = p.seeds ? p.seeds[i] : p.source;
      if (s < 0 || s >= p.n) {
        set_status(ctl, DAWN_ERR_INVALID);
        continue;
      }
      p.state[(size_t)i * p.n + s] = kSourceState;
      const uint32_t deg = (uint32_t)(__ldg(p.row_ptr + s + 1) - __ldg(p.row_ptr + s));
      if (deg == 0) continue;
      p.queue0[(size_t)i * p.n] = make_int2(s, 0);
      p.bitmap0[(size_t)i * p.words + (s >> 5)] = 1u << (s & 31);
      int32_t *tl = p.tiles0 + (size_t)i * p.tiles_cap;
      for (uint32_t tb = 0; tb * (uint32_t)kTile < deg; ++tb) tl[tb] = 0;
      p.tails[i] = ((unsigned long long)deg << 32) | 1ull;
    }
  } else {
    for (long long i = gtid; i < p.nseeds; i += gsize) {
      const int32_t s = p.seeds[i];
      if (s < 0 || s >= p.n) set_status(ctl, DAWN_ERR_INVALID);
      else p.state[s] = kSourceState;
    }
    if (!grid_barrier(ctl, p.wait_limit_ns, &sh.flag)) goto finish;
    // warp-uniform loop: every lane of a warp takes part in the append
    const long long gw = gtid >> 5, nw = gsize >> 5;
    int staged = 0;
    for (long long b = gw * 32; b < p.nseeds; b += nw * 32) {
      const long long i = b + lane;
      int32_t tg[kEdgesPerLane] = {0};
      uint32_t dgs[kEdgesPerLane] = {0};
      unsigned mask = 0;
      if (i < p.nseeds) {
        const int32_t s = p.seeds[i];
        if (s >= 0 && s < p.n) {
          const uint32_t deg = (uint32_t)(__ldg(p.row_ptr + s + 1) - __ldg(p.row_ptr + s));
          if (deg > 0) {
            const uint32_t bit = 1u << (s & 31);
            if (!(atomicOr(p.bitmap0 + (s >> 5), bit) & bit)) {
              mask = 1;
              tg[0] = s;
              dgs[0] = deg;
            }
          }
        }
      }
      stage_entries(sh.wt[warp], staged, mask, tg, dgs);
      if (staged > kStage - 32) flush_entries(p, sh.wt[warp], staged, 0, 0, p.tails);
    }
    flush_entries(p, sh.wt[warp], staged, 0, 0, p.tails);
  }
  if (!grid_barrier(ctl, p.wait_limit_ns, &sh.flag)) goto finish;

  // 3. GOVM steps.
  for (;; ++step) {
    const int cur = (int)(step & 1);
    unsigned long long *tails_cur = p.tails + (size_t)(step % 3) * p.k;
    unsigned long long *tails_next = p.tails + (size_t)((step + 1) % 3) * p.k;
    unsigned long long *tails_old = p.tails + (size_t)((step + 2) % 3) * p.k;
    const int32_t total_tiles = scan_tiles(tails_cur, p.k, sh);
    if (total_tiles == 0) {
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
        tails_old[i] = 0ull;  // read last in the previous step; appended to in the next one
      }
      if (fs) atomicAdd(&ctl->frontier_sum, fs);
      if (es) atomicAdd(&ctl->edges_scanned, es);
    }
    const int32_t gw = blockIdx.x * kWarpsPerBlock + warp;
    const int32_t nw = gridDim.x * kWarpsPerBlock;
    int staged = 0;
    int32_t staged_inst = 0;
    for (int32_t g = gw; g < total_tiles; g += nw) {
      const int32_t inst = find_instance(sh.tprefix, p.k, g);
      const int32_t t = g - sh.tprefix[inst];
      const int32_t tiles_i = sh.tprefix[inst + 1] - sh.tprefix[inst];
      if (staged > 0 && inst != staged_inst) flush_entries(p, sh.wt[warp], staged, staged_inst, cur ^ 1, tails_next);
      staged_inst = inst;
      process_tile<F32>(p, sh.wt[warp], inst, t, __ldcg(tails_cur + inst), tiles_i, cur, staged, updates);
      if (staged > kStage - kTile) flush_entries(p, sh.wt[warp], staged, inst, cur ^ 1, tails_next);
    }
    flush_entries(p, sh.wt[warp], staged, staged_inst, cur ^ 1, tails_next);
    if (!grid_barrier(ctl, p.wait_limit_ns, &sh.flag)) break;
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
  if (quiescent) {
    for (int32_t i = 0; i < p.k; ++i) {
      const unsigned long long *st = p.state + (size_t)i * p.n;
      uint32_t *dist = (uint32_t *)p.dist + (size_t)i * p.n;
      int32_t *par = p.parent ? p.parent + (size_t)i * p.n : nullptr;
      int32_t *pe = p.parent_edge ? p.parent_edge + (size_t)i * p.n : nullptr;
      for (long long v = gtid; v < p.n; v += gsize) {
        const unsigned long long s = __ldcg(st + v);
        const uint32_t key = (uint32_t)(s >> 32);
        const uint32_t e = (uint32_t)s;
        const bool unreachable = key == Key<F32>::inf;
        dist[v] = key;
        if (par) par[v] = unreachable ? -1 : (e == kNoEdge ? (int32_t)v : __ldg(p.src + e));
        if (pe) pe[v] = (unreachable || e == kNoEdge) ? -1 : (int32_t)e;
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
    if (gtid == 0) ctl->steps = (unsigned long long)step;
  }
}

}  // namespace

// Shared memory exceeds the 48 KB static limit: opt in once per kernel.
cudaError_t prepare_kernels() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(govm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(BlockShared));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(govm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BlockShared));
  done = e == cudaSuccess;
  return e;
}

cudaError_t launch_govm(const GovmParams &p, int is_f32, int grid_blocks, cudaStream_t stream) {
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
  if (is_f32) return cudaLaunchKernelEx(&cfg, govm_kernel<true>, p);
  return cudaLaunchKernelEx(&cfg, govm_kernel<false>, p);
}

int govm_max_blocks_per_sm(int is_f32) {
  int nb = 0;
  if (prepare_kernels() != cudaSuccess) return 0;
  const size_t smem = sizeof(BlockShared);
  cudaError_t e = is_f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, govm_kernel<true>, kBlockThreads, smem)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, govm_kernel<false>, kBlockThreads, smem);
  return e == cudaSuccess ? nb : 0;
}

}  // namespace dawn
