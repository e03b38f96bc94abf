// Internal declarations shared by the CUDA translation units of libdawn.
//
// Data layout in device memory (one solver workspace per graph handle, k
// instances):
//   state   u64 [k][n]   alpha, packed (key(dist) << 32) | parent edge.
//                        key(d) is d itself for uint32 weights, the IEEE
//                        bit pattern for non-negative float32 weights and the
//                        offset-binary code for signed int32; all are monotone
//                        in d, so one 64-bit atomicMin updates
//                        distance and parent edge together and keeps the
//                        lexicographically smallest (dist, edge) pair.
//   bitmap  u32 [2][k][words]  beta of Algorithm 2: vertices whose distance
//                        dropped in the current step (one bit per vertex).
//                        Direct steps use both halves: the frontier delta
//                        (the previous step's marks) and this step's marks;
//                        queue steps use the first.
//   queue   uint4[k][n]  delta of Algorithm 2, compacted: one entry per
//                        frontier vertex with an out-edge = (row start,
//                        offset of its first edge in the frontier's virtual
//                        edge list, row start minus that offset (mod 2^32),
//                        vertex id).  No distance is stored: the relax phase
//                        reads the vertex's current key, which is never
//                        above the key it had when the entry was built.
//   tiles   i32 [k][tiles_cap]  entry index owning the first virtual edge of
//                        every kTile-edge tile of the frontier.
//   tails   u64 [2][k]   per-instance frontier size (low 32 bits) and total
//                        out-degree (high 32 bits); one packed atomicAdd
//                        reserves entries and edge offsets together, so the
//                        queue order equals the offset order.
//   cw      uint2[m]     (column, weight bits) of every CSR edge, interleaved
//                        so that each edge is one 8-byte load.
#pragma once

#include <cstdint>

#include "dawn.h"

namespace dawn {

constexpr int kTile = 128;           // virtual edges per warp task
constexpr int kEdgesPerLane = kTile / 32;
constexpr int kBlockThreads = 256;   // persistent kernel block size
constexpr int kWarpsPerBlock = kBlockThreads / 32;
constexpr int kMaxInstancesPerLaunch = 1024;  // per-block prefix over instances lives in shared memory
constexpr uint32_t kNoEdge = 0xFFFFFFFFu;      // parent field of sources and unreachable vertices
constexpr uint32_t kInfKeyU32 = 0xFFFFFFFFu;
constexpr uint32_t kInfKeyF32 = 0x7F800000u;  // +inf
// Direct steps are used (DAWN_FRONTIER_AUTO) when no row has more out-edges
// than this: a warp then expands 32 rows of at most 32 tiles each.
constexpr int32_t kDirectMaxDegree = 128;

// Control block: barrier, status and counters (zeroed before every launch).
struct DeviceCtl {
  unsigned long long bar;  // device-wide barrier: arrivals (bits 0-62), error flag (bit 63)
  int status;
  int stall_flag;  // never set by anyone: the test stall waits on it
  unsigned long long steps;
  unsigned long long frontier_sum;
  unsigned long long edges_scanned;
  unsigned long long updates;
  unsigned long long edges_skipped;  // direct steps: frontier out-edges not relaxed (vertex marked again first)
  unsigned int changed[3];  // Algorithm 1 only: "a path changed in step t" flags, t mod 3
  // Direct steps: "a distance strictly dropped in step t" flags, t mod 3, on
  // a cache line of their own (the barrier counter's line is the hottest).
  alignas(128) unsigned int marks[3];
};

struct GovmParams {
  const int32_t *row_ptr;
  const uint2 *cw;           // per edge: (column, weight bits)
  const int32_t *src;        // tail of every edge
  int32_t n;
  int64_t m;
  int32_t k;                 // instances in this launch
  int32_t roots_mode;        // 0: seeds[i] is the source of instance i; 1: all seeds root instance 0
  const int32_t *seeds;      // device seeds, or null: then `source` is the only seed
  int32_t nseeds;
  int32_t source;
  unsigned long long *state;
  uint32_t *bitmap;
  uint4 *queue;
  int32_t *tiles;
  unsigned long long *tails;  // [2][k]
  int64_t words;             // bitmap words per instance
  int64_t tiles_cap;         // tile slots per instance
  void *dist;                // [k][n] u32 or f32 bits
  int32_t *parent;           // [k][n] or null
  int32_t *parent_edge;      // [k][n] or null
  DeviceCtl *ctl;
  int64_t max_steps;
  unsigned long long wait_limit_ns;
  int test_stall;
  int gsvm;                  // 1: run Algorithm 1 (rescan every reached vertex each step)
  int direct;                // 1: direct steps (frontier read from the bitmap, one barrier per step)
  int skip_remarked;         // direct steps: a frontier vertex marked again in its step is expanded in the next one only
  unsigned long long *trace;  // optional per-step trace [trace_cap][4], null when off
  int32_t trace_cap;
  // Validation verdict of the graph's current weights (written by the
  // validation kernel): [0] error bits, [1] largest |w|.  A solve refuses to
  // run (DAWN_ERR_INVALID) when an error bit is set or n * max|w| reaches
  // vlimit (0: no bound).  This makes deferred validation stream-ordered.
  const unsigned *vflags;
  uint32_t vlimit;
};

// Host-side launchers (govm_kernel.cu).
// ctas_per_sm selects the kernel build (4 or 5 resident CTAs per SM; any
// other value means 5).  The launch is cooperative: grid_blocks must not
// exceed govm_max_blocks_per_sm(wtype, ctas_per_sm) times the SM count.
cudaError_t launch_govm(const GovmParams &p, int wtype, int ctas_per_sm, int grid_blocks, cudaStream_t stream);
int govm_max_blocks_per_sm(int wtype, int ctas_per_sm);

// Small-graph kernel (govm_small.cu): one block per instance with the whole
// solver state in shared memory (and the CSR when it fits).
constexpr int kSmallThreads = 1024;
constexpr int kSmallWarps = kSmallThreads / 32;
struct SmallLayout {  // byte offsets in the block's dynamic shared memory
  size_t state, bitmap, front, scan, hasout, row_ptr, cw, total;
};
// compact: 32-bit keys and 16-bit frontier ids (no parents, weights >= 0,
// n <= 65,536), half the shared memory of the packed form.
__host__ __device__ SmallLayout small_layout(int32_t n, int64_t m, bool csr, bool compact);
size_t small_smem_limit();  // the device's opt-in shared memory per block
cudaError_t launch_govm_small(const GovmParams &p, int wtype, int32_t blocks, bool csr_in_smem, bool compact,
                              cudaStream_t stream);

// Launch limits and current launch options of a handle (dawn_api.cu), for
// the autotuner (dawn_tune.cu), which otherwise uses only the public API.
struct LaunchLimits {
  int sms;              // streaming multiprocessors of the handle's device
  int occupancy4;       // co-resident CTAs per SM of the 4-CTA kernel build
  int occupancy5;       // same for the 5-CTA build
  int32_t max_batch;    // most instances one msssp launch may hold
  int ctas_per_sm;      // current DAWN_OPT_CTAS_PER_SM
  int grid_blocks;      // current DAWN_OPT_GRID_BLOCKS
  int batch;            // current DAWN_OPT_BATCH
  int small_path;       // current DAWN_OPT_SMALL_PATH
  int small_state_fits;  // the small-graph kernel could hold this graph's solver state
  int frontier;         // current DAWN_OPT_FRONTIER
  int auto_frontier;    // the form DAWN_FRONTIER_AUTO gives a single-instance solve (queue or bitmap)
};
int launch_limits(dawn_graph g, LaunchLimits *out);

}  // namespace dawn
