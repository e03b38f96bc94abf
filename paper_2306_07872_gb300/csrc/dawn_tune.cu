// Launch autotuner: picks the kernel (persistent or small-graph), the
// persistent kernel's build (CTAs per SM), grid size and frontier form
// (queue or bitmap steps), and the msssp batch size for one graph and
// workload by timing candidates with CUDA events.  The paper has no counterpart (its launch
// shape is fixed); every solve it times runs through the public API, so a
// tuned configuration is exactly what later solves on the handle use.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "dawn_common.cuh"

namespace {

struct Candidate {
  int ctas;      // DAWN_OPT_CTAS_PER_SM
  int grid;      // DAWN_OPT_GRID_BLOCKS (0 = automatic)
  int batch;     // DAWN_OPT_BATCH (0 = automatic)
  int small;     // DAWN_OPT_SMALL_PATH
  int frontier;  // DAWN_OPT_FRONTIER
};

// Restores a handle's launch options unless released.
struct OptionGuard {
  dawn_graph g;
  int ctas, grid, batch, small, frontier;
  bool armed = true;
  ~OptionGuard() {
    if (!armed) return;
    dawn_set_option(g, DAWN_OPT_CTAS_PER_SM, ctas);
    dawn_set_option(g, DAWN_OPT_GRID_BLOCKS, grid);
    dawn_set_option(g, DAWN_OPT_BATCH, batch);
    dawn_set_option(g, DAWN_OPT_SMALL_PATH, small);
    dawn_set_option(g, DAWN_OPT_FRONTIER, frontier);
  }
};

struct Scratch {
  int32_t *sources = nullptr;
  void *dist = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~Scratch() {
    cudaFree(sources);
    cudaFree(dist);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

int apply(dawn_graph g, const Candidate &c) {
  int rc = dawn_set_option(g, DAWN_OPT_CTAS_PER_SM, c.ctas);
  if (!rc) rc = dawn_set_option(g, DAWN_OPT_GRID_BLOCKS, c.grid);
  if (!rc) rc = dawn_set_option(g, DAWN_OPT_BATCH, c.batch);
  if (!rc) rc = dawn_set_option(g, DAWN_OPT_SMALL_PATH, c.small);
  if (!rc) rc = dawn_set_option(g, DAWN_OPT_FRONTIER, c.frontier);
  return rc;
}

// Grid sizes worth timing for one kernel build: all co-resident CTAs and
// fractions of them, one CTA per SM, and the automatic size (0).
std::vector<int> grid_candidates(int cap, int sms) {
  std::vector<int> v = {0};
  for (int x : {cap, cap * 3 / 4, cap / 2, cap / 4, sms})
    if (x >= 1 && x <= cap && std::find(v.begin(), v.end(), x) == v.end()) v.push_back(x);
  return v;
}

// Batch sizes worth timing (msssp mode): the largest that fits, a half and
// a quarter of it; sizes that give the same launches are timed once.
std::vector<int> batch_candidates(int32_t k, int32_t max_batch) {
  std::vector<int> v = {0};
  std::vector<int32_t> seen = {std::min(k, max_batch)};
  for (int32_t b : {max_batch / 2, max_batch / 4}) {
    const int32_t eff = std::min(k, b);
    if (b >= 1 && std::find(seen.begin(), seen.end(), eff) == seen.end()) {
      seen.push_back(eff);
      v.push_back((int)b);
    }
  }
  return v;
}

}  // namespace

extern "C" int dawn_autotune(dawn_graph g, int mode, const int32_t *sources, int32_t k, int32_t reps,
                             void *stream, dawn_tuning *out) {
  if (!g || !sources || k < 1 || mode < DAWN_TUNE_SSSP || mode > DAWN_TUNE_ROOTS) return DAWN_ERR_INVALID;
  int32_t n = 0;
  int64_t m = 0;
  int wtype = 0;
  int rc = dawn_graph_info(g, &n, &m, &wtype);
  if (rc) return rc;
  for (int32_t i = 0; i < k; ++i)
    if (sources[i] < 0 || sources[i] >= n) return DAWN_ERR_INVALID;
  dawn::LaunchLimits lim;
  if ((rc = dawn::launch_limits(g, &lim))) return rc;
  if (reps <= 0) reps = 3;
  cudaStream_t s = (cudaStream_t)stream;

  // The timed workload.  msssp mode keeps at most 4 GiB of distances.
  int32_t kk = k;
  if (mode == DAWN_TUNE_MSSSP) kk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(k, ((int64_t)1 << 30) / n));
  Scratch sc;
  const size_t dist_rows = mode == DAWN_TUNE_MSSSP ? (size_t)kk : 1;
  if (cudaMalloc((void **)&sc.sources, sizeof(int32_t) * (size_t)k) != cudaSuccess ||
      cudaMalloc(&sc.dist, sizeof(uint32_t) * dist_rows * (size_t)n) != cudaSuccess ||
      cudaEventCreate(&sc.e0) != cudaSuccess || cudaEventCreate(&sc.e1) != cudaSuccess) {
    cudaGetLastError();
    return DAWN_ERR_OOM;
  }
  if (cudaMemcpyAsync(sc.sources, sources, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DAWN_ERR_CUDA;

  auto workload = [&]() -> int {
    if (mode == DAWN_TUNE_MSSSP) return dawn_msssp(g, sc.sources, kk, sc.dist, nullptr, s);
    if (mode == DAWN_TUNE_ROOTS) return dawn_sssp_roots(g, sc.sources, k, sc.dist, nullptr, nullptr, s);
    for (int32_t i = 0; i < k; ++i) {
      const int r = dawn_sssp(g, sources[i], sc.dist, nullptr, nullptr, s);
      if (r) return r;
    }
    return DAWN_OK;
  };

  // The default configuration comes first, so it wins ties; it may run the
  // small-graph kernel, the shapes after it the persistent one, and the
  // small kernel is tried on its own when the solver state fits on-chip.
  std::vector<Candidate> cands = {{5, 0, 0, DAWN_SMALL_AUTO, DAWN_FRONTIER_AUTO}};
  const std::vector<int> batches =
      mode == DAWN_TUNE_MSSSP ? batch_candidates(kk, lim.max_batch) : std::vector<int>{0};
  for (int ctas : {5, 4}) {
    const int cap = (ctas == 4 ? lim.occupancy4 : lim.occupancy5) * lim.sms;
    for (int grid : grid_candidates(cap, lim.sms))
      for (int batch : batches) cands.push_back({ctas, grid, batch, DAWN_SMALL_NEVER, DAWN_FRONTIER_AUTO});
    // a few instances per launch, at the automatic grid size: on large graphs
    // several frontiers fill each step while the instances' states still fit
    // L2 together (R-MAT s22: 8 per launch is 1.09x faster than 64)
    if (mode == DAWN_TUNE_MSSSP)
      for (int batch : {16, 8, 4})
        if (batch < kk && batch < lim.max_batch) cands.push_back({ctas, 0, batch, DAWN_SMALL_NEVER, DAWN_FRONTIER_AUTO});
    // single-instance solves may run either step form: the one the automatic
    // rule does not pick is timed at the automatic grid size
    if (mode != DAWN_TUNE_MSSSP)
      for (int form : {DAWN_FRONTIER_QUEUE, DAWN_FRONTIER_BITMAP})
        if (form != lim.auto_frontier) cands.push_back({ctas, 0, 0, DAWN_SMALL_NEVER, form});
  }
  if (lim.small_state_fits) cands.push_back({5, 0, 0, DAWN_SMALL_WHEN_STATE_FITS, DAWN_FRONTIER_AUTO});

  OptionGuard guard{g, lim.ctas_per_sm, lim.grid_blocks, lim.batch, lim.small_path, lim.frontier};
  float best_ms = 0.0f, default_ms = 0.0f;
  size_t best = 0;
  std::vector<float> t(reps);
  for (size_t c = 0; c < cands.size(); ++c) {
    if ((rc = apply(g, cands[c]))) return rc;
    if ((rc = workload())) return rc;  // warm-up (and workspace growth)
    for (int32_t r = 0; r < reps; ++r) {
      if (cudaEventRecord(sc.e0, s) != cudaSuccess) return DAWN_ERR_CUDA;
      if ((rc = workload())) return rc;
      if (cudaEventRecord(sc.e1, s) != cudaSuccess || cudaEventSynchronize(sc.e1) != cudaSuccess ||
          cudaEventElapsedTime(&t[r], sc.e0, sc.e1) != cudaSuccess)
        return DAWN_ERR_CUDA;
    }
    if ((rc = dawn_status(g, 1))) return rc;
    std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
    const float med = t[reps / 2];
    if (c == 0) default_ms = med;
    if (c == 0 || med < best_ms) {
      best_ms = med;
      best = c;
    }
  }
  if ((rc = apply(g, cands[best]))) return rc;
  guard.armed = false;
  if (out) {
    const Candidate &b = cands[best];
    out->ctas_per_sm = b.ctas;
    out->grid_blocks = b.grid;
    out->batch = b.batch;
    out->small_path = b.small;
    out->frontier = b.frontier;
    out->candidates = (int32_t)cands.size();
    out->best_ms = best_ms;
    out->default_ms = default_ms;
  }
  return DAWN_OK;
}
