/*
 * dawn.h -- C ABI of the GB300 (sm_103a) weighted-DAWN shortest-path library.
 *
 * The library implements the GOVM iteration of weighted DAWN (arxiv
 * 2306.07872, Section 3.4, Algorithm 2): the distance vector alpha is
 * multiplied by the CSR adjacency matrix in the (min, +) semiring, but only
 * the rows of vertices whose distance changed in the previous step (the
 * frontier delta) are expanded; vertices whose distance changes in this step
 * form the next frontier (beta); the iteration stops when a step changes
 * nothing.  This yields single-source shortest paths (SSSP), and multi-source
 * / all-pairs shortest paths as repeated SSSP (Section 3.4, the complexity
 * argument for APSP; Section 1, contribution 5 on MSSP).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns a dawn_status_code value, except dawn_get_trace
 *    (a row count, or a negated code), dawn_status_string and dawn_destroy;
 *    nothing throws across the ABI.
 *  - Arguments checked on the host (sizes, pointers, scalar ids) fail
 *    synchronously.  Arguments that live in device memory (source / root
 *    arrays) are checked by the kernel, which then skips the solve and leaves
 *    the error in the graph's status word: read it with dawn_status().
 *  - Solves are stream ordered: they enqueue work on `stream` (a cudaStream_t,
 *    NULL for the legacy default stream) and return without synchronising.
 *    Device-side failures (step cap, barrier timeout, invalid device input)
 *    are reported through dawn_status().
 *  - Output arrays are caller-allocated DEVICE buffers on the graph's device.
 *  - Distances: uint32 graphs report uint32 distances with 0xFFFFFFFF for
 *    unreachable vertices; float32 graphs report float32 distances, each the
 *    round-to-nearest left fold fl(...fl(0 + w1) + ... + wk) along a shortest
 *    path, with +inf for unreachable vertices; int32 graphs (signed weights,
 *    Section 1 contribution 4) report int32 distances with 0x7FFFFFFF
 *    (INT32_MAX) for unreachable vertices.
 *  - Negative weights (int32 graphs): the iteration is capped at n steps as
 *    in Algorithm 2 (its loop runs at most n steps); without a negative cycle reachable
 *    from a source it converges before the cap, with one the solve reports
 *    DAWN_ERR_NOT_CONVERGED and its outputs are the state after n steps.
 *  - Parents: parent[v] is the tail u of the lowest-index CSR edge e = (u->v)
 *    with fl(dist[u] + w[e]) == dist[v]; parent[source] = source;
 *    parent[unreachable] = -1.  parent_edge[v] is that edge index e, or -1
 *    for sources and unreachable vertices.  (The paper returns distances only;
 *    the parent rule is this library's definition.)
 *  - A graph handle must not be used by two solves that overlap on the GPU
 *    (one stream at a time per handle); solves on different handles may run
 *    concurrently.
 */
#ifndef DAWN_H
#define DAWN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dawn_graph_s *dawn_graph; /* opaque, owned by the library */

typedef enum { DAWN_W_U32 = 0, DAWN_W_F32 = 1, DAWN_W_I32 = 2 } dawn_wtype;

typedef enum {
  DAWN_OK = 0,
  DAWN_ERR_INVALID = 1,       /* bad argument, malformed CSR, bad weight, source out of range */
  DAWN_ERR_OOM = 2,           /* device allocation failed */
  DAWN_ERR_CUDA = 3,          /* a CUDA runtime call failed (launch, copy, ...) */
  DAWN_ERR_NOT_CONVERGED = 4, /* the step cap (n steps, as in Algorithm 2) was reached */
  DAWN_ERR_TIMEOUT = 5,       /* a bounded wait inside the solver ran out; the kernel returned */
  DAWN_ERR_BOUNDS = 6         /* an internal capacity check failed; the kernel returned */
} dawn_status_code;

/* Counters of the last solve call, summed over all its instances (a batched
 * call split into several launches sums all of them). */
typedef struct {
  int64_t steps;         /* GOVM steps executed (frontier non-empty); the most of any launch */
  int64_t frontier_sum;  /* sum over steps of |delta| (frontier vertices, out-degree >= 1) */
  int64_t edges_scanned; /* sum over steps of the frontier's out-edges (edges relaxed) */
  int64_t updates;       /* path updates: vertices whose distance strictly dropped in a step
                            (they enter beta), counted once per step, summed over steps;
                            updates / (reached vertices - sources) is the paper's mu */
  int64_t instances;     /* instances solved by the last call */
  int64_t edges_skipped; /* frontier out-edges (counted in edges_scanned) that bitmap steps did
                            not relax because their vertex was marked again earlier in the
                            same step (DAWN_OPT_SKIP_REMARKED) */
} dawn_stats;

/*
 * Create a graph from a CSR adjacency matrix (Section 3.2: A_CSR.row_ptr,
 * A_CSR.col, A_CSR.value).
 *   n            number of vertices, 1 <= n < 2^31
 *   m            number of edges, 0 <= m < 2^31
 *   row_ptr      int32[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = m
 *   col_idx      int32[m], every entry in [0, n); parallel edges and
 *                self-loops are allowed
 *   weights      uint32[m] (wtype DAWN_W_U32), float32[m] (DAWN_W_F32) or
 *                int32[m] (DAWN_W_I32, may be negative); float weights must
 *                be finite and >= 0; uint32 weights must satisfy
 *                n * max(w) < 0xFFFFFFFF and int32 weights
 *                n * max|w| < 0x7FFFFFFF, so that no path sum can reach the
 *                unreachable sentinel
 *   inputs_on_device  0: the three arrays are host memory; 1: device memory
 *   stream       stream for the copies and the validation kernel
 *   out          receives the handle
 * The library copies the arrays; the caller keeps ownership of its inputs.
 * Validation runs on the device and is synchronous (the call waits for it).
 * Device memory: every buffer of a handle (the graph, the solver workspace,
 * the backward scratch, staging and trace buffers) comes from a stream-ordered
 * memory pool per device that the library owns; creation, solves, the
 * backward pass and destruction never call cudaMalloc or cudaFree, so none of
 * their allocations or frees synchronises the device (dawn_autotune, a setup
 * call, allocates its own timing scratch with cudaMalloc).
 * Memory a handle frees stays in the pool and serves later allocations
 * without mapping new memory; dawn_trim_memory returns it to the devices.
 * Allocations are refused (DAWN_ERR_CUDA) on a stream that is being
 * captured.
 * Errors: DAWN_ERR_INVALID (malformed input), DAWN_ERR_OOM, DAWN_ERR_CUDA.
 */
int dawn_create_graph(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col_idx,
                      const void *weights, int wtype, int inputs_on_device, void *stream,
                      dawn_graph *out);

/*
 * Replace the edge weights (same type and count as at creation), e.g. after
 * a gradient step.  These are the values array of A_CSR (Section 3.2); the
 * paper has no weight update, this is a library addition for training
 * loops.  Same validation and ownership rules as creation.
 *   flags  DAWN_WEIGHTS_ON_DEVICE: `weights` is device memory (else host);
 *          DAWN_WEIGHTS_DEFER_CHECK: do not wait for the validation result.
 *          The call then returns DAWN_OK without synchronising, and a later
 *          solve on the handle refuses invalid weights itself: it writes no
 *          output and reports DAWN_ERR_INVALID in dawn_status (stream
 *          ordered: issue the solve on the same stream, or order the streams).
 * Every solve checks the verdict of the weights in force, so weights that a
 * synchronous call rejected (they have already replaced the old ones) are
 * refused as well until valid weights are set.
 * Device weights are read in place by one stream-ordered kernel that checks
 * them and writes them into the solver's interleaved (column, weight)
 * array: keep them unchanged until `stream` has passed the call.  Host
 * weights are first copied to a device staging buffer of 4 bytes per edge,
 * allocated on the handle's first host-memory call and kept until
 * dawn_destroy (DAWN_ERR_OOM if that allocation fails; the weights in force
 * are then unchanged).
 */
enum { DAWN_WEIGHTS_ON_DEVICE = 1, DAWN_WEIGHTS_DEFER_CHECK = 2 };
int dawn_set_weights(dawn_graph g, const void *weights, int flags, void *stream);

/*
 * Library plumbing with no counterpart in the paper.
 * Pre-size the solver workspace for batches of up to k instances (optional;
 * solves grow it on demand).  Call before capturing solves into a CUDA
 * graph, since growing the workspace allocates device memory.  (Solves by
 * the small-graph kernel keep their state in shared memory and use none.)
 * The workspace is allocated in the order of the handle's last stream (the
 * creation stream, or the stream of its last call), which the call then
 * synchronises.
 */
int dawn_reserve(dawn_graph g, int32_t k);

/*
 * Single-source shortest paths by the GOVM iteration (Algorithm 2).
 *   source       vertex id in [0, n) (checked synchronously)
 *   dist         device uint32[n] or float32[n] (per the graph's weight type)
 *   parent       device int32[n] or NULL
 *   parent_edge  device int32[n] or NULL
 * One kernel launch performs initialisation, every GOVM step and the output,
 * with no host round trip per step: the persistent kernel (device-wide
 * barriers between phases) or, for a graph whose solver state fits in one
 * block's shared memory, the small-graph kernel (one block, block barriers;
 * see DAWN_OPT_SMALL_PATH).
 */
int dawn_sssp(dawn_graph g, int32_t source, void *dist, int32_t *parent, int32_t *parent_edge,
              void *stream);

/*
 * Multi-source shortest paths: k independent SSSP instances, one per source,
 * relaxed together with per-instance frontiers (Section 1, contribution 5;
 * Section 3.5, where the paper parallelises across starting vertices).  APSP
 * is the case sources = 0..n-1.
 *   sources      device int32[k]; an entry outside [0, n) makes the solve
 *                fail with DAWN_ERR_INVALID in dawn_status()
 *   k            number of instances, k >= 1
 *   dist         device [k][n] (row i holds the distances from sources[i])
 *   parent       device int32[k][n] or NULL
 * Large k is processed in chunks of instances (DAWN_OPT_BATCH), each chunk
 * one launch: the persistent kernel, or the small-graph kernel with one block
 * per instance.
 */
int dawn_msssp(dawn_graph g, const int32_t *sources, int32_t k, void *dist, int32_t *parent,
               void *stream);

/*
 * One shortest-path forest grown from several roots at distance 0 (all roots
 * are sources for Algorithm 2's source guard, which never relaxes an edge
 * into a source).  On a graph
 * that is the disjoint union of many graphs with one root each, this solves
 * every graph in one launch.
 *   roots        device int32[k] (duplicates allowed), k >= 1
 *   dist, parent, parent_edge  as for dawn_sssp (parent[root] = root)
 */
int dawn_sssp_roots(dawn_graph g, const int32_t *roots, int32_t k, void *dist, int32_t *parent,
                    int32_t *parent_edge, void *stream);

/*
 * Backward pass of dist with respect to the edge weights (float32 graphs).
 * The paper has no backward pass; this is a library addition that follows
 * from the forward result: the parent tree the GOVM fixpoint defines.
 * dist[v] is the sum of the weights along v's tree path, so for a loss L,
 * dL/dw[e] = sum of dL/ddist[t] over the subtree below tree edge e, and 0 for
 * edges off the tree.  The parent tree from the forward solve is the only
 * saved state.
 *   parent_edge  device int32[n] from dawn_sssp / dawn_sssp_roots
 *   grad_dist    device float32[n] (dL/ddist; entries of unreachable
 *                vertices are ignored)
 *   grad_w       device float32[m], overwritten
 * The tree is processed children before parents (reverse tree order, the
 * reverse of distance order for positive weights): O(n + m) work whatever the
 * number of non-zero dL/ddist entries.  The sums run in float32 in an order
 * that varies from call to call, so the last bits may differ between calls.
 * A parent_edge array that contains a cycle or an edge index outside [0, m)
 * makes the call fail with DAWN_ERR_INVALID in dawn_status().  The first call
 * on a handle allocates 16 bytes per vertex (plus 32) of scratch (make one
 * call before capturing the backward into a CUDA graph).
 */
int dawn_sssp_backward(dawn_graph g, const int32_t *parent_edge, const float *grad_dist, float *grad_w,
                       void *stream);

/*
 * Library plumbing with no counterpart in the paper.
 * Device-side status of the last solve on this handle (DAWN_OK or an error
 * code).  With sync != 0 the call first waits for the last stream used by the
 * handle; with sync == 0 it reads the status without waiting (it may be
 * stale).
 */
int dawn_status(dawn_graph g, int sync);

/* Counters of the last solve (waits for it): steps of Algorithm 2's loop,
 * frontier sizes, edges scanned (the work of Section 3.4's complexity
 * argument) and path updates (mu's numerator, Section 4.2). */
int dawn_get_stats(dawn_graph g, dawn_stats *out);

/*
 * Tuning and test options.
 *   DAWN_OPT_MAX_STEPS     step cap (default n, the step bound of Algorithm 2)
 *   DAWN_OPT_WAIT_LIMIT_NS bound on every in-kernel wait (default 4e9 ns)
 *   DAWN_OPT_GRID_BLOCKS   persistent grid size (0 = automatic: all
 *                          co-resident CTAs for large problems, fewer for
 *                          small ones; larger values are clamped to the
 *                          co-resident count)
 *   DAWN_OPT_CTAS_PER_SM   kernel build: 5 (the default; 48 registers per
 *                          thread, 40 resident warps per SM) or 4 (64
 *                          registers, 32 warps); 0 = default, others invalid
 *   DAWN_OPT_BATCH         instances per persistent launch in dawn_msssp
 *                          (0 = as many as the workspace budget allows, or,
 *                          when fewer than 32 instances' 8-byte-per-vertex
 *                          states fit L2 together, as many as fit and at
 *                          least 4)
 *   DAWN_OPT_TEST_STALL    1: block 0 waits on a flag nothing sets, so the
 *                          bounded waits run out (tests DAWN_ERR_TIMEOUT)
 *   DAWN_OPT_SMALL_PATH    DAWN_SMALL_AUTO (default): a graph whose solver
 *                          state and CSR fit in one block's shared memory
 *                          (about 12 bytes per vertex + 8 per edge within
 *                          the device's opt-in limit, 227 KB on GB300) is
 *                          solved by a kernel with one block per instance
 *                          and everything on-chip, so no step needs a
 *                          device-wide barrier; DAWN_SMALL_NEVER: always the
 *                          persistent kernel; DAWN_SMALL_WHEN_STATE_FITS:
 *                          the small kernel whenever the state fits (the CSR
 *                          is then read from global memory).  Same results.
 *                          A call that wants no parents on a graph of
 *                          non-negative weights with at most 65,536 vertices
 *                          keeps only 32-bit distances there (half the
 *                          shared memory; two instances per SM).
 *   DAWN_OPT_TEST_FAIL_ALLOC  N > 0: the N-th next allocation of this
 *                          handle's workspace (solver, backward scratch,
 *                          trace) fails with DAWN_ERR_OOM without touching
 *                          the device (tests the out-of-memory paths); 0 = off
 *   DAWN_OPT_TRACE_STEPS   record up to `value` per-step trace rows in later
 *                          solves (0 = off, the default); allocates
 *   DAWN_OPT_FRONTIER      how the persistent kernel holds the frontier delta
 *                          between steps.  DAWN_FRONTIER_QUEUE: compacted
 *                          into a queue whose out-edges are cut into
 *                          128-edge tiles (work balanced by edges; two
 *                          device-wide barriers per step).
 *                          DAWN_FRONTIER_BITMAP: left in the bitmap of the
 *                          previous step's marks, from which each warp
 *                          expands the marked vertices of a range directly
 *                          (one barrier per step; a row is expanded by one
 *                          warp, so long rows unbalance it).
 *                          DAWN_FRONTIER_AUTO (default): the bitmap when no
 *                          row has more than 128 out-edges, else the queue.
 *                          Algorithm 1 (DAWN_OPT_GSVM) and launches of
 *                          several instances (dawn_msssp) always use the
 *                          queue.
 *                          Same results; only the time and the step count
 *                          (which may differ by one) depend on it.
 *   DAWN_OPT_SKIP_REMARKED 1 (default): in bitmap steps (DAWN_OPT_FRONTIER),
 *                          a frontier vertex whose distance drops again
 *                          during a step before its own out-edges are
 *                          relaxed is not expanded in that step: it is
 *                          already marked for the next frontier, where it is
 *                          expanded with a distance no larger, so expanding
 *                          it now is redundant.  0: every frontier vertex is
 *                          expanded in its step, as Algorithm 2 lists it.
 *                          Queue steps and Algorithm 1 (DAWN_OPT_GSVM) never
 *                          skip.  Same results; counted in
 *                          dawn_stats.edges_skipped.
 *   DAWN_OPT_GSVM          1: solve with Algorithm 1 (GSVM, Section 3.2) instead
 *                          of Algorithm 2: every step rescans the out-edges of
 *                          every reached vertex and the loop stops after a
 *                          step that changes no path (same distances, more
 *                          work; an ablation of GOVM's frontier).  In this mode
 *                          dawn_stats.updates counts expanded vertices.
 */
enum {
  DAWN_OPT_MAX_STEPS = 1,
  DAWN_OPT_WAIT_LIMIT_NS = 2,
  DAWN_OPT_GRID_BLOCKS = 3,
  DAWN_OPT_TEST_STALL = 4,
  DAWN_OPT_TRACE_STEPS = 5,
  DAWN_OPT_GSVM = 6,
  DAWN_OPT_CTAS_PER_SM = 7,
  DAWN_OPT_BATCH = 8,
  DAWN_OPT_TEST_FAIL_ALLOC = 9,
  DAWN_OPT_SMALL_PATH = 10,
  DAWN_OPT_FRONTIER = 11,
  DAWN_OPT_SKIP_REMARKED = 12
};
enum { DAWN_FRONTIER_AUTO = 0, DAWN_FRONTIER_QUEUE = 1, DAWN_FRONTIER_BITMAP = 2 };
enum { DAWN_SMALL_AUTO = 0, DAWN_SMALL_NEVER = 1, DAWN_SMALL_WHEN_STATE_FITS = 2 };
int dawn_set_option(dawn_graph g, int option, int64_t value);

/*
 * Launch autotuner (the paper has no counterpart; it picks this library's
 * launch shape for a given graph and workload).
 *
 * Times the workload under candidate launch configurations and stores the
 * fastest as the handle's options (DAWN_OPT_CTAS_PER_SM, DAWN_OPT_GRID_BLOCKS
 * and, in DAWN_TUNE_MSSSP mode, DAWN_OPT_BATCH), which then apply to every
 * later solve on the handle.  The candidates are the default options, the
 * two builds of the persistent kernel (4 or 5 CTAs per SM) times the grid
 * sizes {all co-resident CTAs, 3/4, 1/2, 1/4 of them, one per SM, the
 * automatic size}, times, in DAWN_TUNE_MSSSP mode, the batch sizes {largest,
 * 1/2, 1/4 of it}, plus batches of 16, 8 and 4 instances (below k) with each
 * build at the automatic grid size; in the single-instance modes, the step form that
 * DAWN_FRONTIER_AUTO does not pick (queue or bitmap steps, DAWN_OPT_FRONTIER)
 * with each build at the automatic grid size; and the small-graph kernel
 * when the graph's solver state fits in shared memory (DAWN_OPT_SMALL_PATH).  Results do not depend on
 * the configuration (the solver's fixpoint is order-independent); only the
 * time does.
 *   mode     DAWN_TUNE_SSSP: dawn_sssp from each source in turn;
 *            DAWN_TUNE_MSSSP: one dawn_msssp over all k sources;
 *            DAWN_TUNE_ROOTS: one dawn_sssp_roots with the k sources as roots
 *   sources  HOST array of k vertex ids (each in [0, n))
 *   reps     timed repetitions per candidate after one warm-up (<= 0: 3);
 *            the score is the median
 *   out      receives the chosen configuration and its timing (may be NULL)
 * The call is synchronous: it waits for `stream` and allocates scratch
 * output buffers for its duration (DAWN_TUNE_MSSSP: up to 4 GiB, the
 * sources beyond that are not part of the timed workload), so it must not
 * be issued during stream capture.  On an error the options in force
 * before the call are restored and the error is returned.
 */
typedef struct {
  int32_t ctas_per_sm;  /* chosen kernel build (4 or 5) */
  int32_t grid_blocks;  /* chosen DAWN_OPT_GRID_BLOCKS (0 = the automatic size) */
  int32_t batch;        /* chosen DAWN_OPT_BATCH (0 = automatic; always 0 outside DAWN_TUNE_MSSSP) */
  int32_t candidates;   /* configurations timed */
  float best_ms;        /* median workload time with the chosen configuration */
  float default_ms;     /* median workload time with the default options */
  int32_t small_path;   /* chosen DAWN_OPT_SMALL_PATH */
  int32_t frontier;     /* chosen DAWN_OPT_FRONTIER (DAWN_FRONTIER_AUTO unless the other step form won) */
} dawn_tuning;

enum { DAWN_TUNE_SSSP = 0, DAWN_TUNE_MSSSP = 1, DAWN_TUNE_ROOTS = 2 };

int dawn_autotune(dawn_graph g, int mode, const int32_t *sources, int32_t k, int32_t reps, void *stream,
                  dawn_tuning *out);

/*
 * Per-step trace of the last solve (enable with DAWN_OPT_TRACE_STEPS; waits
 * for the solve).  Row i (4 int64 values): device time in ns when step i
 * started (the last row: when the iteration ended), the cumulative frontier
 * size |delta| and cumulative frontier out-edges before step i, and a flag
 * that is 1 on the last row.  Returns the number of rows written (at most
 * cap), 0 when tracing is off, or a negated status code.
 */
int dawn_get_trace(dawn_graph g, int64_t *out, int32_t cap);

/* Basic graph facts: n, m and the weight type (plumbing; no counterpart in
 * the paper). */
int dawn_graph_info(dawn_graph g, int32_t *n, int64_t *m, int *wtype);

/*
 * Allocation-free variant of dawn_sssp (the paper has no counterpart; this is
 * a deployment convenience of the library).
 *
 * For callers that cannot allocate device memory during a call (a memory
 * budget fixed up front, hosts that forbid allocator calls after start-up,
 * or code that must avoid the implicit synchronisation of cudaMalloc /
 * cudaFree), this entry point runs the persistent GOVM kernel of dawn_sssp
 * (Algorithm 2, or Algorithm 1 under DAWN_OPT_GSVM) but takes its whole
 * per-solve workspace from one fixed array of 32 MiB in device global memory
 * that belongs to the library (every GPU that loads the library holds this
 * array until the process exits).  It calls no allocation routine.
 *   g            a graph created earlier with dawn_create_graph
 *   source, dist, parent, parent_edge   as for dawn_sssp
 *   status_out   device int32 or NULL: receives the solve's device-side
 *                status (DAWN_OK or an error code) when the solve ends
 * The solve's status and counters are also copied into the handle, so
 * dawn_status(g, 1), dawn_get_stats and dawn_get_trace report this call like
 * any other solve, and dawn_destroy waits for its stream.
 * Options: DAWN_OPT_MAX_STEPS, DAWN_OPT_WAIT_LIMIT_NS, DAWN_OPT_GRID_BLOCKS,
 * DAWN_OPT_CTAS_PER_SM, DAWN_OPT_FRONTIER, DAWN_OPT_GSVM,
 * DAWN_OPT_TRACE_STEPS (the trace buffer is allocated when the option is
 * set) and DAWN_OPT_TEST_STALL apply as for dawn_sssp.  DAWN_OPT_SMALL_PATH does not: the small-graph kernel is
 * never used, so the results are the same but the time may differ.
 * Limit: the workspace takes R(256) + R(16) + R(8 n) + R(8 ceil(n / 32)) +
 * R(16 n) + R(4 (floor(m / 128) + 2)) bytes, where R(x) rounds x up to a
 * multiple of 256 (about 24.25 bytes per vertex plus 4 bytes per 128 edges
 * plus at most 1.5 KB; with m = 16 n, up to about 1.35 M vertices); a graph
 * whose workspace exceeds 32 MiB (33,554,432 bytes) is rejected with
 * DAWN_ERR_INVALID before anything is enqueued.
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture.  Every call uses
 * the same array and leaves its contents behind (the call clears what must
 * start at zero), so calls that overlap on the GPU, on any stream or handle,
 * race and must not be issued.
 */
int dawn_sssp_noalloc(dawn_graph g, int32_t source, void *dist, int32_t *parent, int32_t *parent_edge,
                      int32_t *status_out, void *stream);

/* Human-readable name of a status code (static string; plumbing). */
const char *dawn_status_string(int code);

/* Free the graph and its device memory.  Waits for the handle's last stream
 * (the stream of its last call, which must still exist), then returns its
 * buffers to the library's pool (see dawn_create_graph), where they stay for
 * later handles until dawn_trim_memory.  NULL is allowed (plumbing). */
void dawn_destroy(dawn_graph g);

/* Return to the devices the memory of the library's pools that no handle
 * holds (memory freed by dawn_destroy, by a workspace that grew, or by a
 * replaced trace buffer).  Handles stay valid; their later allocations map
 * memory again.  A pool that grows while solves run maps new memory, which
 * can stall those solves, so a process that creates and destroys graphs in
 * a loop is best left untrimmed until it idles.  DAWN_ERR_CUDA on a CUDA
 * error (plumbing). */
int dawn_trim_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* DAWN_H */
