/*
 * CPU oracle for weighted DAWN (arxiv 2306.07872) -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, sequential, deliberately slow reference implementations used to
 * check the CUDA path.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's library; the product path never
 * does.  Nothing here is shared with the CUDA sources.
 *
 * Contents (every routine works on a CSR graph row_ptr[n+1], col[m], w[m]):
 *   govm_*      Algorithm 2 (GOVM), Section 3.4, executed step by step.
 *   gsvm_*      Algorithm 1 (GSVM), Section 3.2, executed step by step.
 *   dijkstra_*  Textbook binary-heap Dijkstra (Section 2.1) with lazy deletion.
 *   fw_*        Floyd-Warshall (Section 2.3), dense, for tiny graphs.
 *   parents_*   Parent edge of every vertex by the lowest-edge-index rule.
 *   cert_*      Optimality certificate check (invariants of the fixpoint).
 *   subtree_grad_f64   dL/dw for L = sum_t c_t dist[t] (tree path sums).
 *   dijkstra_f64       float64 Dijkstra for central finite differences.
 *
 * Arithmetic.  Integer weights (uint32) are summed exactly in uint64.  Float
 * weights follow the paper's fp32 weights (Section 4.2 uses 1.0f and
 * [0.0f, 2.0f]): every path value is the left fold fl32(...fl32(0 + w1) ...
 * + wk) with round-to-nearest-even, so results are comparable bit for bit.
 * Compile with -ffp-contract=off (no FMA contraction; only additions occur).
 *
 * Readings of the paper taken here (all are listed in the design notes):
 *   - alpha starts at +inf except alpha[source] = 0, delta = {source},
 *     beta = {}, step = 0 (the paper does not state the initialisation);
 *   - Algorithm 1 tests alpha[j] as a truth value; read here as alpha[j]
 *     being finite (the vertex is reached);
 *   - after each GOVM step delta takes beta's contents and beta is cleared
 *     (the listing copies beta into delta without clearing beta);
 *   - several roots may be given; all start at 0 and the source guard (no
 *     edge is relaxed into a source) covers every root; single-source SSSP
 *     is the case k = 1;
 *   - the loop is capped at n steps, the bound both algorithms state;
 *     a run that reaches the cap reports "not converged".
 *
 * Parity unpinned: the work counters of govm_* / gsvm_* (steps, edges
 * scanned, path updates and so mu = updates / (reached - 1)).  Only mu = 1
 * and one step per BFS level on unit weights are pinned; the paper's own mu
 * values (Section 4.2) were measured on graphs that are not available, and
 * the counters depend on the in-place update order, which the paper leaves
 * open.  Distances, parents and gradients are pinned (tests/test_oracle.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define U64_INF UINT64_MAX

typedef struct {
  int64_t steps;          /* executed iterations of the while loop */
  int64_t frontier_sum;   /* sum over steps of |delta| (vertices with delta[j] and an out-edge) */
  int64_t edges_scanned;  /* inner-loop iterations (edges examined) */
  int64_t updates;        /* successful relaxations (alpha strictly decreased) */
  int64_t reached;        /* vertices with finite alpha at the end (roots included) */
  int64_t multi_updated;  /* vertices updated more than once */
  int64_t converged;      /* 1 if the loop ended because no path changed */
} or_stats;

static uint8_t *mark_roots(int32_t n, const int32_t *roots, int32_t k) {
  uint8_t *is_root = (uint8_t *)calloc((size_t)n, 1);
  if (!is_root) return NULL;
  for (int32_t i = 0; i < k; ++i) is_root[roots[i]] = 1;
  return is_root;
}

static void finish_stats(or_stats *st, int32_t n, const uint8_t *finite, const int32_t *count) {
  st->reached = 0;
  st->multi_updated = 0;
  for (int32_t v = 0; v < n; ++v) {
    if (finite[v]) st->reached++;
    if (count[v] > 1) st->multi_updated++;
  }
}

/* ===================================================================== GOVM */

/*
 * Algorithm 2 (GOVM), Section 3.4.  Each step scans the out-edges of the
 * vertices whose path changed in the previous step (delta) and records the
 * vertices whose path changes now (beta); alpha is updated in place.  The
 * loop stops when a step changes no path.
 */
int govm_u32(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w, const int32_t *roots,
             int32_t k, uint64_t *alpha, or_stats *st) {
  uint8_t *is_root = mark_roots(n, roots, k);
  uint8_t *delta = (uint8_t *)calloc((size_t)n, 1);
  uint8_t *beta = (uint8_t *)calloc((size_t)n, 1);
  int32_t *count = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  if (!is_root || !delta || !beta || !count) { free(is_root); free(delta); free(beta); free(count); return -1; }
  memset(st, 0, sizeof(*st));
  for (int32_t v = 0; v < n; ++v) alpha[v] = U64_INF;
  for (int32_t i = 0; i < k; ++i) { alpha[roots[i]] = 0; delta[roots[i]] = 1; }
  int64_t step = 0;
  while (step < n) {
    step = step + 1;
    int ptr = 0;
    for (int32_t j = 0; j < n; ++j) {
      int32_t start = row_ptr[j], end = row_ptr[j + 1];
      if (delta[j] && start != end) {
        st->frontier_sum++;
        for (int32_t e = start; e < end; ++e) {
          int32_t index = col[e];
          uint64_t value = w[e];
          st->edges_scanned++;
          if (alpha[index] > alpha[j] + value && !is_root[index]) {
            alpha[index] = alpha[j] + value;
            beta[index] = 1;
            count[index]++;
            st->updates++;
            ptr = 1;
          }
        }
      }
    }
    if (!ptr) { st->converged = 1; break; }
    memcpy(delta, beta, (size_t)n); /* delta <= beta */
    memset(beta, 0, (size_t)n);     /* beta <= 0 */
  }
  st->steps = step;
  uint8_t *finite = delta;
  for (int32_t v = 0; v < n; ++v) finite[v] = alpha[v] != U64_INF;
  finish_stats(st, n, finite, count);
  free(is_root); free(delta); free(beta); free(count);
  return st->converged ? 0 : 4;
}

int govm_f32(int32_t n, const int32_t *row_ptr, const int32_t *col, const float *w, const int32_t *roots,
             int32_t k, float *alpha, or_stats *st) {
  uint8_t *is_root = mark_roots(n, roots, k);
  uint8_t *delta = (uint8_t *)calloc((size_t)n, 1);
  uint8_t *beta = (uint8_t *)calloc((size_t)n, 1);
  int32_t *count = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  if (!is_root || !delta || !beta || !count) { free(is_root); free(delta); free(beta); free(count); return -1; }
  memset(st, 0, sizeof(*st));
  for (int32_t v = 0; v < n; ++v) alpha[v] = INFINITY;
  for (int32_t i = 0; i < k; ++i) { alpha[roots[i]] = 0.0f; delta[roots[i]] = 1; }
  int64_t step = 0;
  while (step < n) {
    step = step + 1;
    int ptr = 0;
    for (int32_t j = 0; j < n; ++j) {
      int32_t start = row_ptr[j], end = row_ptr[j + 1];
      if (delta[j] && start != end) {
        st->frontier_sum++;
        for (int32_t e = start; e < end; ++e) {
          int32_t index = col[e];
          float value = w[e];
          st->edges_scanned++;
          float cand = alpha[j] + value;
          if (alpha[index] > cand && !is_root[index]) {
            alpha[index] = cand;
            beta[index] = 1;
            count[index]++;
            st->updates++;
            ptr = 1;
          }
        }
      }
    }
    if (!ptr) { st->converged = 1; break; }
    memcpy(delta, beta, (size_t)n);
    memset(beta, 0, (size_t)n);
  }
  st->steps = step;
  uint8_t *finite = delta;
  for (int32_t v = 0; v < n; ++v) finite[v] = alpha[v] != INFINITY;
  finish_stats(st, n, finite, count);
  free(is_root); free(delta); free(beta); free(count);
  return st->converged ? 0 : 4;
}

/* ===================================================================== GSVM */

/*
 * Algorithm 1 (GSVM), Section 3.2.  Every step rescans the out-edges of all
 * reached vertices (finite alpha) and stops when no path changes.
 */
int gsvm_u32(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w, const int32_t *roots,
             int32_t k, uint64_t *alpha, or_stats *st) {
  uint8_t *is_root = mark_roots(n, roots, k);
  int32_t *count = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  uint8_t *finite = (uint8_t *)calloc((size_t)n, 1);
  if (!is_root || !count || !finite) { free(is_root); free(count); free(finite); return -1; }
  memset(st, 0, sizeof(*st));
  for (int32_t v = 0; v < n; ++v) alpha[v] = U64_INF;
  for (int32_t i = 0; i < k; ++i) alpha[roots[i]] = 0;
  int64_t step = 0;
  while (step < n) {
    step = step + 1;
    int ptr = 0;
    for (int32_t j = 0; j < n; ++j) {
      if (alpha[j] != U64_INF) {
        int32_t start = row_ptr[j], end = row_ptr[j + 1];
        if (start != end) {
          st->frontier_sum++;
          for (int32_t e = start; e < end; ++e) {
            int32_t index = col[e];
            uint64_t value = w[e];
            st->edges_scanned++;
            if (alpha[index] > alpha[j] + value && !is_root[index]) {
              alpha[index] = alpha[j] + value;
              count[index]++;
              st->updates++;
              ptr = 1;
            }
          }
        }
      }
    }
    if (!ptr) { st->converged = 1; break; }
  }
  st->steps = step;
  for (int32_t v = 0; v < n; ++v) finite[v] = alpha[v] != U64_INF;
  finish_stats(st, n, finite, count);
  free(is_root); free(count); free(finite);
  return st->converged ? 0 : 4;
}

int gsvm_f32(int32_t n, const int32_t *row_ptr, const int32_t *col, const float *w, const int32_t *roots,
             int32_t k, float *alpha, or_stats *st) {
  uint8_t *is_root = mark_roots(n, roots, k);
  int32_t *count = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  uint8_t *finite = (uint8_t *)calloc((size_t)n, 1);
  if (!is_root || !count || !finite) { free(is_root); free(count); free(finite); return -1; }
  memset(st, 0, sizeof(*st));
  for (int32_t v = 0; v < n; ++v) alpha[v] = INFINITY;
  for (int32_t i = 0; i < k; ++i) alpha[roots[i]] = 0.0f;
  int64_t step = 0;
  while (step < n) {
    step = step + 1;
    int ptr = 0;
    for (int32_t j = 0; j < n; ++j) {
      if (alpha[j] != INFINITY) {
        int32_t start = row_ptr[j], end = row_ptr[j + 1];
        if (start != end) {
          st->frontier_sum++;
          for (int32_t e = start; e < end; ++e) {
            int32_t index = col[e];
            float cand = alpha[j] + w[e];
            st->edges_scanned++;
            if (alpha[index] > cand && !is_root[index]) {
              alpha[index] = cand;
              count[index]++;
              st->updates++;
              ptr = 1;
            }
          }
        }
      }
    }
    if (!ptr) { st->converged = 1; break; }
  }
  st->steps = step;
  for (int32_t v = 0; v < n; ++v) finite[v] = alpha[v] != INFINITY;
  finish_stats(st, n, finite, count);
  free(is_root); free(count); free(finite);
  return st->converged ? 0 : 4;
}

/* ================================================================= Dijkstra */

/* Binary min-heap of (key, vertex) with lazy deletion (stale entries are
 * skipped when popped). */
typedef struct { double key; int32_t v; } heap_item;
typedef struct { heap_item *a; int64_t size, cap; } heap;

static int heap_push(heap *h, double key, int32_t v) {
  if (h->size == h->cap) {
    int64_t nc = h->cap ? 2 * h->cap : 1024;
    heap_item *na = (heap_item *)realloc(h->a, (size_t)nc * sizeof(heap_item));
    if (!na) return -1;
    h->a = na; h->cap = nc;
  }
  int64_t i = h->size++;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h->a[p].key <= key) break;
    h->a[i] = h->a[p];
    i = p;
  }
  h->a[i].key = key; h->a[i].v = v;
  return 0;
}

static heap_item heap_pop(heap *h) {
  heap_item top = h->a[0];
  heap_item last = h->a[--h->size];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, c = i;
    double ck = last.key;
    if (l < h->size && h->a[l].key < ck) { c = l; ck = h->a[l].key; }
    if (r < h->size && h->a[r].key < ck) { c = r; }
    if (c == i) break;
    h->a[i] = h->a[c];
    i = c;
  }
  if (h->size > 0) h->a[i] = last;
  return top;
}

/* The heap key is the distance converted to double: exact for every uint64
 * below 2^53 and for every float, so the pop order is the distance order. */
int dijkstra_u32(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w, const int32_t *roots,
                 int32_t k, uint64_t *dist) {
  uint8_t *is_root = mark_roots(n, roots, k);
  uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
  if (!is_root || !done) { free(is_root); free(done); return -1; }
  heap h = {0};
  for (int32_t v = 0; v < n; ++v) dist[v] = U64_INF;
  int rc = 0;
  for (int32_t i = 0; i < k; ++i) {
    dist[roots[i]] = 0;
    rc |= heap_push(&h, 0.0, roots[i]);
  }
  while (h.size > 0 && rc == 0) {
    heap_item it = heap_pop(&h);
    int32_t u = it.v;
    if (done[u]) continue;
    done[u] = 1;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t v = col[e];
      if (is_root[v]) continue;
      uint64_t cand = dist[u] + w[e];
      if (cand < dist[v]) {
        dist[v] = cand;
        rc |= heap_push(&h, (double)cand, v);
      }
    }
  }
  free(h.a); free(is_root); free(done);
  return rc;
}

int dijkstra_f32(int32_t n, const int32_t *row_ptr, const int32_t *col, const float *w, const int32_t *roots,
                 int32_t k, float *dist) {
  uint8_t *is_root = mark_roots(n, roots, k);
  uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
  if (!is_root || !done) { free(is_root); free(done); return -1; }
  heap h = {0};
  for (int32_t v = 0; v < n; ++v) dist[v] = INFINITY;
  int rc = 0;
  for (int32_t i = 0; i < k; ++i) {
    dist[roots[i]] = 0.0f;
    rc |= heap_push(&h, 0.0, roots[i]);
  }
  while (h.size > 0 && rc == 0) {
    heap_item it = heap_pop(&h);
    int32_t u = it.v;
    if (done[u]) continue;
    done[u] = 1;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t v = col[e];
      if (is_root[v]) continue;
      float cand = dist[u] + w[e];
      if (cand < dist[v]) {
        dist[v] = cand;
        rc |= heap_push(&h, (double)cand, v);
      }
    }
  }
  free(h.a); free(is_root); free(done);
  return rc;
}

/* float64 weights and distances: used for the central finite differences of
 * the gradient check. */
int dijkstra_f64(int32_t n, const int32_t *row_ptr, const int32_t *col, const double *w, int32_t source,
                 double *dist) {
  uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
  if (!done) return -1;
  heap h = {0};
  for (int32_t v = 0; v < n; ++v) dist[v] = INFINITY;
  dist[source] = 0.0;
  int rc = heap_push(&h, 0.0, source);
  while (h.size > 0 && rc == 0) {
    heap_item it = heap_pop(&h);
    int32_t u = it.v;
    if (done[u]) continue;
    done[u] = 1;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t v = col[e];
      if (v == source) continue;
      double cand = dist[u] + w[e];
      if (cand < dist[v]) {
        dist[v] = cand;
        rc |= heap_push(&h, cand, v);
      }
    }
  }
  free(h.a); free(done);
  return rc;
}

/* =========================================================== Floyd-Warshall */

/* D[i*n+j] = shortest i -> j distance; D[i*n+i] = 0.  Sums are re-associated
 * relative to a left fold, so fp32 results are exact only when every partial
 * sum is exactly representable (e.g. dyadic weights). */
int fw_u32(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w, uint64_t *D) {
  for (int64_t i = 0; i < (int64_t)n * n; ++i) D[i] = U64_INF;
  for (int32_t i = 0; i < n; ++i) D[(int64_t)i * n + i] = 0;
  for (int32_t u = 0; u < n; ++u)
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
      if (col[e] != u && w[e] < D[(int64_t)u * n + col[e]]) D[(int64_t)u * n + col[e]] = w[e];
  for (int32_t kk = 0; kk < n; ++kk)
    for (int32_t i = 0; i < n; ++i) {
      uint64_t dik = D[(int64_t)i * n + kk];
      if (dik == U64_INF) continue;
      for (int32_t j = 0; j < n; ++j) {
        uint64_t dkj = D[(int64_t)kk * n + j];
        if (dkj == U64_INF) continue;
        if (dik + dkj < D[(int64_t)i * n + j]) D[(int64_t)i * n + j] = dik + dkj;
      }
    }
  return 0;
}

int fw_f32(int32_t n, const int32_t *row_ptr, const int32_t *col, const float *w, float *D) {
  for (int64_t i = 0; i < (int64_t)n * n; ++i) D[i] = INFINITY;
  for (int32_t i = 0; i < n; ++i) D[(int64_t)i * n + i] = 0.0f;
  for (int32_t u = 0; u < n; ++u)
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
      if (col[e] != u && w[e] < D[(int64_t)u * n + col[e]]) D[(int64_t)u * n + col[e]] = w[e];
  for (int32_t kk = 0; kk < n; ++kk)
    for (int32_t i = 0; i < n; ++i) {
      float dik = D[(int64_t)i * n + kk];
      if (dik == INFINITY) continue;
      for (int32_t j = 0; j < n; ++j) {
        float s = dik + D[(int64_t)kk * n + j];
        if (s < D[(int64_t)i * n + j]) D[(int64_t)i * n + j] = s;
      }
    }
  return 0;
}

/* ================================================================ parents */

/*
 * Parent edge of every vertex (the paper returns distances only): the
 * lowest CSR edge index e = (u -> v) with fl(dist[u] + w[e]) == dist[v].
 * Roots and unreachable vertices get -1.  Written as the plain definition:
 * one pass over the edges in CSR order, first match wins.
 */
int parents_u32(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w, const int32_t *roots,
                int32_t k, const uint64_t *dist, int32_t *parent_edge) {
  uint8_t *is_root = mark_roots(n, roots, k);
  if (!is_root) return -1;
  for (int32_t v = 0; v < n; ++v) parent_edge[v] = -1;
  for (int32_t u = 0; u < n; ++u) {
    if (dist[u] == U64_INF) continue;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t v = col[e];
      if (is_root[v] || parent_edge[v] != -1) continue;
      if (dist[u] + w[e] == dist[v]) parent_edge[v] = e;
    }
  }
  free(is_root);
  return 0;
}

int parents_f32(int32_t n, const int32_t *row_ptr, const int32_t *col, const float *w, const int32_t *roots,
                int32_t k, const float *dist, int32_t *parent_edge) {
  uint8_t *is_root = mark_roots(n, roots, k);
  if (!is_root) return -1;
  for (int32_t v = 0; v < n; ++v) parent_edge[v] = -1;
  for (int32_t u = 0; u < n; ++u) {
    if (dist[u] == INFINITY) continue;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t v = col[e];
      if (is_root[v] || parent_edge[v] != -1) continue;
      float s = dist[u] + w[e];
      if (s == dist[v]) parent_edge[v] = e;
    }
  }
  free(is_root);
  return 0;
}

/* ============================================================ certificate */

/*
 * Certificate that dist is the exact fixpoint (minimum over walks of the
 * left-fold path value) and parent_edge a valid shortest-path forest:
 *   1  a root has dist != 0 or parent_edge != -1
 *   2  some edge (u -> v), v not a root, has fl(dist[u] + w) < dist[v]
 *   3  a non-root vertex with finite dist has an invalid parent edge
 *      (out of range, wrong head, or fl(dist[tail] + w) != dist[v])
 *   4  an unreachable (infinite) vertex has a parent edge
 *   5  the parent edges contain a cycle
 * Returns 0 when every check passes; *where receives the offending vertex or
 * edge.  Conditions 2 and 3 with 5 imply that dist[v] is both attained by a
 * walk (the tree path) and a lower bound on every walk (fl(+) is monotone),
 * and that infinite dist coincides with unreachability.
 */
static int cert_tree(int32_t n, const int32_t *row_ptr, const uint8_t *is_root,
                     const uint8_t *finite, const int32_t *parent_edge, int64_t *where) {
  /* tail of each parent edge by binary search in row_ptr */
  uint8_t *state = (uint8_t *)calloc((size_t)n, 1); /* 0 new, 1 on path, 2 done */
  int32_t *stack = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!state || !stack) { free(state); free(stack); return -1; }
  int rc = 0;
  for (int32_t v0 = 0; v0 < n && rc == 0; ++v0) {
    if (state[v0] || !finite[v0]) continue;
    int32_t top = 0, v = v0;
    while (!is_root[v] && state[v] == 0) {
      state[v] = 1;
      stack[top++] = v;
      int32_t e = parent_edge[v];
      int32_t lo = 0, hi = n; /* find u with row_ptr[u] <= e < row_ptr[u+1] */
      while (hi - lo > 1) {
        int32_t mid = lo + (hi - lo) / 2;
        if (row_ptr[mid] <= e) lo = mid; else hi = mid;
      }
      v = lo;
    }
    if (!is_root[v] && state[v] == 1) { rc = 5; *where = v; }
    while (top > 0) state[stack[--top]] = 2;
  }
  free(state); free(stack);
  return rc;
}

int cert_u32(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w, const int32_t *roots,
             int32_t k, const uint64_t *dist, const int32_t *parent_edge, int64_t *where) {
  int64_t m = row_ptr[n];
  uint8_t *is_root = mark_roots(n, roots, k);
  uint8_t *finite = (uint8_t *)calloc((size_t)n, 1);
  if (!is_root || !finite) { free(is_root); free(finite); return -1; }
  int rc = 0;
  for (int32_t v = 0; v < n; ++v) finite[v] = dist[v] != U64_INF;
  for (int32_t v = 0; v < n && !rc; ++v)
    if (is_root[v] && (dist[v] != 0 || parent_edge[v] != -1)) { rc = 1; *where = v; }
  for (int32_t u = 0; u < n && !rc; ++u) {
    if (!finite[u]) continue;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
      if (!is_root[col[e]] && dist[u] + w[e] < dist[col[e]]) { rc = 2; *where = e; break; }
  }
  for (int32_t v = 0; v < n && !rc; ++v) {
    if (is_root[v]) continue;
    int32_t e = parent_edge[v];
    if (!finite[v]) { if (e != -1) { rc = 4; *where = v; } continue; }
    if (e < 0 || e >= m || col[e] != v) { rc = 3; *where = v; break; }
    int32_t lo = 0, hi = n;
    while (hi - lo > 1) { int32_t mid = lo + (hi - lo) / 2; if (row_ptr[mid] <= e) lo = mid; else hi = mid; }
    if (!finite[lo] || dist[lo] + w[e] != dist[v]) { rc = 3; *where = v; }
  }
  if (!rc) rc = cert_tree(n, row_ptr, is_root, finite, parent_edge, where);
  free(is_root); free(finite);
  return rc;
}

int cert_f32(int32_t n, const int32_t *row_ptr, const int32_t *col, const float *w, const int32_t *roots,
             int32_t k, const float *dist, const int32_t *parent_edge, int64_t *where) {
  int64_t m = row_ptr[n];
  uint8_t *is_root = mark_roots(n, roots, k);
  uint8_t *finite = (uint8_t *)calloc((size_t)n, 1);
  if (!is_root || !finite) { free(is_root); free(finite); return -1; }
  int rc = 0;
  for (int32_t v = 0; v < n; ++v) finite[v] = dist[v] != INFINITY;
  for (int32_t v = 0; v < n && !rc; ++v)
    if (is_root[v] && (dist[v] != 0.0f || parent_edge[v] != -1)) { rc = 1; *where = v; }
  for (int32_t u = 0; u < n && !rc; ++u) {
    if (!finite[u]) continue;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      float s = dist[u] + w[e];
      if (!is_root[col[e]] && s < dist[col[e]]) { rc = 2; *where = e; break; }
    }
  }
  for (int32_t v = 0; v < n && !rc; ++v) {
    if (is_root[v]) continue;
    int32_t e = parent_edge[v];
    if (!finite[v]) { if (e != -1) { rc = 4; *where = v; } continue; }
    if (e < 0 || e >= m || col[e] != v) { rc = 3; *where = v; break; }
    int32_t lo = 0, hi = n;
    while (hi - lo > 1) { int32_t mid = lo + (hi - lo) / 2; if (row_ptr[mid] <= e) lo = mid; else hi = mid; }
    float s = dist[lo] + w[e];
    if (!finite[lo] || s != dist[v]) { rc = 3; *where = v; }
  }
  if (!rc) rc = cert_tree(n, row_ptr, is_root, finite, parent_edge, where);
  free(is_root); free(finite);
  return rc;
}

/* ================================================================ gradient */

/*
 * Reference gradient of L = sum_v c[v] * dist[v] with respect to the edge
 * weights, in float64.  dist[v] is the sum of the weights on v's tree path,
 * so dL/dw[e] is the sum of c over the subtree hanging below a tree edge e
 * and 0 off the tree.  Vertices are visited in decreasing dist order (order
 * = vertex ids sorted that way by the caller); each adds its accumulated
 * subtree sum to its parent.  parent_edge must describe a tree whose parent
 * has strictly smaller dist than its child.
 */
int subtree_grad_f64(int32_t n, const int32_t *row_ptr, int64_t m, const int32_t *parent_edge,
                     const int32_t *order, const double *c, double *grad_w) {
  double *acc = (double *)malloc((size_t)n * sizeof(double));
  if (!acc) return -1;
  for (int32_t v = 0; v < n; ++v) acc[v] = c[v];
  for (int64_t e = 0; e < m; ++e) grad_w[e] = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t v = order[i];
    int32_t e = parent_edge[v];
    if (e < 0) continue;
    int32_t lo = 0, hi = n;
    while (hi - lo > 1) { int32_t mid = lo + (hi - lo) / 2; if (row_ptr[mid] <= e) lo = mid; else hi = mid; }
    grad_w[e] = acc[v];
    acc[lo] += acc[v];
  }
  free(acc);
  return 0;
}

/* ======================================================== signed weights */

/*
 * Signed integer weights (Section 1 contribution 4: the weighted DAWN
 * handles negative weights).  Distances are exact int64 values; I64_INF marks
 * unreachable vertices.  Algorithm 2 is run as written with the step cap n
 * as the only guard: a run that is still changing after n steps (a negative
 * cycle reachable from a root) reports "not converged".
 */
#define I64_INF INT64_MAX

int govm_i32(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w, const int32_t *roots,
             int32_t k, int64_t *alpha, or_stats *st) {
  uint8_t *is_root = mark_roots(n, roots, k);
  uint8_t *delta = (uint8_t *)calloc((size_t)n, 1);
  uint8_t *beta = (uint8_t *)calloc((size_t)n, 1);
  int32_t *count = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  if (!is_root || !delta || !beta || !count) { free(is_root); free(delta); free(beta); free(count); return -1; }
  memset(st, 0, sizeof(*st));
  for (int32_t v = 0; v < n; ++v) alpha[v] = I64_INF;
  for (int32_t i = 0; i < k; ++i) { alpha[roots[i]] = 0; delta[roots[i]] = 1; }
  int64_t step = 0;
  while (step < n) {
    step = step + 1;
    int ptr = 0;
    for (int32_t j = 0; j < n; ++j) {
      int32_t start = row_ptr[j], end = row_ptr[j + 1];
      if (delta[j] && start != end) {
        st->frontier_sum++;
        for (int32_t e = start; e < end; ++e) {
          int32_t index = col[e];
          int64_t value = w[e];
          st->edges_scanned++;
          if (alpha[index] > alpha[j] + value && !is_root[index]) {
            alpha[index] = alpha[j] + value;
            beta[index] = 1;
            count[index]++;
            st->updates++;
            ptr = 1;
          }
        }
      }
    }
    if (!ptr) { st->converged = 1; break; }
    memcpy(delta, beta, (size_t)n);
    memset(beta, 0, (size_t)n);
  }
  st->steps = step;
  uint8_t *finite = delta;
  for (int32_t v = 0; v < n; ++v) finite[v] = alpha[v] != I64_INF;
  finish_stats(st, n, finite, count);
  free(is_root); free(delta); free(beta); free(count);
  return st->converged ? 0 : 4;
}

/* Textbook Bellman-Ford: n - 1 rounds over every edge, then one more round
 * that detects a reachable negative cycle (returns 4). */
int bellman_ford_i32(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w, const int32_t *roots,
                     int32_t k, int64_t *dist) {
  uint8_t *is_root = mark_roots(n, roots, k);
  if (!is_root) return -1;
  for (int32_t v = 0; v < n; ++v) dist[v] = I64_INF;
  for (int32_t i = 0; i < k; ++i) dist[roots[i]] = 0;
  for (int32_t round = 0; round < n - 1; ++round) {
    int changed = 0;
    for (int32_t u = 0; u < n; ++u) {
      if (dist[u] == I64_INF) continue;
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
        int32_t v = col[e];
        if (!is_root[v] && dist[u] + w[e] < dist[v]) { dist[v] = dist[u] + w[e]; changed = 1; }
      }
    }
    if (!changed) break;
  }
  int rc = 0;
  for (int32_t u = 0; u < n && !rc; ++u) {
    if (dist[u] == I64_INF) continue;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
      if (!is_root[col[e]] && dist[u] + w[e] < dist[col[e]]) { rc = 4; break; }
  }
  free(is_root);
  return rc;
}

int parents_i32(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w, const int32_t *roots,
                int32_t k, const int64_t *dist, int32_t *parent_edge) {
  uint8_t *is_root = mark_roots(n, roots, k);
  if (!is_root) return -1;
  for (int32_t v = 0; v < n; ++v) parent_edge[v] = -1;
  for (int32_t u = 0; u < n; ++u) {
    if (dist[u] == I64_INF) continue;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t v = col[e];
      if (is_root[v] || parent_edge[v] != -1) continue;
      if (dist[u] + w[e] == dist[v]) parent_edge[v] = e;
    }
  }
  free(is_root);
  return 0;
}

int cert_i32(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w, const int32_t *roots,
             int32_t k, const int64_t *dist, const int32_t *parent_edge, int64_t *where) {
  int64_t m = row_ptr[n];
  uint8_t *is_root = mark_roots(n, roots, k);
  uint8_t *finite = (uint8_t *)calloc((size_t)n, 1);
  if (!is_root || !finite) { free(is_root); free(finite); return -1; }
  int rc = 0;
  for (int32_t v = 0; v < n; ++v) finite[v] = dist[v] != I64_INF;
  for (int32_t v = 0; v < n && !rc; ++v)
    if (is_root[v] && (dist[v] != 0 || parent_edge[v] != -1)) { rc = 1; *where = v; }
  for (int32_t u = 0; u < n && !rc; ++u) {
    if (!finite[u]) continue;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
      if (!is_root[col[e]] && dist[u] + w[e] < dist[col[e]]) { rc = 2; *where = e; break; }
  }
  for (int32_t v = 0; v < n && !rc; ++v) {
    if (is_root[v]) continue;
    int32_t e = parent_edge[v];
    if (!finite[v]) { if (e != -1) { rc = 4; *where = v; } continue; }
    if (e < 0 || e >= m || col[e] != v) { rc = 3; *where = v; break; }
    int32_t lo = 0, hi = n;
    while (hi - lo > 1) { int32_t mid = lo + (hi - lo) / 2; if (row_ptr[mid] <= e) lo = mid; else hi = mid; }
    if (!finite[lo] || dist[lo] + w[e] != dist[v]) { rc = 3; *where = v; }
  }
  if (!rc) rc = cert_tree(n, row_ptr, is_root, finite, parent_edge, where);
  free(is_root); free(finite);
  return rc;
}
