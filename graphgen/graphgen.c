/*
 * Seeded synthetic graph generators shared by the CPU oracle tests, the GPU
 * parity tests and the benchmark.  This file holds no shortest-path
 * arithmetic: it only draws graphs, weights, and performs plain structural
 * bookkeeping (sorting, de-duplication, weakly connected components,
 * unweighted reachability) that is used to pick sources and targets.
 *
 * Random numbers come from one counter-based generator: the splitmix64
 * output function (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) applied to key + (ctr + 1) * golden,
 * where key is derived from (seed, stream).  Every draw is therefore a pure
 * function of (seed, stream, ctr) and the graphs are identical on any host
 * and with any number of threads.
 *
 * The workloads stand in for the SNAP / SuiteSparse graphs of the paper's
 * Section 4 (Table 2), which are not available.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t gg_key(uint64_t seed, uint64_t stream) {
  return gg_mix(gg_mix(seed + GG_GOLDEN) ^ (stream * 0xD1B54A32D192ED03ULL + 0x8CB92BA72F3D8DD7ULL));
}

static inline uint64_t gg_at(uint64_t key, uint64_t ctr) { return gg_mix(key + (ctr + 1) * GG_GOLDEN); }

/* uniform double in [0, 1) from the top 53 bits */
static inline double gg_u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* integer in [0, range) by multiply-shift on the top 32 bits (range <= 2^32) */
static inline uint64_t gg_below(uint64_t x, uint64_t range) { return ((x >> 32) * range) >> 32; }

void gg_free(void *p) { free(p); }

/* Raw draws, exposed so that Python-side sampling uses the same generator. */
void gg_draws(uint64_t seed, uint64_t stream, uint64_t ctr0, int64_t count, uint64_t *out) {
  uint64_t key = gg_key(seed, stream);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) out[i] = gg_at(key, ctr0 + (uint64_t)i);
}

/* ---------------------------------------------------------------- sorting */

/* Stable LSD radix sort of 64-bit keys (16 bits per pass) over `bits` low bits. */
static int gg_radix_sort(uint64_t *keys, int64_t n, int bits) {
  if (n <= 1) return 0;
  uint64_t *tmp = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  int64_t *cnt = (int64_t *)malloc(65536 * sizeof(int64_t));
  if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
  uint64_t *src = keys, *dst = tmp;
  for (int shift = 0; shift < bits; shift += 16) {
    memset(cnt, 0, 65536 * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> shift) & 0xFFFF]++;
    int64_t run = 0;
    for (int b = 0; b < 65536; ++b) { int64_t c = cnt[b]; cnt[b] = run; run += c; }
    for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> shift) & 0xFFFF]++] = src[i];
    uint64_t *t = src; src = dst; dst = t;
  }
  if (src != keys) memcpy(keys, src, (size_t)n * sizeof(uint64_t));
  free(tmp); free(cnt);
  return 0;
}

static int gg_bits_for(uint64_t maxkey) {
  int b = 0;
  while (b < 64 && (maxkey >> b)) ++b;
  return b == 0 ? 1 : b;
}

/* Build CSR (row_ptr[n+1], col[m]) from sorted keys (u << kb) | v (payload
 * already stripped).  When `dedup` is set, equal keys are merged. */
static int gg_keys_to_csr(uint64_t *keys, int64_t nk, int32_t n, int kb, int dedup, int32_t **row_ptr_out,
                          int32_t **col_out, int64_t *m_out) {
  int64_t m = 0;
  for (int64_t i = 0; i < nk; ++i)
    if (!dedup || i == 0 || keys[i] != keys[i - 1]) keys[m++] = keys[i];
  int32_t *row_ptr = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  int32_t *col = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  if (!row_ptr || !col) { free(row_ptr); free(col); return -1; }
  for (int64_t i = 0; i < m; ++i) {
    uint64_t u = keys[i] >> kb;
    col[i] = (int32_t)(keys[i] & ((1ULL << kb) - 1));
    row_ptr[u + 1]++;
  }
  for (int32_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
  *row_ptr_out = row_ptr; *col_out = col; *m_out = m;
  return 0;
}

/* -------------------------------------------------------------- R-MAT graph */

/*
 * R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): each of
 * edge_factor * 2^scale draws picks one quadrant per level with probabilities
 * (a, b, c, 1-a-b-c).  Each level consumes a 16-bit slice of a 64-bit draw
 * (four levels per draw), compared against the quadrant thresholds rounded to
 * 1/65536.  Self-loops and duplicates are removed; with `relabel` the vertex
 * ids are permuted by a seeded Fisher-Yates shuffle (stream 1) so that hubs
 * do not cluster at low ids.
 */
int gg_rmat(int scale, int edge_factor, double a, double b, double c, uint64_t seed, int relabel,
            int32_t *n_out, int64_t *m_out, int32_t **row_ptr, int32_t **col) {
  if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
  int32_t n = (int32_t)1 << scale;
  int64_t draws = (int64_t)edge_factor << scale;
  uint32_t ta = (uint32_t)llround(a * 65536.0);
  uint32_t tab = (uint32_t)llround((a + b) * 65536.0);
  uint32_t tabc = (uint32_t)llround((a + b + c) * 65536.0);
  uint64_t *keys = (uint64_t *)malloc((size_t)draws * sizeof(uint64_t));
  if (!keys) return -1;
  uint64_t key = gg_key(seed, 0);
  int per_edge = (scale + 3) / 4;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < draws; ++i) {
    uint64_t u = 0, v = 0;
    int level = 0;
    for (int d = 0; d < per_edge; ++d) {
      uint64_t x = gg_at(key, (uint64_t)i * (uint64_t)per_edge + (uint64_t)d);
      for (int s = 0; s < 4 && level < scale; ++s, ++level) {
        uint32_t r = (uint32_t)((x >> (16 * s)) & 0xFFFF);
        uint64_t bu = 0, bv = 0;
        if (r < ta) { bu = 0; bv = 0; }
        else if (r < tab) { bu = 0; bv = 1; }
        else if (r < tabc) { bu = 1; bv = 0; }
        else { bu = 1; bv = 1; }
        u = (u << 1) | bu;
        v = (v << 1) | bv;
      }
    }
    keys[i] = (u << 32) | v;
  }
  int32_t *perm = NULL;
  if (relabel) {
    perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!perm) { free(keys); return -1; }
    for (int32_t v = 0; v < n; ++v) perm[v] = v;
    uint64_t pk = gg_key(seed, 1);
    for (int32_t i = n - 1; i > 0; --i) {
      int32_t j = (int32_t)gg_below(gg_at(pk, (uint64_t)i), (uint64_t)i + 1);
      int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
  }
  int64_t k = 0;
  for (int64_t i = 0; i < draws; ++i) {
    uint64_t u = keys[i] >> 32, v = keys[i] & 0xFFFFFFFFULL;
    if (u == v) continue;
    if (perm) { u = (uint64_t)perm[u]; v = (uint64_t)perm[v]; }
    keys[k++] = (u << scale) | v;
  }
  free(perm);
  int rc = gg_radix_sort(keys, k, 2 * scale);
  if (rc == 0) rc = gg_keys_to_csr(keys, k, n, scale, 1, row_ptr, col, m_out);
  free(keys);
  *n_out = n;
  return rc;
}

/* ------------------------------------------------------- Erdos-Renyi G(n,M) */

/* G(n, M): the first M distinct directed pairs (u, v), u != v, in draw order
 * of stream 0 (one 64-bit draw per candidate: u from the high half, v from
 * the low half). */
int gg_er(int32_t n, int64_t M, uint64_t seed, int64_t *m_out, int32_t **row_ptr, int32_t **col) {
  if (n < 1 || M < 0) return -1;
  if (n == 1 && M > 0) return -1;
  if ((double)M > (double)n * (double)(n - 1)) return -1;
  int64_t cap = 1;
  while (cap < 2 * M + 16) cap <<= 1;
  uint64_t *set = (uint64_t *)calloc((size_t)cap, sizeof(uint64_t));
  uint64_t *keys = (uint64_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(uint64_t));
  if (!set || !keys) { free(set); free(keys); return -1; }
  uint64_t key = gg_key(seed, 0);
  int kb = gg_bits_for((uint64_t)n - 1);
  int64_t have = 0;
  for (uint64_t ctr = 0; have < M; ++ctr) {
    uint64_t x = gg_at(key, ctr);
    uint64_t u = gg_below(x, (uint64_t)n);
    uint64_t v = gg_below(x << 32, (uint64_t)n);
    if (u == v) continue;
    uint64_t kk = (u << kb) | v;
    uint64_t h = gg_mix(kk) & (uint64_t)(cap - 1);
    int dup = 0;
    while (set[h]) {
      if (set[h] == kk + 1) { dup = 1; break; }
      h = (h + 1) & (uint64_t)(cap - 1);
    }
    if (dup) continue;
    set[h] = kk + 1;
    keys[have++] = kk;
  }
  free(set);
  int rc = gg_radix_sort(keys, M, 2 * kb);
  if (rc == 0) rc = gg_keys_to_csr(keys, M, n, kb, 0, row_ptr, col, m_out);
  free(keys);
  return rc;
}

/* ----------------------------------------------------- grid with shortcuts */

/* side x side 4-neighbour grid, every neighbour pair in both directions
 * (vertex id r*side+c), plus floor(shortcut_frac * grid_edges) directed
 * shortcuts (u, v), u != v, drawn from stream 0.  Parallel edges are kept.
 * is_shortcut[e] marks CSR edge e as a shortcut. */
int gg_grid(int32_t side, double shortcut_frac, uint64_t seed, int64_t *m_out, int32_t **row_ptr,
            int32_t **col, uint8_t **is_shortcut) {
  if (side < 1) return -1;
  int64_t n64 = (int64_t)side * side;
  if (n64 > 0x7FFFFFFF) return -1;
  int32_t n = (int32_t)n64;
  int64_t grid_edges = 4LL * side * (side - 1);
  int64_t ns = (int64_t)floor(shortcut_frac * (double)grid_edges);
  int64_t total = grid_edges + ns;
  uint64_t *keys = (uint64_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(uint64_t));
  if (!keys) return -1;
  int64_t k = 0;
  int kb = gg_bits_for((uint64_t)n - 1);
  for (int32_t r = 0; r < side; ++r)
    for (int32_t c = 0; c < side; ++c) {
      uint64_t u = (uint64_t)r * side + c;
      if (r > 0) keys[k++] = ((u << kb) | (u - side)) << 1;
      if (c > 0) keys[k++] = ((u << kb) | (u - 1)) << 1;
      if (c + 1 < side) keys[k++] = ((u << kb) | (u + 1)) << 1;
      if (r + 1 < side) keys[k++] = ((u << kb) | (u + side)) << 1;
    }
  uint64_t key = gg_key(seed, 0);
  uint64_t ctr = 0;
  for (int64_t i = 0; i < ns && n > 1;) {
    uint64_t x = gg_at(key, ctr++);
    uint64_t u = gg_below(x, (uint64_t)n), v = gg_below(x << 32, (uint64_t)n);
    if (u == v) continue;
    keys[k++] = (((u << kb) | v) << 1) | 1;
    ++i;
  }
  int rc = gg_radix_sort(keys, k, 2 * kb + 1);
  uint8_t *flag = NULL;
  if (rc == 0) {
    flag = (uint8_t *)malloc((size_t)(k > 0 ? k : 1));
    if (!flag) rc = -1;
  }
  if (rc == 0) {
    for (int64_t i = 0; i < k; ++i) { flag[i] = (uint8_t)(keys[i] & 1); keys[i] >>= 1; }
    rc = gg_keys_to_csr(keys, k, n, kb, 0, row_ptr, col, m_out);
  }
  free(keys);
  if (rc != 0) { free(flag); return rc; }
  *is_shortcut = flag;
  return 0;
}

/* ------------------------------------------------------------------ weights */

/* integer weights uniform in [lo, hi], weight of CSR edge e from draw e */
void gg_weights_u32(int64_t m, uint32_t lo, uint32_t hi, uint64_t seed, uint32_t *w) {
  uint64_t key = gg_key(seed, 0);
  uint64_t range = (uint64_t)hi - lo + 1;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) w[e] = lo + (uint32_t)gg_below(gg_at(key, (uint64_t)e), range);
}

/* fp32 weights: round-to-nearest float of lo + (hi - lo) * u, u in [0, 1) */
void gg_weights_f32_uniform(int64_t m, double lo, double hi, uint64_t seed, float *w) {
  uint64_t key = gg_key(seed, 0);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) w[e] = (float)(lo + (hi - lo) * gg_u01(gg_at(key, (uint64_t)e)));
}

/* fp32 weights: round-to-nearest float of exp(ln lo + (ln hi - ln lo) * u) */
void gg_weights_f32_loguniform(int64_t m, double lo, double hi, uint64_t seed, float *w) {
  uint64_t key = gg_key(seed, 0);
  double a = log(lo), b = log(hi);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) w[e] = (float)exp(a + (b - a) * gg_u01(gg_at(key, (uint64_t)e)));
}

/* --------------------------------------------------------- structure helpers */

static int32_t gg_find(int32_t *p, int32_t x) {
  while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
  return x;
}

/* Weakly connected components by union-find (edge direction ignored).
 * label[v] = smallest vertex id of v's component.  Returns the count. */
int32_t gg_wcc(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t *label) {
  for (int32_t v = 0; v < n; ++v) label[v] = v;
  for (int32_t u = 0; u < n; ++u)
    for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t a = gg_find(label, u), b = gg_find(label, col[e]);
      if (a == b) continue;
      if (a < b) label[b] = a; else label[a] = b;
    }
  int32_t comps = 0;
  for (int32_t v = 0; v < n; ++v) {
    label[v] = gg_find(label, v);
    if (label[v] == v) ++comps;
  }
  return comps;
}

/* Vertices reachable from `source` along edge directions (plain BFS, no
 * weights): reach[v] = 1 if reachable.  Returns the count. */
int32_t gg_reachable(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t source, uint8_t *reach) {
  memset(reach, 0, (size_t)n);
  if (source < 0 || source >= n) return 0;
  int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!queue) return -1;
  int32_t head = 0, tail = 0;
  queue[tail++] = source;
  reach[source] = 1;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
      if (!reach[col[e]]) { reach[col[e]] = 1; queue[tail++] = col[e]; }
  }
  free(queue);
  return tail;
}
