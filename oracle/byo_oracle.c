/*
 * byo_oracle.c -- THE ORACLE.  Test infrastructure only.
 *
 * A plain, serial, deliberately slow CPU restatement of what the BYO paper's
 * algorithms compute (Wheatman et al., "BYO: A Unified Framework for
 * Benchmarking Large-Scale Graph Containers", arXiv 2405.11671).  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header or constant with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Conventions
 *   n vertices 0..n-1 (Section 3, "Graphs"); an undirected graph stores both
 *   (u,v) and (v,u); m counts stored (directed) entries.  CSR offsets are
 *   uint64, neighbour ids uint32 sorted ascending.  INF = 0xFFFFFFFF marks an
 *   unreached vertex (level and parent).
 *
 * Every function cites the passage whose definition it writes out.  PageRank
 * and the schedule network are not defined by the paper; the readings used are
 * stated beside them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORA_INF 0xFFFFFFFFu

static int ora_cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

/* Sorted unique keys (u<<32|v) of both directions of every non-loop pair. */
static uint64_t* ora_sym_keys(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t k,
                              uint64_t* count) {
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (2 * k + 1));
  if (!keys) return NULL;
  uint64_t c = 0;
  for (uint64_t i = 0; i < k; ++i) {
    uint32_t u = src[i], v = dst[i];
    if (u == v || u >= n || v >= n) continue;
    keys[c++] = ((uint64_t)u << 32) | v;
    keys[c++] = ((uint64_t)v << 32) | u;
  }
  qsort(keys, c, sizeof(uint64_t), ora_cmp_u64);
  uint64_t w = 0;
  for (uint64_t i = 0; i < c; ++i)
    if (w == 0 || keys[i] != keys[w - 1]) keys[w++] = keys[i];
  *count = w;
  return keys;
}

static void ora_keys_to_csr(uint32_t n, const uint64_t* keys, uint64_t m, uint64_t* off, uint32_t* col) {
  for (uint32_t v = 0; v <= n; ++v) off[v] = 0;
  for (uint64_t i = 0; i < m; ++i) off[(keys[i] >> 32) + 1]++;
  for (uint32_t v = 0; v < n; ++v) off[v + 1] += off[v];
  for (uint64_t i = 0; i < m; ++i) col[i] = (uint32_t)keys[i];
}

/*
 * CSR of the undirected graph given by k raw pairs (Section 3.1: the graph as a
 * sequence of neighbour sets; CSR stores them contiguously, Section 4.2).  A
 * neighbour set holds each neighbour once (sets, Section 3.1), so duplicate
 * pairs collapse; self-loops are dropped; each pair is stored in both
 * directions (undirected graphs, Section 3).  col needs room for 2k entries.
 * Returns m, or UINT64_MAX on bad input / allocation failure.
 */
uint64_t ora_csr_build(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t k,
                       uint64_t* off, uint32_t* col) {
  for (uint64_t i = 0; i < k; ++i)
    if (src[i] >= n || dst[i] >= n) return UINT64_MAX;
  uint64_t m = 0;
  uint64_t* keys = ora_sym_keys(n, src, dst, k, &m);
  if (!keys) return UINT64_MAX;
  ora_keys_to_csr(n, keys, m, off, col);
  free(keys);
  return m;
}

/*
 * Breadth-first search from s (the paper's BFS, Table of algorithms in
 * Section 6.2, built on edgeMap over a frontier vertexSubset, Section 3.2):
 * textbook FIFO queue.  level[v] = hop distance from s or INF; parent[v] = the
 * vertex that first reached v (parent[s] = s), INF when unreached.
 */
void ora_bfs(uint32_t n, const uint64_t* off, const uint32_t* col, uint32_t s, uint32_t* level,
             uint32_t* parent) {
  for (uint32_t v = 0; v < n; ++v) { level[v] = ORA_INF; if (parent) parent[v] = ORA_INF; }
  if (s >= n) return;
  uint32_t* q = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!q) return;
  uint64_t head = 0, tail = 0;
  q[tail++] = s;
  level[s] = 0;
  if (parent) parent[s] = s;
  while (head < tail) {
    uint32_t u = q[head++];
    for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = col[e];
      if (level[v] == ORA_INF) {
        level[v] = level[u] + 1;
        if (parent) parent[v] = u;
        q[tail++] = v;
      }
    }
  }
  free(q);
}

static int ora_has_edge(const uint64_t* off, const uint32_t* col, uint32_t u, uint32_t v) {
  uint64_t lo = off[u], hi = off[u + 1];
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (col[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo < off[u + 1] && col[lo] == v;
}

/*
 * Validity of a BFS parent array against given levels: a BFS tree is not
 * unique, so any parent that is a neighbour one level closer is correct.
 * Returns -1 if valid, else the first offending vertex.
 */
int64_t ora_bfs_check_parents(uint32_t n, const uint64_t* off, const uint32_t* col, uint32_t s,
                              const uint32_t* level, const uint32_t* parent) {
  for (uint32_t v = 0; v < n; ++v) {
    uint32_t p = parent[v];
    if (v == s) { if (p != s || level[v] != 0) return v; continue; }
    if (level[v] == ORA_INF) { if (p != ORA_INF) return v; continue; }
    if (p >= n) return v;
    if (level[p] == ORA_INF || level[p] + 1 != level[v]) return v;
    if (!ora_has_edge(off, col, v, p)) return v;
  }
  return -1;
}

/*
 * Connected components (the paper's connectivity algorithm, Section 6.2):
 * label[v] = the minimum vertex id of v's component.  Vertices are scanned in
 * ascending order and each unlabelled one starts a BFS, so it is the minimum
 * of the component it labels.
 */
void ora_cc(uint32_t n, const uint64_t* off, const uint32_t* col, uint32_t* label) {
  for (uint32_t v = 0; v < n; ++v) label[v] = ORA_INF;
  uint32_t* q = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!q) return;
  for (uint32_t r = 0; r < n; ++r) {
    if (label[r] != ORA_INF) continue;
    uint64_t head = 0, tail = 0;
    q[tail++] = r;
    label[r] = r;
    while (head < tail) {
      uint32_t u = q[head++];
      for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
        uint32_t v = col[e];
        if (label[v] == ORA_INF) { label[v] = r; q[tail++] = v; }
      }
    }
  }
  free(q);
}

/*
 * PageRank (named in the paper's algorithm table, Section 6.2, without a
 * formula).  Reading: p_0(v) = 1/n;
 *   p_{t+1}(v) = (1-d)/n + d * ( sum_{u in N(v)} p_t(u)/deg(u) + D_t/n ),
 *   D_t = sum_{deg(u)=0} p_t(u)   (dangling mass spread uniformly),
 * a fixed number of iterations, resid[t] = sum_v |p_{t+1}(v) - p_t(v)|.
 * FP64 throughout; sums in ascending index order.
 */
void ora_pagerank(uint32_t n, const uint64_t* off, const uint32_t* col, double d, uint32_t iters,
                  double* p, double* resid) {
  if (n == 0) return;
  double* q = (double*)malloc(sizeof(double) * n);
  if (!q) return;
  for (uint32_t v = 0; v < n; ++v) p[v] = 1.0 / (double)n;
  for (uint32_t t = 0; t < iters; ++t) {
    double D = 0.0;
    for (uint32_t u = 0; u < n; ++u)
      if (off[u + 1] == off[u]) D += p[u];
    for (uint32_t v = 0; v < n; ++v) {
      double s = 0.0;
      for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
        uint32_t u = col[e];
        s += p[u] / (double)(off[u + 1] - off[u]);
      }
      q[v] = (1.0 - d) / (double)n + d * (s + D / (double)n);
    }
    double r = 0.0;
    for (uint32_t v = 0; v < n; ++v) { r += fabs(q[v] - p[v]); p[v] = q[v]; }
    if (resid) resid[t] = r;
  }
  free(q);
}

/*
 * Single-source betweenness centrality from s (BC in the paper's table of
 * algorithms, Section 6.2): delta[v] = sum over targets t != s, v of
 * sigma_st(v) / sigma_st, where sigma_st counts the shortest s-t paths and
 * sigma_st(v) those through v.  Computed by Brandes' accumulation (U. Brandes,
 * "A faster algorithm for betweenness centrality", J. Math. Sociology 25(2),
 * 2001): a FIFO BFS from s gives level[] and the path counts sigma[v] (sigma[s]
 * = 1; every edge u-v with level[v] = level[u] + 1 adds sigma[u] to sigma[v]);
 * then, over the vertices in reverse BFS order, every w adds
 * sigma[v] / sigma[w] * (1 + delta[w]) to delta[v] for each neighbour v one
 * level closer to s.  Reading: delta[s] = 0 (the source is not between any
 * pair it ends); unreached vertices get level INF, sigma 0, delta 0.  FP64.
 */
void ora_bc(uint32_t n, const uint64_t* off, const uint32_t* col, uint32_t s, uint32_t* level, double* sigma,
            double* delta) {
  for (uint32_t v = 0; v < n; ++v) { level[v] = ORA_INF; sigma[v] = 0.0; delta[v] = 0.0; }
  if (s >= n) return;
  uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!order) return;
  uint64_t head = 0, tail = 0;
  order[tail++] = s;
  level[s] = 0;
  sigma[s] = 1.0;
  while (head < tail) {
    uint32_t u = order[head++];
    for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = col[e];
      if (level[v] == ORA_INF) {
        level[v] = level[u] + 1;
        order[tail++] = v;
      }
      if (level[v] == level[u] + 1) sigma[v] += sigma[u];
    }
  }
  for (uint64_t i = tail; i-- > 0;) {
    uint32_t w = order[i];
    for (uint64_t e = off[w]; e < off[w + 1]; ++e) {
      uint32_t v = col[e];
      if (level[w] > 0 && level[v] == level[w] - 1) delta[v] += sigma[v] / sigma[w] * (1.0 + delta[w]);
    }
  }
  delta[s] = 0.0;
  free(order);
}

/*
 * Compressed neighbour lists (the paper's compressed graphs, Section 2:
 * difference encoding of each sorted list, the first entry relative to the
 * source vertex, every difference stored as a byte code).  Reading of the
 * layout, which the paper leaves to the cited byte-code work: a value is
 * written in 7-bit groups, least significant first, every byte but the last
 * of a value with the 0x80 bit set; the first difference u0 - v is signed and
 * stored as 2|u0 - v| + (u0 < v); the later ones, u_i - u_(i-1) >= 1, as they
 * are.  Degrees stay in the CSR offsets.  ora_bytecode_encode writes the start
 * of every vertex's bytes to boff[0..n] and the bytes to out (capacity cap)
 * and returns the total, or UINT64_MAX if cap is too small;
 * ora_bytecode_decode writes the neighbour ids back into col (m entries, laid
 * out by off).
 */
static uint64_t ora_put_code(uint64_t w, uint8_t* out, uint64_t at, uint64_t cap) {
  do {
    uint8_t b = (uint8_t)(w & 127u);
    w >>= 7;
    if (w) b |= 128u;
    if (out && at < cap) out[at] = b;
    ++at;
  } while (w);
  return at;
}

uint64_t ora_bytecode_encode(uint32_t n, const uint64_t* off, const uint32_t* col, uint64_t* boff, uint8_t* out,
                             uint64_t cap) {
  uint64_t at = 0;
  for (uint32_t v = 0; v < n; ++v) {
    boff[v] = at;
    for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
      uint64_t w;
      if (e == off[v]) {
        w = col[e] >= v ? 2ull * (col[e] - v) : 2ull * (v - col[e]) + 1;
      } else {
        w = (uint64_t)col[e] - col[e - 1];
      }
      at = ora_put_code(w, out, at, cap);
    }
  }
  boff[n] = at;
  return at <= cap ? at : UINT64_MAX;
}

void ora_bytecode_decode(uint32_t n, const uint64_t* off, const uint64_t* boff, const uint8_t* in, uint32_t* col) {
  for (uint32_t v = 0; v < n; ++v) {
    uint64_t at = boff[v];
    uint64_t prev = 0;
    for (uint64_t e = off[v]; e < off[v + 1]; ++e) {
      uint64_t w = 0;
      int shift = 0;
      uint8_t b;
      do {
        b = in[at++];
        w |= (uint64_t)(b & 127u) << shift;
        shift += 7;
      } while (b & 128u);
      if (e == off[v]) prev = (w & 1) ? (uint64_t)v - (w >> 1) : (uint64_t)v + (w >> 1);
      else prev += w;
      col[e] = (uint32_t)prev;
    }
  }
}

/*
 * Triangle count (Section 4.4: intersections of neighbour sets after a filter).
 * Plain definition: each triangle {u<v<w} is counted once, as the number of
 * w in N(u) and N(v) with w > v, over the pairs u<v that are edges; the lists
 * are sorted, so the intersection is a merge.
 */
uint64_t ora_tc(uint32_t n, const uint64_t* off, const uint32_t* col) {
  uint64_t total = 0;
  for (uint32_t u = 0; u < n; ++u) {
    for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = col[e];
      if (v <= u) continue;
      uint64_t i = off[u], j = off[v];
      while (i < off[u + 1] && col[i] <= v) ++i;
      while (j < off[v + 1] && col[j] <= v) ++j;
      while (i < off[u + 1] && j < off[v + 1]) {
        if (col[i] < col[j]) ++i;
        else if (col[i] > col[j]) ++j;
        else { ++total; ++i; ++j; }
      }
    }
  }
  return total;
}

/*
 * The same count through the filter step of Section 4.4 (keep each edge in one
 * direction, then intersect): every edge {u,v} is kept as u -> v when u
 * precedes v in the order (degree, id), giving out-lists N+(u) in ascending id
 * order.  A triangle a < b < c in that order is then counted exactly once, at
 * the DAG edge a -> b, by c in N+(a) and N+(b).  ora_tc_dag_build writes the
 * out-lists (dag_off[n+1], dag_col[m/2]); ora_tc_dag_count sums
 * |N+(u) intersect N+(v)| over the DAG edges u -> v with lo <= u < hi (a range
 * of centres, so that a test driver may split the sum); both serial.
 */
void ora_tc_dag_build(uint32_t n, const uint64_t* off, const uint32_t* col, uint64_t* dag_off, uint32_t* dag_col) {
  dag_off[0] = 0;
  for (uint32_t u = 0; u < n; ++u) {
    uint64_t du = off[u + 1] - off[u];
    uint64_t w = dag_off[u];
    for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = col[e];
      uint64_t dv = off[v + 1] - off[v];
      if (du < dv || (du == dv && u < v)) dag_col[w++] = v;
    }
    dag_off[u + 1] = w;
  }
}

uint64_t ora_tc_dag_count(const uint64_t* dag_off, const uint32_t* dag_col, uint32_t lo, uint32_t hi) {
  uint64_t total = 0;
  for (uint32_t u = lo; u < hi; ++u) {
    for (uint64_t e = dag_off[u]; e < dag_off[u + 1]; ++e) {
      uint32_t v = dag_col[e];
      uint64_t i = dag_off[u], j = dag_off[v];
      while (i < dag_off[u + 1] && j < dag_off[v + 1]) {
        if (dag_col[i] < dag_col[j]) ++i;
        else if (dag_col[i] > dag_col[j]) ++j;
        else { ++total; ++i; ++j; }
      }
    }
  }
  return total;
}

/* ------------------------------------------------------------------------ */
/* Dynamic graph: the edge set itself, as sorted unique keys (u<<32|v).     */
/* Batch semantics follow the set model (Section 3.1) and the batch update */
/* API (Section 4.2): the library sorts the batch; inserting a present edge */
/* or deleting an absent one changes nothing; self-loops are ignored; each  */
/* pair is applied in both directions.                                     */
typedef struct {
  uint32_t n;
  uint64_t m;
  uint64_t* keys;
} ora_dyn;

ora_dyn* ora_dyn_create(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t k) {
  for (uint64_t i = 0; i < k; ++i)
    if (src[i] >= n || dst[i] >= n) return NULL;
  ora_dyn* g = (ora_dyn*)calloc(1, sizeof(ora_dyn));
  if (!g) return NULL;
  g->n = n;
  g->keys = ora_sym_keys(n, src, dst, k, &g->m);
  if (!g->keys) { free(g); return NULL; }
  return g;
}

void ora_dyn_destroy(ora_dyn* g) {
  if (!g) return;
  free(g->keys);
  free(g);
}

uint64_t ora_dyn_num_edges(const ora_dyn* g) { return g->m; }

/* insert != 0: E <- E u B; insert == 0: E <- E \ B.  Returns 0 or -1. */
int ora_dyn_update(ora_dyn* g, const uint32_t* src, const uint32_t* dst, uint64_t k, int insert) {
  for (uint64_t i = 0; i < k; ++i)
    if (src[i] >= g->n || dst[i] >= g->n) return -1;
  uint64_t b = 0;
  uint64_t* bk = ora_sym_keys(g->n, src, dst, k, &b);
  if (!bk) return -1;
  uint64_t* out = (uint64_t*)malloc(sizeof(uint64_t) * (g->m + (insert ? b : 0) + 1));
  if (!out) { free(bk); return -1; }
  uint64_t i = 0, j = 0, w = 0;
  while (i < g->m || j < b) {
    if (j >= b || (i < g->m && g->keys[i] < bk[j])) { out[w++] = g->keys[i++]; }
    else if (i >= g->m || bk[j] < g->keys[i]) { if (insert) out[w++] = bk[j]; ++j; }
    else { if (insert) out[w++] = g->keys[i]; ++i; ++j; }
  }
  free(bk);
  free(g->keys);
  g->keys = out;
  g->m = w;
  return 0;
}

void ora_dyn_export(const ora_dyn* g, uint64_t* off, uint32_t* col) {
  ora_keys_to_csr(g->n, g->keys, g->m, off, col);
}

/* ------------------------------------------------------------------------ */
/* Schedule network (not in the paper): a fully connected ReLU network      */
/* F -> H1 -> H2 -> K with a weighted softmax cross-entropy loss.           */
/* Parameters packed as W1[H1][F], b1[H1], W2[H2][H1], b2[H2], W3[K][H2],   */
/* b3[K].  Loss L = sum_i w_i * (logsumexp(z_i) - z_i[y_i]) / sum_i w_i.    */
/* Returns L; writes dL/dparams into grad (same packing) and the logits     */
/* into logits (B x K) when those are non-NULL.                            */
double ora_mlp_loss(const double* prm, int F, int H1, int H2, int K, const double* X, const int32_t* y,
                    const double* w, int B, double* grad, double* logits) {
  const double* W1 = prm;
  const double* b1 = W1 + (size_t)H1 * F;
  const double* W2 = b1 + H1;
  const double* b2 = W2 + (size_t)H2 * H1;
  const double* W3 = b2 + H2;
  const double* b3 = W3 + (size_t)K * H2;
  size_t P = (size_t)H1 * F + H1 + (size_t)H2 * H1 + H2 + (size_t)K * H2 + K;
  if (grad) memset(grad, 0, sizeof(double) * P);
  double *gW1 = grad, *gb1 = grad ? gW1 + (size_t)H1 * F : NULL;
  double *gW2 = grad ? gb1 + H1 : NULL, *gb2 = grad ? gW2 + (size_t)H2 * H1 : NULL;
  double *gW3 = grad ? gb2 + H2 : NULL, *gb3 = grad ? gW3 + (size_t)K * H2 : NULL;
  double* h1 = (double*)malloc(sizeof(double) * (H1 + H2 + K + H1 + H2 + K));
  if (!h1) return NAN;
  double* h2 = h1 + H1;
  double* z = h2 + H2;
  double* d1 = z + K;
  double* d2 = d1 + H1;
  double* dz = d2 + H2;
  double wsum = 0.0, L = 0.0;
  for (int i = 0; i < B; ++i) wsum += w ? w[i] : 1.0;
  if (wsum <= 0.0) wsum = 1.0;
  for (int i = 0; i < B; ++i) {
    const double* x = X + (size_t)i * F;
    for (int j = 0; j < H1; ++j) {
      double s = b1[j];
      for (int f = 0; f < F; ++f) s += W1[(size_t)j * F + f] * x[f];
      h1[j] = s > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < H2; ++j) {
      double s = b2[j];
      for (int f = 0; f < H1; ++f) s += W2[(size_t)j * H1 + f] * h1[f];
      h2[j] = s > 0.0 ? s : 0.0;
    }
    double zmax = -INFINITY;
    for (int c = 0; c < K; ++c) {
      double s = b3[c];
      for (int f = 0; f < H2; ++f) s += W3[(size_t)c * H2 + f] * h2[f];
      z[c] = s;
      if (s > zmax) zmax = s;
      if (logits) logits[(size_t)i * K + c] = s;
    }
    double se = 0.0;
    for (int c = 0; c < K; ++c) se += exp(z[c] - zmax);
    double lse = zmax + log(se);
    double wi = (w ? w[i] : 1.0) / wsum;
    L += wi * (lse - z[y[i]]);
    if (!grad) continue;
    for (int c = 0; c < K; ++c) dz[c] = wi * (exp(z[c] - lse) - (c == y[i] ? 1.0 : 0.0));
    for (int f = 0; f < H2; ++f) d2[f] = 0.0;
    for (int c = 0; c < K; ++c) {
      gb3[c] += dz[c];
      for (int f = 0; f < H2; ++f) {
        gW3[(size_t)c * H2 + f] += dz[c] * h2[f];
        d2[f] += W3[(size_t)c * H2 + f] * dz[c];
      }
    }
    for (int f = 0; f < H2; ++f) if (h2[f] <= 0.0) d2[f] = 0.0;
    for (int f = 0; f < H1; ++f) d1[f] = 0.0;
    for (int j = 0; j < H2; ++j) {
      gb2[j] += d2[j];
      for (int f = 0; f < H1; ++f) {
        gW2[(size_t)j * H1 + f] += d2[j] * h1[f];
        d1[f] += W2[(size_t)j * H1 + f] * d2[j];
      }
    }
    for (int f = 0; f < H1; ++f) if (h1[f] <= 0.0) d1[f] = 0.0;
    for (int j = 0; j < H1; ++j) {
      gb1[j] += d1[j];
      for (int f = 0; f < F; ++f) gW1[(size_t)j * F + f] += d1[j] * x[f];
    }
  }
  free(h1);
  return L;
}
