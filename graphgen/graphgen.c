/*
 * graphgen.c -- seeded synthetic graph inputs shared by the oracle tests, the
 * CUDA parity tests and bench.py.
 *
 * This module holds no arithmetic of the graph method itself (no dedup, no
 * symmetrisation, no degree, no traversal): it only draws raw edge lists,
 * sources and update batches from a counter-based generator, so that its output
 * is identical for any thread count and on any host architecture.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014; constants as published by Vigna).  Draw i of a
 * stream seeded with s is the SplitMix64 output after i+1 increments of the
 * state, so every draw is addressable by its index.  Bounded integers use the
 * multiply-high map r*bound >> 64 (Lemire).
 *
 * Generators:
 *   - Erdos-Renyi G(n,m): m ordered pairs uniform on [0,n)^2 (the paper's ER
 *     input, Section 6.2, generated with a fixed edge count).
 *   - RMAT: recursive quadrant choice per bit with probabilities a,b,c,d, no
 *     noise (Chakrabarti et al.; the paper's Kron and rMAT inputs, Section 6.2),
 *     then an optional seeded Fisher-Yates relabelling of the vertex ids.
 *   - 2D grid with independent Bernoulli edge drops and uniform shortcuts.
 *   - Sources: distinct, uniform among vertices that touch a non-loop draw.
 *   - Index draws used to pick deletions among earlier draws.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Draw i (0-based) of the SplitMix64 stream seeded with s. */
uint64_t gg_rand(uint64_t s, uint64_t i) { return gg_mix(s + (i + 1) * GG_GOLDEN); }

/* Seed of the sub-stream `tag` of a base seed. */
uint64_t gg_stream(uint64_t seed, uint64_t tag) { return gg_mix(seed ^ gg_mix(tag + GG_GOLDEN)); }

static inline uint64_t gg_below(uint64_t r, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)r * (unsigned __int128)bound) >> 64);
}

/* Uniform double in [0,1) from draw i: top 53 bits. */
double gg_uniform(uint64_t s, uint64_t i) { return (double)(gg_rand(s, i) >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------------ */
/* tiny parallel-for over [0,k) in contiguous chunks                    */
typedef void (*gg_body_fn)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct { gg_body_fn fn; void* ctx; uint64_t lo, hi; } gg_task;
static void* gg_run(void* p) { gg_task* t = (gg_task*)p; t->fn(t->ctx, t->lo, t->hi); return NULL; }

static void gg_parallel(uint64_t k, int threads, gg_body_fn fn, void* ctx) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  if (k < (1u << 16) || threads == 1) { fn(ctx, 0, k); return; }
  pthread_t th[256];
  gg_task tk[256];
  int started[256];
  for (int t = 0; t < threads; ++t) {
    tk[t].fn = fn; tk[t].ctx = ctx;
    tk[t].lo = k * (uint64_t)t / (uint64_t)threads;
    tk[t].hi = k * (uint64_t)(t + 1) / (uint64_t)threads;
    started[t] = pthread_create(&th[t], NULL, gg_run, &tk[t]) == 0;
    if (!started[t]) gg_run(&tk[t]);
  }
  for (int t = 0; t < threads; ++t) if (started[t]) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------ */
/* Erdos-Renyi G(n, m) pair draws                                       */
typedef struct { uint32_t n; uint64_t s; uint32_t *src, *dst; } gg_er_ctx;
static void gg_er_body(void* p, uint64_t lo, uint64_t hi) {
  gg_er_ctx* c = (gg_er_ctx*)p;
  for (uint64_t i = lo; i < hi; ++i) {
    c->src[i] = (uint32_t)gg_below(gg_rand(c->s, 2 * i), c->n);
    c->dst[i] = (uint32_t)gg_below(gg_rand(c->s, 2 * i + 1), c->n);
  }
}
void gg_er(uint32_t n, uint64_t k, uint64_t seed, uint32_t* src, uint32_t* dst, int threads) {
  gg_er_ctx c = {n, gg_stream(seed, 1), src, dst};
  gg_parallel(k, threads, gg_er_body, &c);
}

/* ------------------------------------------------------------------ */
/* RMAT draws.  Each level uses 32 random bits, compared with the       */
/* cumulative thresholds floor(a*2^32), floor((a+b)*2^32), ...          */
typedef struct {
  int scale; uint64_t s; uint64_t ta, tab, tabc; const uint32_t* perm; uint32_t *src, *dst;
} gg_rmat_ctx;
static void gg_rmat_body(void* p, uint64_t lo, uint64_t hi) {
  gg_rmat_ctx* c = (gg_rmat_ctx*)p;
  const uint64_t per = (uint64_t)(c->scale + 1) / 2;
  for (uint64_t i = lo; i < hi; ++i) {
    uint32_t u = 0, v = 0;
    uint64_t r = 0;
    for (int j = 0; j < c->scale; ++j) {
      if ((j & 1) == 0) r = gg_rand(c->s, i * per + (uint64_t)(j >> 1));
      uint64_t x = (j & 1) ? (r >> 32) : (r & 0xFFFFFFFFULL);
      uint32_t bu, bv;
      if (x < c->ta) { bu = 0; bv = 0; }
      else if (x < c->tab) { bu = 0; bv = 1; }
      else if (x < c->tabc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u |= bu << (c->scale - 1 - j);
      v |= bv << (c->scale - 1 - j);
    }
    if (c->perm) { u = c->perm[u]; v = c->perm[v]; }
    c->src[i] = u;
    c->dst[i] = v;
  }
}

/* Seeded uniform random permutation of [0,n) by Fisher-Yates (Durstenfeld). */
void gg_permutation(uint32_t n, uint64_t seed, uint32_t* perm) {
  uint64_t s = gg_stream(seed, 3);
  for (uint32_t i = 0; i < n; ++i) perm[i] = i;
  for (uint64_t i = n; i > 1; --i) {
    uint64_t j = gg_below(gg_rand(s, i - 1), i);
    uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
  }
}

static uint64_t gg_thresh(double x) {
  if (x <= 0.0) return 0;
  if (x >= 1.0) return 1ULL << 32;
  return (uint64_t)(x * 4294967296.0);
}

/* Returns 0 on success, -1 on bad arguments or allocation failure. */
int gg_rmat(int scale, uint64_t k, double a, double b, double c, uint64_t seed, int permute,
            uint32_t* src, uint32_t* dst, int threads) {
  if (scale < 1 || scale > 31) return -1;
  gg_rmat_ctx ctx;
  ctx.scale = scale;
  ctx.s = gg_stream(seed, 2);
  ctx.ta = gg_thresh(a);
  ctx.tab = gg_thresh(a + b);
  ctx.tabc = gg_thresh(a + b + c);
  ctx.src = src; ctx.dst = dst; ctx.perm = NULL;
  uint32_t* perm = NULL;
  if (permute) {
    uint32_t n = 1u << scale;
    perm = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    if (!perm) return -1;
    gg_permutation(n, seed, perm);
    ctx.perm = perm;
  }
  gg_parallel(k, threads, gg_rmat_body, &ctx);
  free(perm);
  return 0;
}

/* ------------------------------------------------------------------ */
/* rows x cols 4-neighbour grid; vertex id r*cols + c.  Horizontal edge */
/* index r*(cols-1)+c, vertical edge index H + r*cols + c.  Each edge   */
/* is dropped with probability `drop`; then round(shortcut_frac*kept)  */
/* uniform shortcut pairs are appended.  Returns the edge count, or 0   */
/* if `cap` is too small.                                              */
uint64_t gg_grid_capacity(uint32_t rows, uint32_t cols, double shortcut_frac) {
  uint64_t H = (uint64_t)rows * (cols ? cols - 1 : 0);
  uint64_t V = (uint64_t)(rows ? rows - 1 : 0) * cols;
  return H + V + (uint64_t)(shortcut_frac * (double)(H + V)) + 2;
}
uint64_t gg_grid(uint32_t rows, uint32_t cols, double drop, double shortcut_frac, uint64_t seed,
                 uint32_t* src, uint32_t* dst, uint64_t cap) {
  uint64_t H = (uint64_t)rows * (cols ? cols - 1 : 0);
  uint64_t V = (uint64_t)(rows ? rows - 1 : 0) * cols;
  uint64_t sd = gg_stream(seed, 4), ss = gg_stream(seed, 5);
  uint64_t tdrop = gg_thresh(drop);
  uint64_t k = 0;
  for (uint64_t e = 0; e < H + V; ++e) {
    if ((gg_rand(sd, e) & 0xFFFFFFFFULL) < tdrop) continue;
    uint32_t u, v;
    if (e < H) {
      uint64_t r = e / (cols - 1), c = e % (cols - 1);
      u = (uint32_t)(r * cols + c); v = u + 1;
    } else {
      uint64_t f = e - H;
      u = (uint32_t)f; v = (uint32_t)(f + cols);
    }
    if (k >= cap) return 0;
    src[k] = u; dst[k] = v; ++k;
  }
  uint64_t n = (uint64_t)rows * cols;
  double want = shortcut_frac * (double)k;
  uint64_t S = (uint64_t)(want + 0.5);
  for (uint64_t i = 0; i < S; ++i) {
    if (k >= cap) return 0;
    src[k] = (uint32_t)gg_below(gg_rand(ss, 2 * i), n);
    dst[k] = (uint32_t)gg_below(gg_rand(ss, 2 * i + 1), n);
    ++k;
  }
  return k;
}

/* ------------------------------------------------------------------ */
/* `count` distinct sources, uniform among the vertices that are an     */
/* endpoint of at least one draw with src != dst, by a partial          */
/* Fisher-Yates over those vertices listed in ascending order.          */
/* Returns how many were picked, or -1 on allocation failure.          */
int64_t gg_pick_sources(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t k,
                        uint32_t count, uint64_t seed, uint32_t* out) {
  uint8_t* mark = (uint8_t*)calloc(n ? n : 1, 1);
  if (!mark) return -1;
  for (uint64_t i = 0; i < k; ++i) {
    if (src[i] != dst[i] && src[i] < n && dst[i] < n) { mark[src[i]] = 1; mark[dst[i]] = 1; }
  }
  uint64_t L = 0;
  for (uint32_t v = 0; v < n; ++v) L += mark[v];
  uint32_t* list = (uint32_t*)malloc(sizeof(uint32_t) * (L ? L : 1));
  if (!list) { free(mark); return -1; }
  L = 0;
  for (uint32_t v = 0; v < n; ++v) if (mark[v]) list[L++] = v;
  free(mark);
  uint64_t s = gg_stream(seed, 6);
  uint64_t take = count < L ? count : L;
  for (uint64_t i = 0; i < take; ++i) {
    uint64_t j = i + gg_below(gg_rand(s, i), L - i);
    uint32_t t = list[i]; list[i] = list[j]; list[j] = t;
    out[i] = list[i];
  }
  free(list);
  return (int64_t)take;
}

/* idx[i] uniform in [0, pool) for i < count (draws with replacement). */
void gg_pick_indices(uint64_t pool, uint64_t count, uint64_t seed, uint64_t* idx) {
  uint64_t s = gg_stream(seed, 8);
  for (uint64_t i = 0; i < count; ++i) idx[i] = gg_below(gg_rand(s, i), pool);
}
