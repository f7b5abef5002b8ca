// vbins.cuh -- the thread / warp / CTA granularity split of vertex-centric
// kernels (the GPU form of map_neighbors vs parallel_map_neighbors, Section
// 4.2).  The graph keeps its vertices grouped by degree bucket (vorder), so a
// kernel gives low-degree vertices one thread each, mid-degree ones a warp and
// high-degree ones a whole CTA, by splitting its grid into three block ranges.
#pragma once

#include "byo_internal.cuh"

namespace byo {

struct VBins {
  const uint32_t* vorder;
  uint64_t t1;  // vorder[0, t1): one thread per vertex
  uint64_t w1;  // vorder[t1, w1): one warp per vertex
  uint64_t n;   // vorder[w1, n): one CTA per vertex
  uint32_t nbT, nbW, nbC;
};

// Thread bin = degrees < 2^tb, warp bin = degrees < 2^wb, CTA bin = the rest.
inline VBins make_vbins(const byo_graph* g, int tb, int wb, int threads) {
  VBins b;
  b.vorder = g->vorder;
  b.t1 = g->bstart[tb + 1];
  b.w1 = g->bstart[wb + 1];
  b.n = g->n;
  uint64_t cap = (uint64_t)sm_count() * 8;
  auto clampb = [&](uint64_t x) -> uint32_t { return (uint32_t)(x == 0 ? 0 : (x < cap ? x : cap)); };
  b.nbT = clampb((b.t1 + threads - 1) / threads);
  b.nbW = clampb((b.w1 - b.t1 + (threads / 32) - 1) / (threads / 32));
  b.nbC = clampb(b.n - b.w1);
  return b;
}

inline uint32_t vbins_grid(const VBins& b) {
  uint32_t g = b.nbT + b.nbW + b.nbC;
  return g ? g : 1;
}

enum VRole { kRoleThread = 0, kRoleWarp = 1, kRoleCta = 2 };

// Vertex at vorder index i; a null vorder is the identity (a graph whose ids
// are already in degree order).
__device__ __forceinline__ uint32_t vbins_vertex(const VBins& b, uint64_t i) {
  return b.vorder ? __ldg(b.vorder + i) : (uint32_t)i;
}

struct VRange {
  int role;
  uint64_t begin, end, stride;  // vorder indices this block (thread / warp) walks
};

// The vorder indices handled by the calling thread (thread role), warp (warp
// role) or block (CTA role), as a strided range.
__device__ __forceinline__ VRange vbins_range(const VBins& b) {
  VRange r;
  uint32_t blk = blockIdx.x;
  if (blk < b.nbT) {
    r.role = kRoleThread;
    r.begin = (uint64_t)blk * blockDim.x + threadIdx.x;
    r.end = b.t1;
    r.stride = (uint64_t)b.nbT * blockDim.x;
  } else if (blk < b.nbT + b.nbW) {
    r.role = kRoleWarp;
    uint32_t wpb = blockDim.x >> 5;
    r.begin = b.t1 + (uint64_t)(blk - b.nbT) * wpb + (threadIdx.x >> 5);
    r.end = b.w1;
    r.stride = (uint64_t)b.nbW * wpb;
  } else {
    r.role = kRoleCta;
    r.begin = b.w1 + (blk - b.nbT - b.nbW);
    r.end = b.n;
    r.stride = b.nbC;
  }
  return r;
}

}  // namespace byo

namespace byo {

// The CTA bin split into chunks of at most 2^chunk_log neighbours, so that a
// hub's neighbour list is spread over many CTAs instead of one.  Vertices of
// bucket b (degrees < 2^b) get K_b = max(1, 2^(b - chunk_log)) work items each.
struct CtaChunks {
  int b0;                        // first bucket of the CTA bin
  uint32_t chunk_log;
  uint64_t pre[kBuckets + 1];    // work-item prefix over buckets (0 below b0)
  uint64_t vstart[kBuckets + 1]; // vorder index where each bucket starts
  uint64_t items;                // total work items
  uint64_t vbegin;               // vorder index of the first CTA-bin vertex
  uint64_t vcount;               // CTA-bin vertices
};

inline CtaChunks make_cta_chunks(const byo_graph* g, int b0, uint32_t chunk_log) {
  CtaChunks c;
  c.b0 = b0;
  c.chunk_log = chunk_log;
  c.pre[0] = 0;
  for (int b = 0; b < kBuckets; ++b) {
    uint64_t cnt = b >= b0 ? g->bstart[b + 1] - g->bstart[b] : 0;
    uint64_t K = (uint32_t)b > chunk_log ? (1ull << (b - chunk_log)) : 1ull;
    c.pre[b + 1] = c.pre[b] + cnt * K;
  }
  for (int b = 0; b <= kBuckets; ++b) c.vstart[b] = g->bstart[b];
  c.items = c.pre[kBuckets];
  c.vbegin = g->bstart[b0];
  c.vcount = g->n - g->bstart[b0];
  return c;
}

struct ChunkItem {
  uint64_t vidx;   // vorder index of the vertex
  uint64_t first;  // first work item of this vertex
  uint32_t chunk, K;
};

__device__ __forceinline__ ChunkItem chunk_item(const CtaChunks& c, uint64_t j) {
  int lo = c.b0, hi = kBuckets - 1;
  while (lo < hi) {  // largest b with pre[b] <= j
    int mid = (lo + hi + 1) >> 1;
    if (c.pre[mid] <= j) lo = mid;
    else hi = mid - 1;
  }
  const int b = lo;
  const uint64_t K = (uint32_t)b > c.chunk_log ? (1ull << (b - c.chunk_log)) : 1ull;
  const uint64_t r = j - c.pre[b];
  ChunkItem it;
  it.vidx = c.vstart[b] + r / K;
  it.first = c.pre[b] + (r / K) * K;
  it.chunk = (uint32_t)(r % K);
  it.K = (uint32_t)K;
  return it;
}

// [lo, hi) of a vertex's neighbour list covered by one chunk
__device__ __forceinline__ void chunk_range(uint32_t len, uint32_t chunk, uint32_t K, uint32_t* lo, uint32_t* hi) {
  uint32_t per = (len + K - 1) / K;
  uint32_t a = chunk * per;
  *lo = a < len ? a : len;
  *hi = a + per < len ? a + per : len;
}

}  // namespace byo
