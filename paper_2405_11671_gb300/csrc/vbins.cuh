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
