// rank.cuh -- the degree order of a graph's vertices: rank(v) = position of
// (degree(v), v) in ascending lexicographic order, from one radix sort of the
// n keys (degree << lbn | v).  Triangle counting orients its DAG by this order
// (Section 4.4's filter) and PageRank runs on a copy of the graph relabelled by
// it, so that the contributions of high-degree vertices, which most gathers
// read, share a short range of cache lines.
#pragma once

#include "byo_internal.cuh"
#include "prof.cuh"

namespace byo {

template <typename G>
__global__ void degree_keys_kernel(G g, uint32_t n, int lbn, uint64_t* keys) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    keys[v] = ((uint64_t)g.degree((uint32_t)v) << lbn) | v;
}

template <typename K>
__global__ void degree_rank_scatter_kernel(const K* __restrict__ sorted, uint32_t n, K mask, uint32_t* __restrict__ rank) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x)
    rank[sorted[r] & mask] = (uint32_t)r;
}

// Bits of a vertex id (at least 1).
inline int id_bits(uint32_t n) { return n > 1 ? 32 - __builtin_clz(n - 1) : 1; }

// rank[v] for every vertex.  If `sorted_out` is not null it receives the
// sorted keys (n entries, allocated with tmp_alloc on `s`; the caller releases
// them with tmp_free): key r is (degree << id_bits(n)) | vertex of rank r.
template <typename G>
byo_status degree_rank(const byo_graph* g, G view, uint32_t* rank, uint64_t** sorted_out, cudaStream_t s) {
  const uint32_t n = g->n;
  const int lbn = id_bits(n);
  int top = 0;  // highest non-empty degree bucket: degrees < 2^top
  for (int b = 0; b < kBuckets; ++b)
    if (g->bstart[b + 1] > g->bstart[b]) top = b;
  uint64_t *keys = nullptr, *tmp = nullptr, *sorted = nullptr;
  byo_status st = tmp_alloc_t(&keys, n, s, "degree-order keys");
  if (st == BYO_OK) st = tmp_alloc_t(&tmp, n, s, "degree-order keys");
  if (st == BYO_OK) {
    ProfScope ps("degree_rank", s);
    degree_keys_kernel<<<grid_for(n, 256), 256, 0, s>>>(view, n, lbn, keys);
    ::byo::note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_status(e, "degree_keys_kernel");
    if (st == BYO_OK) st = radix_sort_u64(keys, tmp, n, lbn + top, &sorted, s);
    if (st == BYO_OK) {
      degree_rank_scatter_kernel<uint64_t><<<grid_for(n, 256), 256, 0, s>>>(sorted, n, (1ull << lbn) - 1, rank);
      ::byo::note_launch();
      e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_status(e, "degree_rank_scatter_kernel");
    }
  }
  if (st == BYO_OK && sorted_out) {
    *sorted_out = sorted;
    tmp_free(sorted == keys ? tmp : keys, s);
    return BYO_OK;
  }
  tmp_free(keys, s);
  tmp_free(tmp, s);
  return st;
}

}  // namespace byo
