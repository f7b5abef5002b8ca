// cc.cu -- connected components (the paper's connectivity algorithm, Section
// 6.2) as a concurrent union-find.  Every parent pointer goes from a larger id
// to a smaller one (hooks attach the larger root under the smaller), so the
// root of each finished tree is the minimum id of its component and the labels
// come out canonical without a relabelling pass.
//
// The edges are processed in the order of Afforest (Sutton, Ben-Nun and Barak,
// IPDPS 2018), which the paper's comparison with other frameworks credits with
// examining far fewer than all m edges: every vertex is first linked to a
// sample of its neighbours (its first two list entries); the root most of an
// even sample of vertices share is then taken as the large component, and the
// vertices in it at that moment are marked in a bit array.  A final pass
// visits only the unmarked vertices: each links its smaller neighbours, and
// its larger neighbours that are marked.  So an edge between two marked
// vertices needs no link (same component), an edge with one marked end is
// linked from the other end, and an edge between two unmarked vertices is
// linked from its larger end: every edge is covered.  When no component holds
// an eighth of the sample (a batch of many similar graphs) nothing is marked and
// the final pass links every edge from its larger end alone, reading only
// each list's ascending prefix of smaller neighbours.
#include "byo_internal.cuh"
#include "prof.cuh"
#include "container.cuh"
#include "vbins.cuh"

namespace byo {
namespace {

constexpr int kCcThreads = 256;

__device__ __forceinline__ uint32_t cc_find(uint32_t* p, uint32_t x) {
  // path halving; every write stores an ancestor, which stays valid
  while (true) {
    uint32_t px = ld_cg(p + x);
    if (px == x) return x;
    uint32_t gp = ld_cg(p + px);
    if (gp != px) p[x] = gp;
    x = gp;
  }
}

__device__ __forceinline__ void cc_union(uint32_t* p, uint32_t a, uint32_t b) {
  uint32_t ra = cc_find(p, a), rb = cc_find(p, b);
  while (ra != rb) {
    uint32_t hi = ra > rb ? ra : rb;
    uint32_t lo = ra > rb ? rb : ra;
    uint32_t old = atomicCAS(p + hi, hi, lo);
    if (old == hi) return;
    ra = cc_find(p, old);
    rb = cc_find(p, lo);
  }
}

__global__ void cc_identity_kernel(uint32_t* p, uint32_t n) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    p[v] = (uint32_t)v;
}

// sampling round: v is linked to its k-th neighbour
template <typename G>
__global__ void cc_sample_kernel(G g, uint32_t* p, uint32_t k) {
  const uint32_t n = g.num_vertices();
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    Seg s = g.seg((uint32_t)v);
    if (s.len > k) cc_union(p, __ldg(s.p + k), (uint32_t)v);
  }
}

// The root shared by the most of kGiantSample evenly spaced vertices: one
// block finds their roots (read-only walks), sorts them in shared memory and
// takes the longest run.
constexpr int kGiantSample = 1024;

__global__ void __launch_bounds__(kGiantSample) cc_giant_kernel(const uint32_t* p, uint32_t n, uint32_t* giant) {
  __shared__ uint32_t r[kGiantSample];
  __shared__ unsigned long long best;
  const uint32_t t = threadIdx.x;
  {
    uint32_t x = (uint32_t)(((uint64_t)t * n) / kGiantSample), px = ld_cg(p + x);
    while (px != x) {
      x = px;
      px = ld_cg(p + x);
    }
    r[t] = x;
  }
  if (t == 0) best = 0;
  __syncthreads();
  for (uint32_t k = 2; k <= kGiantSample; k <<= 1) {  // bitonic sort, ascending
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const uint32_t q = t ^ j;
      if (q > t) {
        const uint32_t a = r[t], b = r[q];
        if (((t & k) == 0) == (a > b)) {
          r[t] = b;
          r[q] = a;
        }
      }
      __syncthreads();
    }
  }
  if (t == kGiantSample - 1 || r[t] != r[t + 1]) {  // t ends a run: its length by binary search for the start
    uint32_t lo = 0, hi = t;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (r[mid] < r[t]) lo = mid + 1;
      else hi = mid;
    }
    atomicMax(&best, ((unsigned long long)(t - lo + 1) << 32) | r[t]);
  }
  __syncthreads();
  if (t == 0) {
    giant[0] = (uint32_t)(best & 0xFFFFFFFFull);
    giant[1] = (uint32_t)(best >> 32) * 8 >= kGiantSample;  // a component of at least 1/8 of the sample
  }
}

// The vertices whose root is the large component's, one bit each (a snapshot
// taken between the sampling and the final pass).  No vertex is marked when
// no component holds an eighth of the sample (many similar components, as in
// a batch of graphs): the final pass then takes every edge from its larger end.
__global__ void cc_mark_kernel(const uint32_t* p, uint32_t n, const uint32_t* giant_p, uint32_t* marked) {
  const uint32_t giant = __ldg(giant_p), any = __ldg(giant_p + 1);
  const uint32_t nw = (n + 31) / 32;
  for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
       w += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    uint32_t x = (uint32_t)w * 32 + lane_id();
    bool in = false;
    if (x < n) {
      uint32_t px = ld_cg(p + x);
      while (px != x) {
        x = px;
        px = ld_cg(p + x);
      }
      in = any && x == giant;
    }
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, in);
    if (lane_id() == 0) marked[w] = b;
  }
}

__device__ __forceinline__ bool cc_marked(const uint32_t* marked, uint32_t u) {
  return (__ldg(marked + (u >> 5)) >> (u & 31)) & 1u;
}

// Final pass over the unmarked vertices: each links its smaller neighbours and
// its marked larger ones.  Threads, warps or CTA chunks by degree, as in the
// other kernels.
// With nothing marked only the ascending prefix of smaller neighbours is
// read (early exit at the first larger one).
template <typename G>
__global__ void __launch_bounds__(kCcThreads) cc_final_kernel(G g, VBins bins, CtaChunks hubs, uint32_t* p,
                                                              const uint32_t* __restrict__ marked,
                                                              const uint32_t* __restrict__ giant_p) {
  VRange r = vbins_range(bins);
  const uint32_t lane = lane_id();
  const bool any = __ldg(giant_p + 1) != 0;
  if (r.role == kRoleThread) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      if (cc_marked(marked, v)) continue;
      Seg s = g.seg(v);
      for (uint32_t k = 0; k < s.len; ++k) {
        const uint32_t u = __ldg(s.p + k);
        if (u < v) cc_union(p, u, v);
        else if (!any) break;
        else if (cc_marked(marked, u)) cc_union(p, u, v);
      }
    }
  } else if (r.role == kRoleWarp) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      if (cc_marked(marked, v)) continue;
      Seg s = g.seg(v);
      for (uint32_t base = 0; base < s.len; base += 32) {
        const uint32_t k = base + lane;
        const uint32_t u = k < s.len ? __ldg(s.p + k) : kInf;
        if (u < v || (any && k < s.len && cc_marked(marked, u))) cc_union(p, u, v);
        if (!any && __ballot_sync(0xFFFFFFFFu, u >= v) != 0) break;
      }
    }
  } else {
    for (uint64_t j = blockIdx.x - bins.nbT - bins.nbW; j < hubs.items; j += bins.nbC) {
      ChunkItem it = chunk_item(hubs, j);
      uint32_t v = __ldg(bins.vorder + it.vidx);
      if (cc_marked(marked, v)) continue;  // uniform over the block
      Seg s = g.seg(v);
      uint32_t lo, hi;
      chunk_range(s.len, it.chunk, it.K, &lo, &hi);
      for (uint32_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        const uint32_t u = __ldg(s.p + k);
        if (u < v || (any && cc_marked(marked, u))) cc_union(p, u, v);
      }
    }
  }
}

// Between the sampling and the final pass: every entry is pointed at its root
// with path-halving finds, which keeps the final pass's membership test short.
// A racing halving write may leave an entry at an ancestor instead of the
// root, which only costs a longer walk later.
__global__ void cc_flatten_kernel(uint32_t* p, uint32_t n) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    p[v] = cc_find(p, (uint32_t)v);
}

// Final labels.  Each thread writes only its own entry: a path-halving write
// here could land after the owner stored the root and replace it with an
// older ancestor, so the walk only reads.  Entries already finished by their
// owners shorten the walks of the others.
__global__ void cc_compress_kernel(uint32_t* p, uint32_t n) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x = (uint32_t)v;
    uint32_t px = ld_cg(p + x);
    while (px != x) {
      x = px;
      px = ld_cg(p + x);
    }
    p[v] = x;
  }
}

template <typename G>
byo_status run_cc(const byo_graph* g, G view, uint32_t* labels, cudaStream_t s) {
  unsigned grid = (unsigned)((uint64_t)sm_count() * 8);
  uint32_t *giant = nullptr, *marked = nullptr;
  BYO_RETURN_IF(tmp_alloc_t(&giant, 2, s, "CC large-component root"));
  if (tmp_alloc_t(&marked, (g->n + 31) / 32, s, "CC large-component marks") != BYO_OK) {
    tmp_free(giant, s);
    return BYO_ERR_OUT_OF_MEMORY;
  }
  VBins bins = make_vbins(g, 5, 11, kCcThreads);
  CtaChunks hubs = make_cta_chunks(g, 12, 12);  // degrees >= 2048, chunks of <= 4096 ids
  {
    uint64_t cap = (uint64_t)sm_count() * 8;
    bins.nbC = (uint32_t)(hubs.items < cap ? hubs.items : cap);
  }
  byo_status st = BYO_OK;
  {
    ProfScope ps("cc_sample", s);
    cc_identity_kernel<<<grid, kCcThreads, 0, s>>>(labels, g->n);
    cc_sample_kernel<<<grid, kCcThreads, 0, s>>>(view, labels, 0u);
    cc_sample_kernel<<<grid, kCcThreads, 0, s>>>(view, labels, 1u);
    cc_flatten_kernel<<<grid, kCcThreads, 0, s>>>(labels, g->n);
    cc_giant_kernel<<<1, kGiantSample, 0, s>>>(labels, g->n, giant);
    cc_mark_kernel<<<grid, kCcThreads, 0, s>>>(labels, g->n, giant, marked);
    ::byo::note_launch(6);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_status(e, "cc sampling");
  }
  if (st == BYO_OK) {
    ProfScope ps("cc_final", s);
    cc_final_kernel<<<vbins_grid(bins), kCcThreads, 0, s>>>(view, bins, hubs, labels, marked, giant);
    cc_compress_kernel<<<grid, kCcThreads, 0, s>>>(labels, g->n);
    ::byo::note_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_status(e, "cc final pass");
  }
  tmp_free(giant, s);
  tmp_free(marked, s);
  return st;
}

}  // namespace
}  // namespace byo

using namespace byo;

extern "C" byo_status byo_cc(const byo_graph* g, uint32_t* labels, void* stream) {
  clear_error();
  BYO_RETURN_IF(ready_graph(g, static_cast<cudaStream_t>(stream)));
  if (g->n == 0) return BYO_OK;
  if (!labels) {
    set_error("byo_cc: NULL labels");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return with_view(g, [&](auto view) { return run_cc(g, view, labels, s); });
}
