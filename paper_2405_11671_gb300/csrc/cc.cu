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
// even sample of vertices share is then taken as the large component; a final
// pass links every neighbour of the vertices outside that component only.  An edge whose two
// ends are both in the large component needs no link, and an edge with one end
// outside is linked from that end, so every edge is covered.
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
  if (t == 0) *giant = (uint32_t)(best & 0xFFFFFFFFull);
}

// Final pass: the vertices outside the large component link every neighbour
// (the first two again as well; repeated links are no-ops).  Threads, warps or CTA chunks by degree, as in the other kernels.
template <typename G>
__global__ void __launch_bounds__(kCcThreads) cc_final_kernel(G g, VBins bins, CtaChunks hubs, uint32_t* p,
                                                              const uint32_t* giant_p) {
  VRange r = vbins_range(bins);
  const uint32_t lane = lane_id();
  const uint32_t giant = __ldg(giant_p);
  if (r.role == kRoleThread) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      if (cc_find(p, v) == giant) continue;
      Seg s = g.seg(v);
      for (uint32_t k = 0; k < s.len; ++k) cc_union(p, __ldg(s.p + k), v);
    }
  } else if (r.role == kRoleWarp) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      if (__shfl_sync(0xFFFFFFFFu, lane == 0 ? cc_find(p, v) : 0u, 0) == giant) continue;
      Seg s = g.seg(v);
      for (uint32_t k = lane; k < s.len; k += 32) cc_union(p, __ldg(s.p + k), v);
    }
  } else {
    __shared__ uint32_t root_s;
    for (uint64_t j = blockIdx.x - bins.nbT - bins.nbW; j < hubs.items; j += bins.nbC) {
      ChunkItem it = chunk_item(hubs, j);
      uint32_t v = __ldg(bins.vorder + it.vidx);
      if (threadIdx.x == 0) root_s = cc_find(p, v);
      __syncthreads();
      const bool skip = root_s == giant;
      __syncthreads();
      if (skip) continue;
      Seg s = g.seg(v);
      uint32_t lo, hi;
      chunk_range(s.len, it.chunk, it.K, &lo, &hi);
      for (uint32_t k = lo + threadIdx.x; k < hi; k += blockDim.x) cc_union(p, __ldg(s.p + k), v);
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
  uint32_t* giant = nullptr;
  BYO_RETURN_IF(tmp_alloc_t(&giant, 1, s, "CC large-component root"));
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
    ::byo::note_launch(5);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_status(e, "cc sampling");
  }
  if (st == BYO_OK) {
    ProfScope ps("cc_final", s);
    cc_final_kernel<<<vbins_grid(bins), kCcThreads, 0, s>>>(view, bins, hubs, labels, giant);
    cc_compress_kernel<<<grid, kCcThreads, 0, s>>>(labels, g->n);
    ::byo::note_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_status(e, "cc final pass");
  }
  tmp_free(giant, s);
  return st;
}

}  // namespace
}  // namespace byo

using namespace byo;

extern "C" byo_status byo_cc(const byo_graph* g, uint32_t* labels, void* stream) {
  clear_error();
  BYO_RETURN_IF(check_graph(g));
  if (g->n == 0) return BYO_OK;
  if (!labels) {
    set_error("byo_cc: NULL labels");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return with_view(g, [&](auto view) { return run_cc(g, view, labels, s); });
}
