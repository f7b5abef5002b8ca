// cc.cu -- connected components (the paper's connectivity algorithm, Section
// 6.2) as a concurrent union-find over every edge.  Every parent pointer goes
// from a larger id to a smaller one (hooks attach the larger root under the
// smaller), so the root of each finished tree is the minimum id of its
// component and the labels come out canonical without a relabelling pass.
// Because neighbour lists are sorted ascending (CSR, Section 4.2), the
// neighbours below v form a prefix and each undirected edge is visited once,
// from its larger endpoint, with an early exit (map_neighbors_early_exit).
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

// parent[v] = smallest neighbour if it is below v, else v
template <typename G>
__global__ void cc_init_kernel(G g, uint32_t* p) {
  const uint32_t n = g.num_vertices();
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    Seg s = g.seg((uint32_t)v);
    uint32_t first = s.len ? __ldg(s.p) : kInf;
    p[v] = first < v ? first : (uint32_t)v;
  }
}

template <typename G>
__global__ void __launch_bounds__(kCcThreads) cc_hook_kernel(G g, VBins bins, CtaChunks hubs, uint32_t* p) {
  VRange r = vbins_range(bins);
  const uint32_t lane = lane_id();
  if (r.role == kRoleThread) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      for (uint32_t k = 1; k < s.len; ++k) {  // k = 0 was hooked by the init
        uint32_t u = __ldg(s.p + k);
        if (u >= v) break;
        cc_union(p, u, v);
      }
    }
  } else if (r.role == kRoleWarp) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      for (uint32_t base = 1; base < s.len; base += 32) {
        uint32_t k = base + lane;
        uint32_t u = k < s.len ? __ldg(s.p + k) : kInf;
        if (u < v) cc_union(p, u, v);
        if (__ballot_sync(0xFFFFFFFFu, u >= v) != 0) break;
      }
    }
  } else {
    // high degree: chunks of the list spread over CTAs (unions are independent)
    __shared__ int stop;
    for (uint64_t j = blockIdx.x - bins.nbT - bins.nbW; j < hubs.items; j += bins.nbC) {
      ChunkItem it = chunk_item(hubs, j);
      uint32_t v = __ldg(bins.vorder + it.vidx);
      Seg s = g.seg(v);
      uint32_t lo, hi;
      chunk_range(s.len, it.chunk, it.K, &lo, &hi);
      if (lo == 0) lo = 1;  // entry 0 was hooked by the init
      for (uint32_t base = lo; base < hi; base += blockDim.x) {
        if (threadIdx.x == 0) stop = 0;
        __syncthreads();
        uint32_t k = base + threadIdx.x;
        uint32_t u = k < hi ? __ldg(s.p + k) : kInf;
        if (u < v) cc_union(p, u, v);
        else stop = 1;
        __syncthreads();
        if (stop) break;
      }
      __syncthreads();
    }
  }
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
  {
    ProfScope ps("cc_init", s);
    cc_init_kernel<<<grid, kCcThreads, 0, s>>>(view, labels); ::byo::note_launch();
  }
  BYO_CHECK_LAUNCH("cc_init_kernel");
  VBins bins = make_vbins(g, 5, 11, kCcThreads);
  CtaChunks hubs = make_cta_chunks(g, 12, 12);  // degrees >= 2048, chunks of <= 4096 ids
  {
    uint64_t cap = (uint64_t)sm_count() * 8;
    bins.nbC = (uint32_t)(hubs.items < cap ? hubs.items : cap);
  }
  {
    ProfScope ps("cc_hook", s);
    cc_hook_kernel<<<vbins_grid(bins), kCcThreads, 0, s>>>(view, bins, hubs, labels); ::byo::note_launch();
  }
  BYO_CHECK_LAUNCH("cc_hook_kernel");
  {
    ProfScope ps("cc_compress", s);
    cc_compress_kernel<<<grid, kCcThreads, 0, s>>>(labels, g->n); ::byo::note_launch();
  }
  BYO_CHECK_LAUNCH("cc_compress_kernel");
  return BYO_OK;
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
