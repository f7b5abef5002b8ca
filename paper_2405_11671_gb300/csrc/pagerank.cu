// pagerank.cu -- PageRank (named in Section 6.2) as a pull over N(v):
//   p_0 = 1/n,  p_{t+1}(v) = (1-d)/n + d*( sum_{u in N(v)} c_t(u) + D_t/n ),
//   c_t(u) = p_t(u)/deg(u) in FP32,  D_t = sum of p_t over degree-0 vertices.
// Per vertex the gather is summed with Neumaier-compensated FP32 arithmetic
// (lanes of a warp or CTA combine their partial (sum, error) pairs with an
// error-free TwoSum).  The dangling mass D_t and the L1 residual are reduced in
// FP64: per-block partials, then the last block to finish adds them in block
// order (deterministic) and prepares the next iteration's constant term.  The
// next contributions c_{t+1}(v) are written by the same kernel (fused).
//
// The iterations run on a copy of the graph relabelled by degree order
// (rank.cuh), rebuilt by every call: vertices of equal degree class become
// consecutive ids (the degree bins need no index array and are walked in
// order), and the contributions of the high-degree vertices, which most
// gathers read, share a short range of cache lines (L1 and L2 hits).  Each
// vertex keeps its neighbour order, so the sums are the ones of the original
// labels; the ranks are scattered back to the caller's ids at the end.
#include <math.h>

#include "byo_internal.cuh"
#include "prof.cuh"
#include "container.cuh"
#include "vbins.cuh"
#include "rank.cuh"

namespace byo {

struct PrWork {
  uint32_t n = 0;
  // the init + iteration launches of the last call, captured as a CUDA graph
  cudaGraphExec_t exec = nullptr;
  uint64_t exec_version = ~0ull;
  uint32_t exec_iters = 0;
  float exec_damping = 0.f;
  float* exec_ranks = nullptr;
  float2* part = nullptr;      // per hub chunk: compensated partial (sum, error)
  uint64_t part_cap = 0;
  uint32_t* hub_ticket = nullptr;  // per hub: chunks finished this iteration
  uint64_t ticket_cap = 0;
  float* c[2] = {nullptr, nullptr};
  double* partials = nullptr;  // 2 per block
  uint32_t max_blocks = 0;
  double* scal = nullptr;      // [0] = D_t, [1] = residual, [2] = base term
  uint32_t* ticket = nullptr;
  // the relabelled copy: rank[v], CSR (roff, rcol) over ranks, ranks by rank
  uint64_t m_cap = 0;
  uint32_t* rank = nullptr;
  uint32_t* rdeg = nullptr;
  uint64_t* roff = nullptr;
  uint32_t* rcol = nullptr;
  float* rranks = nullptr;
};

void pr_free(PrWork* w) {
  if (!w) return;
  if (w->exec) cudaGraphExecDestroy(w->exec);
  dev_free(w->c[0]);
  dev_free(w->c[1]);
  dev_free(w->part);
  dev_free(w->hub_ticket);
  dev_free(w->partials);
  dev_free(w->scal);
  dev_free(w->ticket);
  dev_free(w->rank);
  dev_free(w->rdeg);
  dev_free(w->roff);
  dev_free(w->rcol);
  dev_free(w->rranks);
  delete w;
}

namespace {

constexpr int kPrThreads = 256;

struct Comp {
  float s, c;
};

__device__ __forceinline__ void neumaier_add(Comp& a, float x) {
  float t = a.s + x;
  if (fabsf(a.s) >= fabsf(x)) a.c += (a.s - t) + x;
  else a.c += (x - t) + a.s;
  a.s = t;
}

// a + b exactly as (sum, error), then fold both errors in
__device__ __forceinline__ Comp comp_merge(Comp a, Comp b) {
  float t = a.s + b.s;
  float bp = t - a.s;
  float e = (a.s - (t - bp)) + (b.s - bp);
  return Comp{t, a.c + b.c + e};
}

__device__ __forceinline__ Comp warp_comp_sum(Comp a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Comp b{__shfl_xor_sync(0xFFFFFFFFu, a.s, o), __shfl_xor_sync(0xFFFFFFFFu, a.c, o)};
    a = comp_merge(a, b);
  }
  return a;
}

__device__ __forceinline__ double block_sum_f64(double x, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
  __syncthreads();
  if (lane_id() == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
  }
  return t;  // valid in thread 0
}

// Last block in: fold the per-block partials in block order.
__device__ __forceinline__ void finish_reduction(double res, double dang, double* partials, double* scal,
                                                 uint32_t* ticket, float damping, uint32_t n) {
  __shared__ double sh[32];
  __shared__ bool last;
  double r = block_sum_f64(res, sh);
  double d = block_sum_f64(dang, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = r;
    partials[2 * blockIdx.x + 1] = d;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  // the whole block folds the partials: thread t the blocks t, t + T, ... in
  // order, then a fixed tree over the threads (deterministic; one thread
  // alone would take thousands of dependent L2 round trips)
  __threadfence();
  double R = 0.0, D = 0.0;
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    R += __ldcg(partials + 2 * b);
    D += __ldcg(partials + 2 * b + 1);
  }
  R = block_sum_f64(R, sh);
  D = block_sum_f64(D, sh);
  if (threadIdx.x == 0) {
    scal[0] = D;
    scal[1] = R;
    scal[2] = (1.0 - (double)damping) / (double)n + (double)damping * D / (double)n;
    *ticket = 0;
  }
}

template <typename G>
__global__ void __launch_bounds__(kPrThreads) pr_init_kernel(G g, float* ranks, float* c, double* partials,
                                                             double* scal, uint32_t* ticket, float damping) {
  const uint32_t n = g.num_vertices();
  const float p0 = (float)(1.0 / (double)n);
  double dang = 0.0;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t d = g.degree((uint32_t)v);
    ranks[v] = p0;
    c[v] = d ? p0 / (float)d : 0.0f;
    if (d == 0) dang += (double)p0;
  }
  finish_reduction(0.0, dang, partials, scal, ticket, damping, n);
}

// L2 eviction priorities: the neighbour ids stream through once per
// iteration (4 bytes per stored edge, gigabytes), the contributions are
// gathered at random (4 bytes per vertex, tens of megabytes): the ids are
// marked evict-first so that they do not push the contributions out of L2,
// and the contributions evict-last.  (The policy registers are pure values;
// the compiler hoists their creation out of the loops.)
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Neighbour ids are read once per iteration: keep them out of L1, which is
// left to the contributions, and first in line for eviction from L2.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) {
  uint32_t x;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(x) : "l"(p), "l"(l2_evict_first()));
  return x;
}

// A contribution: kept in L2 as long as possible.
__device__ __forceinline__ float ld_contrib(const float* p) {
  float x;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(x) : "l"(p), "l"(l2_evict_last()));
  return x;
}

template <typename G>
__device__ __forceinline__ void pr_store(G& g, uint32_t v, uint32_t deg, Comp acc, float d, float base,
                                         float* ranks, float* cn, double& res, double& dang) {
  float s = acc.s + acc.c;
  float pn = fmaf(d, s, base);
  float old = ranks[v];
  ranks[v] = pn;
  // a degree-0 vertex is in no neighbour list, so its contribution is never
  // gathered and is not written
  if (deg) cn[v] = pn / (float)deg;
  res += fabs((double)pn - (double)old);
  if (deg == 0) dang += (double)pn;
}


// Compensated sum of c[ids[k]] for k = first, first+stride, ... < len, with
// eight independent id loads and eight independent gathers in flight per step
// (four, two and one for the tail).
__device__ __forceinline__ void gather_sum(Comp& acc, const uint32_t* __restrict__ ids, uint32_t first, uint32_t len,
                                           uint32_t stride, const float* __restrict__ c) {
  uint32_t k = first;
  for (; k + 7 * stride < len; k += 8 * stride) {
    uint32_t u[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) u[j] = ld_stream(ids + k + j * stride);
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = ld_contrib(c + u[j]);
#pragma unroll
    for (int j = 0; j < 8; ++j) neumaier_add(acc, x[j]);
  }
  if (k + 3 * stride < len) {  // the tail: four, two, one more
    uint32_t u[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = ld_stream(ids + k + j * stride);
    float x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = ld_contrib(c + u[j]);
#pragma unroll
    for (int j = 0; j < 4; ++j) neumaier_add(acc, x[j]);
    k += 4 * stride;
  }
  if (k + stride < len) {
    const uint32_t u0 = ld_stream(ids + k), u1 = ld_stream(ids + k + stride);
    const float x0 = ld_contrib(c + u0), x1 = ld_contrib(c + u1);
    neumaier_add(acc, x0);
    neumaier_add(acc, x1);
    k += 2 * stride;
  }
  if (k < len) neumaier_add(acc, ld_contrib(c + ld_stream(ids + k)));
}

// Low-degree vertices (degree < small_lim) are processed in id order, 32 per
// warp: the warp walks the concatenation of their neighbour lists 32 ids at a
// time (coalesced id reads, 32 independent contribution gathers per step),
// merges the per-lane values of each vertex with a segmented warp scan built
// on the error-free TwoSum, and every lane keeps the compensated sum of its own
// vertex.  Ranks and contributions of those vertices are stored coalesced.
template <typename G>
__device__ __forceinline__ void pr_stream_warp(const G& g, uint32_t v0, uint32_t small_lim, float damping,
                                               float base, const float* __restrict__ c, float* __restrict__ cn,
                                               float* ranks, double& res, double& dang) {
  const uint32_t lane = lane_id();
  const uint32_t n = g.num_vertices();
  const uint32_t v = v0 + lane;
  Seg s{nullptr, 0};
  uint32_t deg = 0;
  if (v < n) {
    s = g.seg(v);
    deg = s.len;
  }
  const uint32_t len = deg < small_lim ? deg : 0;
  uint32_t incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  const uint32_t excl = incl - len;
  Comp acc{0.f, 0.f};
  constexpr int kU = 2;  // chunks of 32 ids per step: kU independent gathers per lane in flight
  for (uint32_t e00 = 0; e00 < total; e00 += 32 * kU) {
    int key[kU];
    uint32_t id[kU];
    float x[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const uint32_t e = e00 + 32 * j + lane;
      int owner = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        int probe = owner + step;
        uint32_t ex = __shfl_sync(0xFFFFFFFFu, excl, probe & 31);
        if (probe < 32 && ex <= e) owner = probe;
      }
      const uint32_t oex = __shfl_sync(0xFFFFFFFFu, excl, owner);
      const uint32_t* op = reinterpret_cast<const uint32_t*>(
          __shfl_sync(0xFFFFFFFFu, reinterpret_cast<unsigned long long>(s.p), owner));
      key[j] = e < total ? owner : 32;
      id[j] = e < total ? ld_stream(op + (e - oex)) : 0u;
    }
#pragma unroll
    for (int j = 0; j < kU; ++j) x[j] = key[j] < 32 ? ld_contrib(c + id[j]) : 0.f;
    for (int j = 0; j < kU; ++j) {
      const uint32_t e0 = e00 + 32 * j;
      if (e0 >= total) break;  // warp-uniform
      Comp val{x[j], 0.f};
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        float ys = __shfl_up_sync(0xFFFFFFFFu, val.s, o);
        float yc = __shfl_up_sync(0xFFFFFFFFu, val.c, o);
        int yk = __shfl_up_sync(0xFFFFFFFFu, key[j], o);
        if ((int)lane >= o && yk == key[j]) val = comp_merge(Comp{ys, yc}, val);
      }
      // this lane's vertex: its ids in this chunk end at lane hi-1-e0
      const uint32_t lo = excl > e0 ? excl : e0;
      const uint32_t hi = (excl + len) < (e0 + 32) ? (excl + len) : (e0 + 32);
      const int srcl = hi > lo ? (int)(hi - 1 - e0) : (int)lane;
      Comp part{__shfl_sync(0xFFFFFFFFu, val.s, srcl), __shfl_sync(0xFFFFFFFFu, val.c, srcl)};
      if (hi > lo) acc = comp_merge(acc, part);
    }
  }
  if (v < n && deg < small_lim) pr_store(g, v, deg, acc, damping, base, ranks, cn, res, dang);
}

template <typename G>
__global__ void __launch_bounds__(kPrThreads, 8) pr_iter_kernel(G g, VBins bins, CtaChunks hubs, uint32_t small_lim,
                                                             uint32_t stream_n, float damping, const float* __restrict__ c,
                                                             float* __restrict__ cn, float* ranks, float2* part,
                                                             uint32_t* hub_ticket, double* partials, double* scal,
                                                             uint32_t* ticket) {
  const uint32_t n = g.num_vertices();
  const float base = (float)__ldcg(scal + 2);
  VRange r = vbins_range(bins);
  const uint32_t lane = lane_id();
  double res = 0.0, dang = 0.0;
  if (r.role == kRoleThread) {
    const uint32_t wpb = blockDim.x >> 5;
    const uint64_t wt = (uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
    const uint64_t nw = (uint64_t)bins.nbT * wpb;
    for (uint64_t v0 = wt * 32; v0 < stream_n; v0 += nw * 32)
      pr_stream_warp(g, (uint32_t)v0, small_lim, damping, base, c, cn, ranks, res, dang);
  } else if (r.role == kRoleWarp) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = vbins_vertex(bins, i);
      Seg s = g.seg(v);
      Comp acc{0.f, 0.f};
      gather_sum(acc, s.p, lane, s.len, 32, c);
      acc = warp_comp_sum(acc);
      if (lane == 0) pr_store(g, v, s.len, acc, damping, base, ranks, cn, res, dang);
    }
  } else {
    // high degree: chunks spread over CTAs; the last chunk of a vertex to finish
    // folds the chunk partials in chunk order and stores the vertex
    __shared__ Comp sh[kPrThreads / 32];
    for (uint64_t j = blockIdx.x - bins.nbT - bins.nbW; j < hubs.items; j += bins.nbC) {
      ChunkItem it = chunk_item(hubs, j);
      uint32_t v = vbins_vertex(bins, it.vidx);
      Seg s = g.seg(v);
      uint32_t lo, hi;
      chunk_range(s.len, it.chunk, it.K, &lo, &hi);
      Comp acc{0.f, 0.f};
      gather_sum(acc, s.p, lo + threadIdx.x, hi, blockDim.x, c);
      acc = warp_comp_sum(acc);
      if (lane == 0) sh[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x < 32) {
        Comp a = lane < (blockDim.x >> 5) ? sh[lane] : Comp{0.f, 0.f};
        a = warp_comp_sum(a);
        if (it.K == 1) {
          if (threadIdx.x == 0) pr_store(g, v, s.len, a, damping, base, ranks, cn, res, dang);
        } else {
          uint32_t* t = hub_ticket + (it.vidx - hubs.vbegin);
          bool last_chunk = false;
          if (threadIdx.x == 0) {
            part[j] = make_float2(a.s, a.c);
            __threadfence();
            last_chunk = atomicAdd(t, 1u) == it.K - 1;
          }
          // the last chunk to finish folds the vertex's chunk partials: lane
          // l the chunks l, l + 32, ... in order, then the warp's fixed tree
          if (__shfl_sync(0xFFFFFFFFu, last_chunk, 0)) {
            __threadfence();
            Comp tot{0.f, 0.f};
            for (uint32_t q = lane; q < it.K; q += 32) {
              const float2 pq = __ldcg(part + it.first + q);
              tot = comp_merge(tot, Comp{pq.x, pq.y});
            }
            tot = warp_comp_sum(tot);
            if (threadIdx.x == 0) {
              pr_store(g, v, s.len, tot, damping, base, ranks, cn, res, dang);
              *t = 0;
            }
          }
        }
      }
      __syncthreads();
    }
  }
  finish_reduction(res, dang, partials, scal, ticket, damping, n);
}

// ---------------------------------------------------------------- relabelled copy
// degree of rank r, from the sorted (degree << lbn | v) keys
__global__ void pr_rdeg_kernel(const uint64_t* __restrict__ sorted, uint32_t n, int lbn, uint32_t* __restrict__ rdeg) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x)
    rdeg[r] = (uint32_t)(sorted[r] >> lbn);
}

__global__ void pr_set_last_kernel(uint64_t* off, uint32_t n, uint64_t total) { off[n] = total; }

// rcol[roff[rank v] + k] = rank(k-th neighbour of v): thread, warp or CTA per
// vertex by degree, neighbour order kept.
template <typename G>
__global__ void __launch_bounds__(kPrThreads) pr_relabel_kernel(G g, VBins bins, const uint32_t* __restrict__ rank,
                                                                const uint64_t* __restrict__ roff,
                                                                uint32_t* __restrict__ rcol) {
  VRange r = vbins_range(bins);
  const uint32_t lane = lane_id();
  uint32_t first = 0, step = 1;
  if (r.role == kRoleWarp) {
    first = lane;
    step = 32;
  } else if (r.role == kRoleCta) {
    first = threadIdx.x;
    step = blockDim.x;
  }
  for (uint64_t i = r.begin; i < r.end; i += r.stride) {
    const uint32_t v = vbins_vertex(bins, i);
    const Seg sg = g.seg(v);
    uint32_t* out = rcol + roff[__ldg(rank + v)];
    // eight ids, then their eight ranks, in flight before the stores
    for (uint32_t k = first; k < sg.len; k += 8 * step) {
      uint32_t u[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) u[j] = k + j * step < sg.len ? ld_stream(sg.p + k + j * step) : 0u;
      uint32_t ru[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) ru[j] = k + j * step < sg.len ? __ldg(rank + u[j]) : 0u;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (k + j * step < sg.len) out[k + j * step] = ru[j];
    }
  }
}

// the caller's ranks, by vertex id
__global__ void pr_unrelabel_kernel(const uint32_t* __restrict__ rank, const float* __restrict__ rranks, uint32_t n,
                                    float* __restrict__ ranks) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    ranks[v] = rranks[__ldg(rank + v)];
}

byo_status ensure_pr_work(byo_graph* g, uint32_t blocks, uint64_t parts, uint64_t hubs) {
  if (g->pr && g->pr->max_blocks >= blocks && g->pr->part_cap >= parts && g->pr->ticket_cap >= hubs &&
      g->pr->m_cap >= g->m)
    return BYO_OK;
  if (g->pr) {
    pr_free(g->pr);
    g->pr = nullptr;
  }
  PrWork* w = new (std::nothrow) PrWork();
  if (!w) {
    set_error("host allocation failed");
    return BYO_ERR_OUT_OF_MEMORY;
  }
  w->n = g->n;
  w->max_blocks = blocks;
  byo_status st = dev_alloc_t(&w->c[0], g->n, "PageRank contributions");
  if (st == BYO_OK) st = dev_alloc_t(&w->c[1], g->n, "PageRank contributions");
  if (st == BYO_OK) st = dev_alloc_t(&w->partials, 2ull * blocks, "PageRank partials");
  w->part_cap = parts + 64;
  w->ticket_cap = hubs + 64;
  if (st == BYO_OK) st = dev_alloc_t(&w->part, w->part_cap, "PageRank hub partials");
  if (st == BYO_OK) st = dev_alloc_t(&w->hub_ticket, w->ticket_cap, "PageRank hub tickets");
  if (st == BYO_OK) {
    cudaError_t e = cudaMemset(w->hub_ticket, 0, sizeof(uint32_t) * w->ticket_cap);
    if (e != cudaSuccess) st = cuda_status(e, "cudaMemset");
  }
  w->m_cap = g->m + (g->dyn ? g->m / 8 : 0);  // headroom for later inserts
  if (st == BYO_OK) st = dev_alloc_t(&w->rank, g->n, "PageRank degree order");
  if (st == BYO_OK) st = dev_alloc_t(&w->rdeg, g->n, "PageRank relabelled degrees");
  if (st == BYO_OK) st = dev_alloc_t(&w->roff, g->n + 1ull, "PageRank relabelled offsets");
  if (st == BYO_OK) st = dev_alloc_t(&w->rcol, w->m_cap + 8, "PageRank relabelled neighbours");
  if (st == BYO_OK) st = dev_alloc_t(&w->rranks, g->n, "PageRank ranks by degree order");
  if (st == BYO_OK) st = dev_alloc_t(&w->scal, 4, "PageRank scalars");
  if (st == BYO_OK) st = dev_alloc_t(&w->ticket, 1, "PageRank ticket");
  if (st == BYO_OK) {
    cudaError_t e = cudaMemset(w->ticket, 0, sizeof(uint32_t));
    if (e != cudaSuccess) st = cuda_status(e, "cudaMemset");
  }
  if (st != BYO_OK) {
    pr_free(w);
    return st;
  }
  g->pr = w;
  return BYO_OK;
}

template <typename G>
byo_status run_pr(byo_graph* g, G view, float damping, uint32_t iters, float* ranks, double* host_residual,
                  cudaStream_t s) {
  constexpr int kSmallBucket = 8;  // degree < 256 goes to the warp stream
  const uint32_t n = g->n;
  // bins of the relabelled copy: bucket b holds the ranks [bstart[b], bstart[b+1])
  VBins bins = make_vbins(g, kSmallBucket, 10, kPrThreads);
  bins.vorder = nullptr;
  const uint32_t stream_n = (uint32_t)bins.t1;
  {
    uint64_t want = ((uint64_t)stream_n + 32ull * (kPrThreads / 32) - 1) / (32ull * (kPrThreads / 32));
    uint64_t cap = (uint64_t)sm_count() * 8;
    bins.nbT = (uint32_t)(want < cap ? (want ? want : 1) : cap);
  }
  // degrees >= 1024 in chunks of at most 65,536 ids: a CTA sums a whole list
  // (few partials and tickets), only the largest hubs are split over CTAs
  CtaChunks hubs = make_cta_chunks(g, 11, 16);
  {
    uint64_t cap = (uint64_t)sm_count() * 8;
    bins.nbC = (uint32_t)(hubs.items < cap ? hubs.items : cap);
  }
  uint32_t grid = vbins_grid(bins);
  uint32_t init_grid = (uint32_t)sm_count() * 4;
  BYO_RETURN_IF(ensure_pr_work(g, grid > init_grid ? grid : init_grid, hubs.items, hubs.vcount));
  PrWork* w = g->pr;
  // the relabelled copy
  {
    ProfScope ps("pr_relabel", s);
    uint64_t* sorted = nullptr;
    BYO_RETURN_IF(degree_rank(g, view, w->rank, &sorted, s));
    pr_rdeg_kernel<<<grid_for(n, 256), 256, 0, s>>>(sorted, n, id_bits(n), w->rdeg);
    ::byo::note_launch();
    tmp_free(sorted, s);
    BYO_CHECK_LAUNCH("pr_rdeg_kernel");
    BYO_RETURN_IF(scan_u32_to_u64(w->rdeg, w->roff, n, nullptr, s));
    pr_set_last_kernel<<<1, 1, 0, s>>>(w->roff, n, g->m);
    ::byo::note_launch();
    VBins fb = make_vbins(g, 4, 10, kPrThreads);
    pr_relabel_kernel<<<vbins_grid(fb), kPrThreads, 0, s>>>(view, fb, w->rank, w->roff, w->rcol);
    ::byo::note_launch();
    BYO_CHECK_LAUNCH("pr_relabel_kernel");
  }
  const CsrView<uint64_t> rv{n, g->m, w->roff, w->rcol};
  auto launch_all = [&]() -> byo_status {
    {
      ProfScope ps("pr_init", s);
      pr_init_kernel<<<init_grid, kPrThreads, 0, s>>>(rv, w->rranks, w->c[0], w->partials, w->scal, w->ticket,
                                                       damping);
      ::byo::note_launch();
    }
    BYO_CHECK_LAUNCH("pr_init_kernel");
    for (uint32_t t = 0; t < iters; ++t) {
      ProfScope ps("pr_iter", s);
      pr_iter_kernel<<<grid, kPrThreads, 0, s>>>(rv, bins, hubs, 1u << kSmallBucket, stream_n, damping, w->c[t & 1],
                                                 w->c[(t + 1) & 1], w->rranks, w->part, w->hub_ticket, w->partials,
                                                 w->scal, w->ticket);
      ::byo::note_launch();
      BYO_CHECK_LAUNCH("pr_iter_kernel");
    }
    pr_unrelabel_kernel<<<grid_for(n, 256), 256, 0, s>>>(w->rank, w->rranks, n, ranks);
    ::byo::note_launch();
    BYO_CHECK_LAUNCH("pr_unrelabel_kernel");
    return BYO_OK;
  };
  // On a non-default stream (stream capture needs one) and with profiling
  // off, the iterations run as one CUDA graph, captured once per (graph
  // version, iterations, damping, output) and replayed.
  if (s != nullptr && !profiling_on()) {
    if (!(w->exec && w->exec_version == g->version && w->exec_iters == iters && w->exec_damping == damping &&
          w->exec_ranks == ranks)) {
      if (w->exec) {
        cudaGraphExecDestroy(w->exec);
        w->exec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      BYO_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      byo_status st = launch_all();
      cudaError_t e = cudaStreamEndCapture(s, &graph);
      if (st != BYO_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&w->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        w->exec = nullptr;
        return cuda_status(e, "cudaGraphInstantiate");
      }
      w->exec_version = g->version;
      w->exec_iters = iters;
      w->exec_damping = damping;
      w->exec_ranks = ranks;
    } else {
      note_launch(2 + iters);  // the replay launches the same kernels
    }
    BYO_CUDA(cudaGraphLaunch(w->exec, s));
  } else {
    BYO_RETURN_IF(launch_all());
  }
  if (host_residual) {
    double r = 0.0;
    BYO_CUDA(cudaMemcpyAsync(&r, w->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    BYO_CUDA(cudaStreamSynchronize(s));
    *host_residual = iters ? r : 0.0;
  }
  return BYO_OK;
}

}  // namespace
}  // namespace byo

using namespace byo;

extern "C" byo_status byo_pagerank(const byo_graph* gc, float damping, uint32_t iters, float* ranks,
                                   double* host_residual, void* stream) {
  clear_error();
  BYO_RETURN_IF(ready_graph(gc, static_cast<cudaStream_t>(stream)));
  byo_graph* g = const_cast<byo_graph*>(gc);
  if (!(damping >= 0.0f && damping <= 1.0f)) {
    set_error("byo_pagerank: damping must be in [0, 1]");
    return BYO_ERR_INVALID_ARG;
  }
  if (g->n == 0) {
    if (host_residual) *host_residual = 0.0;
    return BYO_OK;
  }
  if (!ranks) {
    set_error("byo_pagerank: NULL ranks");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return with_view(g, [&](auto view) { return run_pr(g, view, damping, iters, ranks, host_residual, s); });
}
