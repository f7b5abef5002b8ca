// pagerank.cu -- PageRank (named in Section 6.2) as a pull over N(v):
//   p_0 = 1/n,  p_{t+1}(v) = (1-d)/n + d*( sum_{u in N(v)} c_t(u) + D_t/n ),
//   c_t(u) = p_t(u)/deg(u) in FP32,  D_t = sum of p_t over degree-0 vertices.
// Per vertex the gather is summed with Neumaier-compensated FP32 arithmetic
// (lanes of a warp or CTA combine their partial (sum, error) pairs with an
// error-free TwoSum).  The dangling mass D_t and the L1 residual are reduced in
// FP64: per-block partials, then the last block to finish adds them in block
// order (deterministic) and prepares the next iteration's constant term.  The
// next contributions c_{t+1}(v) are written by the same kernel (fused).
#include <math.h>

#include "byo_internal.cuh"
#include "prof.cuh"
#include "container.cuh"
#include "vbins.cuh"

namespace byo {

struct PrWork {
  uint32_t n = 0;
  float* c[2] = {nullptr, nullptr};
  double* partials = nullptr;  // 2 per block
  uint32_t max_blocks = 0;
  double* scal = nullptr;      // [0] = D_t, [1] = residual, [2] = base term
  uint32_t* ticket = nullptr;
};

void pr_free(PrWork* w) {
  if (!w) return;
  dev_free(w->c[0]);
  dev_free(w->c[1]);
  dev_free(w->partials);
  dev_free(w->scal);
  dev_free(w->ticket);
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
  if (threadIdx.x == 0) {
    __threadfence();
    double R = 0.0, D = 0.0;
    for (uint32_t b = 0; b < gridDim.x; ++b) {
      R += __ldcg(partials + 2 * b);
      D += __ldcg(partials + 2 * b + 1);
    }
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

template <typename G>
__device__ __forceinline__ void pr_store(G& g, uint32_t v, uint32_t deg, Comp acc, float d, float base,
                                         float* ranks, float* cn, double& res, double& dang) {
  float s = acc.s + acc.c;
  float pn = fmaf(d, s, base);
  float old = ranks[v];
  ranks[v] = pn;
  cn[v] = deg ? pn / (float)deg : 0.0f;
  res += fabs((double)pn - (double)old);
  if (deg == 0) dang += (double)pn;
}

template <typename G>
__global__ void __launch_bounds__(kPrThreads) pr_iter_kernel(G g, VBins bins, float damping,
                                                             const float* __restrict__ c, float* __restrict__ cn,
                                                             float* ranks, double* partials, double* scal,
                                                             uint32_t* ticket) {
  const uint32_t n = g.num_vertices();
  const float base = (float)__ldcg(scal + 2);
  VRange r = vbins_range(bins);
  const uint32_t lane = lane_id();
  double res = 0.0, dang = 0.0;
  if (r.role == kRoleThread) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      Comp acc{0.f, 0.f};
      for (uint32_t k = 0; k < s.len; ++k) neumaier_add(acc, __ldg(c + __ldg(s.p + k)));
      pr_store(g, v, s.len, acc, damping, base, ranks, cn, res, dang);
    }
  } else if (r.role == kRoleWarp) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      Comp acc{0.f, 0.f};
      for (uint32_t k = lane; k < s.len; k += 32) neumaier_add(acc, __ldg(c + __ldg(s.p + k)));
      acc = warp_comp_sum(acc);
      if (lane == 0) pr_store(g, v, s.len, acc, damping, base, ranks, cn, res, dang);
    }
  } else {
    __shared__ Comp sh[kPrThreads / 32];
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      Comp acc{0.f, 0.f};
      for (uint32_t k = threadIdx.x; k < s.len; k += blockDim.x) neumaier_add(acc, __ldg(c + __ldg(s.p + k)));
      acc = warp_comp_sum(acc);
      if (lane == 0) sh[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x < 32) {
        Comp a = lane < (blockDim.x >> 5) ? sh[lane] : Comp{0.f, 0.f};
        a = warp_comp_sum(a);
        if (threadIdx.x == 0) pr_store(g, v, s.len, a, damping, base, ranks, cn, res, dang);
      }
      __syncthreads();
    }
  }
  finish_reduction(res, dang, partials, scal, ticket, damping, n);
}

byo_status ensure_pr_work(byo_graph* g, uint32_t blocks) {
  if (g->pr && g->pr->max_blocks >= blocks) return BYO_OK;
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

template <typename OffT>
byo_status run_pr(byo_graph* g, float damping, uint32_t iters, float* ranks, double* host_residual,
                  cudaStream_t s) {
  CsrView<OffT> view{g->n, g->m, static_cast<const OffT*>(g->off), g->col};
  VBins bins = make_vbins(g, 4, 10, kPrThreads);
  uint32_t grid = vbins_grid(bins);
  uint32_t init_grid = (uint32_t)sm_count() * 4;
  BYO_RETURN_IF(ensure_pr_work(g, grid > init_grid ? grid : init_grid));
  PrWork* w = g->pr;
  {
    ProfScope ps("pr_init", s);
    pr_init_kernel<<<init_grid, kPrThreads, 0, s>>>(view, ranks, w->c[0], w->partials, w->scal, w->ticket, damping); ::byo::note_launch();
  }
  BYO_CHECK_LAUNCH("pr_init_kernel");
  for (uint32_t t = 0; t < iters; ++t) {
    ProfScope ps("pr_iter", s);
    pr_iter_kernel<<<grid, kPrThreads, 0, s>>>(view, bins, damping, w->c[t & 1], w->c[(t + 1) & 1], ranks,
                                               w->partials, w->scal, w->ticket); ::byo::note_launch();
    BYO_CHECK_LAUNCH("pr_iter_kernel");
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
  BYO_RETURN_IF(check_graph(gc));
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
  return g->off64 ? run_pr<uint64_t>(g, damping, iters, ranks, host_residual, s)
                  : run_pr<uint32_t>(g, damping, iters, ranks, host_residual, s);
}
