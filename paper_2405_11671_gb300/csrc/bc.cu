// bc.cu -- single-source betweenness centrality (BC in the paper's table of
// algorithms, Section 6.2), by Brandes' accumulation (U. Brandes, "A faster
// algorithm for betweenness centrality", J. Math. Sociology 25(2), 2001):
//   levels    the BFS of bfs.cu from the source (hop distances);
//   forward   sigma(v) = sum of sigma(u) over the neighbours u one level
//             closer (sigma(s) = 1): the number of shortest s-v paths;
//   backward  delta(v) = sum over the neighbours w one level deeper of
//             sigma(v) / sigma(w) * (1 + delta(w)), from the deepest level up;
//             delta(s) = 0.
// Both sweeps are pulls over the container's neighbour lists, level by level:
// every vertex gathers from its own list, so no value is accumulated by
// atomics and the result does not depend on scheduling.  The vertices of a
// level are grouped first (a counting sort by level), split into light
// (degree < kHeavy: eight lanes per vertex) and heavy vertices (a whole CTA
// per vertex).  FP64 throughout: path counts are exact below 2^53.
#include <vector>

#include "byo_internal.cuh"
#include "container.cuh"
#include "prof.cuh"

namespace byo {
namespace {

constexpr int kBcThreads = 256;
constexpr uint32_t kHeavy = 256;  // degree at which a vertex gets a whole CTA
constexpr int kGroup = 8;         // lanes per light vertex

__global__ void bc_init_kernel(uint32_t n, uint32_t src, const uint32_t* __restrict__ level, double* sigma,
                               double* delta, uint32_t* maxl) {
  uint32_t mx = 0;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    sigma[v] = v == src ? 1.0 : 0.0;
    delta[v] = 0.0;
    const uint32_t l = level[v];
    if (l != kInf && l > mx) mx = l;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xFFFFFFFFu, mx, o));
  if (lane_id() == 0 && mx) atomicMax(maxl, mx);
}

// Levels below kBcSmemLevels are counted in shared memory and reach the
// global counters once per CTA (a few popular levels hold most vertices, and
// one address takes about 1.5 G atomics/s); deeper levels, which a deep
// graph spreads thinly, count directly.
constexpr uint32_t kBcSmemLevels = 64;
constexpr int kBcItems = 8;  // vertices per thread per scatter tile

// per level: how many vertices (cnt) and how many of them are light (lcnt)
template <typename G>
__global__ void bc_hist_kernel(G g, const uint32_t* __restrict__ level, uint32_t* cnt, uint32_t* lcnt) {
  __shared__ uint32_t sc[kBcSmemLevels], sl[kBcSmemLevels];
  for (uint32_t i = threadIdx.x; i < kBcSmemLevels; i += blockDim.x) sc[i] = sl[i] = 0;
  __syncthreads();
  const uint32_t n = g.num_vertices();
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t l = level[v];
    if (l == kInf) continue;
    const bool light = g.degree((uint32_t)v) < kHeavy;
    if (l < kBcSmemLevels) {
      atomicAdd(&sc[l], 1u);
      if (light) atomicAdd(&sl[l], 1u);
    } else {
      atomicAdd(cnt + l, 1u);
      if (light) atomicAdd(lcnt + l, 1u);
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kBcSmemLevels; i += blockDim.x) {
    if (sc[i]) atomicAdd(cnt + i, sc[i]);
    if (sl[i]) atomicAdd(lcnt + i, sl[i]);
  }
}

// vertices grouped by level: light ones from the start of their level's range,
// heavy ones from its end.  Per tile of blockDim * kBcItems vertices a CTA
// counts its vertices per level, reserves each level's run with one atomic,
// and places them from shared cursors.
template <typename G>
__global__ void bc_scatter_kernel(G g, const uint32_t* __restrict__ level, const uint64_t* __restrict__ lstart,
                                  uint32_t* lcur, uint32_t* hcur, uint32_t* order) {
  __shared__ uint32_t cl[kBcSmemLevels], ch[kBcSmemLevels], bl[kBcSmemLevels], bh[kBcSmemLevels];
  const uint32_t n = g.num_vertices();
  const uint64_t tile = (uint64_t)blockDim.x * kBcItems;
  for (uint64_t t0 = (uint64_t)blockIdx.x * tile; t0 < n; t0 += (uint64_t)gridDim.x * tile) {
    for (uint32_t i = threadIdx.x; i < kBcSmemLevels; i += blockDim.x) cl[i] = ch[i] = 0;
    __syncthreads();
    uint32_t lv[kBcItems];
    bool light[kBcItems];
#pragma unroll
    for (int k = 0; k < kBcItems; ++k) {
      const uint64_t v = t0 + (uint64_t)k * blockDim.x + threadIdx.x;
      lv[k] = v < n ? level[v] : kInf;
      light[k] = lv[k] != kInf && g.degree((uint32_t)v) < kHeavy;
      if (lv[k] < kBcSmemLevels) atomicAdd(light[k] ? &cl[lv[k]] : &ch[lv[k]], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kBcSmemLevels; i += blockDim.x) {
      bl[i] = cl[i] ? atomicAdd(lcur + i, cl[i]) : 0u;
      bh[i] = ch[i] ? atomicAdd(hcur + i, ch[i]) : 0u;
      cl[i] = 0;
      ch[i] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBcItems; ++k) {
      const uint32_t l = lv[k];
      if (l == kInf) continue;
      const uint64_t v = t0 + (uint64_t)k * blockDim.x + threadIdx.x;
      uint64_t at;
      if (l < kBcSmemLevels) {
        if (light[k]) at = lstart[l] + bl[l] + atomicAdd(&cl[l], 1u);
        else at = lstart[l + 1] - 1 - (bh[l] + atomicAdd(&ch[l], 1u));
      } else {
        if (light[k]) at = lstart[l] + atomicAdd(lcur + l, 1u);
        else at = lstart[l + 1] - 1 - atomicAdd(hcur + l, 1u);
      }
      order[at] = (uint32_t)v;
    }
    __syncthreads();
  }
}

// The gathered value of neighbour u: forward sigma(u), backward
// ratio(u) = (1 + delta(u)) / sigma(u) (kept per vertex, so that a gather
// divides nothing).  Only neighbours at level `want` count.
template <bool kForward>
__device__ __forceinline__ double bc_value(uint32_t u, const double* __restrict__ sigma,
                                           const double* __restrict__ ratio) {
  return kForward ? __ldcg(sigma + u) : __ldcg(ratio + u);
}

// whether u is at the level the sweep gathers from: its bit in `inlvl`, a
// bitmap of that level's vertices (n/8 bytes, L2-resident where the level
// array is not)
__device__ __forceinline__ bool bc_in(const uint32_t* __restrict__ inlvl, uint32_t u) {
  return (__ldg(inlvl + (u >> 5)) >> (u & 31)) & 1u;
}

// Sum over the ids p[k], k = first, first + stride, ... < len, of the values
// of those at the gathered level: four ids, their four bits and then their
// values in flight per step.
template <bool kForward>
__device__ __forceinline__ double bc_gather(const uint32_t* __restrict__ p, uint32_t first, uint32_t len,
                                            uint32_t stride, const uint32_t* __restrict__ inlvl,
                                            const double* __restrict__ sigma, const double* __restrict__ ratio) {
  double acc = 0.0;
  uint32_t k = first;
  for (; k + 3 * stride < len; k += 4 * stride) {
    uint32_t u[4];
    bool in[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = __ldg(p + k + j * stride);
#pragma unroll
    for (int j = 0; j < 4; ++j) in[j] = bc_in(inlvl, u[j]);
    double x[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = in[j] ? bc_value<kForward>(u[j], sigma, ratio) : 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) acc += x[j];
  }
  for (; k < len; k += stride) {
    const uint32_t u = __ldg(p + k);
    if (bc_in(inlvl, u)) acc += bc_value<kForward>(u, sigma, ratio);
  }
  return acc;
}

// the source's bit: level 0, gathered by the first forward level
__global__ void bc_source_bit_kernel(uint32_t* bits, uint32_t src) { bits[src >> 5] = 1u << (src & 31); }

// forward: sigma(v), and the ratio a vertex without deeper neighbours keeps;
// backward: delta(v) = sigma(v) * sum, and v's ratio for the level above
template <bool kForward>
__device__ __forceinline__ void bc_store(uint32_t v, double acc, double* sigma, double* delta, double* ratio) {
  if (kForward) {
    sigma[v] = acc;
    ratio[v] = 1.0 / acc;
  } else {
    const double sv = __ldcg(sigma + v);
    const double dv = sv * acc;
    delta[v] = dv;
    ratio[v] = (1.0 + dv) / sv;
  }
}

// One level of a sweep.  Blocks [0, light_blocks) take the level's light
// vertices, eight lanes each; the remaining blocks take its heavy vertices,
// one CTA each.  Level membership comes from two bitmaps by level parity
// (bits + (l & 1) * nw): the kernel of level l reads the other parity's
// bitmap (the gathered level, l - 1 forward, l + 1 backward), sets its own
// vertices' bits in its parity's bitmap for the next kernel, and clears from
// that bitmap the level two steps back, whose last reader was the previous
// kernel.  No kernel reads the bitmap it writes.
template <typename G, bool kForward>
__global__ void __launch_bounds__(kBcThreads) bc_level_kernel(G g, const uint32_t* __restrict__ order,
                                                              const uint64_t* __restrict__ lstart,
                                                              const uint32_t* __restrict__ lcnt, uint32_t l,
                                                              uint32_t light_blocks, uint32_t* bits, uint32_t nw,
                                                              uint32_t L, double* sigma, double* delta, double* ratio) {
  const uint64_t begin = lstart[l], end = lstart[l + 1];
  const uint32_t* __restrict__ inlvl = bits + (size_t)((l & 1) ^ 1) * nw;
  uint32_t* own = bits + (size_t)(l & 1) * nw;
  const bool clear = kForward ? l >= 2 : l + 2 < L;
  if (clear) {
    const uint32_t lc = kForward ? l - 2 : l + 2;
    for (uint64_t i = lstart[lc] + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < lstart[lc + 1];
         i += (uint64_t)gridDim.x * blockDim.x) {
      const uint32_t v = order[i];
      atomicAnd(own + (v >> 5), ~(1u << (v & 31)));
    }
  }
  const uint64_t mid = begin + lcnt[l];
  if (blockIdx.x < light_blocks) {
    const uint32_t lane = threadIdx.x & (kGroup - 1);
    const uint64_t grp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / kGroup;
    const uint64_t ngrp = (uint64_t)light_blocks * blockDim.x / kGroup;
    // every group runs the same number of rounds (the shuffles need all lanes)
    for (uint64_t i0 = begin; i0 < mid; i0 += ngrp) {
      const uint64_t i = i0 + grp;
      double acc = 0.0;
      uint32_t v = 0;
      if (i < mid) {
        v = order[i];
        const Seg s = g.seg(v);
        acc = bc_gather<kForward>(s.p, lane, s.len, kGroup, inlvl, sigma, ratio);
      }
#pragma unroll
      for (int o = kGroup / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o, kGroup);
      if (i < mid && lane == 0) {
        bc_store<kForward>(v, acc, sigma, delta, ratio);
        atomicOr(own + (v >> 5), 1u << (v & 31));
      }
    }
  } else {
    __shared__ double red[kBcThreads / 32];
    for (uint64_t i = mid + (blockIdx.x - light_blocks); i < end; i += gridDim.x - light_blocks) {
      const uint32_t v = order[i];
      const Seg s = g.seg(v);
      double acc = bc_gather<kForward>(s.p, threadIdx.x, s.len, blockDim.x, inlvl, sigma, ratio);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
      if (lane_id() == 0) red[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kBcThreads / 32; ++w) t += red[w];
        bc_store<kForward>(v, t, sigma, delta, ratio);
        atomicOr(own + (v >> 5), 1u << (v & 31));
      }
      __syncthreads();
    }
  }
}

template <typename G>
byo_status run_bc(const byo_graph* g, G view, uint32_t src, uint32_t* level, double* sigma, double* delta,
                  cudaStream_t s) {
  const uint32_t n = g->n;
  uint32_t* maxl = nullptr;
  BYO_RETURN_IF(tmp_alloc_t(&maxl, 1, s, "BC depth"));
  byo_status st = BYO_OK;
  uint32_t depth = 0;
  {
    ProfScope ps("bc_init", s);
    cudaMemsetAsync(maxl, 0, sizeof(uint32_t), s);
    bc_init_kernel<<<grid_for(n, kBcThreads), kBcThreads, 0, s>>>(n, src, level, sigma, delta, maxl);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&depth, maxl, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "bc_init_kernel");
  }
  tmp_free(maxl, s);
  BYO_RETURN_IF(st);
  if (depth == 0) return BYO_OK;  // the source reaches nothing
  const uint64_t L = (uint64_t)depth + 1;
  uint32_t *cnt = nullptr, *lcnt = nullptr, *cur = nullptr, *order = nullptr;
  uint64_t* lstart = nullptr;
  double* ratio = nullptr;
  st = tmp_alloc_t(&cnt, L + 1, s, "BC level counts");
  if (st == BYO_OK) st = tmp_alloc_t(&ratio, n, s, "BC ratios");
  if (st == BYO_OK) st = tmp_alloc_t(&lcnt, L, s, "BC light counts");
  if (st == BYO_OK) st = tmp_alloc_t(&cur, 2 * L, s, "BC cursors");
  if (st == BYO_OK) st = tmp_alloc_t(&lstart, L + 1, s, "BC level starts");
  if (st == BYO_OK) st = tmp_alloc_t(&order, n, s, "BC level order");
  const uint32_t nw = (n + 31) / 32;
  uint32_t* bits = nullptr;  // two level bitmaps, by level parity
  if (st == BYO_OK) st = tmp_alloc_t(&bits, 2ull * nw, s, "BC level bits");
  if (st == BYO_OK) {
    cudaMemsetAsync(bits, 0, sizeof(uint32_t) * 2ull * nw, s);
    bc_source_bit_kernel<<<1, 1, 0, s>>>(bits, src);
    note_launch();
  }
  std::vector<uint64_t> hstart;
  std::vector<uint32_t> hlight;  // light vertices per level
  if (st == BYO_OK) {
    ProfScope ps("bc_group", s);
    cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (L + 1), s);
    cudaMemsetAsync(lcnt, 0, sizeof(uint32_t) * L, s);
    cudaMemsetAsync(cur, 0, sizeof(uint32_t) * 2 * L, s);
    const uint32_t gb = (uint32_t)sm_count() * 4;  // CTAs for the two grouping passes
    bc_hist_kernel<G><<<gb, kBcThreads, 0, s>>>(view, level, cnt, lcnt);
    note_launch();
    st = scan_u32_to_u64(cnt, lstart, L + 1, nullptr, s);
    if (st == BYO_OK) {
      bc_scatter_kernel<G><<<gb, kBcThreads, 0, s>>>(view, level, lstart, cur, cur + L, order);
      note_launch();
      hstart.resize(L + 1);
      hlight.resize(L);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hstart.data(), lstart, sizeof(uint64_t) * (L + 1), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hlight.data(), lcnt, sizeof(uint32_t) * L, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_status(e, "bc grouping");
    }
  }
  if (st == BYO_OK) {
    const uint32_t cap = (uint32_t)sm_count() * 8;
    auto blocks = [&](uint64_t c) {
      uint64_t want = (c * kGroup + kBcThreads - 1) / kBcThreads;
      return (uint32_t)(want < cap ? (want ? want : 1) : cap);
    };
    // heavy vertices (degree >= kHeavy, most of the edges on skewed graphs):
    // a CTA each, as many CTAs as the level has of them, up to 8 per SM
    auto heavy_blocks = [&](uint32_t l) {
      const uint64_t h = hstart[l + 1] - hstart[l] - hlight[l];
      return (uint32_t)(h < cap ? (h ? h : 1) : cap);
    };
    // the level kernel also clears level lc's bits: at least a thread per
    // cleared vertex up to the cap, or a small level's kernel would clear a
    // large level with a handful of CTAs (the extra CTAs join the heavy part)
    auto grid = [&](uint32_t l, uint32_t lb, uint64_t lc) {
      const uint32_t g = lb + heavy_blocks(l);
      if (lc >= L) return g;
      const uint64_t c = (hstart[lc + 1] - hstart[lc] + kBcThreads - 1) / kBcThreads;
      const uint32_t cb = (uint32_t)(c < cap ? c : cap);
      return g > cb ? g : cb;
    };
    {
      ProfScope ps("bc_forward", s);
      for (uint32_t l = 1; l < L; ++l) {
        const uint32_t lb = blocks(hlight[l]);
        bc_level_kernel<G, true><<<grid(l, lb, l >= 2 ? l - 2 : L), kBcThreads, 0, s>>>(
            view, order, lstart, lcnt, l, lb, bits, nw, (uint32_t)L, sigma, delta, ratio);
        note_launch();
      }
    }
    {
      ProfScope ps("bc_backward", s);
      for (uint32_t l = depth; l-- > 1;) {  // the deepest level has no deeper neighbour; delta(s) stays 0
        const uint32_t lb = blocks(hlight[l]);
        bc_level_kernel<G, false><<<grid(l, lb, l + 2 < L ? l + 2 : L), kBcThreads, 0, s>>>(
            view, order, lstart, lcnt, l, lb, bits, nw, (uint32_t)L, sigma, delta, ratio);
        note_launch();
      }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "bc sweeps");
  }
  tmp_free(cnt, s);
  tmp_free(lcnt, s);
  tmp_free(cur, s);
  tmp_free(lstart, s);
  tmp_free(order, s);
  tmp_free(bits, s);
  tmp_free(ratio, s);
  return st;
}

}  // namespace
}  // namespace byo

using namespace byo;

extern "C" byo_status byo_bc(const byo_graph* gc, uint32_t source, uint32_t* levels, double* sigma, double* delta,
                             void* stream) {
  clear_error();
  BYO_RETURN_IF(ready_graph(gc, static_cast<cudaStream_t>(stream)));
  if (!sigma || !delta) {
    set_error("byo_bc: NULL sigma or delta");
    return BYO_ERR_INVALID_ARG;
  }
  if (source >= gc->n) {
    set_error("byo_bc: source %u is >= n (%u)", source, gc->n);
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* lv = levels;
  if (!lv) BYO_RETURN_IF(tmp_alloc_t(&lv, gc->n, s, "BC levels"));
  byo_status st = byo_bfs(gc, &source, 1, lv, nullptr, nullptr, stream);
  if (st == BYO_OK) {
    clear_error();
    st = with_view(gc, [&](auto view) { return run_bc(gc, view, source, lv, sigma, delta, s); });
  }
  if (!levels) tmp_free(lv, s);
  return st;
}
