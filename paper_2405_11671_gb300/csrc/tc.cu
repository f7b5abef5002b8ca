// tc.cu -- triangle counting by filter-then-intersect (Section 4.4: a filter
// builds a smaller DAG first, then neighbour sets are intersected).
//
// Filter: each edge is kept once, from the endpoint of lower rank, where
// rank(v) = (degree(v), v) in lexicographic order; N+(v) stays sorted by id.
// Count: the number of triangles is the sum over DAG edges u->v of
// |N+(u) intersect N+(v)|.  For every u, N+(u) is staged in shared memory by a
// TMA bulk copy (cp.async.bulk, completion on an mbarrier; no multicast), then
// the ids of N+(v) for all v in N+(u) are walked 32 at a time by a warp
// (edge-balanced across the warp) and looked up in shared memory.  u with |N+(u)| <= kLightMax: one warp each; the staged N+(u) is
// loaded into an open-addressing hash set in the warp's shared memory and each
// id of N+(v) costs one or two probes.  Larger u: one CTA each (taken from a
// work counter), N+(u) staged in windows of kWindow ids, each hashed the same
// way into the CTA's shared memory.
#include <stdlib.h>

#include "byo_internal.cuh"
#include "prof.cuh"
#include "container.cuh"
#include "vbins.cuh"

namespace byo {

constexpr uint32_t kLightMax = 256;   // capacity of a warp's shared-memory slice (ids)
constexpr uint32_t kWindow = 8192;    // capacity of a CTA's shared-memory window (ids)
constexpr int kTcThreads = 256;

// The light/heavy split and the window length can be lowered (never raised)
// with BYO_TC_LIGHT_MAX / BYO_TC_WINDOW, so that small test graphs exercise
// the CTA path and multi-window intersections.
static uint32_t env_cap(const char* name, uint32_t cap) {
  const char* e = getenv(name);
  if (!e || !*e) return cap;
  long long v = atoll(e);
  if (v < 4) v = 4;
  return v < (long long)cap ? (uint32_t)v : cap;
}

struct TcWork {
  uint32_t n = 0;
  uint64_t half_cap = 0;        // capacity of dag_col (undirected edges)
  uint64_t* dag_off = nullptr;  // n + 1
  uint32_t* dag_col = nullptr;  // m/2 + 8
  uint32_t* outdeg = nullptr;   // n
  uint32_t* light = nullptr;    // n
  uint32_t* heavy = nullptr;    // n
  uint32_t* ctr = nullptr;      // [0] light count, [1] heavy count, [2] light cursor, [3] error, [4] heavy cursor
  unsigned long long* count = nullptr;
};

void tc_free(TcWork* w) {
  if (!w) return;
  dev_free(w->dag_off);
  dev_free(w->dag_col);
  dev_free(w->outdeg);
  dev_free(w->light);
  dev_free(w->heavy);
  dev_free(w->ctr);
  dev_free(w->count);
  delete w;
}

namespace {

// ---------------------------------------------------------------- TMA / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase to complete; false (and the error word set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, uint32_t* err, uint64_t limit_ns) {
  if (mbar_test(bar, phase)) return true;
  uint64_t t0 = globaltimer();
  while (!mbar_test(bar, phase)) {
    if (globaltimer() - t0 > limit_ns) {
      atomicCAS(err, 0u, (uint32_t)BYO_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// ---------------------------------------------------------------- filter
template <typename G>
__device__ __forceinline__ bool rank_lt(const G& g, uint32_t a, uint32_t da, uint32_t b) {
  uint32_t db = g.degree(b);
  return da < db || (da == db && a < b);
}

template <typename G>
__global__ void __launch_bounds__(kTcThreads) tc_outdeg_kernel(G g, VBins bins, uint32_t* outdeg) {
  VRange r = vbins_range(bins);
  const uint32_t lane = lane_id();
  if (r.role == kRoleThread) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      uint32_t c = 0;
      for (uint32_t k = 0; k < s.len; ++k) c += rank_lt(g, v, s.len, __ldg(s.p + k));
      outdeg[v] = c;
    }
  } else if (r.role == kRoleWarp) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      uint32_t c = 0;
      for (uint32_t k = lane; k < s.len; k += 32) c += rank_lt(g, v, s.len, __ldg(s.p + k));
      c = __reduce_add_sync(0xFFFFFFFFu, c);
      if (lane == 0) outdeg[v] = c;
    }
  } else {
    __shared__ uint32_t part[kTcThreads / 32];
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      uint32_t c = 0;
      for (uint32_t k = threadIdx.x; k < s.len; k += blockDim.x) c += rank_lt(g, v, s.len, __ldg(s.p + k));
      c = __reduce_add_sync(0xFFFFFFFFu, c);
      if (lane == 0) part[threadIdx.x >> 5] = c;
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) t += part[w];
        outdeg[v] = t;
      }
      __syncthreads();
    }
  }
}

template <typename G>
__global__ void __launch_bounds__(kTcThreads) tc_fill_kernel(G g, VBins bins, const uint64_t* __restrict__ dag_off,
                                                             uint32_t* __restrict__ dag_col) {
  VRange r = vbins_range(bins);
  const uint32_t lane = lane_id();
  if (r.role == kRoleThread) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      uint64_t o = dag_off[v];
      for (uint32_t k = 0; k < s.len; ++k) {
        uint32_t u = __ldg(s.p + k);
        if (rank_lt(g, v, s.len, u)) dag_col[o++] = u;
      }
    }
  } else if (r.role == kRoleWarp) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      uint64_t o = dag_off[v];
      for (uint32_t base = 0; base < s.len; base += 32) {
        uint32_t k = base + lane;
        uint32_t u = k < s.len ? __ldg(s.p + k) : 0;
        bool keep = k < s.len && rank_lt(g, v, s.len, u);
        uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        if (keep) dag_col[o + __popc(bal & lanemask_lt())] = u;
        o += __popc(bal);
      }
    }
  } else {
    __shared__ uint32_t wcnt[kTcThreads / 32];
    __shared__ uint32_t wpre[kTcThreads / 32 + 1];
    const uint32_t nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      uint64_t o = dag_off[v];
      for (uint32_t base = 0; base < s.len; base += blockDim.x) {
        uint32_t k = base + threadIdx.x;
        uint32_t u = k < s.len ? __ldg(s.p + k) : 0;
        bool keep = k < s.len && rank_lt(g, v, s.len, u);
        uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        if (lane == 0) wcnt[w] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
          wpre[0] = 0;
          for (uint32_t j = 0; j < nw; ++j) wpre[j + 1] = wpre[j] + wcnt[j];
        }
        __syncthreads();
        if (keep) dag_col[o + wpre[w] + __popc(bal & lanemask_lt())] = u;
        o += wpre[nw];
        __syncthreads();
      }
    }
  }
}

__global__ void tc_set_last_kernel(uint64_t* dag_off, uint32_t n, uint64_t total) { dag_off[n] = total; }

__global__ void tc_classify_kernel(const uint64_t* __restrict__ dag_off, uint32_t n, uint32_t light_max,
                                   uint32_t* light, uint32_t* heavy, uint32_t* ctr) {
  const uint32_t lane = lane_id();
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t u = base + threadIdx.x;
    uint64_t od = u < n ? dag_off[u + 1] - dag_off[u] : 0;
    bool l = od >= 2 && od <= light_max;
    bool h = od > light_max;
    uint32_t bl = __ballot_sync(0xFFFFFFFFu, l), bh = __ballot_sync(0xFFFFFFFFu, h);
    uint32_t pl = 0, ph = 0;
    if (lane == 0 && bl) pl = atomicAdd(ctr + 0, __popc(bl));
    if (lane == 0 && bh) ph = atomicAdd(ctr + 1, __popc(bh));
    pl = __shfl_sync(0xFFFFFFFFu, pl, 0);
    ph = __shfl_sync(0xFFFFFFFFu, ph, 0);
    if (l) light[pl + __popc(bl & lanemask_lt())] = (uint32_t)u;
    if (h) heavy[ph + __popc(bh & lanemask_lt())] = (uint32_t)u;
  }
}

// ---------------------------------------------------------------- intersect
// Open-addressing hash set in shared memory (linear probing, empty = INF,
// multiplicative hashing); the table has at least twice as many slots as keys.
struct SmemHash {
  const uint32_t* t;
  uint32_t mask, shift;
  __device__ __forceinline__ bool contains(uint32_t x) const {
    uint32_t h = (x * 0x9E3779B1u) >> shift;
    while (true) {
      uint32_t y = t[h];
      if (y == x) return true;
      if (y == kInf) return false;
      h = (h + 1) & mask;
    }
  }
};


// The warp walks the concatenation of N+(v) for the 32 (or fewer) v held by
// its lanes and counts the ids w in [lo_id, hi_id] that the set contains.
template <typename Set>
__device__ __forceinline__ uint64_t warp_count_group(const uint64_t* __restrict__ dag_off,
                                                     const uint32_t* __restrict__ dag_col, uint32_t v, bool has_v,
                                                     const Set& set, uint32_t lo_id, uint32_t hi_id) {
  const uint32_t lane = lane_id();
  uint64_t vb = 0;
  uint32_t len = 0;
  if (has_v) {
    vb = dag_off[v];
    len = (uint32_t)(dag_off[v + 1] - vb);
  }
  uint32_t incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  uint32_t excl = incl - len;
  uint64_t hits = 0;
  for (uint32_t e0 = 0; e0 < total; e0 += 32) {
    uint32_t e = e0 + lane;
    int owner = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      int probe = owner + step;
      uint32_t ex = __shfl_sync(0xFFFFFFFFu, excl, probe & 31);
      if (probe < 32 && ex <= e) owner = probe;
    }
    uint32_t oex = __shfl_sync(0xFFFFFFFFu, excl, owner);
    uint64_t ob = __shfl_sync(0xFFFFFFFFu, vb, owner);
    if (e < total) {
      uint32_t w = __ldg(dag_col + ob + (e - oex));
      if (w >= lo_id && w <= hi_id && set.contains(w)) ++hits;
    }
  }
  return hits;
}

constexpr uint32_t kSlice = kLightMax + 8;  // staged N+(u) (+ alignment slack), ids
constexpr uint32_t kTable = 2 * kLightMax;   // hash slots per warp
constexpr size_t kLightSmem = (size_t)(kTcThreads / 32) * (kSlice + kTable) * sizeof(uint32_t);

__global__ void __launch_bounds__(kTcThreads) tc_light_kernel(const uint64_t* __restrict__ dag_off,
                                                              const uint32_t* __restrict__ dag_col,
                                                              const uint32_t* __restrict__ light, uint32_t* ctr,
                                                              unsigned long long* count, uint64_t limit_ns) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ __align__(8) uint64_t bar[kTcThreads / 32];
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t* buf = smem + (size_t)w * (kSlice + kTable);
  uint32_t* table = buf + kSlice;
  const uint32_t nlight = __ldcg(ctr + 0);
  uint32_t* err = ctr + 3;
  if (lane == 0) mbar_init(&bar[w], 1);
  __syncwarp();
  uint32_t phase = 0;
  uint64_t hits = 0;
  while (true) {
    uint32_t idx = 0;
    if (lane == 0) idx = atomicAdd(ctr + 2, 1u);
    idx = __shfl_sync(0xFFFFFFFFu, idx, 0);
    if (idx >= nlight) break;
    uint32_t u = __ldg(light + idx);
    uint64_t beg = dag_off[u], end = dag_off[u + 1];
    uint64_t a0 = beg & ~3ull, a1 = (end + 3) & ~3ull;
    uint32_t head = (uint32_t)(beg - a0), len = (uint32_t)(end - beg);
    __syncwarp();  // every lane is done with the previous u's slice and table
    bool ok = true;
    if (lane == 0) {
      bulk_load(buf, dag_col + a0, (uint32_t)((a1 - a0) * 4), &bar[w]);
      ok = mbar_wait(&bar[w], phase, err, limit_ns);
    }
    if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) return;
    mbar_wait(&bar[w], phase, err, limit_ns);  // completed: every lane observes the phase
    phase ^= 1;
    const uint32_t* list = buf + head;
    // hash set of N+(u): 2^b >= 2 len slots
    uint32_t bits = 32 - __clz(2 * len - 1);
    if (bits < 5) bits = 5;
    const uint32_t slots = 1u << bits;
    for (uint32_t i = lane; i < slots; i += 32) table[i] = kInf;
    __syncwarp();
    for (uint32_t k = lane; k < len; k += 32) {
      uint32_t x = list[k];
      uint32_t h = (x * 0x9E3779B1u) >> (32 - bits);
      while (atomicCAS(table + h, kInf, x) != kInf) h = (h + 1) & (slots - 1);
    }
    __syncwarp();
    SmemHash set{table, slots - 1, 32 - bits};
    const uint32_t lo_id = list[0], hi_id = list[len - 1];
    for (uint32_t k0 = 0; k0 < len; k0 += 32) {
      uint32_t k = k0 + lane;
      bool has = k < len;
      uint32_t v = has ? list[k] : 0;
      hits += warp_count_group(dag_off, dag_col, v, has, set, lo_id, hi_id);
    }
  }
  uint64_t t = hits;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
  if (lane == 0 && t) atomicAdd(count, (unsigned long long)t);
}

constexpr uint32_t kHeavyTable = 2 * kWindow;
constexpr size_t kHeavySmem = (size_t)(kWindow + 8 + kHeavyTable) * sizeof(uint32_t);

__global__ void __launch_bounds__(kTcThreads) tc_heavy_kernel(const uint64_t* __restrict__ dag_off,
                                                              const uint32_t* __restrict__ dag_col,
                                                              const uint32_t* __restrict__ heavy, uint32_t* ctr,
                                                              unsigned long long* count, uint32_t window,
                                                              uint64_t limit_ns) {
  extern __shared__ __align__(16) uint32_t win[];
  uint32_t* table = win + kWindow + 8;
  __shared__ __align__(8) uint64_t bar;
  __shared__ bool ok_s;
  __shared__ uint32_t idx_s;
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t nheavy = __ldcg(ctr + 1);
  uint32_t* err = ctr + 3;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  uint64_t hits = 0;
  while (true) {
    if (threadIdx.x == 0) idx_s = atomicAdd(ctr + 4, 1u);
    __syncthreads();
    const uint32_t idx = idx_s;
    if (idx >= nheavy) break;
    uint32_t u = __ldg(heavy + idx);
    uint64_t beg = dag_off[u], end = dag_off[u + 1];
    for (uint64_t wb = beg; wb < end; wb += window) {
      uint64_t we = wb + window < end ? wb + window : end;
      uint64_t a0 = wb & ~3ull, a1 = (we + 3) & ~3ull;
      uint32_t head = (uint32_t)(wb - a0), wlen = (uint32_t)(we - wb);
      __syncthreads();  // every thread is done with the previous window and table
      if (threadIdx.x == 0) {
        bulk_load(win, dag_col + a0, (uint32_t)((a1 - a0) * 4), &bar);
        ok_s = mbar_wait(&bar, phase, err, limit_ns);
      }
      __syncthreads();
      if (!ok_s) return;
      mbar_wait(&bar, phase, err, limit_ns);  // completed: every thread observes the phase
      phase ^= 1;
      const uint32_t* list = win + head;
      uint32_t bits = 32 - __clz(2 * wlen - 1);
      if (bits < 5) bits = 5;
      const uint32_t slots = 1u << bits;
      for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) table[i] = kInf;
      __syncthreads();
      for (uint32_t k = threadIdx.x; k < wlen; k += blockDim.x) {
        uint32_t x = list[k];
        uint32_t h = (x * 0x9E3779B1u) >> (32 - bits);
        while (atomicCAS(table + h, kInf, x) != kInf) h = (h + 1) & (slots - 1);
      }
      __syncthreads();
      SmemHash set{table, slots - 1, 32 - bits};
      uint32_t lo_id = list[0], hi_id = list[wlen - 1];
      for (uint64_t k0 = beg + (uint64_t)w * 32; k0 < end; k0 += (uint64_t)nw * 32) {
        uint64_t k = k0 + lane;
        bool has = k < end;
        uint32_t v = has ? __ldg(dag_col + k) : 0;
        hits += warp_count_group(dag_off, dag_col, v, has, set, lo_id, hi_id);
      }
    }
  }
  uint64_t t = hits;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
  if (lane == 0 && t) atomicAdd(count, (unsigned long long)t);
}

byo_status ensure_tc_work(byo_graph* g) {
  if (g->tc && g->tc->half_cap >= g->m / 2) return BYO_OK;
  if (g->tc) {  // the dynamic container grew
    tc_free(g->tc);
    g->tc = nullptr;
  }
  TcWork* w = new (std::nothrow) TcWork();
  if (!w) {
    set_error("host allocation failed");
    return BYO_ERR_OUT_OF_MEMORY;
  }
  w->n = g->n;
  w->half_cap = g->m / 2 + (g->dyn ? g->m / 8 : 0);  // headroom for later inserts
  byo_status st = dev_alloc_t(&w->dag_off, g->n + 1ull, "TC DAG offsets");
  if (st == BYO_OK) st = dev_alloc_t(&w->dag_col, w->half_cap + 8, "TC DAG neighbours");
  if (st == BYO_OK) st = dev_alloc_t(&w->outdeg, g->n, "TC out-degrees");
  if (st == BYO_OK) st = dev_alloc_t(&w->light, g->n, "TC light list");
  if (st == BYO_OK) st = dev_alloc_t(&w->heavy, g->n, "TC heavy list");
  if (st == BYO_OK) st = dev_alloc_t(&w->ctr, 8, "TC counters");
  if (st == BYO_OK) st = dev_alloc_t(&w->count, 1, "TC count");
  if (st == BYO_OK) {
    cudaError_t e = cudaMemset(w->dag_col, 0, sizeof(uint32_t) * (w->half_cap + 8));
    if (e != cudaSuccess) st = cuda_status(e, "cudaMemset");
  }
  if (st != BYO_OK) {
    tc_free(w);
    return st;
  }
  g->tc = w;
  return BYO_OK;
}

template <typename G>
byo_status run_tc(byo_graph* g, G view, uint64_t* host_count, cudaStream_t s) {
  BYO_RETURN_IF(ensure_tc_work(g));
  TcWork* w = g->tc;
  VBins bins = make_vbins(g, 4, 10, kTcThreads);
  {
    ProfScope ps("tc_outdeg", s);
    tc_outdeg_kernel<<<vbins_grid(bins), kTcThreads, 0, s>>>(view, bins, w->outdeg); ::byo::note_launch();
  }
  BYO_CHECK_LAUNCH("tc_outdeg_kernel");
  BYO_RETURN_IF(scan_u32_to_u64(w->outdeg, w->dag_off, g->n, nullptr, s));
  tc_set_last_kernel<<<1, 1, 0, s>>>(w->dag_off, g->n, g->m / 2); ::byo::note_launch();
  BYO_CHECK_LAUNCH("tc_set_last_kernel");
  {
    ProfScope ps("tc_fill", s);
    tc_fill_kernel<<<vbins_grid(bins), kTcThreads, 0, s>>>(view, bins, w->dag_off, w->dag_col); ::byo::note_launch();
  }
  BYO_CHECK_LAUNCH("tc_fill_kernel");
  BYO_CUDA(cudaMemsetAsync(w->ctr, 0, 8 * sizeof(uint32_t), s));
  BYO_CUDA(cudaMemsetAsync(w->count, 0, sizeof(unsigned long long), s));
  unsigned grid = (unsigned)sm_count() * 4;
  tc_classify_kernel<<<grid, 256, 0, s>>>(w->dag_off, g->n, env_cap("BYO_TC_LIGHT_MAX", kLightMax), w->light,
                                          w->heavy, w->ctr); ::byo::note_launch();
  BYO_CHECK_LAUNCH("tc_classify_kernel");
  uint64_t limit = timeout_ns();
  int per_sm = 0;
  BYO_CUDA(cudaFuncSetAttribute(tc_light_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLightSmem));
  BYO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_light_kernel, kTcThreads, kLightSmem));
  {
    ProfScope ps("tc_light", s);
    tc_light_kernel<<<(unsigned)(sm_count() * (per_sm > 0 ? per_sm : 1)), kTcThreads, kLightSmem, s>>>(
      w->dag_off, w->dag_col, w->light, w->ctr, w->count, limit); ::byo::note_launch();
  }
  BYO_CHECK_LAUNCH("tc_light_kernel");
  size_t dyn = kHeavySmem;
  BYO_CUDA(cudaFuncSetAttribute(tc_heavy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  {
    ProfScope ps("tc_heavy", s);
    tc_heavy_kernel<<<(unsigned)sm_count() * 2, kTcThreads, dyn, s>>>(w->dag_off, w->dag_col, w->heavy, w->ctr,
                                                                    w->count, env_cap("BYO_TC_WINDOW", kWindow),
                                                                    limit); ::byo::note_launch();
  }
  BYO_CHECK_LAUNCH("tc_heavy_kernel");
  uint32_t err = 0;
  unsigned long long c = 0;
  BYO_CUDA(cudaMemcpyAsync(&c, w->count, sizeof(c), cudaMemcpyDeviceToHost, s));
  BYO_CUDA(cudaMemcpyAsync(&err, w->ctr + 3, sizeof(err), cudaMemcpyDeviceToHost, s));
  BYO_CUDA(cudaStreamSynchronize(s));
  if (err) {
    set_error("byo_tc: a TMA completion wait exceeded BYO_TIMEOUT_MS");
    return BYO_ERR_TIMEOUT;
  }
  *host_count = c;
  return BYO_OK;
}

}  // namespace
}  // namespace byo

using namespace byo;

extern "C" byo_status byo_tc(const byo_graph* gc, uint64_t* host_count, void* stream) {
  clear_error();
  BYO_RETURN_IF(check_graph(gc));
  if (!host_count) {
    set_error("byo_tc: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  byo_graph* g = const_cast<byo_graph*>(gc);
  *host_count = 0;
  if (g->n == 0 || g->m == 0) return BYO_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return with_view(g, [&](auto view) { return run_tc(g, view, host_count, s); });
}
