// graph.cu -- error plumbing, allocation helpers, and the static CSR
// container: build (Section 3.1 neighbour sets stored contiguously, Section
// 4.2), num_vertices / num_edges / degree (Section 4.2, kept as metadata as in
// Section 4.3), export, destroy.
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include <atomic>

#include "byo_internal.cuh"
#include "prof.cuh"
#include "container.cuh"

namespace byo {

// ---------------------------------------------------------------- errors
static thread_local char g_err[512] = "";
// device allocations made by the current public call (see inject_alloc_failure)
static thread_local long long t_allocs_in_call = 0;

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() {
  g_err[0] = 0;
  t_allocs_in_call = 0;
}

byo_status cuda_status(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return BYO_ERR_OUT_OF_MEMORY;
  return BYO_ERR_CUDA;
}

// Allocation-failure injection for tests of the error paths: with
// BYO_FAULT_INJECT=alloc:K in the environment, the K-th device allocation
// (cudaMalloc or cudaMallocAsync) that a public call makes is not made and
// reports OUT_OF_MEMORY, as a full device would.  The count restarts at every
// public call (clear_error).  Only the host side is involved.
static bool inject_alloc_failure() {
  const char* e = getenv("BYO_FAULT_INJECT");
  if (!e || strncmp(e, "alloc:", 6) != 0) return false;
  const long long k = atoll(e + 6);
  return k > 0 && ++t_allocs_in_call == k;
}

byo_status dev_alloc(void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (inject_alloc_failure()) {
    set_error("cudaMalloc(%zu bytes) for %s: injected failure (BYO_FAULT_INJECT)", bytes, what);
    return BYO_ERR_OUT_OF_MEMORY;
  }
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("cudaMalloc(%zu bytes) for %s: %s", bytes, what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BYO_ERR_OUT_OF_MEMORY : BYO_ERR_CUDA;
  }
  return BYO_OK;
}
void dev_free(void* p) {
  if (p) cudaFree(p);
}

// Scratch comes from the device's stream-ordered memory pool.  The pool keeps
// up to a quarter of the device memory mapped between calls (the default
// releases everything at each synchronisation), so that the multi-GB scratch
// of a large graph is not mapped again by every call.  Set once per device;
// it lasts as long as the process.
static void keep_pool_warm() {
  static std::atomic<uint64_t> done_mask{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) {
    cudaGetLastError();
    return;
  }
  if (done_mask.load() & (1ull << dev)) return;
  done_mask.fetch_or(1ull << dev);
  cudaMemPool_t pool;
  size_t free_b = 0, total_b = 0;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
    uint64_t keep = (uint64_t)total_b / 4;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
}

byo_status tmp_alloc(void** p, size_t bytes, cudaStream_t s, const char* what) {
  *p = nullptr;
  if (inject_alloc_failure()) {
    set_error("cudaMallocAsync(%zu bytes) for %s: injected failure (BYO_FAULT_INJECT)", bytes, what);
    return BYO_ERR_OUT_OF_MEMORY;
  }
  keep_pool_warm();
  cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("cudaMallocAsync(%zu bytes) for %s: %s", bytes, what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BYO_ERR_OUT_OF_MEMORY : BYO_ERR_CUDA;
  }
  return BYO_OK;
}
void tmp_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

int sm_count() {
  int dev = 0, c = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
  return c > 0 ? c : 1;
}

uint64_t timeout_ns() {
  const char* e = getenv("BYO_TIMEOUT_MS");
  uint64_t ms = 10000;
  if (e && *e) {
    long long v = atoll(e);
    if (v > 0) ms = (uint64_t)v;
  }
  return ms * 1000000ull;
}

byo_status check_graph(const byo_graph* g) {
  if (!g) {
    set_error("graph handle is NULL");
    return BYO_ERR_INVALID_ARG;
  }
  return BYO_OK;
}

byo_status ready_graph(const byo_graph* gc, cudaStream_t s) {
  BYO_RETURN_IF(check_graph(gc));
  if (gc->comp) {
    set_error("a compressed container supports BFS, degree, export and space queries only");
    return BYO_ERR_UNSUPPORTED;
  }
  byo_graph* g = const_cast<byo_graph*>(gc);
  if (!g->buckets_stale) return BYO_OK;
  BYO_RETURN_IF(rebuild_buckets(g, s));
  g->buckets_stale = false;
  return BYO_OK;
}

// ---------------------------------------------------------------- kernels
namespace {

__global__ void make_keys_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t k,
                                 uint32_t n, int lb, bool sym, uint64_t* __restrict__ keys, uint32_t* bad) {
  const uint64_t sentinel = (lb == 32) ? ~0ull : ((1ull << (2 * lb)) - 1);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t u = src[i], v = dst[i];
    uint64_t a = sentinel, b = sentinel;
    if (u >= n || v >= n) {
      atomicOr(bad, 1u);
    } else if (u != v) {
      a = ((uint64_t)u << lb) | v;
      b = ((uint64_t)v << lb) | u;
    }
    if (sym) {
      keys[2 * i] = a;
      keys[2 * i + 1] = b;
    } else {
      keys[i] = a;
    }
  }
}

// Unique pairs of the sorted keys, in tiles of kUniqTile keys striped over
// the CTA (key tile0 + r * kUniqThreads + t is thread t's key of round r).
// Key i is kept iff it is valid (not the sentinel of a dropped self loop) and
// differs from key i - 1: the first copy of each pair.
constexpr int kUniqThreads = 512;
constexpr int kUniqRounds = 8;
constexpr int kUniqWarps = kUniqThreads / 32;
constexpr uint64_t kUniqTile = (uint64_t)kUniqThreads * kUniqRounds;

struct UniqKey {
  uint64_t x;     // the key (the sentinel past the end)
  uint64_t prev;  // key i - 1 (meaningless for i = 0)
  bool keep;      // first copy of a valid key
};

__device__ __forceinline__ UniqKey uniq_key(const uint64_t* __restrict__ keys, uint64_t i, uint64_t cnt,
                                            uint64_t sentinel) {
  UniqKey u;
  u.x = i < cnt ? __ldg(keys + i) : sentinel;
  u.prev = __shfl_up_sync(0xFFFFFFFFu, u.x, 1);
  if (lane_id() == 0) u.prev = (i > 0 && i < cnt) ? __ldg(keys + i - 1) : ~u.x;
  u.keep = u.x != sentinel && (i == 0 || u.prev != u.x);
  return u;
}

__global__ void __launch_bounds__(kUniqThreads) unique_count_kernel(const uint64_t* __restrict__ keys, uint64_t cnt,
                                                                     uint64_t sentinel,
                                                                     uint32_t* __restrict__ tile_counts) {
  __shared__ uint32_t wsum[kUniqWarps];
  const uint64_t tile0 = (uint64_t)blockIdx.x * kUniqTile;
  uint32_t c = 0;
#pragma unroll
  for (int r = 0; r < kUniqRounds; ++r)
    c += __popc(__ballot_sync(0xFFFFFFFFu, uniq_key(keys, tile0 + (uint64_t)r * kUniqThreads + threadIdx.x, cnt,
                                                    sentinel).keep));
  if (lane_id() == 0) wsum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t t = threadIdx.x < kUniqWarps ? wsum[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
    if (threadIdx.x == 0) tile_counts[blockIdx.x] = t;
  }
}

// Writes the kept keys of each tile from position tile_offs[tile] on, in key
// order: col[p] = destination, rows[p] = source (if rows is not null), and,
// if off is not null, the CSR offsets: off[s] = p for every row s in
// (source of key i - 1, source of key i] when kept key i starts a row, and
// off[s] = m for every s after the source of the last valid key.  Consecutive
// lanes write consecutive positions.
template <typename OffT>
__global__ void __launch_bounds__(kUniqThreads) unique_write_kernel(const uint64_t* __restrict__ keys, uint64_t cnt,
                                                                     uint64_t sentinel, int lb,
                                                                     const uint64_t* __restrict__ tile_offs,
                                                                     uint64_t m, uint32_t n,
                                                                     uint32_t* __restrict__ col,
                                                                     uint32_t* __restrict__ rows,
                                                                     OffT* __restrict__ off) {
  __shared__ uint32_t wsum[kUniqRounds * kUniqWarps];  // kept keys per (round, warp), then their exclusive scan
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  const uint64_t tile0 = (uint64_t)blockIdx.x * kUniqTile;
  const uint64_t lowmask = (lb == 32) ? 0xFFFFFFFFull : ((1ull << lb) - 1);
  UniqKey u[kUniqRounds];
  uint32_t ball[kUniqRounds];
#pragma unroll
  for (int r = 0; r < kUniqRounds; ++r) {
    u[r] = uniq_key(keys, tile0 + (uint64_t)r * kUniqThreads + threadIdx.x, cnt, sentinel);
    ball[r] = __ballot_sync(0xFFFFFFFFu, u[r].keep);
    if (lane == 0) wsum[r * kUniqWarps + w] = __popc(ball[r]);
  }
  __syncthreads();
  if (w == 0) {  // exclusive scan of the kUniqRounds * kUniqWarps counts, in key order
    constexpr int kPer = kUniqRounds * kUniqWarps / 32;
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      v[j] = wsum[lane * kPer + j];
      sum += v[j];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if ((int)lane >= o) incl += y;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      wsum[lane * kPer + j] = run;
      run += v[j];
    }
  }
  __syncthreads();
  const uint64_t base = tile_offs[blockIdx.x];
#pragma unroll
  for (int r = 0; r < kUniqRounds; ++r) {
    const uint64_t i = tile0 + (uint64_t)r * kUniqThreads + threadIdx.x;
    const uint64_t x = u[r].x;
    if (u[r].keep) {
      const uint64_t p = base + wsum[r * kUniqWarps + w] + __popc(ball[r] & lanemask_lt());
      const uint32_t src = (uint32_t)(x >> lb);
      col[p] = (uint32_t)(x & lowmask);
      if (rows) rows[p] = src;
      if (off) {
        // key i - 1 is valid (keys are sorted and the sentinel is the largest)
        const uint64_t lo = i == 0 ? 0 : ((u[r].prev >> lb) + 1);
        for (uint64_t s = lo; s <= src; ++s) off[s] = (OffT)p;
      }
    }
    if (off && x != sentinel && (i + 1 >= cnt || __ldg(keys + i + 1) == sentinel)) {
      for (uint64_t s = (x >> lb) + 1; s <= n; ++s) off[s] = (OffT)m;
    }
  }
}

// Keys for grouping vertices by degree bucket, ascending id inside a bucket:
// (v << kBucketBits) | bucket, written in id order, so that one stable radix
// pass over the bucket field gives the order.
constexpr int kBucketBits = 6;
static_assert(kBuckets <= (1 << kBucketBits), "degree buckets 0..32 fit the bucket field");

template <typename G>
__global__ void bucket_keys_kernel(G g, uint64_t* keys, unsigned long long* hist) {
  __shared__ uint32_t h[kBuckets];  // a CTA counts at most its grid-stride share of n < 2^32
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t n = g.num_vertices();
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    int b = degree_bucket(g.degree((uint32_t)v));
    keys[v] = (v << kBucketBits) | (uint64_t)b;
    atomicAdd(&h[b], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// bucket starts = exclusive scan of the bucket sizes (kBuckets + 1 entries)
__global__ void bucket_starts_kernel(const unsigned long long* __restrict__ hist, uint64_t* bstart) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint64_t acc = 0;
  for (int b = 0; b < kBuckets; ++b) {
    bstart[b] = acc;
    acc += hist[b];
  }
  bstart[kBuckets] = acc;
}

__global__ void high_bits_kernel(const uint64_t* __restrict__ keys, uint64_t n, int shift, uint32_t* out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)(keys[i] >> shift);
}

__global__ void low32_kernel(const uint64_t* __restrict__ keys, uint64_t n, int lb, uint32_t* out) {
  const uint64_t lowmask = (lb == 32) ? 0xFFFFFFFFull : ((1ull << lb) - 1);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)(keys[i] & lowmask);
}

// symmetry check: (u,v) present => (v,u) present
template <typename OffT>
__global__ void symmetric_kernel(const OffT* __restrict__ off, const uint32_t* __restrict__ col,
                                 const uint32_t* __restrict__ rows, uint64_t m, uint32_t* bad) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t u = rows[p], v = col[p];
    uint64_t lo = off[v], hi = off[v + 1];
    while (lo < hi) {
      uint64_t mid = (lo + hi) >> 1;
      if (col[mid] < u) lo = mid + 1;
      else hi = mid;
    }
    if (!(lo < off[v + 1] && col[lo] == u)) atomicOr(bad, 1u);
  }
}

template <typename G>
__global__ void degree_kernel(G g, const uint32_t* __restrict__ vs, uint64_t k, uint32_t* out, uint32_t* bad) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v = vs ? vs[i] : (uint32_t)i;
    if (v >= g.num_vertices()) {
      atomicOr(bad, 1u);
      out[i] = 0;
    } else {
      out[i] = g.degree(v);
    }
  }
}

template <typename G>
__global__ void degrees_kernel(G g, uint32_t* deg) {
  const uint32_t n = g.num_vertices();
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    deg[v] = g.degree((uint32_t)v);
}

// one warp per vertex copies its list to col[off[v]...]
template <typename G>
__global__ void export_col_kernel(G g, const uint64_t* __restrict__ off, uint32_t* __restrict__ col) {
  const uint32_t n = g.num_vertices();
  const uint32_t lane = lane_id();
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = w0; v < n; v += nw) {
    Seg sg = g.seg((uint32_t)v);
    uint64_t o = off[v];
    for (uint32_t i = lane; i < sg.len; i += 32) col[o + i] = __ldg(sg.p + i);
  }
}

__global__ void set_last_u64_kernel(uint64_t* a, uint64_t i, uint64_t v) { a[i] = v; }

}  // namespace

unsigned grid_for(uint64_t work, int threads) {
  uint64_t b = (work + threads - 1) / threads;
  uint64_t cap = (uint64_t)sm_count() * 16;
  if (b > cap) b = cap;
  if (b == 0) b = 1;
  return (unsigned)b;
}

namespace {

int bits_for(uint32_t n) {
  int lb = 1;
  while (lb < 32 && (1ull << lb) < (uint64_t)n) ++lb;
  return lb;
}

// The sorted keys (source << lb | destination) of the k pairs, and of their
// reverses if sym; self loops become the sentinel, which sorts last.  *keys
// and *tmp are the two key buffers (cnt entries each, released by the
// caller); *sorted is the one holding the result.
byo_status sorted_pair_keys(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t k, bool sym, int lb,
                            cudaStream_t s, uint64_t** keys, uint64_t** tmp, uint64_t** sorted) {
  const uint64_t cnt = sym ? 2 * k : k;
  *keys = *tmp = *sorted = nullptr;
  uint32_t* bad = nullptr;
  byo_status st = tmp_alloc_t(&bad, 4, s, "flag");
  if (st == BYO_OK) st = tmp_alloc_t(keys, cnt, s, "edge keys");
  if (st == BYO_OK) st = tmp_alloc_t(tmp, cnt, s, "edge keys tmp");
  if (st == BYO_OK) {
    cudaMemsetAsync(bad, 0, 16, s);
    if (k) {
      make_keys_kernel<<<grid_for(k, 256), 256, 0, s>>>(src, dst, k, n, lb, sym, *keys, bad);
      ::byo::note_launch();
    }
    cudaError_t e = cudaGetLastError();
    uint32_t hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "make_keys_kernel");
    else if (hbad) {
      set_error("a vertex id is >= n (%u)", n);
      st = BYO_ERR_INVALID_ARG;
    }
  }
  if (st == BYO_OK) st = radix_sort_u64(*keys, *tmp, cnt, 2 * lb, sorted, s);
  tmp_free(bad, s);
  return st;
}

uint64_t pair_sentinel(int lb) { return (lb == 32) ? ~0ull : ((1ull << (2 * lb)) - 1); }

// First output position of each tile's kept keys (*tile_offs, released by the
// caller) and the number of kept keys *m (read back to the host).
byo_status unique_positions(const uint64_t* sorted, uint64_t cnt, int lb, cudaStream_t s, uint64_t** tile_offs,
                            uint64_t* m) {
  *tile_offs = nullptr;
  *m = 0;
  const uint64_t ntiles = (cnt + kUniqTile - 1) / kUniqTile;
  if (ntiles == 0) return BYO_OK;
  uint32_t* counts = nullptr;
  BYO_RETURN_IF(tmp_alloc_t(&counts, ntiles, s, "unique counts"));
  byo_status st = tmp_alloc_t(tile_offs, ntiles, s, "unique positions");
  if (st == BYO_OK) {
    unique_count_kernel<<<(unsigned)ntiles, kUniqThreads, 0, s>>>(sorted, cnt, pair_sentinel(lb), counts);
    ::byo::note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_status(e, "unique_count_kernel");
  }
  if (st == BYO_OK) st = scan_u32_to_u64(counts, *tile_offs, ntiles, m, s);
  tmp_free(counts, s);
  return st;
}

template <typename OffT>
byo_status unique_write(const uint64_t* sorted, uint64_t cnt, int lb, const uint64_t* tile_offs, uint64_t m,
                        uint32_t n, uint32_t* col, uint32_t* rows, OffT* off, cudaStream_t s) {
  const uint64_t ntiles = (cnt + kUniqTile - 1) / kUniqTile;
  if (ntiles == 0 || m == 0) return BYO_OK;
  unique_write_kernel<OffT><<<(unsigned)ntiles, kUniqThreads, 0, s>>>(sorted, cnt, pair_sentinel(lb), lb, tile_offs,
                                                                       m, n, col, rows, off);
  ::byo::note_launch();
  BYO_CHECK_LAUNCH("unique_write_kernel");
  return BYO_OK;
}

template <typename G>
byo_status build_buckets(byo_graph* g, G view, cudaStream_t s) {
  uint32_t n = g->n;
  uint64_t *keys = nullptr, *tmp = nullptr, *sorted = nullptr;
  unsigned long long* hist = nullptr;
  BYO_RETURN_IF(tmp_alloc_t(&keys, n, s, "bucket keys"));
  byo_status st = tmp_alloc_t(&tmp, n, s, "bucket keys tmp");
  if (st == BYO_OK) st = tmp_alloc_t(&hist, kBuckets, s, "bucket histogram");
  if (st == BYO_OK && !g->vorder) st = dev_alloc_t(&g->vorder, n, "vertex order");
  if (st == BYO_OK && !g->d_bstart) st = dev_alloc_t(&g->d_bstart, kBuckets + 1, "bucket starts");
  if (st == BYO_OK) {
    ProfScope ps("buckets_keys", s);
    cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kBuckets, s);
    bucket_keys_kernel<G><<<grid_for(n, 256), 256, 0, s>>>(view, keys, hist); ::byo::note_launch();
    bucket_starts_kernel<<<1, 32, 0, s>>>(hist, g->d_bstart); ::byo::note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_status(e, "bucket_keys_kernel");
  }
  if (st == BYO_OK) {
    ProfScope ps("buckets_sort", s);
    st = radix_sort_u64(keys, tmp, n, kBucketBits, &sorted, s);
  }
  if (st == BYO_OK) {
    ProfScope ps("buckets_order", s);
    high_bits_kernel<<<grid_for(n, 256), 256, 0, s>>>(sorted, n, kBucketBits, g->vorder); ::byo::note_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g->bstart, g->d_bstart, sizeof(uint64_t) * (kBuckets + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "degree buckets");
  }
  tmp_free(keys, s);
  tmp_free(tmp, s);
  tmp_free(hist, s);
  return st;
}

void graph_free(byo_graph* g) {
  if (!g) return;
  dev_free(g->off);
  dev_free(g->col);
  dev_free(g->vorder);
  dev_free(g->d_bstart);
  bfs_free(g->bfs);
  pr_free(g->pr);
  tc_free(g->tc);
  dyn_free(g->dyn);
  comp_free(g->comp);
  if (g->member_base) cudaFree(g->member_base);
  delete[] g->member_base_host;
  dev_free(g->ms_seen);
  dev_free(g->ms_ctl);
  dev_free(g->ms_src);
  delete g;
}

byo_status build_csr(byo_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t k, bool sym, cudaStream_t s) {
  const uint32_t n = g->n;
  const int lb = bits_for(n > 1 ? n : 2);
  const uint64_t cnt = sym ? 2 * k : k;
  uint64_t *keys = nullptr, *tmp = nullptr, *sorted = nullptr, *tile_offs = nullptr;
  uint32_t *rows = nullptr, *bad = nullptr;
  uint64_t m = 0;
  byo_status st = sorted_pair_keys(n, src, dst, k, sym, lb, s, &keys, &tmp, &sorted);
  if (st == BYO_OK) st = unique_positions(sorted, cnt, lb, s, &tile_offs, &m);
  if (st == BYO_OK) {
    g->m = m;
    g->off64 = (g->flags & BYO_OFFSETS64) || m >= (1ull << 32);
    st = dev_alloc(&g->off, (size_t)(n + 1) * (g->off64 ? 8 : 4) + 16, "CSR offsets");
  }
  if (st == BYO_OK) st = dev_alloc_t(&g->col, m + 4, "CSR neighbours");
  if (st == BYO_OK && !sym && m) st = tmp_alloc_t(&rows, m, s, "sorted rows");
  if (st == BYO_OK) {
    cudaMemsetAsync(g->col + m, 0, 16, s);
    if (m == 0) cudaMemsetAsync(g->off, 0, (size_t)(n + 1) * (g->off64 ? 8 : 4), s);
    st = g->off64 ? unique_write<uint64_t>(sorted, cnt, lb, tile_offs, m, n, g->col, rows,
                                           static_cast<uint64_t*>(g->off), s)
                  : unique_write<uint32_t>(sorted, cnt, lb, tile_offs, m, n, g->col, rows,
                                           static_cast<uint32_t*>(g->off), s);
  }
  tmp_free(keys, s);
  tmp_free(tmp, s);
  tmp_free(tile_offs, s);
  if (st == BYO_OK && !sym && m) st = tmp_alloc_t(&bad, 1, s, "flag");
  if (st == BYO_OK && !sym && m) {
    cudaMemsetAsync(bad, 0, 4, s);
    if (g->off64)
      symmetric_kernel<uint64_t><<<grid_for(m, 256), 256, 0, s>>>(static_cast<uint64_t*>(g->off), g->col, rows, m, bad);
    else
      symmetric_kernel<uint32_t><<<grid_for(m, 256), 256, 0, s>>>(static_cast<uint32_t*>(g->off), g->col, rows, m, bad);
    ::byo::note_launch();
    cudaError_t e = cudaGetLastError();
    uint32_t hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "symmetric_kernel");
    else if (hbad) {
      set_error("byo_graph_build: input is not symmetric and BYO_SYMMETRIZE was not given");
      st = BYO_ERR_NOT_SYMMETRIC;
    }
  }
  tmp_free(rows, s);
  tmp_free(bad, s);
  if (st == BYO_OK) st = rebuild_buckets(g, s);
  if (st == BYO_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "byo_graph_build");
  }
  return st;
}

}  // namespace

byo_status sort_unique_pairs(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t k, bool sym,
                             cudaStream_t s, uint32_t** rows_out, uint32_t** cols_out, uint64_t* count) {
  *rows_out = *cols_out = nullptr;
  *count = 0;
  const int lb = bits_for(n > 1 ? n : 2);
  const uint64_t cnt = sym ? 2 * k : k;
  uint64_t *keys = nullptr, *tmp = nullptr, *sorted = nullptr, *tile_offs = nullptr;
  uint32_t *rows = nullptr, *cols = nullptr;
  uint64_t m = 0;
  byo_status st = sorted_pair_keys(n, src, dst, k, sym, lb, s, &keys, &tmp, &sorted);
  if (st == BYO_OK) st = unique_positions(sorted, cnt, lb, s, &tile_offs, &m);
  if (st == BYO_OK) st = tmp_alloc_t(&rows, m + 4, s, "sorted rows");
  if (st == BYO_OK) st = tmp_alloc_t(&cols, m + 4, s, "sorted cols");
  if (st == BYO_OK) st = unique_write<uint32_t>(sorted, cnt, lb, tile_offs, m, n, cols, rows, nullptr, s);
  tmp_free(keys, s);
  tmp_free(tmp, s);
  tmp_free(tile_offs, s);
  if (st != BYO_OK) {
    tmp_free(rows, s);
    tmp_free(cols, s);
    return st;
  }
  *rows_out = rows;
  *cols_out = cols;
  *count = m;
  return BYO_OK;
}

byo_status rebuild_buckets(byo_graph* g, cudaStream_t s) {
  ++g->version;
  return with_view(g, [&](auto view) { return build_buckets(g, view, s); });
}

}  // namespace byo

using namespace byo;

extern "C" {

const char* byo_last_error(void) { return g_err; }

byo_sched byo_sched_default(void) {
  byo_sched s;
  s.mode = BYO_SCHED_HEURISTIC;
  s.thr_thread = 16;
  s.thr_warp = 1024;
  s.alpha = 15.0f;
  s.beta = 18.0f;
  s.mlp = nullptr;
  s.action = 1;
  s.flags = 0;
  return s;
}

byo_status byo_graph_build(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t k, uint32_t flags,
                           void* stream, byo_graph** out) {
  clear_error();
  if (!out) {
    set_error("byo_graph_build: out is NULL");
    return BYO_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (k > 0 && (!src || !dst)) {
    set_error("byo_graph_build: NULL edge arrays with k = %llu", (unsigned long long)k);
    return BYO_ERR_INVALID_ARG;
  }
  if ((flags & BYO_COMPRESSED) && !(flags & BYO_CSR)) {
    set_error("byo_graph_build: BYO_COMPRESSED applies to BYO_CSR only");
    return BYO_ERR_INVALID_ARG;
  }
  if ((flags & BYO_DYN_NO_INLINE) && !(flags & BYO_DYNAMIC)) {
    set_error("byo_graph_build: BYO_DYN_NO_INLINE applies to BYO_DYNAMIC only");
    return BYO_ERR_INVALID_ARG;
  }
  if ((flags & BYO_DYN_HASH) && !(flags & BYO_DYNAMIC)) {
    set_error("byo_graph_build: BYO_DYN_HASH applies to BYO_DYNAMIC only");
    return BYO_ERR_INVALID_ARG;
  }
  if (!(flags & (BYO_CSR | BYO_DYNAMIC)) || (flags & BYO_CSR && flags & BYO_DYNAMIC)) {
    set_error("byo_graph_build: exactly one of BYO_CSR / BYO_DYNAMIC is required");
    return BYO_ERR_INVALID_ARG;
  }
  if (n == 0xFFFFFFFFu) {
    set_error("byo_graph_build: n must be < 2^32 - 1 (0xFFFFFFFF is the INF marker)");
    return BYO_ERR_INVALID_ARG;
  }
  if (k > (1ull << 36)) {
    set_error("byo_graph_build: k too large");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  byo_graph* g = new (std::nothrow) byo_graph();
  if (!g) {
    set_error("byo_graph_build: host allocation failed");
    return BYO_ERR_OUT_OF_MEMORY;
  }
  g->n = n;
  g->flags = flags;
  cudaGetDevice(&g->device);
  byo_status st;
  {
    ProfScope ps("csr_build", s);
    st = build_csr(g, src, dst, k, (flags & BYO_SYMMETRIZE) != 0, s);
    if (st == BYO_OK && (flags & BYO_DYNAMIC)) st = dyn_from_csr(g, s);
    if (st == BYO_OK && (flags & BYO_COMPRESSED)) st = comp_from_csr(g, s);
  }
  if (st != BYO_OK) {
    cudaStreamSynchronize(s);
    graph_free(g);
    return st;
  }
  *out = g;
  return BYO_OK;
}

byo_status byo_graph_destroy(byo_graph* g) {
  clear_error();
  if (!g) return BYO_OK;
  cudaDeviceSynchronize();
  graph_free(g);
  return BYO_OK;
}

byo_status byo_space(const byo_graph* g, uint64_t* host_bytes, void* stream) {
  clear_error();
  BYO_RETURN_IF(check_graph(g));
  if (!host_bytes) {
    set_error("byo_space: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  if (g->dyn) return dyn_space(g, host_bytes, static_cast<cudaStream_t>(stream));
  if (g->comp) {  // degree offsets, byte offsets and the code bytes
    *host_bytes = (uint64_t)(g->n + 1ull) * ((g->off64 ? 8u : 4u) + 8u) + comp_bytes(g);
    return BYO_OK;
  }
  *host_bytes = (uint64_t)(g->n + 1ull) * (g->off64 ? 8u : 4u) + 4ull * g->m;
  return BYO_OK;
}

byo_status byo_num_vertices(const byo_graph* g, uint32_t* host_n) {
  clear_error();
  BYO_RETURN_IF(check_graph(g));
  if (!host_n) {
    set_error("byo_num_vertices: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  *host_n = g->n;
  return BYO_OK;
}

byo_status byo_num_edges(const byo_graph* g, uint64_t* host_m) {
  clear_error();
  BYO_RETURN_IF(check_graph(g));
  if (!host_m) {
    set_error("byo_num_edges: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  *host_m = g->m;
  return BYO_OK;
}

byo_status byo_degree(const byo_graph* g, const uint32_t* vs, uint64_t k, uint32_t* out, void* stream) {
  clear_error();
  BYO_RETURN_IF(check_graph(g));
  if (!vs) k = g->n;
  if (k && !out) {
    set_error("byo_degree: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  if (k == 0) return BYO_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* bad = nullptr;
  BYO_RETURN_IF(tmp_alloc_t(&bad, 1, s, "flag"));
  cudaMemsetAsync(bad, 0, 4, s);
  with_view(g, [&](auto view) {
    degree_kernel<<<grid_for(k, 256), 256, 0, s>>>(view, vs, k, out, bad);
    return BYO_OK;
  });
  ::byo::note_launch();
  cudaError_t e = cudaGetLastError();
  uint32_t hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s);
  tmp_free(bad, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "byo_degree");
  if (hbad) {
    set_error("byo_degree: a vertex id is >= n");
    return BYO_ERR_INVALID_ARG;
  }
  return BYO_OK;
}

byo_status byo_graph_export_csr(const byo_graph* g, uint64_t* offsets, uint32_t* col, void* stream) {
  clear_error();
  BYO_RETURN_IF(check_graph(g));
  if (!offsets || (g->m && !col)) {
    set_error("byo_graph_export_csr: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // offsets = exclusive scan of the degrees, then one warp per vertex copies its list
  uint32_t* deg = nullptr;
  BYO_RETURN_IF(tmp_alloc_t(&deg, g->n + 1ull, s, "export degrees"));
  byo_status st = with_view(g, [&](auto view) {
    degrees_kernel<<<grid_for(g->n, 256), 256, 0, s>>>(view, deg);
    ::byo::note_launch();
    return BYO_OK;
  });
  if (st == BYO_OK) st = scan_u32_to_u64(deg, offsets, g->n, nullptr, s);
  if (st == BYO_OK) {
    set_last_u64_kernel<<<1, 1, 0, s>>>(offsets, g->n, g->m);
    ::byo::note_launch();
    if (g->comp) {
      st = comp_export(g, offsets, col, s);
    } else {
      st = with_view(g, [&](auto view) {
        export_col_kernel<<<grid_for((uint64_t)g->n * 32, 256), 256, 0, s>>>(view, offsets, col);
        ::byo::note_launch();
        return BYO_OK;
      });
      if (st == BYO_OK && g->dyn && g->dyn->hashed) st = dyn_sort_lists(g, offsets, col, s);
    }
  }
  tmp_free(deg, s);
  BYO_RETURN_IF(st);
  BYO_CHECK_LAUNCH("byo_graph_export_csr");
  return BYO_OK;
}

}  // extern "C"
