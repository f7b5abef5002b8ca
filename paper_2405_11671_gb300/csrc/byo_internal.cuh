// byo_internal.cuh -- shared declarations of libbyo.so (host structs, error
// plumbing, device helpers).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/byo.h"

namespace byo {

// ---------------------------------------------------------------- constants
constexpr uint32_t kInf = 0xFFFFFFFFu;
// Degree buckets: bucket(0) = 0, bucket(d) = 1 + floor(log2 d) for d >= 1, so
// bucket b >= 1 holds degrees [2^(b-1), 2^b).  33 buckets cover uint32 degrees.
constexpr int kBuckets = 33;
constexpr int kWarp = 32;

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();
byo_status cuda_status(cudaError_t e, const char* what);

#define BYO_CUDA(call)                                                     \
  do {                                                                     \
    cudaError_t _e = (call);                                               \
    if (_e != cudaSuccess) return ::byo::cuda_status(_e, #call);           \
  } while (0)

#define BYO_CHECK_LAUNCH(what)                                             \
  do {                                                                     \
    cudaError_t _e = cudaGetLastError();                                   \
    if (_e != cudaSuccess) return ::byo::cuda_status(_e, what);            \
  } while (0)

#define BYO_RETURN_IF(st)                                                  \
  do {                                                                     \
    byo_status _s = (st);                                                  \
    if (_s != BYO_OK) return _s;                                           \
  } while (0)

// Device allocation that reports OUT_OF_MEMORY through the error string.
byo_status dev_alloc(void** p, size_t bytes, const char* what);
template <typename T>
inline byo_status dev_alloc_t(T** p, size_t count, const char* what) {
  return dev_alloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16, what);
}
void dev_free(void* p);
// Stream-ordered temporaries (cudaMallocAsync / cudaFreeAsync on stream s).
byo_status tmp_alloc(void** p, size_t bytes, cudaStream_t s, const char* what);
template <typename T>
inline byo_status tmp_alloc_t(T** p, size_t count, cudaStream_t s, const char* what) {
  return tmp_alloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16, s, what);
}
void tmp_free(void* p, cudaStream_t s);

int sm_count();
uint64_t timeout_ns();

// ---------------------------------------------------------------- scan / sort
// Exclusive scan of n uint32 flags/counts into uint64 (out may alias nothing).
// *host_total (nullable) receives the total and synchronises the stream.
byo_status scan_u32_to_u64(const uint32_t* in, uint64_t* out, uint64_t n, uint64_t* host_total, cudaStream_t s);
byo_status scan_u64_inplace(uint64_t* data, uint64_t n, cudaStream_t s);
// LSD radix sort of n uint64 keys on bits [0, bits).  Uses keys and tmp
// (both n entries); *sorted points at whichever holds the result.
byo_status radix_sort_u64(uint64_t* keys, uint64_t* tmp, uint64_t n, int bits, uint64_t** sorted, cudaStream_t s);

// ---------------------------------------------------------------- workspaces
struct BfsWork;
struct PrWork;
struct TcWork;
struct DynStore;
struct CompStore;
struct SchedParams;

}  // namespace byo

// The graph handle.  Static CSR: off (uint32 or uint64, n+1), col (m + 4
// padding entries, 16-byte aligned).  vorder lists the vertices grouped by
// degree bucket, ascending inside each bucket; bstart[b] is where bucket b
// starts in vorder (host copy and device copy).
struct byo_graph {
  uint32_t n = 0;
  uint64_t m = 0;
  uint64_t version = 0;  // bumped whenever the structure changes (cached launch plans depend on it)
  bool buckets_stale = false;  // vorder/bstart lag the degrees (see ready_graph)
  uint32_t flags = 0;
  bool off64 = false;
  int device = 0;
  void* off = nullptr;
  uint32_t* col = nullptr;
  uint32_t* vorder = nullptr;
  uint64_t bstart[byo::kBuckets + 1] = {0};
  uint64_t* d_bstart = nullptr;
  byo::BfsWork* bfs = nullptr;
  byo::PrWork* pr = nullptr;
  byo::TcWork* tc = nullptr;
  byo::DynStore* dyn = nullptr;  // set for BYO_DYNAMIC (then off/col are unused)
  byo::CompStore* comp = nullptr;  // set for BYO_COMPRESSED (then col is unused; off gives the degrees)
  // batch of graphs (byo_batch_build): member i owns ids [member_base[i], member_base[i+1])
  uint32_t members = 0;
  uint32_t* member_base = nullptr;       // device
  uint32_t* member_base_host = nullptr;  // host
  // multi-source BFS scratch
  unsigned long long* ms_seen = nullptr;  // seen, frontier, next words (3n)
  void* ms_ctl = nullptr;
  uint32_t* ms_src = nullptr;
  uint64_t ms_src_cap = 0;
};

namespace byo {
void bfs_free(BfsWork* w);
void pr_free(PrWork* w);
void tc_free(TcWork* w);
void dyn_free(DynStore* d);
void comp_free(CompStore* c);
// Compressed container (compressed.cu): encode g's CSR into byte codes and
// release the neighbour ids; decode into col laid out by offsets; BFS.
byo_status comp_from_csr(byo_graph* g, cudaStream_t s);
byo_status comp_export(const byo_graph* g, const uint64_t* offsets, uint32_t* col, cudaStream_t s);
byo_status comp_bfs(const byo_graph* g, const uint32_t* sources, uint32_t ns, uint32_t* levels, uint32_t* parents,
                    const SchedParams& sp, cudaStream_t s);
uint64_t comp_bytes(const byo_graph* g);
byo_status check_graph(const byo_graph* g);
// check_graph, then re-derive the degree buckets on stream s if a batch update
// could not (it ran out of memory after applying the batch).
byo_status ready_graph(const byo_graph* g, cudaStream_t s);
// Sorted, unique (row, col) pairs of k raw pairs (both directions when sym,
// self-loops dropped).  *rows and *cols are stream-ordered temporaries of
// *count + 4 entries that the caller releases with tmp_free.  Ids >= n give
// BYO_ERR_INVALID_ARG.  Synchronises the stream.
byo_status sort_unique_pairs(uint32_t n, const uint32_t* src, const uint32_t* dst, uint64_t k, bool sym,
                             cudaStream_t s, uint32_t** rows, uint32_t** cols, uint64_t* count);
// Recompute vorder / bstart from the container's current degrees.
byo_status rebuild_buckets(byo_graph* g, cudaStream_t s);
// Fill g->dyn from the CSR just built in g (then releases the CSR arrays).
byo_status dyn_from_csr(byo_graph* g, cudaStream_t s);
// Bytes of a dynamic container's records and held pool blocks (synchronises).
byo_status dyn_space(const byo_graph* g, uint64_t* host_bytes, cudaStream_t s);
// Sort each list of an exported CSR (off, col) ascending: the hash-indexed
// dynamic container keeps its lists in insertion order.
byo_status dyn_sort_lists(const byo_graph* g, const uint64_t* off, uint32_t* col, cudaStream_t s);
unsigned grid_for(uint64_t work, int threads);
}  // namespace byo

// ================================================================ device side
namespace byo {

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// L2-only loads for data that other SMs write during the same kernel.
__device__ __forceinline__ uint32_t ld_cg(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint64_t ld_cg(const unsigned long long* p) { return __ldcg(p); }

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int degree_bucket(uint32_t d) { return d == 0 ? 0 : 32 - __clz(d); }

// Grid-wide barrier for a cooperative launch.  One 64-bit arrival counter
// that only grows within a launch: the k-th barrier of a launch of B CTAs
// takes the arrivals numbered [kB, (k+1)B), because no CTA can arrive at a
// barrier before all B have arrived at the one before it.  So each CTA's
// thread 0 adds one (acquire-release, which also publishes what the CTA wrote
// before the barrier) and waits until the counter reaches the next multiple of
// B above the number its add returned; the last to arrive does not wait.
// The counter must be zero when a launch starts (reset_barrier).  A wait
// is bounded by `limit_ns`; on timeout the error word is set and false is
// returned (the caller leaves its loop and exits).
struct GridBar {
  unsigned long long arrive;
  uint32_t pad[30];
};

__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long* p, unsigned long long v) {
  unsigned long long r;
  asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(v) : "memory");
  return r;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_barrier(GridBar* bar, uint32_t nblocks, uint32_t* err, uint64_t limit_ns) {
  __shared__ uint32_t ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t ok = 1;
    const unsigned long long old = atom_add_acq_rel(&bar->arrive, 1ull);
    const unsigned long long target = (old / nblocks + 1) * nblocks;
    if (old + 1 != target) {
      uint64_t t0 = globaltimer();
      uint32_t spins = 0;
      while (ld_acquire(&bar->arrive) < target) {
        if (++spins > 64) {
          spins = 0;
          if (ld_cg(err) != 0 || globaltimer() - t0 > limit_ns) {
            atomicCAS(err, 0u, (uint32_t)BYO_ERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Clears the arrival counter of `bar` on stream `s`; called before each
// cooperative launch that synchronises through it.
inline cudaError_t reset_barrier(GridBar* bar, cudaStream_t s) {
  return cudaMemsetAsync(&bar->arrive, 0, sizeof(bar->arrive), s);
}

}  // namespace byo
