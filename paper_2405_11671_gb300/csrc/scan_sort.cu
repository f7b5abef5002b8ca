// scan_sort.cu -- device-wide exclusive scan and LSD radix sort of 64-bit
// keys.  Used to build the CSR (sort of packed (src, dst) keys, then unique),
// to group vertices by degree bucket, and to pre-process update batches (the
// library sorts unsorted batches, Section 4.2).
#include <vector>

#include "byo_internal.cuh"
#include "prof.cuh"

namespace byo {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if ((int)lane_id() >= o) x += y;
  }
  return x;
}

// Exclusive scan of one value per thread across the CTA (1024 threads).
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t x) {
  __shared__ uint64_t warp_sums[kScanThreads / 32];
  uint64_t inc = warp_inclusive_scan(x);
  int w = threadIdx.x >> 5;
  if (lane_id() == 31) warp_sums[w] = inc;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    uint64_t s = lane_id() < (uint32_t)nw ? warp_sums[lane_id()] : 0;
    uint64_t si = warp_inclusive_scan(s);
    if (lane_id() < (uint32_t)nw) warp_sums[lane_id()] = si - s;
  }
  __syncthreads();
  return warp_sums[w] + inc - x;
}

template <typename In>
__global__ void tile_reduce_kernel(const In* in, uint64_t n, uint64_t* tile_sums) {
  uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += (uint64_t)in[base + i];
  __shared__ uint64_t red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  if (lane_id() == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint64_t t = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = t;
  }
}

// Exclusive scan of a tile, offset by tile_offsets[tile] (nullable = 0).
// in and out may alias.
template <typename In>
__global__ void tile_scan_kernel(const In* in, uint64_t* out, uint64_t n, const uint64_t* tile_offsets) {
  uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint64_t v[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? (uint64_t)in[base + i] : 0;
    s += v[i];
  }
  uint64_t run = block_exclusive_scan(s);
  if (tile_offsets) run += tile_offsets[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

__global__ void read_total_kernel(const uint64_t* scanned, const uint64_t* tile_sums_scanned, uint64_t ntiles,
                                  const uint64_t* last_tile_sum, uint64_t* total) {
  *total = tile_sums_scanned[ntiles - 1] + *last_tile_sum;
}

template <typename In>
byo_status scan_impl(const In* in, uint64_t* out, uint64_t n, uint64_t* host_total, cudaStream_t s) {
  if (n == 0) {
    if (host_total) *host_total = 0;
    return BYO_OK;
  }
  uint64_t ntiles = (n + kScanTile - 1) / kScanTile;
  uint64_t* sums = nullptr;
  BYO_RETURN_IF(tmp_alloc_t(&sums, ntiles + 2, s, "scan tile sums"));
  tile_reduce_kernel<In><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, sums); ::byo::note_launch();
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    tmp_free(sums, s);
    return cuda_status(le, "tile_reduce_kernel");
  }
  // keep the last tile's sum to form the total after the in-place scan
  uint64_t* last = sums + ntiles;
  cudaMemcpyAsync(last, sums + ntiles - 1, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
  byo_status st = BYO_OK;
  if (ntiles > 1) st = scan_u64_inplace(sums, ntiles, s);
  else cudaMemsetAsync(sums, 0, sizeof(uint64_t), s);
  if (st != BYO_OK) {
    tmp_free(sums, s);
    return st;
  }
  tile_scan_kernel<In><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, out, n, sums); ::byo::note_launch();
  le = cudaGetLastError();
  if (le == cudaSuccess && host_total) {
    uint64_t* tot = sums + ntiles + 1;
    read_total_kernel<<<1, 1, 0, s>>>(out, sums, ntiles, last, tot); ::byo::note_launch();
    le = cudaMemcpyAsync(host_total, tot, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (le == cudaSuccess) le = cudaStreamSynchronize(s);
  }
  tmp_free(sums, s);
  if (le != cudaSuccess) return cuda_status(le, "scan");
  return BYO_OK;
}

// ---------------------------------------------------------------- radix sort
constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 8;  // keys per lane
constexpr int kWarpKeys = 32 * kSortRounds;
constexpr uint64_t kSortTile = (uint64_t)kSortWarps * kWarpKeys;
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                                  int shift, uint32_t mask, uint32_t* hist,
                                                                  uint64_t ntiles) {
  __shared__ uint32_t h[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kSortTile + threadIdx.x;
  uint64_t k[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {  // all loads in flight before the first count
    const uint64_t idx = base + (uint64_t)r * kSortThreads;
    k[r] = idx < n ? __ldg(keys + idx) : 0;
  }
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r)
    if (base + (uint64_t)r * kSortThreads < n) atomicAdd(&h[(uint32_t)(k[r] >> shift) & mask], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) hist[(uint64_t)d * ntiles + blockIdx.x] = h[d];
}

// One tile of kSortTile keys per CTA.  Each key's rank among the tile's keys
// of its digit comes from per-bit ballots and per-warp digit counters; the tile
// is then reordered by digit in shared memory (stable: warps, then rounds,
// then lanes in order) and written out run by run, so that consecutive
// threads store consecutive addresses of a digit's output range.
constexpr size_t kScatterSmem = (size_t)kSortTile * sizeof(uint64_t);
static_assert(kRadix == 1 << 8, "the scatter ranks keys with one ballot per bit of an 8-bit digit");

__global__ void __launch_bounds__(kSortThreads, 2) radix_scatter_kernel(const uint64_t* __restrict__ keys,
                                                                     uint64_t* __restrict__ out, uint64_t n,
                                                                     int shift, uint32_t mask,
                                                                     const uint64_t* __restrict__ offs,
                                                                     uint64_t ntiles) {
  extern __shared__ __align__(16) uint64_t sk[];  // the tile, reordered by digit
  __shared__ uint32_t cnt[kSortWarps][kRadix];
  __shared__ uint32_t start[kRadix];              // tile-local start of each digit
  __shared__ uint64_t gbase[kRadix];              // output index of the digit's tile-local position 0
  const int w = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += blockDim.x) (&cnt[0][0])[i] = 0;
  __syncthreads();
  const uint64_t tile0 = (uint64_t)blockIdx.x * kSortTile;
  const uint64_t base = tile0 + (uint64_t)w * kWarpKeys;
  uint64_t k[kSortRounds];
  uint32_t rank[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    uint64_t idx = base + (uint64_t)r * 32 + lane;
    bool valid = idx < n;
    k[r] = valid ? keys[idx] : 0;
    uint32_t d = valid ? ((uint32_t)(k[r] >> shift) & mask) : 0u;
    // the valid lanes holding the same digit: one ballot per digit bit (a warp
    // match instruction is several times slower)
    uint32_t peers = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const uint32_t bb = __ballot_sync(0xFFFFFFFFu, (d >> b) & 1u);
      peers &= ((d >> b) & 1u) ? bb : ~bb;
    }
    uint32_t before = __popc(peers & lanemask_lt());
    uint32_t c = valid ? cnt[w][d] : 0;
    rank[r] = c + before;
    __syncwarp();
    if (valid && before == 0) cnt[w][d] = c + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive offsets over the warps, and the digit's tile total
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kSortWarps; ++ww) {
      uint32_t t = cnt[ww][d];
      cnt[ww][d] = run;
      run += t;
    }
    start[d] = run;  // total for now
    gbase[d] = offs[(uint64_t)d * ntiles + blockIdx.x];
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan of the digit totals (256 = 8 per lane)
    uint32_t v[kRadix / 32], sum = 0;
#pragma unroll
    for (int j = 0; j < kRadix / 32; ++j) {
      v[j] = start[lane * (kRadix / 32) + j];
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
    for (int j = 0; j < kRadix / 32; ++j) {
      start[lane * (kRadix / 32) + j] = run;
      gbase[lane * (kRadix / 32) + j] -= run;  // now the output index of tile-local position 0 of the digit
      run += v[j];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    uint64_t idx = base + (uint64_t)r * 32 + lane;
    if (idx < n) {
      uint32_t d = (uint32_t)(k[r] >> shift) & mask;
      sk[start[d] + cnt[w][d] + rank[r]] = k[r];
    }
  }
  __syncthreads();
  const uint32_t count = (uint32_t)(n - tile0 < kSortTile ? n - tile0 : kSortTile);
  for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) {
    const uint64_t key = sk[i];
    out[gbase[(uint32_t)(key >> shift) & mask] + i] = key;
  }
}

}  // namespace

byo_status scan_u32_to_u64(const uint32_t* in, uint64_t* out, uint64_t n, uint64_t* host_total, cudaStream_t s) {
  return scan_impl<uint32_t>(in, out, n, host_total, s);
}

byo_status scan_u64_inplace(uint64_t* data, uint64_t n, cudaStream_t s) {
  return scan_impl<uint64_t>(data, data, n, nullptr, s);
}

byo_status radix_sort_u64(uint64_t* keys, uint64_t* tmp, uint64_t n, int bits, uint64_t** sorted, cudaStream_t s) {
  *sorted = keys;
  if (n <= 1 || bits <= 0) return BYO_OK;
  uint64_t ntiles = (n + kSortTile - 1) / kSortTile;
  uint32_t* hist = nullptr;
  uint64_t* offs = nullptr;
  BYO_RETURN_IF(tmp_alloc_t(&hist, (uint64_t)kRadix * ntiles, s, "radix histogram"));
  byo_status st = tmp_alloc_t(&offs, (uint64_t)kRadix * ntiles, s, "radix offsets");
  if (st != BYO_OK) {
    tmp_free(hist, s);
    return st;
  }
  {
    cudaError_t e = cudaFuncSetAttribute(radix_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kScatterSmem);
    if (e != cudaSuccess) st = cuda_status(e, "radix_scatter_kernel shared memory");
  }
  uint64_t* a = keys;
  uint64_t* b = tmp;
  for (int shift = 0; shift < bits && st == BYO_OK; shift += 8) {
    int w = bits - shift < 8 ? bits - shift : 8;
    uint32_t mask = (1u << w) - 1u;
    radix_hist_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(a, n, shift, mask, hist, ntiles); ::byo::note_launch();
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
      st = cuda_status(le, "radix_hist_kernel");
      break;
    }
    st = scan_u32_to_u64(hist, offs, (uint64_t)kRadix * ntiles, nullptr, s);
    if (st != BYO_OK) break;
    radix_scatter_kernel<<<(unsigned)ntiles, kSortThreads, kScatterSmem, s>>>(a, b, n, shift, mask, offs, ntiles);
    ::byo::note_launch();
    le = cudaGetLastError();
    if (le != cudaSuccess) {
      st = cuda_status(le, "radix_scatter_kernel");
      break;
    }
    uint64_t* t = a;
    a = b;
    b = t;
  }
  tmp_free(hist, s);
  tmp_free(offs, s);
  *sorted = a;
  return st;
}

}  // namespace byo
