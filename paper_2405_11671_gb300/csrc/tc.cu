// tc.cu -- triangle counting by filter-then-intersect (Section 4.4: a filter
// builds a smaller DAG first, then neighbour sets are intersected).
//
// Filter: each edge is kept once, from the endpoint of lower rank, where
// rank(v) = (degree(v), v) in lexicographic order.  The DAG is stored in rank
// space: vertex v becomes its position in that order (a radix sort of the
// (degree, id) keys), so that N+(r) holds only ids above r and the out-lists
// of high-degree vertices fall in the short range of top ranks.
// Count: the number of triangles is the sum over DAG edges u->v of
// |N+(u) intersect N+(v)| (the count does not depend on the labels).  Each
// edge is intersected from the side with the shorter out-list: N+(c) of a
// "centre" c is put into a shared-memory set and the out-lists of its
// partners (out-neighbours p with d+(p) <= d+(c), in-neighbours p with d+(p) <
// d+(c)) are walked 32 ids at a time by a warp (edge-balanced across the warp)
// and probed.  Centres with |N+(c)| <= kLightMax: one warp each; N+(c) is
// staged by a TMA bulk copy (cp.async.bulk, completion on an mbarrier; no
// multicast) and loaded into an open-addressing hash set in the warp's shared
// memory.  Larger centres: one CTA each (taken from a work counter); when the
// rank range above c fits the CTA's shared memory, N+(c) becomes a bitmap of
// that range (one probe per id, no collisions), otherwise it is staged in
// windows of kWindow ids, each hashed into the CTA's shared memory.
// Out-lists of kSortedMin..kSortedMax ids are sorted by rank after the filter
// (bitonic networks: one warp per list up to kWarpSortMax ids, in registers,
// one CTA per longer list, in shared memory), so that the walk of an
// in-neighbour p's out-list for a centre c skips the ids at or below c, which
// N+(c) cannot hold: the lane holding p finds where they end by binary search.
#include <stdlib.h>

#include "byo_internal.cuh"
#include "prof.cuh"
#include "container.cuh"
#include "vbins.cuh"
#include "rank.cuh"

namespace byo {

constexpr uint32_t kLightMax = 256;   // capacity of a warp's shared-memory slice (ids)
constexpr uint32_t kWindow = 2048;    // capacity of a CTA's shared-memory window (ids)
constexpr int kTcThreads = 256;
constexpr uint32_t kSortedMin = 32;       // shorter out-lists are walked in concatenation, never trimmed
constexpr uint32_t kWarpSortMax = 1024;   // longest out-list sorted by one warp
constexpr uint32_t kSortedMax = 16384;    // longest out-list sorted at all (by one CTA)

// The light/heavy split, the window length, the bitmap range and the sorted
// out-list lengths can be lowered (never raised) with BYO_TC_LIGHT_MAX /
// BYO_TC_WINDOW / BYO_TC_BITMAP_BITS / BYO_TC_WARP_SORT_MAX / BYO_TC_SORT_MAX,
// so that small test graphs exercise the CTA path, the hashed windows,
// multi-window intersections, both sorts and unsorted long out-lists.
static uint32_t env_cap(const char* name, uint32_t cap) {
  const char* e = getenv(name);
  if (!e || !*e) return cap;
  long long v = atoll(e);
  if (v < 4) v = 4;
  return v < (long long)cap ? (uint32_t)v : cap;
}

// A DAG row in rank space: N+(r) = dag[off, off + dplus), N-(r) = dag[off +
// dplus, off + len); one 16-byte load gives a partner's walked list.
struct __align__(16) RowInfo {
  uint64_t off;
  uint32_t dplus, len;
};

struct TcWork {
  uint32_t n = 0;
  uint64_t cap = 0;             // capacity of dag (stored entries)
  RowInfo* row = nullptr;       // n + 1, rank-indexed: where each DAG row starts, |N+|, |row|
  uint64_t* roff = nullptr;     // n + 1: row starts (scan of the degrees in rank order)
  uint32_t* dag = nullptr;      // cap + 8: row r = N+(r) then N-(r), rank ids
  uint32_t* rdeg = nullptr;     // n: degree of rank r
  uint32_t* rank = nullptr;     // n: vertex id -> position in (degree, id) order
  uint32_t* cnt_l = nullptr;    // n: light task counts
  uint32_t* cnt_h = nullptr;    // n: heavy task counts
  uint64_t* pos_l = nullptr;    // n + 1
  uint64_t* pos_h = nullptr;    // n + 1
  uint32_t* ctr = nullptr;      // [2] light cursor, [3] error, [4] heavy cursor
  unsigned long long* count = nullptr;
  unsigned long long* work = nullptr;  // [0] sum d+(c)^2, [1] sum d-(c) d+(c), [2] sum over edges of the shorter out-list
  unsigned long long host_work[3] = {0, 0, 0};
};

void tc_free(TcWork* w) {
  if (!w) return;
  dev_free(w->row);
  dev_free(w->roff);
  dev_free(w->dag);
  dev_free(w->rdeg);
  dev_free(w->rank);
  dev_free(w->cnt_l);
  dev_free(w->cnt_h);
  dev_free(w->pos_l);
  dev_free(w->pos_h);
  dev_free(w->ctr);
  dev_free(w->count);
  dev_free(w->work);
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
// One pass over every neighbour list: the ranks of v's higher-rank neighbours
// (N+) go to the front of row rank(v) of the DAG, those of the lower-rank ones
// (N-) to its back, both in v's stored neighbour order; the row's RowInfo
// records |N+|.  Rows are laid out in rank order (row starts = a scan of the
// degrees in rank order), so no counting pass is needed.
template <typename G>
__global__ void __launch_bounds__(kTcThreads) tc_fill_kernel(G g, VBins bins, const uint32_t* __restrict__ rank,
                                                             const uint64_t* __restrict__ roff,
                                                             uint32_t* __restrict__ dag, RowInfo* __restrict__ row) {
  VRange r = vbins_range(bins);
  const uint32_t lane = lane_id();
  if (r.role == kRoleThread) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      const uint32_t rv = __ldg(rank + v);
      const uint64_t b = roff[rv];
      uint64_t o = b, q = b + s.len;
      for (uint32_t k = 0; k < s.len; k += 8) {  // eight ids and their ranks in flight before the stores
        uint32_t u[8], ru[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) u[j] = k + j < s.len ? __ldg(s.p + k + j) : 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) ru[j] = k + j < s.len ? __ldg(rank + u[j]) : 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (k + j >= s.len) break;
          if (ru[j] > rv) dag[o++] = ru[j];
          else dag[--q] = ru[j];
        }
      }
      row[rv] = RowInfo{b, (uint32_t)(o - b), s.len};
    }
  } else if (r.role == kRoleWarp) {
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      const uint32_t rv = __ldg(rank + v);
      const uint64_t b = roff[rv];
      uint64_t o = b, q = b + s.len;
      for (uint32_t base = 0; base < s.len; base += 128) {  // four chunks' ranks in flight before the stores
        uint32_t ru[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t k = base + 32 * j + lane;
          ru[j] = k < s.len ? __ldg(s.p + k) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) ru[j] = base + 32 * j + lane < s.len ? __ldg(rank + ru[j]) : 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t k = base + 32 * j + lane;
          bool keep = k < s.len && ru[j] > rv;
          bool back = k < s.len && !keep;
          uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep), bbk = __ballot_sync(0xFFFFFFFFu, back);
          if (keep) dag[o + __popc(bal & lanemask_lt())] = ru[j];
          if (back) dag[q - 1 - __popc(bbk & lanemask_lt())] = ru[j];
          o += __popc(bal);
          q -= __popc(bbk);
        }
      }
      if (lane == 0) row[rv] = RowInfo{b, (uint32_t)(o - b), s.len};
    }
  } else {
    __shared__ uint32_t wcnt[2][kTcThreads / 32];
    __shared__ uint32_t wpre[2][kTcThreads / 32 + 1];
    const uint32_t nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    for (uint64_t i = r.begin; i < r.end; i += r.stride) {
      uint32_t v = __ldg(bins.vorder + i);
      Seg s = g.seg(v);
      const uint32_t rv = __ldg(rank + v);
      const uint64_t b = roff[rv];
      uint64_t o = b, q = b + s.len;
      for (uint32_t base = 0; base < s.len; base += blockDim.x) {
        uint32_t k = base + threadIdx.x;
        uint32_t ru = k < s.len ? __ldg(rank + __ldg(s.p + k)) : 0;
        bool keep = k < s.len && ru > rv;
        bool back = k < s.len && !keep;
        uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep), bbk = __ballot_sync(0xFFFFFFFFu, back);
        if (lane == 0) {
          wcnt[0][w] = __popc(bal);
          wcnt[1][w] = __popc(bbk);
        }
        __syncthreads();
        if (threadIdx.x < 2) {
          wpre[threadIdx.x][0] = 0;
          for (uint32_t j = 0; j < nw; ++j) wpre[threadIdx.x][j + 1] = wpre[threadIdx.x][j] + wcnt[threadIdx.x][j];
        }
        __syncthreads();
        if (keep) dag[o + wpre[0][w] + __popc(bal & lanemask_lt())] = ru;
        if (back) dag[q - 1 - wpre[1][w] - __popc(bbk & lanemask_lt())] = ru;
        o += wpre[0][nw];
        q -= wpre[1][nw];
        __syncthreads();
      }
      if (threadIdx.x == 0) row[rv] = RowInfo{b, (uint32_t)(o - b), s.len};
    }
  }
}

// ---------------------------------------------------------------- sorted out-lists
// Ascending bitonic sorting network over buf[0, S) (S a power of two) by
// `lanes` threads, this one numbered t; the stages are ordered by a warp
// (kCta = false) or CTA barrier.
template <bool kCta>
__device__ __forceinline__ void bitonic_sort(uint32_t* buf, uint32_t S, uint32_t t, uint32_t lanes) {
  for (uint32_t k = 2; k <= S; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t q = t; q < S / 2; q += lanes) {  // pair q: (i, i + j), i = q with a zero inserted at bit j
        const uint32_t i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
        const uint32_t l = i | j;
        const uint32_t a = buf[i], b = buf[l];
        if ((a > b) == ((i & k) == 0)) {
          buf[i] = b;
          buf[l] = a;
        }
      }
      if (kCta) __syncthreads();
      else __syncwarp();
    }
}

__host__ __device__ __forceinline__ uint32_t pow2_at_least(uint32_t d) {
  uint32_t s = 1;
  while (s < d) s <<= 1;
  return s;
}

// One warp sorts an out-list of d <= 32 R ids held in registers: element
// e = 32 r + lane is v[r] of that lane, padded with kInf.  Stages that pair
// elements less than 32 apart exchange them between lanes, the others between
// a lane's registers.
template <int R>
__device__ __forceinline__ void warp_sort_list(uint32_t* p, uint32_t d) {
  const uint32_t lane = lane_id();
  uint32_t v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = r * 32 + lane < d ? p[r * 32 + lane] : kInf;
#pragma unroll
  for (uint32_t k = 2; k <= 32u * R; k <<= 1) {
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int r2 = r | (int)(j / 32);
          if (r2 != r) {
            const bool asc = ((uint32_t)(r * 32) & k) == 0;  // k >= 64: the lane bits do not matter
            const uint32_t a = v[r], b = v[r2];
            v[r] = asc ? min(a, b) : max(a, b);
            v[r2] = asc ? max(a, b) : min(a, b);
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t o = __shfl_xor_sync(0xFFFFFFFFu, v[r], j);
          const bool asc = ((r * 32 + lane) & k) == 0, lower = (lane & j) == 0;
          v[r] = asc == lower ? min(v[r], o) : max(v[r], o);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r * 32 + lane < d) p[r * 32 + lane] = v[r];
}

// Out-lists of kSortedMin..wmax ids, one warp each: the warp reads the row
// records of 32 rows at a time and sorts the ones in range in registers.
__global__ void __launch_bounds__(kTcThreads) tc_sort_warp_kernel(const RowInfo* __restrict__ row,
                                                                 uint32_t* __restrict__ dag, uint32_t n,
                                                                 uint32_t wmax) {
  const uint32_t lane = lane_id();
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r0 = gw * 32; r0 < n; r0 += nw * 32) {
    uint64_t off = 0;
    uint32_t d = 0;
    if (r0 + lane < n) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(row + r0 + lane));
      off = ((uint64_t)q.y << 32) | q.x;
      d = q.z;
    }
    uint32_t todo = __ballot_sync(0xFFFFFFFFu, d >= kSortedMin && d <= wmax);
    while (todo) {
      const int l = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t dl = __shfl_sync(0xFFFFFFFFu, d, l);
      uint32_t* p = dag + __shfl_sync(0xFFFFFFFFu, off, l);
      switch (pow2_at_least(dl)) {
        case 32: warp_sort_list<1>(p, dl); break;
        case 64: warp_sort_list<2>(p, dl); break;
        case 128: warp_sort_list<4>(p, dl); break;
        case 256: warp_sort_list<8>(p, dl); break;
        case 512: warp_sort_list<16>(p, dl); break;
        default: warp_sort_list<32>(p, dl); break;  // 1024 = kWarpSortMax
      }
    }
  }
}

// degree of rank r, from the sorted (degree << lbn | v) keys
__global__ void tc_rdeg_kernel(const uint64_t* __restrict__ sorted, uint32_t n, int lbn, uint32_t* __restrict__ rdeg) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x)
    rdeg[r] = (uint32_t)(sorted[r] >> lbn);
}

__global__ void tc_set_last_kernel(uint64_t* off, uint32_t n, uint64_t total) { off[n] = total; }

// Work items.  Every DAG edge a->b is intersected from the side with the
// shorter out-list: at centre a (walk N+(b), probe N+(a)) when d+(b) <= d+(a),
// else at centre b (walk N+(a), probe N+(b)).  A warp task is one centre c
// (whose N+(c) is hashed) with d+(c) <= light_max and a chunk of at most
// kPartners partners: kind 0 takes partners from N+(c), kind 1 from N-(c).  A
// CTA task is a whole larger centre (kind 2): its warps take groups of 32
// partners, first from N+(c) then from N-(c), from a shared counter.
constexpr uint32_t kPartners = 512;

struct TcTask {
  uint32_t c, kind, lo, hi;
};

__device__ __forceinline__ uint32_t chunks(uint32_t len) { return (len + kPartners - 1) / kPartners; }

// Intersection work of the DAG: the out-list lengths every method must read
// (sum over edges a->b of d+(a) + d+(b) = sum_c d+(c)^2 + d-(c) d+(c)) and the
// ids this implementation walks: per edge a->b the shorter out-list, d+(b) at
// centre a when d+(b) <= d+(a), else N+(a) at centre b (only its ids above b
// when N+(a) is sorted: kSortedMin <= d+(a) <= smax), nothing when the walked
// side is the single-entry list of a (the rules of tc_task_count_kernel and
// tc_task_fill_kernel below).  One thread per
// vertex over its out-list (out-lists are short in this order); runs after
// the sorts.
__global__ void tc_work_kernel(const RowInfo* __restrict__ row, const uint32_t* __restrict__ dag, uint32_t n,
                               uint32_t smax, unsigned long long* work) {
  unsigned long long sq = 0, io = 0, mn = 0;
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (uint64_t)gridDim.x * blockDim.x) {
    const RowInfo ra = row[a];
    const unsigned long long da = ra.dplus;
    sq += da * da;
    io += (unsigned long long)(ra.len - ra.dplus) * da;
    if (da < 2) continue;
    const bool sorted = da >= kSortedMin && da <= smax;
    for (uint64_t i = ra.off; i < ra.off + da; ++i) {
      const unsigned long long db = row[dag[i]].dplus;
      mn += db <= da ? db : (sorted ? da - 1 - (i - ra.off) : da);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_down_sync(0xFFFFFFFFu, sq, o);
    io += __shfl_down_sync(0xFFFFFFFFu, io, o);
    mn += __shfl_down_sync(0xFFFFFFFFu, mn, o);
  }
  if (lane_id() == 0) {
    atomicAdd(work + 0, sq);
    atomicAdd(work + 1, io);
    atomicAdd(work + 2, mn);
  }
}

__global__ void tc_task_count_kernel(const RowInfo* __restrict__ row, uint32_t n, uint32_t light_max,
                                     uint32_t* cnt_light, uint32_t* cnt_heavy) {
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (uint64_t)gridDim.x * blockDim.x) {
    const RowInfo rc = row[c];
    const uint32_t dp = rc.dplus, dm = rc.len - rc.dplus;
    // kind 0 needs two out-neighbours; kind 1 a partner with 2 <= d+(p) < d+(c)
    uint32_t t = (dp >= 2 ? chunks(dp) : 0) + (dp >= 3 ? chunks(dm) : 0);
    cnt_light[c] = dp <= light_max ? t : 0;
    cnt_heavy[c] = dp <= light_max ? 0 : 1;  // one task per CTA centre
  }
}

__global__ void tc_task_fill_kernel(const RowInfo* __restrict__ row, uint32_t n, uint32_t light_max,
                                    const uint64_t* __restrict__ pos_light, const uint64_t* __restrict__ pos_heavy,
                                    TcTask* light, TcTask* heavy) {
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (uint64_t)gridDim.x * blockDim.x) {
    const RowInfo rc = row[c];
    const uint32_t dp = rc.dplus, dm = rc.len - rc.dplus;
    if (dp > light_max) {
      heavy[pos_heavy[c]] = TcTask{(uint32_t)c, 2u, 0u, dp};
      continue;
    }
    TcTask* out = light + pos_light[c];
    if (dp >= 2)
      for (uint32_t lo = 0; lo < dp; lo += kPartners) *out++ = TcTask{(uint32_t)c, 0u, lo, min(dp, lo + kPartners)};
    if (dp >= 3)
      for (uint32_t lo = 0; lo < dm; lo += kPartners) *out++ = TcTask{(uint32_t)c, 1u, lo, min(dm, lo + kPartners)};
  }
}

// Out-lists of more than lo and at most hi ids, one CTA each, in dynamic
// shared memory of pow2_at_least(hi) words.  Every out-list longer than wmax
// is a CTA centre (wmax is at least the light/heavy split), so the CTA tasks
// list them.  Two launches: up to kSortMidMax ids with many small CTAs, the
// longer lists with room for kSortedMax ids.
constexpr uint32_t kSortMidMax = 4096;

__global__ void __launch_bounds__(kTcThreads) tc_sort_cta_kernel(const RowInfo* __restrict__ row,
                                                                uint32_t* __restrict__ dag,
                                                                const TcTask* __restrict__ tasks, uint64_t ntasks,
                                                                uint32_t lo, uint32_t hi) {
  extern __shared__ __align__(16) uint32_t cbuf[];
  for (uint64_t t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const RowInfo ri = row[tasks[t].c];
    const uint32_t d = ri.dplus;
    if (d <= lo || d > hi) continue;
    uint32_t* p = dag + ri.off;
    const uint32_t S = pow2_at_least(d);
    for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) cbuf[i] = i < d ? p[i] : kInf;
    __syncthreads();
    bitonic_sort<true>(cbuf, S, threadIdx.x, blockDim.x);
    for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) p[i] = cbuf[i];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- intersect
// Open-addressing hash set in shared memory (linear probing, empty = INF,
// multiplicative hashing) over ids in [lo, hi]; the table has at least twice
// (warp kernel: four times) as many slots as keys, so that most absent ids
// cost one probe.
struct SmemHash {
  const uint32_t* t;
  uint32_t mask, shift, lo, hi;
  __device__ __forceinline__ bool contains(uint32_t x) const {
    if (x < lo || x > hi) return false;
    uint32_t h = (x * 0x9E3779B1u) >> shift;
    while (true) {
      uint32_t y = t[h];
      if (y == x) return true;
      if (y == kInf) return false;
      h = (h + 1) & mask;
    }
  }
};

// Bitmap over the rank range [base, base + nbits) in shared memory.
struct SmemBits {
  const uint32_t* b;
  uint32_t base, nbits;
  __device__ __forceinline__ uint32_t contains(uint32_t x) const {
    const uint32_t i = x - base;  // wraps for x < base
    const uint32_t in = i < nbits;
    const uint32_t word = b[(in ? i : 0u) >> 5];  // no branch: out-of-range ids read word 0
    return __funnelshift_r(word, 0u, i) & in;     // the shift takes i mod 32
  }
};

// The warp walks the lists dag_col[vb .. vb+len) held by its lanes (len = 0
// for lanes without a partner) and counts the ids the set contains.  Lists of
// 32 ids or more are walked one at a time by the whole warp (coalesced, eight
// loads in flight per lane, no bookkeeping per id); the shorter ones are
// concatenated and walked 32 ids at a time, each lane finding the list its id
// belongs to by a 5-step search over the lanes' prefix sums.
template <typename Set>
__device__ __forceinline__ uint32_t warp_count_group(const uint32_t* __restrict__ dag_col, uint64_t vb, uint32_t len,
                                                     const Set& set) {
  const uint32_t lane = lane_id();
  uint32_t hits = 0;
  uint32_t longs = __ballot_sync(0xFFFFFFFFu, len >= 32);
  while (longs) {
    const int l = __ffs(longs) - 1;
    longs &= longs - 1;
    const uint64_t b = __shfl_sync(0xFFFFFFFFu, vb, l);
    const uint32_t ln = __shfl_sync(0xFFFFFFFFu, len, l);
    const uint32_t* p = dag_col + b;
    uint32_t k = lane;
    for (; k + 224 < ln; k += 256) {
      uint32_t w[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = __ldg(p + k + 32 * j);
#pragma unroll
      for (int j = 0; j < 8; ++j) hits += set.contains(w[j]);
    }
    if (k + 96 < ln) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = __ldg(p + k + 32 * j);
#pragma unroll
      for (int j = 0; j < 4; ++j) hits += set.contains(w[j]);
      k += 128;
    }
    for (; k < ln; k += 32) hits += set.contains(__ldg(p + k));
  }
  const uint32_t slen = len >= 32 ? 0 : len;
  uint32_t incl = slen;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  const uint32_t excl = incl - slen;
  for (uint32_t e0 = 0; e0 < total; e0 += 32) {
    const uint32_t e = e0 + lane;
    int owner = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      int probe = owner + step;
      uint32_t ex = __shfl_sync(0xFFFFFFFFu, excl, probe & 31);
      if (probe < 32 && ex <= e) owner = probe;
    }
    const uint32_t oex = __shfl_sync(0xFFFFFFFFu, excl, owner);
    const uint64_t ob = __shfl_sync(0xFFFFFFFFu, vb, owner);
    if (e < total) hits += set.contains(__ldg(dag_col + ob + (e - oex)));
  }
  return hits;
}

// 16-byte vector loads of the DAG (read-only during the count; the DAG
// allocation is padded, so a vector that starts inside a list stays inside it)
__device__ __forceinline__ uint4 ld_dag4(const uint32_t* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }

// ids x[0..3] of a vector whose first id sits at list position `pos` (may be
// negative at the list's start), counted if inside [0, len)
template <typename Set>
__device__ __forceinline__ uint32_t count_vec(const Set& set, uint4 q, int pos, int len) {
  uint32_t h = 0;
  h += set.contains(q.x) & (uint32_t)(pos >= 0 && pos < len);
  h += set.contains(q.y) & (uint32_t)(pos + 1 >= 0 && pos + 1 < len);
  h += set.contains(q.z) & (uint32_t)(pos + 2 >= 0 && pos + 2 < len);
  h += set.contains(q.w) & (uint32_t)(pos + 3 >= 0 && pos + 3 < len);
  return h;
}

constexpr uint32_t kWarpListMin = 1024;  // lists at least this long are walked by the whole warp
constexpr int kVecU = 2;                 // vectors in flight per lane

// warp_count_group for the light centres, whose partners' lists are mostly
// short: the warp walks the lists dag_col[vb .. vb+len) held by its lanes
// (len = 0 for lanes without a partner) and counts the ids the set contains.
// Every list is read in aligned 16-byte vectors (4 ids).  Lists of kWarpListMin ids
// or more are walked one at a time by the whole warp; all the others are
// concatenated at vector granularity and walked together, each lane finding
// the list its vector belongs to by a 5-step search over the lanes' prefix
// sums, so the lists of a group are read in a few rounds instead of one round
// each.
template <typename Set>
__device__ __forceinline__ uint32_t warp_count_group_vec(const uint32_t* __restrict__ dag_col, uint64_t vb,
                                                         uint32_t len, const Set& set) {
  const uint32_t lane = lane_id();
  uint32_t hits = 0;
  uint32_t longs = __ballot_sync(0xFFFFFFFFu, len >= kWarpListMin);
  while (longs) {
    const int l = __ffs(longs) - 1;
    longs &= longs - 1;
    const uint64_t b = __shfl_sync(0xFFFFFFFFu, vb, l);
    const int ln = (int)__shfl_sync(0xFFFFFFFFu, len, l);
    const uint32_t* al = dag_col + (b & ~3ull);
    const int head = (int)(b & 3ull);
    for (int v0 = 0; 4 * v0 < head + ln; v0 += 32 * 4) {
      uint4 q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int vi = v0 + 32 * u + (int)lane;
        q[u] = 4 * vi < head + ln ? ld_dag4(al + 4 * vi) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) hits += count_vec(set, q[u], 4 * (v0 + 32 * u + (int)lane) - head, ln);
    }
  }
  const uint32_t slen = len >= kWarpListMin ? 0u : len;
  const uint64_t a0 = vb & ~3ull;
  const uint32_t head = (uint32_t)(vb - a0);
  const uint32_t nv = slen ? (head + slen + 3) >> 2 : 0u;
  uint32_t incl = nv;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  const uint32_t excl = incl - nv;
  for (uint32_t e0 = 0; e0 < total; e0 += 32 * kVecU) {
    uint4 q[kVecU];
    int pos[kVecU], ln[kVecU];
#pragma unroll
    for (int u = 0; u < kVecU; ++u) {
      const uint32_t e = e0 + 32 * u + lane;
      int owner = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        int probe = owner + step;
        uint32_t ex = __shfl_sync(0xFFFFFFFFu, excl, probe & 31);
        if (probe < 32 && ex <= e) owner = probe;
      }
      const uint32_t oex = __shfl_sync(0xFFFFFFFFu, excl, owner);
      const uint64_t oa = __shfl_sync(0xFFFFFFFFu, a0, owner);
      const uint32_t oh = __shfl_sync(0xFFFFFFFFu, head, owner);
      const uint32_t ol = __shfl_sync(0xFFFFFFFFu, slen, owner);
      const uint32_t vi = e - oex;
      const bool ok = e < total;
      q[u] = ok ? ld_dag4(dag_col + oa + 4ull * vi) : make_uint4(0u, 0u, 0u, 0u);
      pos[u] = (int)(4 * vi) - (int)oh;
      ln[u] = ok ? (int)ol : 0;
    }
#pragma unroll
    for (int u = 0; u < kVecU; ++u) hits += count_vec(set, q[u], pos[u], ln[u]);
  }
  return hits;
}

// A lane's partner p: its out-list, kept only on the side that walks the
// shorter list (kind 0: d+(p) <= d+(c); kind 1: d+(p) < d+(c)).  A kind-1
// partner's out-list holds c itself, which N+(c) does not, so one of length 1
// cannot meet N+(c) and is skipped; a sorted one (kSortedMin..smax ids) keeps
// only its ids above c (a binary search by the lane).
__device__ __forceinline__ void partner_list(const RowInfo* __restrict__ row, const uint32_t* __restrict__ dag_col,
                                             bool has, uint32_t p, uint32_t kind, uint32_t c, uint32_t dc,
                                             uint32_t smax, uint64_t* vb, uint32_t* len) {
  *vb = 0;
  *len = 0;
  if (!has) return;
  const uint4 q = __ldg(reinterpret_cast<const uint4*>(row + p));  // off (2 words), dplus, len
  const uint32_t d = q.z;
  if (kind == 0 ? d <= dc : (d < dc && d >= 2)) {
    uint64_t b = ((uint64_t)q.y << 32) | q.x;
    uint32_t lo = 0;
    if (kind == 1 && d >= kSortedMin && d <= smax) {
      uint32_t hi = d;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(dag_col + b + mid) > c) hi = mid;
        else lo = mid + 1;
      }
    }
    *vb = b + lo;
    *len = d - lo;
  }
}

// Walks the partners [t.lo, t.hi) of a task with `warps` warps (this one is
// warp `w`) and counts the ids of their out-lists that `set` contains.  The
// partner ids and out-list bounds of the next two groups are loaded while the
// current group is walked.
template <typename Set>
__device__ __forceinline__ uint64_t walk_partners(const RowInfo* __restrict__ row,
                                                  const uint32_t* __restrict__ dag_col, const uint32_t* partners,
                                                  const TcTask& t, uint32_t dc, uint32_t smax, uint32_t w,
                                                  uint32_t warps, const Set& set) {
  const uint32_t lane = lane_id(), step = warps * 32;
  uint64_t hits = 0;
  uint32_t k0 = t.lo + w * 32;
  bool has = k0 + lane < t.hi;
  uint32_t p = has ? __ldg(partners + k0 + lane) : 0;
  uint64_t vb;
  uint32_t len;
  partner_list(row, dag_col, has, p, t.kind, t.c, dc, smax, &vb, &len);
  bool has1 = k0 + step + lane < t.hi;
  uint32_t p1 = has1 ? __ldg(partners + k0 + step + lane) : 0;
  for (; k0 < t.hi; k0 += step) {
    uint64_t vb1;
    uint32_t len1;
    partner_list(row, dag_col, has1, p1, t.kind, t.c, dc, smax, &vb1, &len1);  // group k0 + step
    const bool has2 = k0 + 2 * step + lane < t.hi;
    const uint32_t p2 = has2 ? __ldg(partners + k0 + 2 * step + lane) : 0;
    hits += warp_count_group_vec(dag_col, vb, len, set);
    vb = vb1;
    len = len1;
    has1 = has2;
    p1 = p2;
  }
  return hits;
}

constexpr uint32_t kSlice = kLightMax + 8;  // staged N+(u) (+ alignment slack), ids
constexpr uint32_t kTable = 4 * kLightMax;   // hash slots per warp (load factor <= 1/4)
constexpr size_t kLightSmem = (size_t)(kTcThreads / 32) * (kSlice + kTable) * sizeof(uint32_t);

__global__ void __launch_bounds__(kTcThreads, 5) tc_light_kernel(const RowInfo* __restrict__ row,
                                                              const uint32_t* __restrict__ dag_col,
                                                              const TcTask* __restrict__ tasks, uint64_t ntasks,
                                                              uint32_t* ctr, unsigned long long* count,
                                                              uint32_t smax, uint64_t limit_ns) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ __align__(8) uint64_t bar[kTcThreads / 32];
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t* buf = smem + (size_t)w * (kSlice + kTable);
  uint32_t* table = buf + kSlice;
  uint32_t* err = ctr + 3;
  if (lane == 0) mbar_init(&bar[w], 1);
  __syncwarp();
  uint32_t phase = 0;
  uint32_t have = kInf;  // centre whose N+ is staged and hashed in this warp's slice
  uint32_t head = 0, dc = 0, bits = 5, lo = 0, hi = 0;
  uint64_t hits = 0;
  while (true) {
    uint32_t idx = 0;
    if (lane == 0) idx = atomicAdd(ctr + 2, 1u);
    idx = __shfl_sync(0xFFFFFFFFu, idx, 0);
    if (idx >= ntasks) break;
    const TcTask t = tasks[idx];
    const uint32_t c = t.c;
    if (c != have) {
      const RowInfo rc = row[c];
      uint64_t beg = rc.off, end = rc.off + rc.dplus;
      uint64_t a0 = beg & ~3ull, a1 = (end + 3) & ~3ull;
      head = (uint32_t)(beg - a0);
      dc = (uint32_t)(end - beg);
      // every lane is done with the previous slice and table, and its reads
      // are ordered before the bulk copy's writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      bool ok = true;
      if (lane == 0) {
        bulk_load(buf, dag_col + a0, (uint32_t)((a1 - a0) * 4), &bar[w]);
        ok = mbar_wait(&bar[w], phase, err, limit_ns);
      }
      if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) return;
      mbar_wait(&bar[w], phase, err, limit_ns);  // completed: every lane observes the phase
      phase ^= 1;
      // hash set of N+(c): 2^bits >= 4 d+(c) slots (few probes for absent ids)
      bits = 32 - __clz(4 * dc - 1);
      if (bits < 5) bits = 5;
      const uint32_t slots = 1u << bits;
      for (uint32_t i = lane; i < slots; i += 32) table[i] = kInf;
      __syncwarp();
      uint32_t mn = kInf, mx = 0;
      for (uint32_t k = lane; k < dc; k += 32) {
        uint32_t x = buf[head + k];
        mn = min(mn, x);
        mx = max(mx, x);
        uint32_t h = (x * 0x9E3779B1u) >> (32 - bits);
        while (atomicCAS(table + h, kInf, x) != kInf) h = (h + 1) & (slots - 1);
      }
      lo = __reduce_min_sync(0xFFFFFFFFu, mn);
      hi = __reduce_max_sync(0xFFFFFFFFu, mx);
      __syncwarp();
      have = c;
    }
    SmemHash set{table, (1u << bits) - 1, 32 - bits, lo, hi};
    const RowInfo rc = row[c];
    const uint32_t* partners = dag_col + rc.off + (t.kind == 0 ? 0u : rc.dplus);
    hits += walk_partners(row, dag_col, partners, t, dc, smax, 0, 1, set);
  }
  uint64_t sum = hits;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
  if (lane == 0 && sum) atomicAdd(count, (unsigned long long)sum);
}

constexpr uint32_t kHeavyTable = 2 * kWindow;
constexpr uint32_t kHeavyWords = kWindow + 8 + kHeavyTable;  // 32-bit words of dynamic shared memory
constexpr uint32_t kBitmapBits = 32 * (kHeavyWords & ~3u);   // bitmap capacity of the same memory
constexpr size_t kHeavySmem = (size_t)kHeavyWords * sizeof(uint32_t);

// The partners of group g of a CTA centre: groups [0, g0) hold N+(c) in 32s,
// groups [g0, gt) hold N-(c).  Returns this lane's partner (has = false past
// the end of the list) and its kind.
struct CentreGroups {
  const uint32_t* out;  // N+(c)
  const uint32_t* in;   // N-(c)
  uint32_t c, dc, dm, g0, gt, smax;
  __device__ __forceinline__ uint32_t partner(uint32_t g, bool* has, uint32_t* kind) const {
    const uint32_t lane = lane_id();
    if (g < g0) {
      const uint32_t k = g * 32 + lane;
      *kind = 0;
      *has = k < dc;
      return *has ? __ldg(out + k) : 0u;
    }
    const uint32_t k = (g - g0) * 32 + lane;
    *kind = 1;
    *has = k < dm;
    return *has ? __ldg(in + k) : 0u;
  }
};

__device__ __forceinline__ uint32_t grab_group(uint32_t* gctr) {
  uint32_t g = 0;
  if (lane_id() == 0) g = atomicAdd(gctr, 1u);
  return __shfl_sync(0xFFFFFFFFu, g, 0);
}

// A warp's share of a CTA centre: groups taken from the CTA's counter until
// they run out.  The partner ids of the group after next and the out-list
// bounds of the next group are loaded while the current group is walked.
template <typename Set>
__device__ __forceinline__ uint32_t walk_groups(const RowInfo* __restrict__ row,
                                                const uint32_t* __restrict__ dag_col, const CentreGroups& cg,
                                                uint32_t* gctr, const Set& set) {
  uint32_t g = grab_group(gctr);
  if (g >= cg.gt) return 0;
  bool has;
  uint32_t kind;
  uint32_t p = cg.partner(g, &has, &kind);
  uint64_t vb;
  uint32_t len;
  partner_list(row, dag_col, has, p, kind, cg.c, cg.dc, cg.smax, &vb, &len);
  uint32_t gn = grab_group(gctr);
  bool hasn = false;
  uint32_t kindn = 0, pn = gn < cg.gt ? cg.partner(gn, &hasn, &kindn) : 0u;
  uint32_t hits = 0;
  while (true) {
    uint64_t vbn;
    uint32_t lenn;
    partner_list(row, dag_col, hasn, pn, kindn, cg.c, cg.dc, cg.smax, &vbn, &lenn);
    const uint32_t gnn = gn < cg.gt ? grab_group(gctr) : cg.gt;
    bool hasnn = false;
    uint32_t kindnn = 0, pnn = gnn < cg.gt ? cg.partner(gnn, &hasnn, &kindnn) : 0u;
    hits += warp_count_group(dag_col, vb, len, set);
    if (gn >= cg.gt) break;
    vb = vbn;
    len = lenn;
    gn = gnn;
    hasn = hasnn;
    kindn = kindnn;
    pn = pnn;
  }
  return hits;
}

// One CTA per centre, the largest centres (highest ranks) first.  Bitmap mode
// (the n - 1 - c ranks above c fit in `bitmap_bits`): N+(c) is set into a
// bitmap of that range, read straight from the DAG.  Hash mode: N+(c) is
// staged by TMA in windows of `window` ids, each hashed.
__global__ void __launch_bounds__(kTcThreads, 6) tc_heavy_kernel(const RowInfo* __restrict__ row,
                                                              const uint32_t* __restrict__ dag_col,
                                                              const TcTask* __restrict__ tasks, uint64_t ntasks,
                                                              uint32_t n, uint32_t* ctr, unsigned long long* count,
                                                              uint32_t window, uint32_t bitmap_bits,
                                                              uint32_t smax, uint64_t limit_ns) {
  extern __shared__ __align__(16) uint32_t win[];
  uint32_t* table = win + kWindow + 8;
  __shared__ __align__(8) uint64_t bar;
  __shared__ bool ok_s;
  __shared__ uint32_t idx_s, lo_s, hi_s, gctr;
  const uint32_t lane = lane_id();
  uint32_t* err = ctr + 3;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  uint64_t hits = 0;
  while (true) {
    if (threadIdx.x == 0) idx_s = atomicAdd(ctr + 4, 1u);
    __syncthreads();  // also: every thread is done with the previous centre
    const uint32_t idx = idx_s;
    if (idx >= ntasks) break;
    const uint32_t c = tasks[ntasks - 1 - idx].c;
    const RowInfo rc = row[c];
    const uint64_t beg = rc.off, end = rc.off + rc.dplus, ib = end;
    const uint32_t dc = rc.dplus, dm = rc.len - rc.dplus;
    const uint32_t g0 = (dc + 31) / 32;
    const CentreGroups cg{dag_col + beg, dag_col + ib, c, dc, dm, g0, g0 + (dm + 31) / 32, smax};
    const uint32_t above = n - 1 - c;  // N+(c) lies in the ranks (c, n)
    if (above <= bitmap_bits) {
      const uint32_t words = (above + 127) / 128 * 4;
      uint4* w4 = reinterpret_cast<uint4*>(win);
      for (uint32_t i = threadIdx.x; i < words / 4; i += blockDim.x) w4[i] = make_uint4(0u, 0u, 0u, 0u);
      if (threadIdx.x == 0) gctr = 0;
      __syncthreads();  // idx_s is read by every thread before thread 0 rewrites it
      for (uint32_t k = threadIdx.x; k < dc; k += blockDim.x) {
        const uint32_t x = __ldg(dag_col + beg + k) - (c + 1);
        atomicOr(win + (x >> 5), 1u << (x & 31));
      }
      __syncthreads();
      hits += walk_groups(row, dag_col, cg, &gctr, SmemBits{win, c + 1, above});
      continue;
    }
    for (uint64_t wb = beg; wb < end; wb += window) {
      uint64_t we = wb + window < end ? wb + window : end;
      uint64_t a0 = wb & ~3ull, a1 = (we + 3) & ~3ull;
      uint32_t head = (uint32_t)(wb - a0), wlen = (uint32_t)(we - wb);
      // every thread is done with the previous window, table or bitmap, and
      // its shared-memory accesses are ordered before the bulk copy's writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        lo_s = kInf;
        hi_s = 0;
        gctr = 0;
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
      uint32_t mn = kInf, mx = 0;
      for (uint32_t k = threadIdx.x; k < wlen; k += blockDim.x) {
        uint32_t x = list[k];
        mn = min(mn, x);
        mx = max(mx, x);
        uint32_t h = (x * 0x9E3779B1u) >> (32 - bits);
        while (atomicCAS(table + h, kInf, x) != kInf) h = (h + 1) & (slots - 1);
      }
      mn = __reduce_min_sync(0xFFFFFFFFu, mn);
      mx = __reduce_max_sync(0xFFFFFFFFu, mx);
      if (lane == 0) {
        atomicMin(&lo_s, mn);
        atomicMax(&hi_s, mx);
      }
      __syncthreads();
      hits += walk_groups(row, dag_col, cg, &gctr, SmemHash{table, slots - 1, 32 - bits, lo_s, hi_s});
    }
  }
  uint64_t sum = hits;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
  if (lane == 0 && sum) atomicAdd(count, (unsigned long long)sum);
}

byo_status ensure_tc_work(byo_graph* g) {
  if (g->tc && g->tc->cap >= g->m) return BYO_OK;
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
  w->cap = g->m + (g->dyn ? g->m / 4 : 0);  // headroom for later inserts
  byo_status st = dev_alloc_t(&w->row, g->n + 1ull, "TC DAG rows");
  if (st == BYO_OK) st = dev_alloc_t(&w->roff, g->n + 1ull, "TC DAG row starts");
  if (st == BYO_OK) st = dev_alloc_t(&w->dag, w->cap + 8, "TC DAG");
  if (st == BYO_OK) st = dev_alloc_t(&w->rdeg, g->n, "TC degrees by rank");
  if (st == BYO_OK) st = dev_alloc_t(&w->rank, g->n, "TC ranks");
  if (st == BYO_OK) st = dev_alloc_t(&w->cnt_l, g->n, "TC task counts");
  if (st == BYO_OK) st = dev_alloc_t(&w->cnt_h, g->n, "TC task counts");
  if (st == BYO_OK) st = dev_alloc_t(&w->pos_l, g->n + 1ull, "TC task offsets");
  if (st == BYO_OK) st = dev_alloc_t(&w->pos_h, g->n + 1ull, "TC task offsets");
  if (st == BYO_OK) st = dev_alloc_t(&w->ctr, 8, "TC counters");
  if (st == BYO_OK) st = dev_alloc_t(&w->count, 1, "TC count");
  if (st == BYO_OK) st = dev_alloc_t(&w->work, 4, "TC work counters");
  if (st == BYO_OK) {
    cudaError_t e = cudaMemset(w->dag, 0, sizeof(uint32_t) * (w->cap + 8));
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
byo_status run_tc(byo_graph* g, G view, uint64_t* host_count, bool want_work, cudaStream_t s) {
  BYO_RETURN_IF(ensure_tc_work(g));
  TcWork* w = g->tc;
  const uint32_t n = g->n;
  VBins bins = make_vbins(g, 4, 10, kTcThreads);
  // rank(v) = position of (degree(v), v) in ascending order; the DAG rows are
  // laid out in rank order, row r holding deg(r) entries
  {
    uint64_t* sorted = nullptr;
    BYO_RETURN_IF(degree_rank(g, view, w->rank, &sorted, s));
    tc_rdeg_kernel<<<grid_for(n, 256), 256, 0, s>>>(sorted, n, id_bits(n), w->rdeg);
    ::byo::note_launch();
    tmp_free(sorted, s);
    BYO_CHECK_LAUNCH("tc_rdeg_kernel");
    BYO_RETURN_IF(scan_u32_to_u64(w->rdeg, w->roff, n, nullptr, s));
    tc_set_last_kernel<<<1, 1, 0, s>>>(w->roff, n, g->m);
    ::byo::note_launch();
  }
  {
    ProfScope ps("tc_fill", s);
    tc_fill_kernel<<<vbins_grid(bins), kTcThreads, 0, s>>>(view, bins, w->rank, w->roff, w->dag, w->row);
    ::byo::note_launch();
  }
  BYO_CHECK_LAUNCH("tc_fill_kernel");
  // tasks
  const uint32_t light_max = env_cap("BYO_TC_LIGHT_MAX", kLightMax);
  uint32_t wmax = env_cap("BYO_TC_WARP_SORT_MAX", kWarpSortMax);
  if (wmax < light_max) wmax = light_max;  // longer out-lists are CTA centres, listed by the CTA tasks
  const uint32_t smax = env_cap("BYO_TC_SORT_MAX", kSortedMax);
  tc_task_count_kernel<<<grid_for(n, 256), 256, 0, s>>>(w->row, n, light_max, w->cnt_l, w->cnt_h);
  ::byo::note_launch();
  BYO_CHECK_LAUNCH("tc_task_count_kernel");
  uint64_t nl = 0, nh = 0;
  BYO_RETURN_IF(scan_u32_to_u64(w->cnt_l, w->pos_l, n, &nl, s));
  BYO_RETURN_IF(scan_u32_to_u64(w->cnt_h, w->pos_h, n, &nh, s));
  TcTask *tl = nullptr, *th = nullptr;
  byo_status st = tmp_alloc_t(&tl, nl + 1, s, "TC light tasks");
  if (st == BYO_OK) st = tmp_alloc_t(&th, nh + 1, s, "TC heavy tasks");
  if (st == BYO_OK) {
    tc_task_fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(w->row, n, light_max, w->pos_l, w->pos_h, tl,
                                                         th);
    ::byo::note_launch();
    cudaMemsetAsync(w->ctr, 0, 8 * sizeof(uint32_t), s);
    cudaMemsetAsync(w->count, 0, sizeof(unsigned long long), s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_status(e, "tc_task_fill_kernel");
  }
  if (st == BYO_OK) {  // sort the out-lists the walks may trim
    cudaError_t e;
    {
      ProfScope ps("tc_sort", s);
      tc_sort_warp_kernel<<<sm_count() * 4, kTcThreads, 0, s>>>(w->row, w->dag, n, wmax < smax ? wmax : smax);
      ::byo::note_launch();
      e = cudaGetLastError();
    }
    const uint32_t mid = smax < kSortMidMax ? smax : kSortMidMax;
    const uint32_t tiers[2][3] = {{wmax, mid, 8}, {mid, smax, 2}};  // lo, hi, CTAs per SM
    for (const auto& tier : tiers) {
      if (e != cudaSuccess || !nh || tier[1] <= tier[0]) continue;
      const size_t smem = (size_t)pow2_at_least(tier[1]) * sizeof(uint32_t);
      e = cudaFuncSetAttribute(tc_sort_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) break;
      ProfScope ps("tc_sort_cta", s);
      const uint64_t cap = (uint64_t)sm_count() * tier[2];
      tc_sort_cta_kernel<<<(unsigned)(nh < cap ? nh : cap), kTcThreads, smem, s>>>(w->row, w->dag, th, nh, tier[0],
                                                                                    tier[1]);
      ::byo::note_launch();
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = cuda_status(e, "tc_sort");
  }
  if (st == BYO_OK && want_work) {
    cudaMemsetAsync(w->work, 0, 4 * sizeof(unsigned long long), s);
    tc_work_kernel<<<grid_for(n, 256), 256, 0, s>>>(w->row, w->dag, n, smax, w->work);
    ::byo::note_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w->host_work, w->work, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_status(e, "tc_work_kernel");
  }
  const uint64_t limit = timeout_ns();
  if (st == BYO_OK && nl) {
    int per_sm = 0;
    cudaError_t e = cudaFuncSetAttribute(tc_light_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLightSmem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_light_kernel, kTcThreads, kLightSmem);
    if (e == cudaSuccess) {
      ProfScope ps("tc_light", s);
      tc_light_kernel<<<(unsigned)(sm_count() * (per_sm > 0 ? per_sm : 1)), kTcThreads, kLightSmem, s>>>(
          w->row, w->dag, tl, nl, w->ctr, w->count, smax, limit);
      ::byo::note_launch();
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = cuda_status(e, "tc_light_kernel");
  }
  if (st == BYO_OK && nh) {
    int per_sm = 0;
    cudaError_t e = cudaFuncSetAttribute(tc_heavy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHeavySmem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_heavy_kernel, kTcThreads, kHeavySmem);
    if (e == cudaSuccess) {
      ProfScope ps("tc_heavy", s);
      tc_heavy_kernel<<<(unsigned)(sm_count() * (per_sm > 0 ? per_sm : 1)), kTcThreads, kHeavySmem, s>>>(
          w->row, w->dag, th, nh, n, w->ctr, w->count, env_cap("BYO_TC_WINDOW", kWindow),
          env_cap("BYO_TC_BITMAP_BITS", kBitmapBits), smax, limit);
      ::byo::note_launch();
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = cuda_status(e, "tc_heavy_kernel");
  }
  uint32_t err = 0;
  unsigned long long c = 0;
  if (st == BYO_OK) {
    cudaError_t e = cudaMemcpyAsync(&c, w->count, sizeof(c), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, w->ctr + 3, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "byo_tc");
  }
  tmp_free(tl, s);
  tmp_free(th, s);
  BYO_RETURN_IF(st);
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
  BYO_RETURN_IF(ready_graph(gc, static_cast<cudaStream_t>(stream)));
  if (!host_count) {
    set_error("byo_tc: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  byo_graph* g = const_cast<byo_graph*>(gc);
  *host_count = 0;
  if (g->n == 0 || g->m == 0) return BYO_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return with_view(g, [&](auto view) { return run_tc(g, view, host_count, false, s); });
}

extern "C" byo_status byo_tc_work(const byo_graph* gc, uint64_t* host_work3, void* stream) {
  clear_error();
  BYO_RETURN_IF(ready_graph(gc, static_cast<cudaStream_t>(stream)));
  if (!host_work3) {
    set_error("byo_tc_work: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  byo_graph* g = const_cast<byo_graph*>(gc);
  host_work3[0] = host_work3[1] = host_work3[2] = 0;
  if (g->n == 0 || g->m == 0) return BYO_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint64_t count = 0;
  BYO_RETURN_IF(with_view(g, [&](auto view) { return run_tc(g, view, &count, true, s); }));
  for (int i = 0; i < 3; ++i) host_work3[i] = g->tc->host_work[i];
  return BYO_OK;
}
