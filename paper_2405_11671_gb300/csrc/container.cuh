// container.cuh -- device side of the GraphContainer API (Section 4.2):
// num_vertices(), num_edges(), degree(i) and map_neighbors(i, f) with its
// early-exit and parallel variants, as views that the algorithm kernels are
// written against once.  A neighbour list is exposed as contiguous segments
// of ascending uint32 ids so that kernels can read it with 16-byte vector
// loads; the static CSR has one segment per vertex.
#pragma once

#include "byo_internal.cuh"

namespace byo {

struct Seg {
  const uint32_t* p;
  uint32_t len;
};

template <typename OffT>
struct CsrView {
  uint32_t n;
  uint64_t m;
  const OffT* off;
  const uint32_t* col;

  __device__ __forceinline__ uint32_t num_vertices() const { return n; }
  __device__ __forceinline__ uint64_t num_edges() const { return m; }
  __device__ __forceinline__ uint64_t begin(uint32_t v) const { return (uint64_t)__ldg(off + v); }
  __device__ __forceinline__ uint32_t degree(uint32_t v) const {
    return (uint32_t)(__ldg(off + v + 1) - __ldg(off + v));
  }
  __device__ __forceinline__ Seg seg(uint32_t v) const {
    OffT a = __ldg(off + v), b = __ldg(off + v + 1);
    return Seg{col + a, (uint32_t)(b - a)};
  }
  __device__ __forceinline__ uint32_t nbr(uint32_t v, uint32_t i) const { return __ldg(col + __ldg(off + v) + i); }

  // map_neighbors(v, f): f(u) for every neighbour in ascending order.
  template <typename F>
  __device__ __forceinline__ void map_neighbors(uint32_t v, F&& f) const {
    Seg s = seg(v);
    for (uint32_t i = 0; i < s.len; ++i) f(__ldg(s.p + i));
  }
  // map_neighbors_early_exit(v, f): stops after the first f(u) == true;
  // returns the index of that neighbour or the degree.
  template <typename F>
  __device__ __forceinline__ uint32_t map_neighbors_early_exit(uint32_t v, F&& f) const {
    Seg s = seg(v);
    for (uint32_t i = 0; i < s.len; ++i)
      if (f(__ldg(s.p + i))) return i;
    return s.len;
  }
};

// 16-byte aligned vector read of the neighbour ids [i, i+4) of a segment,
// where the first id of the vector may lie before the segment start: the
// caller masks with seg_valid().  `base` is the segment start rounded down
// to 16 bytes.  The container allocations are padded so that reading the
// rounded-up tail stays inside them.
__device__ __forceinline__ uint4 ld_nc_v4(const uint32_t* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }

__device__ __forceinline__ const uint32_t* align16_down(const uint32_t* p) {
  return reinterpret_cast<const uint32_t*>(reinterpret_cast<uintptr_t>(p) & ~uintptr_t(15));
}

}  // namespace byo

namespace byo {

// ---------------------------------------------------------------- dynamic container
// Blocked adjacency with an inline head (the inline optimisation of Section
// 4.1, here ~12 ids next to the vertex record).  A vertex with at most
// kInline neighbours keeps them in its 64-byte record; a larger one keeps all
// of them, ascending, in a run of 2^cls blocks of 32 ids (128 bytes each) from
// a device pool.  Either way the list is ONE contiguous segment, so every
// algorithm kernel runs unchanged over both containers; it is ascending except
// in the hash-indexed variant (BYO_DYN_HASH), which keeps insertion order and
// finds an id through a per-run hash index instead (DHB's design, Section 5.2).
constexpr uint32_t kInline = 12;
constexpr uint32_t kBlockIds = 32;
constexpr uint32_t kNoRun = 0xFFFFFFFFu;
constexpr uint32_t kHashSlots = 2 * kBlockIds;  // index slots per pool block (load <= 1/2 from live ids)
constexpr uint32_t kTomb = 0xFFFFFFFEu;         // a deleted index key (ids are below n <= 0xFFFFFFFE)

struct __align__(64) DynVertex {
  uint32_t deg;
  uint32_t cls;  // kNoRun when the list is inline
  uint64_t run;  // first block of the run (block index into the pool)
  uint32_t inl[kInline];  // the inline list; in the hash-indexed variant a run list keeps its index's tombstone count in inl[0]
};

struct DynView {
  uint32_t n;
  uint64_t m;
  const DynVertex* vtx;
  const uint32_t* pool;
  uint32_t icap;  // lists of at most icap ids are inline (kInline, or 0 without the inline head)

  __device__ __forceinline__ uint32_t num_vertices() const { return n; }
  __device__ __forceinline__ uint64_t num_edges() const { return m; }
  __device__ __forceinline__ uint32_t degree(uint32_t v) const { return __ldg(&vtx[v].deg); }
  __device__ __forceinline__ Seg seg(uint32_t v) const {
    uint32_t d = __ldg(&vtx[v].deg);
    const uint32_t* p = d <= icap ? vtx[v].inl : pool + __ldg(&vtx[v].run) * kBlockIds;
    return Seg{p, d};
  }
  template <typename F>
  __device__ __forceinline__ void map_neighbors(uint32_t v, F&& f) const {
    Seg s = seg(v);
    for (uint32_t i = 0; i < s.len; ++i) f(__ldg(s.p + i));
  }
  template <typename F>
  __device__ __forceinline__ uint32_t map_neighbors_early_exit(uint32_t v, F&& f) const {
    Seg s = seg(v);
    for (uint32_t i = 0; i < s.len; ++i)
      if (f(__ldg(s.p + i))) return i;
    return s.len;
  }
};

constexpr int kClasses = 27;  // run sizes 2^0 .. 2^26 blocks

struct DynStore {
  DynVertex* vtx = nullptr;        // n + 1 records (the spare keeps vector tail reads inside)
  uint32_t* pool = nullptr;        // pool_blocks * 32 ids
  uint64_t pool_blocks = 0;
  unsigned long long* bump = nullptr;  // next free block (device)
  uint32_t* stacks[kClasses] = {nullptr};  // free runs per class
  uint64_t stack_cap[kClasses] = {0};
  long long* tops = nullptr;       // kClasses stack tops (device)
  uint32_t icap = kInline;         // inline capacity: kInline, or 0 (BYO_DYN_NO_INLINE)
  // BYO_DYN_HASH: lists unsorted; the run at block r (class c, 32 * 2^c ids)
  // has an open-addressing index of 64 * 2^c slots at [64 r, 64 (r + 2^c)):
  // hkey holds an id (kInf empty, kTomb deleted), hpos its position in the list
  bool hashed = false;
  uint32_t* hkey = nullptr;        // 64 * pool_blocks slots
  uint32_t* hpos = nullptr;        // 64 * pool_blocks slots
  uint32_t* vcnt = nullptr;        // n batch counters of the semisort (zero between batches)
  uint32_t* vslot = nullptr;       // n: vertex -> its group in the current batch
};

inline DynView dyn_view(const byo_graph* g) { return DynView{g->n, g->m, g->dyn->vtx, g->dyn->pool, g->dyn->icap}; }

// Call f with the device view of g's container.
template <typename F>
inline byo_status with_view(const byo_graph* g, F&& f) {
  if (g->dyn) return f(dyn_view(g));
  if (g->off64) return f(CsrView<uint64_t>{g->n, g->m, static_cast<const uint64_t*>(g->off), g->col});
  return f(CsrView<uint32_t>{g->n, g->m, static_cast<const uint32_t*>(g->off), g->col});
}

}  // namespace byo
