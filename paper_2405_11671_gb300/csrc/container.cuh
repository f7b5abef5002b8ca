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
