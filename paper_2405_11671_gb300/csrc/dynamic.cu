// dynamic.cu -- the dynamic blocked-adjacency container and its batch updates
// (insert_sorted_batch / delete_sorted_batch of Section 4.2; the library sorts
// the batch itself, as BYO does).
//
// Layout (container.cuh): a 64-byte record per vertex holding the degree and
// either up to kInline ids inline (the inline optimisation of Section 4.1) or
// the location of a run of 2^cls blocks of 32 ids in a device pool.  Free runs
// are kept on one stack per size class and reused; the pool grows (copy to a
// larger allocation) before an update that might not fit.
//
// A batch is applied in data-parallel passes, all on the device:
//   1. symmetrise, drop self-loops, sort and unique the pairs (radix sort);
//   2. split the sorted batch into per-vertex segments;
//   3. mark each batch id as effective (insert: absent from the list; delete:
//      present) by binary search in the vertex's current list, and scan marks;
//   4. new degree per affected vertex, scan -> slots of a merge buffer;
//   5. write each merged list into the buffer: every old id and every
//      effective batch id computes its output rank with one binary search;
//   6. choose storage for the new list (inline, keep the run, pop a free run of
//      the right class, or bump-allocate), copy the list back, free old runs;
//   7. update m and the degree-bucket order used by the algorithm kernels.
#include <memory>

#include "byo_internal.cuh"
#include "container.cuh"
#include "prof.cuh"

namespace byo {

void dyn_free(DynStore* d) {
  if (!d) return;
  dev_free(d->vtx);
  dev_free(d->pool);
  dev_free(d->bump);
  for (int c = 0; c < kClasses; ++c) dev_free(d->stacks[c]);
  dev_free(d->tops);
  dev_free(d->hkey);
  dev_free(d->hpos);
  dev_free(d->vcnt);
  dev_free(d->vslot);
  delete d;
}

namespace {


__host__ __device__ inline uint32_t run_class(uint32_t deg) {
  // smallest c with (2^c blocks * 32 ids) >= deg
  uint32_t blocks = (deg + kBlockIds - 1) / kBlockIds;
  uint32_t c = 0;
  while ((1u << c) < blocks) ++c;
  return c;
}

__device__ __forceinline__ uint32_t lower_bound(const uint32_t* a, uint32_t len, uint32_t x) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- initial load
template <typename OffT>
__global__ void dyn_blocks_kernel(const OffT* __restrict__ off, uint32_t n, uint32_t icap, uint32_t* blocks) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t d = (uint32_t)(off[v + 1] - off[v]);
    blocks[v] = d <= icap ? 0u : (1u << run_class(d));
  }
}

template <typename OffT>
__global__ void dyn_load_kernel(const OffT* __restrict__ off, const uint32_t* __restrict__ col, uint32_t n,
                                uint32_t icap, bool hashed, const uint64_t* __restrict__ first_block, DynVertex* vtx,
                                uint32_t* pool) {
  const uint32_t lane = lane_id();
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = w0; v < n; v += nw) {
    uint64_t b = off[v];
    uint32_t d = (uint32_t)(off[v + 1] - b);
    DynVertex* r = vtx + v;
    if (d <= icap) {
      if (lane < kInline) r->inl[lane] = lane < d ? col[b + lane] : kInf;
      if (lane == 0) {
        r->deg = d;
        r->cls = kNoRun;
        r->run = 0;
      }
    } else {
      uint64_t run = first_block[v];
      uint32_t* dst = pool + run * kBlockIds;
      for (uint32_t i = lane; i < d; i += 32) dst[i] = col[b + i];
      if (lane < kInline) r->inl[lane] = lane == 0 && hashed ? 0u : kInf;  // no tombstones yet
      if (lane == 0) {
        r->deg = d;
        r->cls = run_class(d);
        r->run = run;
      }
    }
  }
}

// ---------------------------------------------------------------- batch passes
// seg_start[a] = first batch index of the a-th affected vertex; seg_v[a] = the vertex
__global__ void seg_flags_kernel(const uint32_t* __restrict__ rows, uint64_t B, uint32_t* flags) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (uint64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || rows[i] != rows[i - 1]) ? 1u : 0u;
}

__global__ void seg_fill_kernel(const uint32_t* __restrict__ rows, const uint32_t* __restrict__ flags,
                                const uint64_t* __restrict__ idx, uint64_t B, uint64_t A, uint64_t* seg_start,
                                uint32_t* seg_v) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (uint64_t)gridDim.x * blockDim.x) {
    if (flags[i]) {
      seg_start[idx[i]] = i;
      seg_v[idx[i]] = rows[i];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) seg_start[A] = B;
}

// mark[i] = 1 if batch entry i changes the list (insert: absent; delete: present)
__global__ void mark_kernel(DynView g, const uint32_t* __restrict__ rows, const uint32_t* __restrict__ cols,
                            uint64_t B, bool insert, uint32_t* mark) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (uint64_t)gridDim.x * blockDim.x) {
    Seg s = g.seg(rows[i]);
    uint32_t x = cols[i];
    uint32_t p = lower_bound(s.p, s.len, x);
    bool present = p < s.len && __ldg(s.p + p) == x;
    mark[i] = (insert ? !present : present) ? 1u : 0u;
  }
}

__global__ void newdeg_kernel(DynView g, const uint64_t* __restrict__ seg_start, const uint32_t* __restrict__ seg_v,
                              const uint64_t* __restrict__ mrank, uint64_t A, bool insert, uint32_t* newdeg,
                              long long* delta) {
  long long dsum = 0;
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t d = g.degree(seg_v[a]);
    uint32_t c = (uint32_t)(mrank[seg_start[a + 1]] - mrank[seg_start[a]]);
    uint32_t nd = insert ? d + c : d - c;
    newdeg[a] = nd;
    dsum += (long long)nd - (long long)d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xFFFFFFFFu, dsum, o);
  if (lane_id() == 0 && dsum) atomicAdd((unsigned long long*)delta, (unsigned long long)dsum);
}

// Long lists are split into chunks of kChunkIds ids, one warp task each, so
// that a high-degree vertex (which a batch of uniformly chosen edges touches
// every time) does not leave one warp working on it long after the others.
constexpr uint32_t kChunkIds = 4096;

// chunks per affected vertex: cm by the old list (merge), cc by the new one (copy-back)
__global__ void chunk_count_kernel(DynView g, const uint32_t* __restrict__ seg_v, const uint32_t* __restrict__ newdeg,
                                   uint64_t A, uint32_t* cm, uint32_t* cc) {
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t d = g.degree(seg_v[a]), nd = newdeg[a];
    cm[a] = d > kChunkIds ? (d + kChunkIds - 1) / kChunkIds : 1u;
    cc[a] = nd > kChunkIds ? (nd + kChunkIds - 1) / kChunkIds : 1u;
  }
}

// item[j] = the affected vertex of chunk task j (starts = scan of the counts)
__global__ void chunk_expand_kernel(const uint64_t* __restrict__ start, uint64_t A, uint32_t* item) {
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x)
    for (uint64_t j = start[a]; j < start[a + 1]; ++j) item[j] = (uint32_t)a;
}

// One warp per chunk task writes its part of a merged list into buf[toff[a] ...]:
// the old ids of the chunk, and (chunk 0 of an insert) the effective batch ids.
__global__ void merge_kernel(DynView g, const uint32_t* __restrict__ cols, const uint64_t* __restrict__ seg_start,
                             const uint32_t* __restrict__ seg_v, const uint32_t* __restrict__ mark,
                             const uint64_t* __restrict__ mrank, const uint64_t* __restrict__ toff,
                             const uint32_t* __restrict__ item, const uint64_t* __restrict__ cstart, uint64_t NC,
                             bool insert, uint32_t* __restrict__ buf) {
  const uint32_t lane = lane_id();
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t t = w0; t < NC; t += nw) {
    const uint32_t a = item[t];
    const uint32_t c = (uint32_t)(t - cstart[a]);
    const uint32_t v = seg_v[a];
    const Seg s = g.seg(v);
    const uint64_t b0 = seg_start[a], b1 = seg_start[a + 1];
    const uint32_t blen = (uint32_t)(b1 - b0);
    const uint32_t* bcol = cols + b0;
    const uint64_t r0 = mrank[b0];
    uint32_t* out = buf + toff[a];
    const uint32_t i1 = min(s.len, (c + 1) * kChunkIds);
    // old ids
    for (uint32_t i = c * kChunkIds + lane; i < i1; i += 32) {
      uint32_t x = __ldg(s.p + i);
      uint32_t j = lower_bound(bcol, blen, x);  // batch ids < x
      uint32_t marked_before = (uint32_t)(mrank[b0 + j] - r0);
      if (insert) {
        out[i + marked_before] = x;
      } else {
        bool gone = j < blen && __ldg(bcol + j) == x;
        if (!gone) out[i - marked_before] = x;
      }
    }
    // effective batch ids (insert only)
    if (insert && c == 0) {
      for (uint32_t q = lane; q < blen; q += 32) {
        if (mark[b0 + q]) {
          uint32_t y = __ldg(bcol + q);
          uint32_t k = lower_bound(s.p, s.len, y);  // old ids < y
          out[(uint32_t)(mrank[b0 + q] - r0) + k] = y;
        }
      }
    }
  }
}

// Storage for each new list.  Pops may drive a stack top below zero; the
// fix-up kernel clamps it.  Frees happen in a later kernel (no concurrent
// push and pop).
__global__ void alloc_kernel(DynVertex* vtx, const uint32_t* __restrict__ seg_v, const uint32_t* __restrict__ newdeg,
                             uint64_t A, uint32_t icap, uint32_t* const* stacks, long long* tops,
                             unsigned long long* bump, uint64_t* new_run, uint32_t* new_cls, uint64_t* free_run,
                             uint32_t* free_cls) {
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x) {
    const DynVertex r = vtx[seg_v[a]];
    const uint32_t nd = newdeg[a];
    uint32_t oc = r.cls;
    uint64_t orun = r.run;
    free_run[a] = ~0ull;
    free_cls[a] = kNoRun;
    if (nd <= icap) {
      new_cls[a] = kNoRun;
      new_run[a] = 0;
      if (oc != kNoRun) {
        free_run[a] = orun;
        free_cls[a] = oc;
      }
      continue;
    }
    uint32_t c = run_class(nd);
    if (oc != kNoRun && oc >= c && oc <= c + 1) {  // keep the run (fits, not oversized)
      new_cls[a] = oc;
      new_run[a] = orun;
      continue;
    }
    uint64_t run;
    long long t = atomicAdd((unsigned long long*)(tops + c), (unsigned long long)(-1ll));
    if (t > 0) run = stacks[c][t - 1];
    else run = atomicAdd(bump, 1ull << c);
    new_cls[a] = c;
    new_run[a] = run;
    if (oc != kNoRun) {
      free_run[a] = orun;
      free_cls[a] = oc;
    }
  }
}

__global__ void clamp_tops_kernel(long long* tops) {
  if (threadIdx.x < kClasses && tops[threadIdx.x] < 0) tops[threadIdx.x] = 0;
}

// One warp per chunk task copies its part of a merged list to the new
// storage; chunk 0 also writes the inline ids and the vertex record.
__global__ void copyback_kernel(DynVertex* vtx, uint32_t* pool, const uint32_t* __restrict__ seg_v,
                                const uint32_t* __restrict__ newdeg, const uint64_t* __restrict__ new_run,
                                const uint32_t* __restrict__ new_cls, const uint64_t* __restrict__ toff,
                                const uint32_t* __restrict__ buf, const uint32_t* __restrict__ item,
                                const uint64_t* __restrict__ cstart, uint64_t NC, uint32_t icap) {
  const uint32_t lane = lane_id();
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t t = w0; t < NC; t += nw) {
    const uint32_t a = item[t];
    const uint32_t c = (uint32_t)(t - cstart[a]);
    DynVertex* r = vtx + seg_v[a];
    const uint32_t nd = newdeg[a];
    const uint32_t* src = buf + toff[a];
    if (nd <= icap) {
      if (lane < kInline) r->inl[lane] = lane < nd ? src[lane] : kInf;
    } else {
      uint32_t* dst = pool + new_run[a] * kBlockIds;
      const uint32_t i1 = min(nd, (c + 1) * kChunkIds);
      for (uint32_t i = c * kChunkIds + lane; i < i1; i += 32) dst[i] = src[i];
    }
    __syncwarp();
    if (lane == 0 && c == 0) {
      r->deg = nd;
      r->cls = new_cls[a];
      r->run = nd <= icap ? 0 : new_run[a];
    }
  }
}

__global__ void free_kernel(const uint64_t* __restrict__ free_run, const uint32_t* __restrict__ free_cls, uint64_t A,
                            uint32_t* const* stacks, long long* tops, const uint64_t* __restrict__ cap) {
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t c = free_cls[a];
    if (c == kNoRun || c >= (uint32_t)kClasses) continue;
    long long t = (long long)atomicAdd((unsigned long long*)(tops + c), 1ull);
    if ((uint64_t)t < cap[c]) stacks[c][t] = (uint32_t)free_run[a];
    else atomicAdd((unsigned long long*)(tops + c), (unsigned long long)(-1ll));  // full: the run is dropped
  }
}

// worst-case pool blocks a batch may bump-allocate
__global__ void need_kernel(const uint32_t* __restrict__ newdeg, uint64_t A, uint32_t icap, unsigned long long* need) {
  unsigned long long s = 0;
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x)
    if (newdeg[a] > icap) s += 1ull << run_class(newdeg[a]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  if (lane_id() == 0 && s) atomicAdd(need, s);
}

byo_status alloc_stacks(DynStore* d) {
  for (int c = 0; c < kClasses; ++c) {
    uint64_t cap = d->pool_blocks >> c;
    if (cap > (1ull << 24)) cap = 1ull << 24;
    if (cap < 16) cap = 16;
    d->stack_cap[c] = cap;
    BYO_RETURN_IF(dev_alloc_t(&d->stacks[c], cap, "free-run stack"));
  }
  return BYO_OK;
}

// Grow the pool to at least `blocks` (copying the used part); stacks keep
// their run indices, which stay valid in the larger pool.
byo_status grow_pool(DynStore* d, uint64_t used, uint64_t blocks, cudaStream_t s) {
  uint32_t* np = nullptr;
  BYO_RETURN_IF(dev_alloc_t(&np, blocks * kBlockIds, "dynamic pool"));
  uint32_t *nk = nullptr, *npos = nullptr;
  if (d->hashed) {  // the index arrays grow with the pool (64 slots per block)
    byo_status st = dev_alloc_t(&nk, blocks * kHashSlots, "hash index keys");
    if (st == BYO_OK) st = dev_alloc_t(&npos, blocks * kHashSlots, "hash index positions");
    if (st != BYO_OK) {
      dev_free(np);
      dev_free(nk);
      return st;
    }
  }
  if (used) BYO_CUDA(cudaMemcpyAsync(np, d->pool, used * kBlockIds * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  if (d->hashed && used) {
    BYO_CUDA(cudaMemcpyAsync(nk, d->hkey, used * kHashSlots * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    BYO_CUDA(cudaMemcpyAsync(npos, d->hpos, used * kHashSlots * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
  BYO_CUDA(cudaStreamSynchronize(s));
  dev_free(d->pool);
  d->pool = np;
  if (d->hashed) {
    dev_free(d->hkey);
    dev_free(d->hpos);
    d->hkey = nk;
    d->hpos = npos;
  }
  d->pool_blocks = blocks;
  return BYO_OK;
}

template <typename OffT>
byo_status load_from_csr(byo_graph* g, DynStore* d, cudaStream_t s) {
  const OffT* off = static_cast<const OffT*>(g->off);
  uint32_t* blocks = nullptr;
  uint64_t* first = nullptr;
  uint64_t total = 0;
  byo_status st = tmp_alloc_t(&blocks, g->n + 1ull, s, "run sizes");
  if (st == BYO_OK) st = tmp_alloc_t(&first, g->n + 1ull, s, "run starts");
  if (st == BYO_OK) {
    dyn_blocks_kernel<OffT><<<grid_for(g->n, 256), 256, 0, s>>>(off, g->n, d->icap, blocks);
    note_launch();
    st = scan_u32_to_u64(blocks, first, g->n, &total, s);
  }
  if (st == BYO_OK) {
    // room for the runs plus the same again for growth
    d->pool_blocks = total * 2 + 4096;
    st = dev_alloc_t(&d->pool, d->pool_blocks * kBlockIds, "dynamic pool");
  }
  if (st == BYO_OK) st = alloc_stacks(d);
  if (st == BYO_OK) {
    cudaMemsetAsync(d->tops, 0, sizeof(long long) * kClasses, s);
    cudaMemcpyAsync(d->bump, &total, sizeof(total), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(d->vtx + g->n, 0, sizeof(DynVertex), s);
    dyn_load_kernel<OffT><<<grid_for((uint64_t)g->n * 32, 256), 256, 0, s>>>(off, g->col, g->n, d->icap, d->hashed,
                                                                               first, d->vtx, d->pool);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "dynamic load");
  }
  tmp_free(blocks, s);
  tmp_free(first, s);
  return st;
}

// ---------------------------------------------------------------- hash-indexed variant
// BYO_DYN_HASH: the hashed-blocks container of DHB (Section 5.2) fed by the
// semisort-only batch form of Section 4.1 (group the batch by source, order
// nothing).  Records, inline head and pool runs are the ones above; a list is
// kept dense in insertion order, and a list held in a run of C ids has an
// open-addressing index of 2C slots (linear probing, multiplicative hash):
// hkey the id (kInf empty, kTomb deleted), hpos the id's position in the list.
// One warp owns each vertex the batch touches, so no two warps ever update
// one list or one index and nothing waits on another thread.
//   insert: plan per vertex (stay inline; insert in place; rebuild the index
//     in place when tombstones crowd it; move to a larger run), allocate,
//     clear and fill the moved or rebuilt indexes (chunk tasks), then the
//     vertex's warp probes the index for each batch id: a CAS that takes an
//     empty slot admits a new id, appended at the end of the list; meeting
//     the id itself means it is present (or a duplicate in the batch);
//   delete: the vertex's warp turns the keys it finds into tombstones, then
//     fills the holes below the new degree with the ids that survive above
//     it and re-points their index entries; a list that falls to the inline
//     capacity goes back inline and frees its run.
// Live ids plus tombstones never exceed 3/4 of an index's slots (the plan
// rebuilds or moves before an insert could pass that; deletes only turn live
// keys into tombstones), so every probe meets an empty slot within the index.
enum : uint32_t { kActInline = 0, kActKeep = 1, kActRebuild = 2, kActMove = 3 };

__device__ __forceinline__ uint32_t hslot(uint32_t x, uint32_t c) {  // index of class c: 2^(c+6) slots
  return (x * 2654435769u) >> (26 - c);
}
__device__ __forceinline__ uint32_t hmask(uint32_t c) { return 0xFFFFFFFFu >> (26 - c); }

// Both directions of each pair; self-loops, and pairs with an id >= n (which
// also set *bad), get the row kInf and are skipped by the semisort.
__global__ void hsym_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t k, uint32_t n,
                            uint32_t* rows, uint32_t* cols, uint32_t* bad) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t u = src[i], v = dst[i];
    const bool ok = u < n && v < n;
    if (!ok) *bad = 1u;
    const bool keep = ok && u != v;
    rows[2 * i] = keep ? u : kInf;
    cols[2 * i] = v;
    rows[2 * i + 1] = keep ? v : kInf;
    cols[2 * i + 1] = u;
  }
}

// Semisort, pass 1: count the entries per source; the first entry of a
// source gives it a group slot (one atomic per warp for the slots).
__global__ void hhist_kernel(const uint32_t* __restrict__ rows, uint64_t B, uint32_t* vcnt, uint32_t* vslot,
                             uint32_t* aff, unsigned long long* nA) {
  const uint32_t lane = lane_id();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; i0 < B; i0 += stride) {
    const uint64_t i = i0 + lane;
    const uint32_t r = i < B ? rows[i] : kInf;
    const bool first = r != kInf && atomicAdd(vcnt + r, 1u) == 0u;
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, first);
    uint32_t base = 0;
    if (lane == 0 && m) base = (uint32_t)atomicAdd(nA, (unsigned long long)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (first) {
      const uint32_t a = base + __popc(m & lanemask_lt());
      aff[a] = r;
      vslot[r] = a;
    }
  }
}

// group sizes (gcnt[A] = 0, so that a scan of A + 1 entries ends with the total)
__global__ void hgcount_kernel(const uint32_t* __restrict__ aff, uint64_t A, const uint32_t* __restrict__ vcnt,
                               uint32_t* gcnt) {
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x)
    gcnt[a] = vcnt[aff[a]];
  if (blockIdx.x == 0 && threadIdx.x == 0) gcnt[A] = 0;
}

// Semisort, pass 2: each entry takes a place in its source's group by
// counting the source's counter back down (which leaves it zero again).
__global__ void hscatter_kernel(const uint32_t* __restrict__ rows, const uint32_t* __restrict__ cols, uint64_t B,
                                uint32_t* vcnt, const uint32_t* __restrict__ vslot, const uint64_t* __restrict__ gstart,
                                uint32_t* gcols) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t r = rows[i];
    if (r == kInf) continue;
    const uint64_t p = gstart[vslot[r]] + atomicSub(vcnt + r, 1u) - 1u;
    gcols[p] = cols[i];
  }
}

// Insert plan per affected vertex from an upper bound on its new degree
// (old degree + group size, at most n): the action, the class of the run the
// list will live in, and the pool blocks moves may take (*need).
__global__ void hplan_kernel(const DynVertex* __restrict__ vtx, const uint32_t* __restrict__ aff,
                             const uint64_t* __restrict__ gstart, uint64_t A, uint32_t n, uint32_t icap, uint32_t* act,
                             uint32_t* new_cls, unsigned long long* need) {
  unsigned long long sum = 0;
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x) {
    const DynVertex& r = vtx[aff[a]];
    const uint32_t cls = r.cls;
    const uint64_t raw = (uint64_t)r.deg + (gstart[a + 1] - gstart[a]);
    const uint64_t ub = raw < n ? raw : n;  // no list holds more than n - 1 ids
    uint32_t ac, c = kNoRun;
    if (cls == kNoRun) {
      ac = raw <= icap ? kActInline : kActMove;  // inline inserts take one batch id per lane
    } else {
      const uint64_t C = (uint64_t)kBlockIds << cls;
      if (ub > C) ac = kActMove;
      else ac = ub + r.inl[0] <= C + C / 2 ? kActKeep : kActRebuild;
      c = cls;
    }
    if (ac == kActMove) {
      c = run_class((uint32_t)ub);
      sum += 1ull << c;
    }
    act[a] = ac;
    new_cls[a] = c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xFFFFFFFFu, sum, o);
  if (lane_id() == 0 && sum) atomicAdd(need, sum);
}

// Runs for moved lists (a free run of the class, else bump-allocated); the
// old run of a moved list is freed after the batch.  Pops may drive a stack
// top below zero; clamp_tops_kernel fixes it up.
__global__ void halloc_kernel(const DynVertex* __restrict__ vtx, const uint32_t* __restrict__ aff,
                              const uint32_t* __restrict__ act, const uint32_t* __restrict__ new_cls, uint64_t A,
                              uint32_t* const* stacks, long long* tops, unsigned long long* bump, uint64_t* new_run,
                              uint64_t* free_run, uint32_t* free_cls) {
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x) {
    const DynVertex& r = vtx[aff[a]];
    free_run[a] = ~0ull;
    free_cls[a] = kNoRun;
    if (act[a] != kActMove) {
      new_run[a] = r.run;
      continue;
    }
    const uint32_t c = new_cls[a];
    uint64_t run;
    const long long t = atomicAdd((unsigned long long*)(tops + c), (unsigned long long)(-1ll));
    if (t > 0) run = stacks[c][t - 1];
    else run = atomicAdd(bump, 1ull << c);
    new_run[a] = run;
    if (r.cls != kNoRun) {
      free_run[a] = r.run;
      free_cls[a] = r.cls;
    }
  }
}

// chunk tasks per affected vertex: index slots to clear (moved and rebuilt
// lists), ids to enter into an index (the same lists; with act == NULL every
// run list, for the initial build, where a = the vertex itself)
__global__ void htask_count_kernel(const DynVertex* __restrict__ vtx, const uint32_t* __restrict__ aff,
                                   const uint32_t* __restrict__ act, const uint32_t* __restrict__ new_cls, uint64_t A,
                                   uint32_t* nclear, uint32_t* nfill) {
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = aff ? aff[a] : (uint32_t)a;
    const bool build = act ? (act[a] == kActRebuild || act[a] == kActMove) : vtx[v].cls != kNoRun;
    const uint32_t d = vtx[v].deg;
    if (nclear) {
      const uint64_t H = build ? (uint64_t)kHashSlots << new_cls[a] : 0;
      nclear[a] = (uint32_t)((H + kChunkIds - 1) / kChunkIds);
    }
    nfill[a] = build ? (d + kChunkIds - 1) / kChunkIds : 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (nclear) nclear[A] = 0;
    nfill[A] = 0;
  }
}

// one warp per task: kChunkIds index slots of a moved or rebuilt list set empty
__global__ void hclear_kernel(const uint32_t* __restrict__ item, const uint64_t* __restrict__ tstart, uint64_t NT,
                              const uint64_t* __restrict__ new_run, const uint32_t* __restrict__ new_cls,
                              uint32_t* hkey) {
  const uint32_t lane = lane_id();
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t t = w0; t < NT; t += nw) {
    const uint32_t a = item[t];
    const uint64_t ch = t - tstart[a];
    uint32_t* key = hkey + new_run[a] * kHashSlots;
    const uint64_t H = (uint64_t)kHashSlots << new_cls[a];
    const uint64_t hi = min(H, (ch + 1) * kChunkIds);
    for (uint64_t i = ch * kChunkIds + lane; i < hi; i += 32) key[i] = kInf;
  }
}

// One warp per task: kChunkIds ids of a list are copied to its new run (a
// moved list) and entered into the run's index.  Without act/new_run (the
// initial build) the list stays where the record says.
__global__ void hfill_kernel(const DynVertex* __restrict__ vtx, uint32_t* pool, uint32_t* hkey, uint32_t* hpos,
                             const uint32_t* __restrict__ aff, const uint64_t* __restrict__ new_run,
                             const uint32_t* __restrict__ new_cls, const uint32_t* __restrict__ item,
                             const uint64_t* __restrict__ tstart, uint64_t NT, uint32_t* err) {
  const uint32_t lane = lane_id();
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t t = w0; t < NT; t += nw) {
    const uint32_t a = item[t];
    const uint64_t ch = t - tstart[a];
    const uint32_t v = aff ? aff[a] : a;
    const DynVertex& r = vtx[v];
    const uint32_t d = r.deg;
    const uint32_t* from = r.cls == kNoRun ? r.inl : pool + r.run * kBlockIds;
    const uint64_t run = new_run ? new_run[a] : r.run;
    const uint32_t c = new_cls ? new_cls[a] : r.cls;
    uint32_t* to = pool + run * kBlockIds;
    uint32_t* key = hkey + run * kHashSlots;
    uint32_t* pos = hpos + run * kHashSlots;
    const uint32_t mask = hmask(c);
    const uint32_t hi = (uint32_t)min((uint64_t)d, (ch + 1) * kChunkIds);
    for (uint32_t i = (uint32_t)(ch * kChunkIds) + lane; i < hi; i += 32) {
      const uint32_t x = from[i];
      if (from != to) to[i] = x;
      uint32_t h = hslot(x, c);
      bool placed = false;
      for (uint64_t it = 0; it <= mask; ++it) {
        if (atomicCAS(key + h, kInf, x) == kInf) {
          pos[h] = i;
          placed = true;
          break;
        }
        h = (h + 1) & mask;
      }
      if (!placed) *err = 1u;
    }
  }
}

// adds the threads' degree changes into *delta, one atomic per block
__device__ __forceinline__ void block_add_delta(long long dsum, long long* delta) {
  __shared__ long long bsum;
  if (threadIdx.x == 0) bsum = 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xFFFFFFFFu, dsum, o);
  __syncthreads();
  if (lane_id() == 0 && dsum) atomicAdd((unsigned long long*)&bsum, (unsigned long long)dsum);
  __syncthreads();
  if (threadIdx.x == 0 && bsum) atomicAdd((unsigned long long*)delta, (unsigned long long)bsum);
}

// Groups of at most kSmallGroup ids (most of a batch of scattered pairs) are
// applied by one thread each; larger ones by a warp (mid[]) or, above
// kWarpGroupMax ids, by a CTA (huge[]).
constexpr uint32_t kSmallGroup = 4;

__global__ void hsplit_kernel(const uint64_t* __restrict__ gstart, uint64_t A, uint32_t warp_max, uint32_t* mid,
                              uint32_t* nmid, uint32_t* huge, uint32_t* nhuge) {
  const uint32_t lane = lane_id();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t a0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; a0 < A; a0 += stride) {
    const uint64_t a = a0 + lane;
    const uint64_t gs = a < A ? gstart[a + 1] - gstart[a] : 0;
    const bool m1 = gs > kSmallGroup && gs <= warp_max, m2 = gs > warp_max;
    const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, m1), b2 = __ballot_sync(0xFFFFFFFFu, m2);
    uint32_t base1 = 0, base2 = 0;
    if (lane == 0 && b1) base1 = atomicAdd(nmid, (uint32_t)__popc(b1));
    if (lane == 0 && b2) base2 = atomicAdd(nhuge, (uint32_t)__popc(b2));
    base1 = __shfl_sync(0xFFFFFFFFu, base1, 0);
    base2 = __shfl_sync(0xFFFFFFFFu, base2, 0);
    if (m1) mid[base1 + __popc(b1 & lanemask_lt())] = (uint32_t)a;
    if (m2) huge[base2 + __popc(b2 & lanemask_lt())] = (uint32_t)a;
  }
}

// the slot *h of key y in an index of class c; false if y is not there
__device__ __forceinline__ bool hfind(const uint32_t* key, uint32_t y, uint32_t c, uint32_t* h) {
  const uint32_t mask = hmask(c);
  uint32_t at = hslot(y, c);
  for (uint64_t it = 0; it <= mask; ++it) {
    const uint32_t k = key[at];
    if (k == y) {
      *h = at;
      return true;
    }
    if (k == kInf) return false;
    at = (at + 1) & mask;
  }
  return false;
}

// One thread applies a small insert group to a list it alone owns.
__device__ void hinsert_thread(DynVertex* r, uint32_t* pool, uint32_t* hkey, uint32_t* hpos,
                               const uint32_t* __restrict__ gcols, uint64_t g0, uint64_t g1, uint32_t ac, uint32_t c,
                               uint64_t run, uint32_t icap, uint64_t* free_run, uint32_t* free_cls, uint64_t a,
                               long long& dsum, uint32_t* err) {
  const uint32_t d0 = r->deg, cls0 = r->cls;
  uint32_t d = d0;
  if (ac == kActInline) {
    for (uint64_t i = g0; i < g1; ++i) {
      const uint32_t x = gcols[i];
      bool dup = false;
      for (uint32_t j = 0; j < d; ++j) dup |= r->inl[j] == x;
      if (!dup) r->inl[d++] = x;
    }
  } else {
    uint32_t* ids = pool + run * kBlockIds;
    uint32_t* key = hkey + run * kHashSlots;
    uint32_t* pos = hpos + run * kHashSlots;
    const uint32_t mask = hmask(c);
    for (uint64_t i = g0; i < g1; ++i) {
      const uint32_t x = gcols[i];
      uint32_t h = hslot(x, c);
      bool done = false;
      for (uint64_t it = 0; it <= mask; ++it) {
        const uint32_t k = key[h];
        if (k == x) {
          done = true;
          break;
        }
        if (k == kInf) {
          key[h] = x;
          pos[h] = d;
          ids[d++] = x;
          done = true;
          break;
        }
        h = (h + 1) & mask;
      }
      if (!done) *err = 1u;
    }
    if (ac == kActMove && cls0 == kNoRun && d <= icap) {  // stays within the inline capacity
      for (uint32_t j = 0; j < kInline; ++j) r->inl[j] = j < d ? ids[j] : kInf;
      free_run[a] = run;
      free_cls[a] = c;
    } else {
      if (ac == kActMove) {
        r->cls = c;
        r->run = run;
      }
      if (ac != kActKeep) r->inl[0] = 0;
    }
  }
  r->deg = d;
  dsum += (long long)d - (long long)d0;
}

// One thread applies a small delete group: each found id becomes a tombstone
// and the list's last id moves into its place.
__device__ void hdelete_thread(DynVertex* r, uint32_t* pool, uint32_t* hkey, uint32_t* hpos,
                               const uint32_t* __restrict__ gcols, uint64_t g0, uint64_t g1, uint32_t icap,
                               uint64_t* free_run, uint32_t* free_cls, uint64_t a, long long& dsum, uint32_t* err) {
  const uint32_t d0 = r->deg, cls = r->cls;
  uint32_t d = d0;
  free_run[a] = ~0ull;
  free_cls[a] = kNoRun;
  if (cls == kNoRun) {
    for (uint64_t i = g0; i < g1; ++i) {
      const uint32_t x = gcols[i];
      for (uint32_t j = 0; j < d; ++j)
        if (r->inl[j] == x) {
          r->inl[j] = r->inl[d - 1];
          r->inl[d - 1] = kInf;
          --d;
          break;
        }
    }
  } else {
    const uint64_t run = r->run;
    uint32_t* ids = pool + run * kBlockIds;
    uint32_t* key = hkey + run * kHashSlots;
    uint32_t* pos = hpos + run * kHashSlots;
    uint32_t tombs = r->inl[0];
    for (uint64_t i = g0; i < g1; ++i) {
      uint32_t h;
      if (!hfind(key, gcols[i], cls, &h)) continue;
      key[h] = kTomb;
      const uint32_t p = pos[h];
      const uint32_t last = d - 1;
      if (p != last) {
        const uint32_t y = ids[last];
        ids[p] = y;
        uint32_t hy;
        if (hfind(key, y, cls, &hy)) pos[hy] = p;
        else *err = 1u;
      }
      --d;
      ++tombs;
    }
    if (d <= icap) {  // back inline; the run is freed
      for (uint32_t j = 0; j < kInline; ++j) r->inl[j] = j < d ? ids[j] : kInf;
      r->cls = kNoRun;
      r->run = 0;
      free_run[a] = run;
      free_cls[a] = cls;
    } else {
      r->inl[0] = tombs;
    }
  }
  r->deg = d;
  dsum += (long long)d - (long long)d0;
}

// A team of threads applying one group: a warp (groups of kSmallGroup + 1 ..
// kWarpGroupMax ids) or a whole CTA (larger groups: a hub's share of a batch).
constexpr uint32_t kWarpGroupMax = 256;

template <bool kCta>
struct Team {
  uint32_t* sh;  // kCta: one word per warp of the CTA
  __device__ __forceinline__ uint32_t id() const { return kCta ? threadIdx.x : lane_id(); }
  __device__ __forceinline__ uint32_t size() const { return kCta ? blockDim.x : 32u; }
  __device__ __forceinline__ void sync() const {
    if (kCta) __syncthreads();
    else __syncwarp();
  }
  // rank of this thread among the team's threads with f set (in id order),
  // and their number; a barrier of the team
  __device__ __forceinline__ uint32_t scan(bool f, uint32_t* total) const {
    const uint32_t m = __ballot_sync(0xFFFFFFFFu, f);
    if (!kCta) {
      *total = __popc(m);
      return __popc(m & lanemask_lt());
    }
    const uint32_t w = threadIdx.x >> 5;
    __syncthreads();  // the previous scan's readers are done with sh
    if (lane_id() == 0) sh[w] = __popc(m);
    __syncthreads();
    uint32_t before = 0, tot = 0;
    for (uint32_t i = 0; i < (blockDim.x >> 5); ++i) {
      const uint32_t c = sh[i];
      before += i < w ? c : 0u;
      tot += c;
    }
    *total = tot;
    return before + __popc(m & lanemask_lt());
  }
};

// A team applies an insert group to a list that is in, or moves into, a run:
// a CAS that takes an empty slot admits a new id, appended at the list's end.
template <bool kCta>
__device__ void hinsert_team(const Team<kCta>& T, DynVertex* r, uint32_t* pool, uint32_t* hkey, uint32_t* hpos,
                             const uint32_t* __restrict__ gcols, uint64_t g0, uint64_t g1, uint32_t ac, uint32_t c,
                             uint64_t run, uint32_t icap, uint64_t* free_run, uint32_t* free_cls, uint64_t a,
                             long long& dsum, uint32_t* err) {
  const uint32_t t = T.id();
  const uint32_t d0 = r->deg, cls0 = r->cls;
  uint32_t* ids = pool + run * kBlockIds;
  uint32_t* key = hkey + run * kHashSlots;
  uint32_t* pos = hpos + run * kHashSlots;
  const uint32_t mask = hmask(c);
  uint32_t d = d0;
  for (uint64_t i0 = g0; i0 < g1; i0 += T.size()) {
    const uint64_t i = i0 + t;
    uint32_t x = kInf, slot = 0;
    bool fresh = false;
    if (i < g1) {
      x = gcols[i];
      uint32_t h = hslot(x, c);
      bool done = false;
      for (uint64_t it = 0; it <= mask; ++it) {
        const uint32_t k = ld_cg(key + h);
        if (k == x) {
          done = true;
          break;
        }
        if (k == kInf) {
          const uint32_t o = atomicCAS(key + h, kInf, x);
          if (o == kInf) {
            fresh = done = true;
            slot = h;
            break;
          }
          if (o == x) {
            done = true;
            break;
          }
        }
        h = (h + 1) & mask;
      }
      if (!done) *err = 1u;
    }
    uint32_t cnt;
    const uint32_t rk = T.scan(fresh, &cnt);
    if (fresh) {
      ids[d + rk] = x;
      pos[slot] = d + rk;
    }
    d += cnt;
  }
  T.sync();
  if (ac == kActMove && cls0 == kNoRun && d <= icap) {
    // an inline list the plan moved (upper bound) that stays within the
    // inline capacity: back inline, and the new run is freed
    const uint32_t y = t < d ? ids[t] : kInf;
    T.sync();
    if (t < kInline) r->inl[t] = y;
    if (t == 0) {
      free_run[a] = run;
      free_cls[a] = c;
    }
  } else if (t == 0) {
    if (ac == kActMove) {
      r->cls = c;
      r->run = run;
    }
    if (ac != kActKeep) r->inl[0] = 0;  // a fresh index has no tombstones
  }
  if (t == 0) {
    r->deg = d;
    dsum += (long long)d - (long long)d0;
  }
}

// A team applies a delete group.  Run lists: found keys become tombstones;
// the holes below the new degree are filled with the ids that survive above
// it, whose index entries follow.  s1, s2, s3: scratch with one entry per
// batch entry (freed positions, the holes among them, the surviving tail
// positions), each group in its own slice.
template <bool kCta>
__device__ void hdelete_team(const Team<kCta>& T, DynVertex* r, uint32_t* pool, uint32_t* hkey, uint32_t* hpos,
                             const uint32_t* __restrict__ gcols, uint64_t g0, uint64_t g1, uint32_t icap, uint32_t* s1,
                             uint32_t* s2, uint32_t* s3, uint64_t* free_run, uint32_t* free_cls, uint64_t a,
                             long long& dsum, uint32_t* err) {
  const uint32_t t = T.id(), ts = T.size();
  const uint32_t d0 = r->deg, cls = r->cls;
  uint32_t d;
  if (t == 0) {
    free_run[a] = ~0ull;
    free_cls[a] = kNoRun;
  }
  if (cls == kNoRun) {  // inline: thread j checks the j-th id against the group
    const uint32_t y = t < d0 ? r->inl[t] : kInf;
    bool keep = t < d0;
    if (keep)
      for (uint64_t i = g0; i < g1; ++i)
        if (gcols[i] == y) {
          keep = false;
          break;
        }
    const uint32_t rk = T.scan(keep, &d);
    if (keep) r->inl[rk] = y;
    T.sync();
    if (t >= d && t < kInline) r->inl[t] = kInf;
  } else {
    const uint64_t run = r->run;
    uint32_t* ids = pool + run * kBlockIds;
    uint32_t* key = hkey + run * kHashSlots;
    uint32_t* pos = hpos + run * kHashSlots;
    const uint32_t mask = hmask(cls);
    uint32_t ndel = 0;
    // 1: found ids become tombstones; s1 = the position each one freed
    for (uint64_t i0 = g0; i0 < g1; i0 += ts) {
      const uint64_t i = i0 + t;
      uint32_t p = kInf;
      if (i < g1) {
        const uint32_t x = gcols[i];
        uint32_t h = hslot(x, cls);
        for (uint64_t it = 0; it <= mask; ++it) {
          const uint32_t k = ld_cg(key + h);
          if (k == kInf) break;
          if (k == x) {
            if (atomicCAS(key + h, x, kTomb) == x) p = pos[h];
            break;
          }
          h = (h + 1) & mask;
        }
        s1[i] = p;
      }
      uint32_t c;
      T.scan(p != kInf, &c);
      ndel += c;
    }
    d = d0 - ndel;
    T.sync();
    // 2: mark the freed positions
    for (uint64_t i = g0 + t; i < g1; i += ts) {
      const uint32_t p = s1[i];
      if (p != kInf) ids[p] = kInf;
    }
    T.sync();
    // 3: holes (freed positions below d) and survivors (ids left in [d, d0))
    uint32_t nh = 0, ns = 0;
    for (uint64_t i0 = g0; i0 < g1; i0 += ts) {
      const uint64_t i = i0 + t;
      const uint32_t p = i < g1 ? s1[i] : kInf;
      const bool hole = p < d;
      uint32_t c;
      const uint32_t rk = T.scan(hole, &c);
      if (hole) s2[g0 + nh + rk] = p;
      nh += c;
    }
    for (uint32_t q0 = d; q0 < d0; q0 += ts) {
      const uint32_t q = q0 + t;
      const bool live = q < d0 && ids[q] != kInf;
      uint32_t c;
      const uint32_t rk = T.scan(live, &c);
      if (live) s3[g0 + ns + rk] = q;
      ns += c;
    }
    if (ns != nh) {
      if (t == 0) *err = 1u;
      nh = ns < nh ? ns : nh;
    }
    T.sync();
    // 4: survivors move into the holes; their index entries follow
    for (uint32_t k = t; k < nh; k += ts) {
      const uint32_t p = s2[g0 + k], q = s3[g0 + k];
      const uint32_t y = ids[q];
      ids[p] = y;
      uint32_t h = hslot(y, cls);
      bool found = false;
      for (uint64_t it = 0; it <= mask; ++it) {
        if (ld_cg(key + h) == y) {
          pos[h] = p;
          found = true;
          break;
        }
        h = (h + 1) & mask;
      }
      if (!found) *err = 1u;
    }
    T.sync();
    if (d <= icap) {  // back inline; the run is freed
      const uint32_t y = t < d ? ids[t] : kInf;
      T.sync();
      if (t < kInline) r->inl[t] = y;
      if (t == 0) {
        r->cls = kNoRun;
        r->run = 0;
        free_run[a] = run;
        free_cls[a] = cls;
      }
    } else if (t == 0) {
      r->inl[0] += ndel;  // tombstones
    }
  }
  if (t == 0) {
    r->deg = d;
    dsum += (long long)d - (long long)d0;
  }
}

// Inserts: small groups a thread each, mid-sized ones a warp each (mid[]),
// the largest a CTA each (huge[]).
__global__ void hinsert_kernel(DynVertex* vtx, uint32_t* pool, uint32_t* hkey, uint32_t* hpos,
                               const uint32_t* __restrict__ aff, const uint64_t* __restrict__ gstart,
                               const uint32_t* __restrict__ gcols, const uint32_t* __restrict__ act,
                               const uint64_t* __restrict__ new_run, const uint32_t* __restrict__ new_cls, uint64_t A,
                               const uint32_t* __restrict__ mid, const uint32_t* __restrict__ nmid,
                               const uint32_t* __restrict__ huge, const uint32_t* __restrict__ nhuge, uint32_t icap,
                               uint64_t* free_run, uint32_t* free_cls, long long* delta, uint32_t* err) {
  __shared__ uint32_t sh[32];
  const uint32_t lane = lane_id();
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  long long dsum = 0;
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t g0 = gstart[a], g1 = gstart[a + 1];
    if (g1 - g0 <= kSmallGroup)
      hinsert_thread(vtx + aff[a], pool, hkey, hpos, gcols, g0, g1, act[a], new_cls[a], new_run[a], icap, free_run,
                     free_cls, a, dsum, err);
  }
  const Team<false> W{nullptr};
  const uint32_t NM = *nmid;
  for (uint64_t b = w0; b < NM; b += nw) {
    const uint32_t a = mid[b];
    DynVertex* r = vtx + aff[a];
    const uint64_t g0 = gstart[a], g1 = gstart[a + 1];
    if (act[a] == kActInline) {  // d0 + group size <= icap <= kInline: one id per lane
      const uint32_t d0 = r->deg;
      const uint32_t gs = (uint32_t)(g1 - g0);
      const uint32_t x = lane < gs ? gcols[g0 + lane] : kInf;
      bool fresh = lane < gs;
      for (uint32_t j = 0; j < d0; ++j)
        if (r->inl[j] == x) fresh = false;
      for (uint32_t j = 0; j < 32; ++j) {
        const uint32_t y = __shfl_sync(0xFFFFFFFFu, x, j);
        if (j < lane && y == x) fresh = false;
      }
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, fresh);
      __syncwarp();
      if (fresh) r->inl[d0 + __popc(m & lanemask_lt())] = x;
      if (lane == 0) {
        r->deg = d0 + __popc(m);
        dsum += __popc(m);
      }
    } else {
      hinsert_team(W, r, pool, hkey, hpos, gcols, g0, g1, act[a], new_cls[a], new_run[a], icap, free_run, free_cls, a,
                   dsum, err);
    }
  }
  const Team<true> C{sh};
  const uint32_t NH = *nhuge;
  for (uint64_t b = blockIdx.x; b < NH; b += gridDim.x) {  // never an inline action (group > kInline)
    const uint32_t a = huge[b];
    hinsert_team(C, vtx + aff[a], pool, hkey, hpos, gcols, gstart[a], gstart[a + 1], act[a], new_cls[a], new_run[a],
                 icap, free_run, free_cls, a, dsum, err);
    __syncthreads();  // the record is written before the CTA moves on
  }
  block_add_delta(dsum, delta);
}

// Deletes: small groups a thread each, mid-sized ones a warp each, the
// largest a CTA each.
__global__ void hdelete_kernel(DynVertex* vtx, uint32_t* pool, uint32_t* hkey, uint32_t* hpos,
                               const uint32_t* __restrict__ aff, const uint64_t* __restrict__ gstart,
                               const uint32_t* __restrict__ gcols, uint64_t A, const uint32_t* __restrict__ mid,
                               const uint32_t* __restrict__ nmid, const uint32_t* __restrict__ huge,
                               const uint32_t* __restrict__ nhuge, uint32_t icap, uint32_t* s1, uint32_t* s2,
                               uint32_t* s3, uint64_t* free_run, uint32_t* free_cls, long long* delta, uint32_t* err) {
  __shared__ uint32_t sh[32];
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  long long dsum = 0;
  for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < A; a += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t g0 = gstart[a], g1 = gstart[a + 1];
    if (g1 - g0 <= kSmallGroup)
      hdelete_thread(vtx + aff[a], pool, hkey, hpos, gcols, g0, g1, icap, free_run, free_cls, a, dsum, err);
  }
  const Team<false> W{nullptr};
  const uint32_t NM = *nmid;
  for (uint64_t b = w0; b < NM; b += nw) {
    const uint32_t a = mid[b];
    hdelete_team(W, vtx + aff[a], pool, hkey, hpos, gcols, gstart[a], gstart[a + 1], icap, s1, s2, s3, free_run,
                 free_cls, a, dsum, err);
  }
  const Team<true> C{sh};
  const uint32_t NH = *nhuge;
  for (uint64_t b = blockIdx.x; b < NH; b += gridDim.x) {
    const uint32_t a = huge[b];
    hdelete_team(C, vtx + aff[a], pool, hkey, hpos, gcols, gstart[a], gstart[a + 1], icap, s1, s2, s3, free_run,
                 free_cls, a, dsum, err);
    __syncthreads();
  }
  block_add_delta(dsum, delta);
}

// Enter every run list of a freshly loaded container into its index.
byo_status build_hash_index(byo_graph* g, DynStore* d, uint64_t used_blocks, cudaStream_t s) {
  const uint32_t n = g->n;
  uint32_t *nfill = nullptr, *item = nullptr, *err = nullptr;
  uint64_t* tstart = nullptr;
  uint64_t NT = 0;
  byo_status st = dev_alloc_t(&d->hkey, d->pool_blocks * kHashSlots, "hash index keys");
  if (st == BYO_OK) st = dev_alloc_t(&d->hpos, d->pool_blocks * kHashSlots, "hash index positions");
  if (st == BYO_OK) st = dev_alloc_t(&d->vcnt, n + 1ull, "semisort counters");
  if (st == BYO_OK) st = dev_alloc_t(&d->vslot, n + 1ull, "semisort slots");
  if (st == BYO_OK) st = tmp_alloc_t(&nfill, n + 1ull, s, "index fill tasks");
  if (st == BYO_OK) st = tmp_alloc_t(&tstart, n + 1ull, s, "index fill starts");
  if (st == BYO_OK) st = tmp_alloc_t(&err, 1, s, "index error");
  if (st == BYO_OK) {
    cudaMemsetAsync(d->vcnt, 0, sizeof(uint32_t) * (n + 1ull), s);
    cudaMemsetAsync(d->hkey, 0xFF, sizeof(uint32_t) * used_blocks * kHashSlots, s);
    cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
    htask_count_kernel<<<grid_for(n, 256), 256, 0, s>>>(d->vtx, nullptr, nullptr, nullptr, n, nullptr, nfill);
    note_launch();
    st = scan_u32_to_u64(nfill, tstart, n + 1ull, &NT, s);
  }
  if (st == BYO_OK) st = tmp_alloc_t(&item, NT + 1, s, "index fill items");
  if (st == BYO_OK && NT) {
    chunk_expand_kernel<<<grid_for(n, 256), 256, 0, s>>>(tstart, n, item);
    hfill_kernel<<<grid_for(NT * 32, 256), 256, 0, s>>>(d->vtx, d->pool, d->hkey, d->hpos, nullptr, nullptr, nullptr,
                                                         item, tstart, NT, err);
    note_launch(2);
  }
  if (st == BYO_OK) {
    uint32_t herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "hash index build");
    else if (herr) {
      set_error("hash index build: an index ran out of slots");
      st = BYO_ERR_CUDA;
    }
  }
  tmp_free(nfill, s);
  tmp_free(tstart, s);
  tmp_free(item, s);
  tmp_free(err, s);
  return st;
}

// A batch on the hash-indexed variant: symmetrise, semisort by source, then
// the insert or delete passes above.
byo_status apply_batch_hashed(byo_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t k, bool insert,
                              cudaStream_t s) {
  DynStore* d = g->dyn;
  const uint32_t n = g->n;
  const uint64_t B = 2 * k;
  const uint64_t Amax = B < n ? B : n;
  uint32_t *rows = nullptr, *cols = nullptr, *flag = nullptr, *aff = nullptr, *gcnt = nullptr, *gcols = nullptr;
  uint32_t *act = nullptr, *new_cls = nullptr, *free_cls = nullptr, *nclear = nullptr, *nfill = nullptr;
  uint32_t *item_c = nullptr, *item_f = nullptr, *s1 = nullptr, *s2 = nullptr, *s3 = nullptr;
  uint64_t *gstart = nullptr, *new_run = nullptr, *free_run = nullptr, *cstart = nullptr, *fstart = nullptr;
  unsigned long long *nA = nullptr, *need = nullptr;
  long long* delta = nullptr;
  uint32_t** d_stacks = nullptr;
  uint64_t* d_cap = nullptr;
  uint32_t *mid = nullptr, *huge = nullptr, *nsplit = nullptr;  // nsplit: [mid count, huge count]
  uint64_t A = 0, NTC = 0, NTF = 0;
  uint32_t hflag[2] = {0, 0};  // [0]: an id >= n in the batch, [1]: an index inconsistency
  std::unique_ptr<ProfScope> phase(new ProfScope("dyn_semisort", s));
  byo_status st = tmp_alloc_t(&rows, B, s, "batch rows");
  if (st == BYO_OK) st = tmp_alloc_t(&cols, B, s, "batch cols");
  if (st == BYO_OK) st = tmp_alloc_t(&flag, 2, s, "batch flags");
  if (st == BYO_OK) st = tmp_alloc_t(&nA, 1, s, "group count");
  if (st == BYO_OK) st = tmp_alloc_t(&aff, Amax + 1, s, "group vertices");
  if (st == BYO_OK) st = tmp_alloc_t(&delta, 1, s, "edge delta");
  if (st == BYO_OK) {
    cudaMemsetAsync(flag, 0, 2 * sizeof(uint32_t), s);
    cudaMemsetAsync(nA, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(delta, 0, sizeof(long long), s);
    // semisort: count per source (rows of invalid pairs are skipped), group
    // starts, scatter into groups
    hsym_kernel<<<grid_for(k, 256), 256, 0, s>>>(src, dst, k, n, rows, cols, flag);
    hhist_kernel<<<grid_for(B, 256), 256, 0, s>>>(rows, B, d->vcnt, d->vslot, aff, nA);
    note_launch(2);
    unsigned long long hA = 0;
    cudaError_t e = cudaMemcpyAsync(&hA, nA, sizeof(hA), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflag, flag, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = cuda_status(e, "batch semisort");
    } else if (hflag[0]) {  // nothing applied; the counters must be zero between batches
      cudaMemsetAsync(d->vcnt, 0, sizeof(uint32_t) * (n + 1ull), s);
      set_error("batch: vertex id >= n");
      st = BYO_ERR_INVALID_ARG;
    }
    A = hA;
  }
  if (st == BYO_OK && A > 0) {
    st = tmp_alloc_t(&gcnt, A + 1, s, "group sizes");
    if (st == BYO_OK) st = tmp_alloc_t(&gstart, A + 1, s, "group starts");
    if (st == BYO_OK) st = tmp_alloc_t(&gcols, B + 1, s, "grouped batch");
    if (st == BYO_OK) st = tmp_alloc_t(&mid, A + 1, s, "warp groups");
    if (st == BYO_OK) st = tmp_alloc_t(&huge, A + 1, s, "CTA groups");
    if (st == BYO_OK) st = tmp_alloc_t(&nsplit, 2, s, "group split counts");
    if (st == BYO_OK) {
      hgcount_kernel<<<grid_for(A, 256), 256, 0, s>>>(aff, A, d->vcnt, gcnt);
      note_launch();
      st = scan_u32_to_u64(gcnt, gstart, A + 1, nullptr, s);
    }
    if (st == BYO_OK) {
      cudaMemsetAsync(nsplit, 0, 2 * sizeof(uint32_t), s);
      hsplit_kernel<<<grid_for(A, 256), 256, 0, s>>>(gstart, A, kWarpGroupMax, mid, nsplit, huge, nsplit + 1);
      note_launch();
      hscatter_kernel<<<grid_for(B, 256), 256, 0, s>>>(rows, cols, B, d->vcnt, d->vslot, gstart, gcols);
      note_launch();
    } else {
      cudaMemsetAsync(d->vcnt, 0, sizeof(uint32_t) * (n + 1ull), s);  // the counters must be zero between batches
    }
  }
  if (st == BYO_OK && A > 0) st = tmp_alloc_t(&free_run, A + 1, s, "freed runs");
  if (st == BYO_OK && A > 0) st = tmp_alloc_t(&free_cls, A + 1, s, "freed classes");
  if (st == BYO_OK && A > 0) st = tmp_alloc_t(&d_stacks, kClasses, s, "stack table");
  if (st == BYO_OK && A > 0) st = tmp_alloc_t(&d_cap, kClasses, s, "stack capacities");
  if (st == BYO_OK && A > 0) {
    cudaMemcpyAsync(d_stacks, d->stacks, sizeof(uint32_t*) * kClasses, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_cap, d->stack_cap, sizeof(uint64_t) * kClasses, cudaMemcpyHostToDevice, s);
  }
  phase.reset(new ProfScope("dyn_hash_plan", s));
  if (st == BYO_OK && A > 0 && insert) {
    st = tmp_alloc_t(&act, A + 1, s, "actions");
    if (st == BYO_OK) st = tmp_alloc_t(&new_cls, A + 1, s, "new classes");
    if (st == BYO_OK) st = tmp_alloc_t(&new_run, A + 1, s, "new runs");
    if (st == BYO_OK) st = tmp_alloc_t(&need, 1, s, "need");
    if (st == BYO_OK) {
      cudaMemsetAsync(need, 0, sizeof(unsigned long long), s);
      hplan_kernel<<<grid_for(A, 256), 256, 0, s>>>(d->vtx, aff, gstart, A, n, d->icap, act, new_cls, need);
      note_launch();
      unsigned long long hneed = 0, hbump = 0;
      cudaError_t e = cudaMemcpyAsync(&hneed, need, sizeof(hneed), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&hbump, d->bump, sizeof(hbump), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) st = cuda_status(e, "pool check");
      else if (hbump + hneed > d->pool_blocks) st = grow_pool(d, hbump, (hbump + hneed) * 3 / 2 + 4096, s);
    }
    if (st == BYO_OK) st = tmp_alloc_t(&nclear, A + 1, s, "clear tasks");
    if (st == BYO_OK) st = tmp_alloc_t(&nfill, A + 1, s, "fill tasks");
    if (st == BYO_OK) st = tmp_alloc_t(&cstart, A + 1, s, "clear task starts");
    if (st == BYO_OK) st = tmp_alloc_t(&fstart, A + 1, s, "fill task starts");
    if (st == BYO_OK) {
      halloc_kernel<<<grid_for(A, 256), 256, 0, s>>>(d->vtx, aff, act, new_cls, A, d_stacks, d->tops, d->bump,
                                                      new_run, free_run, free_cls);
      clamp_tops_kernel<<<1, 32, 0, s>>>(d->tops);
      htask_count_kernel<<<grid_for(A, 256), 256, 0, s>>>(d->vtx, aff, act, new_cls, A, nclear, nfill);
      note_launch(3);
      st = scan_u32_to_u64(nclear, cstart, A + 1, &NTC, s);
    }
    if (st == BYO_OK) st = scan_u32_to_u64(nfill, fstart, A + 1, &NTF, s);
    if (st == BYO_OK) st = tmp_alloc_t(&item_c, NTC + 1, s, "clear task items");
    if (st == BYO_OK) st = tmp_alloc_t(&item_f, NTF + 1, s, "fill task items");
    phase.reset(new ProfScope("dyn_hash_index", s));
    if (st == BYO_OK) {
      if (NTC) {
        chunk_expand_kernel<<<grid_for(A, 256), 256, 0, s>>>(cstart, A, item_c);
        hclear_kernel<<<grid_for(NTC * 32, 256), 256, 0, s>>>(item_c, cstart, NTC, new_run, new_cls, d->hkey);
        note_launch(2);
      }
      if (NTF) {
        chunk_expand_kernel<<<grid_for(A, 256), 256, 0, s>>>(fstart, A, item_f);
        hfill_kernel<<<grid_for(NTF * 32, 256), 256, 0, s>>>(d->vtx, d->pool, d->hkey, d->hpos, aff, new_run, new_cls,
                                                              item_f, fstart, NTF, flag + 1);
        note_launch(2);
      }
      phase.reset(new ProfScope("dyn_hash_apply", s));
      hinsert_kernel<<<grid_for(A, 256), 256, 0, s>>>(d->vtx, d->pool, d->hkey, d->hpos, aff, gstart, gcols, act,
                                                       new_run, new_cls, A, mid, nsplit, huge, nsplit + 1, d->icap,
                                                       free_run, free_cls, delta, flag + 1);
      note_launch();
    }
  }
  if (st == BYO_OK && A > 0 && !insert) {
    st = tmp_alloc_t(&s1, B + 1, s, "freed positions");
    if (st == BYO_OK) st = tmp_alloc_t(&s2, B + 1, s, "holes");
    if (st == BYO_OK) st = tmp_alloc_t(&s3, B + 1, s, "survivors");
    phase.reset(new ProfScope("dyn_hash_apply", s));
    if (st == BYO_OK) {
      hdelete_kernel<<<grid_for(A, 256), 256, 0, s>>>(d->vtx, d->pool, d->hkey, d->hpos, aff, gstart, gcols, A, mid,
                                                       nsplit, huge, nsplit + 1, d->icap, s1, s2, s3, free_run,
                                                       free_cls, delta, flag + 1);
      note_launch();
    }
  }
  if (st == BYO_OK && A > 0) {
    free_kernel<<<grid_for(A, 256), 256, 0, s>>>(free_run, free_cls, A, d_stacks, d->tops, d_cap);
    note_launch();
    long long hdelta = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hdelta, delta, sizeof(hdelta), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflag + 1, flag + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = cuda_status(e, "hashed batch apply");
    } else {
      g->m = (uint64_t)((long long)g->m + hdelta);
      if (hflag[1]) {
        set_error("hashed batch apply: a hash index ran out of slots or lost an id");
        st = BYO_ERR_CUDA;
      }
    }
  }
  tmp_free(rows, s);
  tmp_free(cols, s);
  tmp_free(flag, s);
  tmp_free(nA, s);
  tmp_free(aff, s);
  tmp_free(delta, s);
  tmp_free(gcnt, s);
  tmp_free(gstart, s);
  tmp_free(gcols, s);
  tmp_free(act, s);
  tmp_free(new_cls, s);
  tmp_free(new_run, s);
  tmp_free(need, s);
  tmp_free(free_run, s);
  tmp_free(free_cls, s);
  tmp_free(d_stacks, s);
  tmp_free(d_cap, s);
  tmp_free(nclear, s);
  tmp_free(nfill, s);
  tmp_free(cstart, s);
  tmp_free(fstart, s);
  tmp_free(item_c, s);
  tmp_free(item_f, s);
  tmp_free(s1, s);
  tmp_free(s2, s);
  tmp_free(s3, s);
  tmp_free(mid, s);
  tmp_free(huge, s);
  tmp_free(nsplit, s);
  phase.reset();
  if (A > 0 && st == BYO_OK) {
    ProfScope ps("dyn_buckets", s);
    g->buckets_stale = true;
    st = rebuild_buckets(g, s);
    if (st == BYO_OK) g->buckets_stale = false;
  }
  return st;
}

byo_status apply_batch(byo_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t k, bool insert,
                       cudaStream_t s) {
  DynStore* d = g->dyn;
  if (d->hashed) return apply_batch_hashed(g, src, dst, k, insert, s);
  uint32_t *rows = nullptr, *cols = nullptr;
  uint64_t B = 0;
  {
    ProfScope ps("dyn_sort", s);
    BYO_RETURN_IF(sort_unique_pairs(g->n, src, dst, k, true, s, &rows, &cols, &B));
  }
  if (B == 0) {
    tmp_free(rows, s);
    tmp_free(cols, s);
    return BYO_OK;
  }
  const DynView view = dyn_view(g);
  uint32_t *flags = nullptr, *seg_v = nullptr, *mark = nullptr, *newdeg = nullptr, *buf = nullptr;
  uint32_t *new_cls = nullptr, *free_cls = nullptr;
  uint32_t *cm = nullptr, *cc = nullptr, *item_m = nullptr, *item_c = nullptr;
  uint64_t *mstart = nullptr, *cstart = nullptr;
  uint64_t NM = 0, NCC = 0;
  uint64_t *idx = nullptr, *seg_start = nullptr, *mrank = nullptr, *toff = nullptr;
  uint64_t *new_run = nullptr, *free_run = nullptr;
  long long* delta = nullptr;
  unsigned long long* need = nullptr;
  uint32_t** d_stacks = nullptr;
  uint64_t* d_cap = nullptr;
  uint64_t A = 0, T = 0;
  byo_status st = tmp_alloc_t(&flags, B + 1, s, "segment flags");
  if (st == BYO_OK) st = tmp_alloc_t(&idx, B + 1, s, "segment index");
  if (st == BYO_OK) {
    seg_flags_kernel<<<grid_for(B, 256), 256, 0, s>>>(rows, B, flags);
    note_launch();
    st = scan_u32_to_u64(flags, idx, B, &A, s);
  }
  if (st == BYO_OK) st = tmp_alloc_t(&seg_start, A + 1, s, "segment starts");
  if (st == BYO_OK) st = tmp_alloc_t(&seg_v, A + 1, s, "segment vertices");
  if (st == BYO_OK) {
    seg_fill_kernel<<<grid_for(B, 256), 256, 0, s>>>(rows, flags, idx, B, A, seg_start, seg_v);
    note_launch();
    st = tmp_alloc_t(&mark, B + 1, s, "marks");
  }
  if (st == BYO_OK) st = tmp_alloc_t(&mrank, B + 1, s, "mark ranks");
  if (st == BYO_OK) {
    mark_kernel<<<grid_for(B, 256), 256, 0, s>>>(view, rows, cols, B, insert, mark);
    note_launch();
    cudaMemsetAsync(mark + B, 0, sizeof(uint32_t), s);
    st = scan_u32_to_u64(mark, mrank, B + 1, nullptr, s);  // mrank[B] = total marks
  }
  if (st == BYO_OK) st = tmp_alloc_t(&newdeg, A + 1, s, "new degrees");
  if (st == BYO_OK) st = tmp_alloc_t(&toff, A + 1, s, "merge offsets");
  if (st == BYO_OK) st = tmp_alloc_t(&delta, 1, s, "edge delta");
  if (st == BYO_OK) {
    cudaMemsetAsync(delta, 0, sizeof(long long), s);
    newdeg_kernel<<<grid_for(A, 256), 256, 0, s>>>(view, seg_start, seg_v, mrank, A, insert, newdeg, delta);
    note_launch();
    st = scan_u32_to_u64(newdeg, toff, A, &T, s);
  }
  if (st == BYO_OK) st = tmp_alloc_t(&buf, T + 1, s, "merge buffer");
  // chunk tasks of the merge (old lists) and of the copy-back (new lists)
  if (st == BYO_OK) st = tmp_alloc_t(&cm, A + 1, s, "merge chunk counts");
  if (st == BYO_OK) st = tmp_alloc_t(&cc, A + 1, s, "copy chunk counts");
  if (st == BYO_OK) st = tmp_alloc_t(&mstart, A + 1, s, "merge chunk starts");
  if (st == BYO_OK) st = tmp_alloc_t(&cstart, A + 1, s, "copy chunk starts");
  if (st == BYO_OK) {
    chunk_count_kernel<<<grid_for(A, 256), 256, 0, s>>>(view, seg_v, newdeg, A, cm, cc);
    note_launch();
    cudaMemsetAsync(cm + A, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(cc + A, 0, sizeof(uint32_t), s);
    st = scan_u32_to_u64(cm, mstart, A + 1, &NM, s);  // mstart[A] = all merge tasks
  }
  if (st == BYO_OK) st = scan_u32_to_u64(cc, cstart, A + 1, &NCC, s);
  if (st == BYO_OK) st = tmp_alloc_t(&item_m, NM + 1, s, "merge chunk tasks");
  if (st == BYO_OK) st = tmp_alloc_t(&item_c, NCC + 1, s, "copy chunk tasks");
  if (st == BYO_OK) {
    chunk_expand_kernel<<<grid_for(A, 256), 256, 0, s>>>(mstart, A, item_m);
    chunk_expand_kernel<<<grid_for(A, 256), 256, 0, s>>>(cstart, A, item_c);
    note_launch(2);
    merge_kernel<<<grid_for(NM * 32, 256), 256, 0, s>>>(view, cols, seg_start, seg_v, mark, mrank, toff, item_m,
                                                         mstart, NM, insert, buf);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_status(e, "merge_kernel");
  }
  // make sure the pool can take the worst case of this batch before allocating
  if (st == BYO_OK) st = tmp_alloc_t(&need, 1, s, "need");
  if (st == BYO_OK) {
    cudaMemsetAsync(need, 0, sizeof(unsigned long long), s);
    need_kernel<<<grid_for(A, 256), 256, 0, s>>>(newdeg, A, d->icap, need);
    note_launch();
    unsigned long long hneed = 0, hbump = 0;
    cudaError_t e = cudaMemcpyAsync(&hneed, need, sizeof(hneed), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbump, d->bump, sizeof(hbump), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "pool check");
    else if (hbump + hneed > d->pool_blocks) st = grow_pool(d, hbump, (hbump + hneed) * 3 / 2 + 4096, s);
  }
  if (st == BYO_OK) st = tmp_alloc_t(&new_run, A + 1, s, "new runs");
  if (st == BYO_OK) st = tmp_alloc_t(&free_run, A + 1, s, "freed runs");
  if (st == BYO_OK) st = tmp_alloc_t(&new_cls, A + 1, s, "new classes");
  if (st == BYO_OK) st = tmp_alloc_t(&free_cls, A + 1, s, "freed classes");
  if (st == BYO_OK) st = tmp_alloc_t(&d_stacks, kClasses, s, "stack table");
  if (st == BYO_OK) st = tmp_alloc_t(&d_cap, kClasses, s, "stack capacities");
  if (st == BYO_OK) {
    cudaMemcpyAsync(d_stacks, d->stacks, sizeof(uint32_t*) * kClasses, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_cap, d->stack_cap, sizeof(uint64_t) * kClasses, cudaMemcpyHostToDevice, s);
    alloc_kernel<<<grid_for(A, 256), 256, 0, s>>>(d->vtx, seg_v, newdeg, A, d->icap, d_stacks, d->tops, d->bump,
                                                   new_run, new_cls, free_run, free_cls);
    clamp_tops_kernel<<<1, 32, 0, s>>>(d->tops);
    copyback_kernel<<<grid_for(NCC * 32, 256), 256, 0, s>>>(d->vtx, d->pool, seg_v, newdeg, new_run, new_cls, toff,
                                                             buf, item_c, cstart, NCC, d->icap);
    free_kernel<<<grid_for(A, 256), 256, 0, s>>>(free_run, free_cls, A, d_stacks, d->tops, d_cap);
    note_launch(4);
    long long hdelta = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hdelta, delta, sizeof(hdelta), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "batch apply");
    else g->m = (uint64_t)((long long)g->m + hdelta);
  }
  tmp_free(rows, s);
  tmp_free(cols, s);
  tmp_free(flags, s);
  tmp_free(idx, s);
  tmp_free(seg_start, s);
  tmp_free(seg_v, s);
  tmp_free(mark, s);
  tmp_free(mrank, s);
  tmp_free(newdeg, s);
  tmp_free(toff, s);
  tmp_free(buf, s);
  tmp_free(delta, s);
  tmp_free(need, s);
  tmp_free(new_run, s);
  tmp_free(free_run, s);
  tmp_free(new_cls, s);
  tmp_free(free_cls, s);
  tmp_free(d_stacks, s);
  tmp_free(d_cap, s);
  tmp_free(cm, s);
  tmp_free(cc, s);
  tmp_free(mstart, s);
  tmp_free(cstart, s);
  tmp_free(item_m, s);
  tmp_free(item_c, s);
  // the batch is applied; if the buckets cannot be re-derived now (no memory
  // for the sort), the next call that reads them does it
  if (st == BYO_OK) {
    ProfScope ps("dyn_buckets", s);
    g->buckets_stale = true;
    st = rebuild_buckets(g, s);
    if (st == BYO_OK) g->buckets_stale = false;
  }
  return st;
}

}  // namespace

__global__ void dyn_space_kernel(const DynVertex* __restrict__ vtx, uint32_t n, unsigned long long* blocks) {
  unsigned long long b = 0;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = vtx[v].cls;
    if (c != kNoRun) b += 1ull << c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xFFFFFFFFu, b, o);
  if (lane_id() == 0 && b) atomicAdd(blocks, b);
}

byo_status dyn_space(const byo_graph* g, uint64_t* host_bytes, cudaStream_t s) {
  unsigned long long* blocks = nullptr;
  BYO_RETURN_IF(tmp_alloc_t(&blocks, 1, s, "space counter"));
  unsigned long long hb = 0;
  cudaMemsetAsync(blocks, 0, sizeof(unsigned long long), s);
  dyn_space_kernel<<<grid_for(g->n, 256), 256, 0, s>>>(g->dyn->vtx, g->n, blocks);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, blocks, sizeof(hb), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  tmp_free(blocks, s);
  if (e != cudaSuccess) return cuda_status(e, "byo_space");
  // a block holds 32 ids; the hash-indexed variant adds its 64 index slots (key and position)
  const uint64_t per_block = kBlockIds * sizeof(uint32_t) + (g->dyn->hashed ? kHashSlots * 2 * sizeof(uint32_t) : 0);
  *host_bytes = sizeof(DynVertex) * ((uint64_t)g->n + 1) + (uint64_t)hb * per_block;
  return BYO_OK;
}

__global__ void dyn_sort_keys_kernel(const uint64_t* __restrict__ off, const uint32_t* __restrict__ col, uint32_t n,
                                     uint64_t* keys) {
  const uint32_t lane = lane_id();
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = w0; v < n; v += nw)
    for (uint64_t i = off[v] + lane; i < off[v + 1]; i += 32) keys[i] = (v << 32) | col[i];
}

__global__ void dyn_sort_cols_kernel(const uint64_t* __restrict__ keys, uint64_t m, uint32_t* col) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    col[i] = (uint32_t)keys[i];
}

byo_status dyn_sort_lists(const byo_graph* g, const uint64_t* off, uint32_t* col, cudaStream_t s) {
  const uint64_t m = g->m;
  if (m == 0) return BYO_OK;
  uint64_t *keys = nullptr, *tmp = nullptr, *sorted = nullptr;
  byo_status st = tmp_alloc_t(&keys, m, s, "export sort keys");
  if (st == BYO_OK) st = tmp_alloc_t(&tmp, m, s, "export sort scratch");
  if (st == BYO_OK) {
    dyn_sort_keys_kernel<<<grid_for((uint64_t)g->n * 32, 256), 256, 0, s>>>(off, col, g->n, keys);
    note_launch();
    const int idb = g->n > 1 ? 32 - __builtin_clz(g->n - 1) : 1;
    st = radix_sort_u64(keys, tmp, m, 32 + idb, &sorted, s);
  }
  if (st == BYO_OK) {
    dyn_sort_cols_kernel<<<grid_for(m, 256), 256, 0, s>>>(sorted, m, col);
    note_launch();
  }
  tmp_free(keys, s);
  tmp_free(tmp, s);
  return st;
}

byo_status dyn_from_csr(byo_graph* g, cudaStream_t s) {
  if (g->n > (1u << 31)) {  // a list of up to n - 1 ids must fit a run of at most 2^26 blocks
    set_error("dynamic containers hold at most 2^31 vertices");
    return BYO_ERR_UNSUPPORTED;
  }
  DynStore* d = new (std::nothrow) DynStore();
  if (!d) {
    set_error("host allocation failed");
    return BYO_ERR_OUT_OF_MEMORY;
  }
  d->icap = (g->flags & BYO_DYN_NO_INLINE) ? 0u : kInline;
  d->hashed = (g->flags & BYO_DYN_HASH) != 0;
  byo_status st = dev_alloc_t(&d->vtx, g->n + 1ull, "vertex records");
  if (st == BYO_OK) st = dev_alloc_t(&d->bump, 1, "pool cursor");
  if (st == BYO_OK) st = dev_alloc_t(&d->tops, kClasses, "stack tops");
  if (st == BYO_OK) st = g->off64 ? load_from_csr<uint64_t>(g, d, s) : load_from_csr<uint32_t>(g, d, s);
  if (st == BYO_OK && d->hashed) st = build_hash_index(g, d, d->pool_blocks, s);
  if (st != BYO_OK) {
    dyn_free(d);
    return st;
  }
  g->dyn = d;
  dev_free(g->off);
  dev_free(g->col);
  g->off = nullptr;
  g->col = nullptr;
  return rebuild_buckets(g, s);
}

}  // namespace byo

using namespace byo;

static byo_status batch_entry(byo_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t k, void* stream,
                              bool insert) {
  clear_error();
  BYO_RETURN_IF(check_graph(g));
  if (!g->dyn) {
    set_error("batch updates need a BYO_DYNAMIC container");
    return BYO_ERR_UNSUPPORTED;
  }
  if (k == 0) return BYO_OK;
  if (!src || !dst) {
    set_error("NULL batch arrays");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ProfScope ps(insert ? "dyn_insert" : "dyn_delete", s);
  return apply_batch(g, src, dst, k, insert, s);
}

extern "C" byo_status byo_insert_batch(byo_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t k,
                                       void* stream) {
  return batch_entry(g, src, dst, k, stream, true);
}

extern "C" byo_status byo_delete_batch(byo_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t k,
                                       void* stream) {
  return batch_entry(g, src, dst, k, stream, false);
}
