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
                                uint32_t icap, const uint64_t* __restrict__ first_block, DynVertex* vtx,
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
      if (lane < kInline) r->inl[lane] = kInf;
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
  if (used) BYO_CUDA(cudaMemcpyAsync(np, d->pool, used * kBlockIds * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  BYO_CUDA(cudaStreamSynchronize(s));
  dev_free(d->pool);
  d->pool = np;
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
    dyn_load_kernel<OffT><<<grid_for((uint64_t)g->n * 32, 256), 256, 0, s>>>(off, g->col, g->n, d->icap, first,
                                                                               d->vtx, d->pool);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "dynamic load");
  }
  tmp_free(blocks, s);
  tmp_free(first, s);
  return st;
}

byo_status apply_batch(byo_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t k, bool insert,
                       cudaStream_t s) {
  DynStore* d = g->dyn;
  uint32_t *rows = nullptr, *cols = nullptr;
  uint64_t B = 0;
  BYO_RETURN_IF(sort_unique_pairs(g->n, src, dst, k, true, s, &rows, &cols, &B));
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
  *host_bytes = sizeof(DynVertex) * ((uint64_t)g->n + 1) + (uint64_t)hb * kBlockIds * sizeof(uint32_t);
  return BYO_OK;
}

byo_status dyn_from_csr(byo_graph* g, cudaStream_t s) {
  DynStore* d = new (std::nothrow) DynStore();
  if (!d) {
    set_error("host allocation failed");
    return BYO_ERR_OUT_OF_MEMORY;
  }
  d->icap = (g->flags & BYO_DYN_NO_INLINE) ? 0u : kInline;
  byo_status st = dev_alloc_t(&d->vtx, g->n + 1ull, "vertex records");
  if (st == BYO_OK) st = dev_alloc_t(&d->bump, 1, "pool cursor");
  if (st == BYO_OK) st = dev_alloc_t(&d->tops, kClasses, "stack tops");
  if (st == BYO_OK) st = g->off64 ? load_from_csr<uint64_t>(g, d, s) : load_from_csr<uint32_t>(g, d, s);
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
