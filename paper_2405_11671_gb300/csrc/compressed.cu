// compressed.cu -- the compressed static container (the paper's compressed
// graphs, Section 2 and Section 6.5: each sorted neighbour list difference-
// encoded and the differences written as byte codes), and BFS over it.
//
// Format (the one of the oracle's byte codes): for vertex v with neighbours
// u_0 < u_1 < ..., the first value is 2|u_0 - v| + (u_0 < v), the later ones
// the gaps u_i - u_(i-1) >= 1; each value in 7-bit groups, least significant
// first, the 0x80 bit set on every byte but a value's last.  The CSR offsets
// stay (degrees), beside byte offsets boff[n+1] into the code bytes.
//
// A list cannot be read at an arbitrary position, only decoded in order, so
// the kernels here walk lists in two ways:
//   - a lane decodes its own list value by value (short lists, pull scans);
//   - a warp decodes a list 32 bytes at a time: a ballot over the stop bits
//     (bytes below 0x80 end a value) finds the values that end in the window,
//     each lane shifts its byte into place and a 4-step segmented sum over the
//     shuffles assembles the values, a warp scan of the gaps gives the ids;
//     the next window starts after the window's last complete value.
// BFS over the container is its own persistent cooperative kernel (the
// uncompressed one reads lists at arbitrary positions): push levels give each
// frontier vertex a warp; pull levels give each unvisited vertex a lane that
// decodes until the first frontier neighbour, and hand lists without one in
// their first 16 values to the whole warp; the direction follows the Beamer
// rule of the schedule.
#include "byo_internal.cuh"
#include "container.cuh"
#include "prof.cuh"
#include "sched.cuh"

namespace byo {

// A list is decoded from its start; so that several warps can share a long
// list, every kCkptValues-th value of it has a checkpoint: where its code
// starts and the id before it.
constexpr uint32_t kCkptValues = 4096;
struct Ckpt {
  uint64_t byte;  // absolute offset of the value's first code byte
  uint32_t prev;  // the id before it
  uint32_t pad;
};

struct CompStore {
  uint64_t* boff = nullptr;   // n+1 byte offsets
  uint8_t* bytes = nullptr;   // boff[n] bytes + 48 of padding
  uint64_t nbytes = 0;
  // vertices with checkpoints ((degree-1)/kCkptValues of them), ascending,
  // and the index of each one's first checkpoint in ck
  uint32_t* ckv = nullptr;
  uint64_t* ckfirst = nullptr;
  uint64_t nckv = 0;
  Ckpt* ck = nullptr;
  uint64_t nck = 0;
  // BFS scratch (first use)
  uint32_t* vis = nullptr;    // visited bits
  uint32_t* fb = nullptr;     // two frontier bit arrays
  uint32_t* queue = nullptr;  // two queues of n
  uint2* spill = nullptr;     // push chunk tasks (nck + 1)
  void* ctl = nullptr;
};

void comp_free(CompStore* c) {
  if (!c) return;
  dev_free(c->boff);
  dev_free(c->bytes);
  dev_free(c->ckv);
  dev_free(c->ckfirst);
  dev_free(c->ck);
  dev_free(c->vis);
  dev_free(c->fb);
  dev_free(c->queue);
  dev_free(c->spill);
  dev_free(c->ctl);
  delete c;
}

namespace {

constexpr int kCompThreads = 256;

__device__ __forceinline__ uint32_t code_len(uint64_t w) {
  uint32_t l = 1;
  while (w >= 128) {
    w >>= 7;
    ++l;
  }
  return l;
}

// value i of v's list (sorted ids p[0..len)): the signed first difference or a gap
__device__ __forceinline__ uint64_t code_value(const uint32_t* p, uint32_t i, uint32_t v) {
  const uint32_t u = __ldg(p + i);
  if (i == 0) return u >= v ? 2ull * (u - v) : 2ull * (v - u) + 1;
  return (uint64_t)u - __ldg(p + i - 1);
}

// bytes of each vertex's codes (a warp per vertex)
template <typename OffT>
__global__ void comp_size_kernel(CsrView<OffT> g, uint32_t* size) {
  const uint32_t lane = lane_id();
  for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n;
       v += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    const Seg s = g.seg((uint32_t)v);
    uint32_t t = 0;
    for (uint32_t i = lane; i < s.len; i += 32) t += code_len(code_value(s.p, i, (uint32_t)v));
    t = __reduce_add_sync(0xFFFFFFFFu, t);
    if (lane == 0) size[v] = t;
  }
}

// the codes of each vertex (a warp per vertex, 32 values per step: a warp
// scan of the code lengths places every lane's bytes)
// checkpoints per vertex (one at each value kCkptValues, 2 kCkptValues, ...
// below the degree) and whether it has any
template <typename OffT>
__global__ void comp_ckcount_kernel(CsrView<OffT> g, uint32_t* cnt, uint32_t* has) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t d = g.degree((uint32_t)v);
    cnt[v] = d ? (d - 1) / kCkptValues : 0u;
    has[v] = cnt[v] ? 1u : 0u;
  }
}

// the list of vertices with checkpoints and their first checkpoint
__global__ void comp_cklist_kernel(uint32_t n, const uint32_t* __restrict__ has, const uint64_t* __restrict__ hpos,
                                   const uint64_t* __restrict__ first, uint32_t* ckv, uint64_t* ckfirst) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    if (has[v]) {
      ckv[hpos[v]] = (uint32_t)v;
      ckfirst[hpos[v]] = first[v];
    }
}

// index in ck of the checkpoint before value c * kCkptValues of u's list (c >= 1)
__device__ __forceinline__ uint64_t ckpt_index(const uint32_t* __restrict__ ckv, const uint64_t* __restrict__ ckfirst,
                                               uint64_t nckv, uint32_t u, uint32_t c) {
  uint64_t lo = 0, hi = nckv;  // first entry >= u
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(ckv + mid) < u) lo = mid + 1;
    else hi = mid;
  }
  return __ldg(ckfirst + lo) + c - 1;
}

template <typename OffT>
__global__ void comp_write_kernel(CsrView<OffT> g, const uint64_t* __restrict__ boff, uint8_t* bytes,
                                  const uint64_t* __restrict__ ckoff, Ckpt* ck) {  // ckoff: per vertex, first checkpoint
  static_assert(kCkptValues % 32 == 0, "checkpoints fall on the 32-value steps");
  const uint32_t lane = lane_id();
  for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n;
       v += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    const Seg s = g.seg((uint32_t)v);
    uint64_t at = boff[v];
    for (uint32_t i0 = 0; i0 < s.len; i0 += 32) {
      if (i0 > 0 && i0 % kCkptValues == 0 && lane == 0)
        ck[ckoff[v] + i0 / kCkptValues - 1] = Ckpt{at, __ldg(s.p + i0 - 1), 0u};
      const uint32_t i = i0 + lane;
      uint64_t w = i < s.len ? code_value(s.p, i, (uint32_t)v) : 0;
      const uint32_t l = i < s.len ? code_len(w) : 0u;
      uint32_t incl = l;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      uint64_t pos = at + incl - l;
      for (uint32_t k = 0; k < l; ++k) {
        uint8_t b = (uint8_t)(w & 127u);
        w >>= 7;
        if (k + 1 < l) b |= 128u;
        bytes[pos + k] = b;
      }
      at += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
  }
}

// One 32-byte window of a list's codes, decoded by the whole warp.  The
// window starts at byte p (a value boundary, value index ci of the list);
// prev is the last id decoded so far (unused for ci = 0).  Returns the mask
// of lanes that end a value inside the window; such a lane gets its id.  *p,
// *ci and *prev move past the window's last complete value.
__device__ __forceinline__ uint32_t warp_decode_window(const uint8_t* __restrict__ bytes, uint64_t* p, uint64_t end,
                                                       uint32_t v, uint64_t* ci, uint32_t* prev, uint32_t* id) {
  const uint32_t lane = lane_id();
  const bool valid = *p + lane < end;
  const uint32_t b = valid ? (uint32_t)__ldg(bytes + *p + lane) : 0x80u;
  const uint32_t T = __ballot_sync(0xFFFFFFFFu, valid && !(b & 0x80u));
  if (T == 0) return 0;
  const uint32_t below = T & lanemask_lt();
  const int prev_t = below ? 31 - __clz(below) : -1;  // the lane before this value's first byte
  const uint32_t pos = (uint32_t)((int)lane - prev_t - 1);
  const uint64_t own = (uint64_t)(b & 127u) << (7 * (pos < 5 ? pos : 0));
  uint64_t w = own;
#pragma unroll
  for (int o = 1; o <= 4; ++o) {
    const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, own, o);
    if ((int)lane - o > prev_t) w += y;
  }
  const bool term = (T >> lane) & 1u;
  const uint64_t c = *ci + __popc(below);  // the value index of a terminating lane
  uint32_t base = *prev;
  if (*ci == 0) {
    const int f = __ffs(T) - 1;  // the list's first value: relative to v, signed
    const uint64_t w0 = __shfl_sync(0xFFFFFFFFu, w, f);
    base = (w0 & 1) ? v - (uint32_t)(w0 >> 1) : v + (uint32_t)(w0 >> 1);
  }
  uint32_t gap = (term && c > 0) ? (uint32_t)w : 0u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, gap, o);
    if ((int)lane >= o) gap += y;
  }
  *id = base + gap;
  const int last = 31 - __clz(T);
  *prev = __shfl_sync(0xFFFFFFFFu, *id, last);
  *p += (uint64_t)last + 1;
  *ci += __popc(T);
  return T;
}

// Up to four values of one list, decoded by one lane from a 32-byte register
// window that starts at the 16-byte boundary below byte *p (two vector loads;
// the code bytes are padded so the window stays inside the allocation).
// Values that end inside the window are taken, at most four and at most the
// d - *ci left; *p, *ci and *prev move past the last one.  Returns how many.
__device__ __forceinline__ uint32_t lane_decode4(const uint8_t* __restrict__ bytes, uint64_t* p, uint32_t v,
                                                 uint64_t* ci, uint64_t d, uint32_t* prev, uint32_t* id0,
                                                 uint32_t* id1, uint32_t* id2, uint32_t* id3) {
  const uint64_t a0 = *p & ~15ull;
  const uint32_t o = (uint32_t)(*p - a0);
  const uint4 q0 = __ldg(reinterpret_cast<const uint4*>(bytes + a0));
  const uint4 q1 = __ldg(reinterpret_cast<const uint4*>(bytes + a0 + 16));
  const uint32_t wd[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
  const uint32_t want = (uint32_t)min((uint64_t)4, d - *ci);
  uint64_t acc = 0;
  uint32_t sh = 0, nv = 0, end = o, cur = *prev;
#pragma unroll
  for (uint32_t j = 0; j < 32; ++j) {
    const uint32_t b = (wd[j >> 2] >> (8 * (j & 3))) & 255u;
    if (j >= o && nv < want) {
      acc |= (uint64_t)(b & 127u) << sh;
      sh += 7;
      if (!(b & 128u)) {
        cur = (*ci + nv == 0) ? ((acc & 1) ? v - (uint32_t)(acc >> 1) : v + (uint32_t)(acc >> 1))
                              : cur + (uint32_t)acc;
        if (nv == 0) *id0 = cur;
        else if (nv == 1) *id1 = cur;
        else if (nv == 2) *id2 = cur;
        else *id3 = cur;
        ++nv;
        acc = 0;
        sh = 0;
        end = j + 1;
      }
    }
  }
  *p = a0 + end;
  *ci += nv;
  *prev = cur;
  return nv;
}

// the decoded lists, laid out by the CSR offsets (export)
template <typename OffT>
__global__ void comp_decode_kernel(const OffT* __restrict__ off, uint32_t n, const uint64_t* __restrict__ boff,
                                   const uint8_t* __restrict__ bytes, const uint64_t* __restrict__ out_off,
                                   uint32_t* __restrict__ col) {
  for (uint64_t v = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n;
       v += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    uint64_t p = boff[v], ci = 0;
    const uint64_t end = boff[v + 1];
    const uint64_t o = out_off[v];
    const uint64_t d = (uint64_t)(off[v + 1] - off[v]);
    uint32_t prev = 0, id = 0;
    while (ci < d) {
      const uint64_t c0 = ci;
      const uint32_t T = warp_decode_window(bytes, &p, end, (uint32_t)v, &ci, &prev, &id);
      if (T == 0) break;  // cannot happen for a well-formed list
      if ((T >> lane_id()) & 1u) col[o + c0 + __popc(T & lanemask_lt())] = id;
    }
  }
}

// ------------------------------------------------------------------ BFS
struct CompCtl {
  GridBar bar;
  uint32_t err;
  uint32_t levels;
  unsigned long long nq[2];    // queue length, by level parity
  unsigned long long mq[2];    // degree sum of the queue
  unsigned long long nspill[2];  // push chunk tasks of long lists, by level parity
};

template <typename OffT>
struct CompBfsArgs {
  const OffT* off;
  const uint64_t* boff;
  const uint8_t* bytes;
  uint32_t n;
  uint64_t m;
  uint32_t src;
  uint32_t* level;
  uint32_t* parent;
  uint32_t* vis;
  uint32_t* fb;
  uint32_t* queue;  // [2][n]
  CompCtl* ctl;
  const uint32_t* ckv;      // checkpointed vertices (ascending), their first checkpoint, the checkpoints
  const uint64_t* ckfirst;
  uint64_t nckv;
  const Ckpt* ck;
  uint2* spill;             // push chunk tasks (vertex, chunk >= 1); room for every checkpoint
  float alpha, beta;
  uint64_t limit_ns;
  uint32_t nw;
};

// Warp-collective: the `cand` lanes claim vertex x (parent u) for level
// next_level; winners get level/parent, go to the next queue and add their
// degree to the next level's edge count (one atomic per warp each).
// Winners of a warp waiting for their queue slots: the queue counter takes
// every warp's reservations, so a warp reserves for at least
// kCompStage - 31 winners at a time.
constexpr uint32_t kCompStage = 128;
struct CompStage {
  uint32_t x[kCompStage];
  uint32_t n;
};

template <typename OffT>
__device__ __noinline__ void comp_stage_flush(const CompBfsArgs<OffT>& a, CompStage& W, int nxt) {
  const uint32_t lane = lane_id();
  const uint32_t ns = W.n;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&a.ctl->nq[nxt], (unsigned long long)ns);
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  for (uint32_t i = lane; i < ns; i += 32) a.queue[(size_t)nxt * a.n + base + i] = W.x[i];
  __syncwarp();
  if (lane == 0) W.n = 0;
  __syncwarp();
}

// Stages the lanes with `won` (vertex x); warp-collective.
template <typename OffT>
__device__ __forceinline__ void comp_stage_add(const CompBfsArgs<OffT>& a, CompStage& W, bool won, uint32_t x,
                                               int nxt) {
  const uint32_t m = __ballot_sync(0xFFFFFFFFu, won);
  if (m == 0) return;
  const uint32_t n0 = W.n;
  if (won) W.x[n0 + __popc(m & lanemask_lt())] = x;
  __syncwarp();
  const uint32_t n1 = n0 + __popc(m);
  if (lane_id() == 0) W.n = n1;
  __syncwarp();
  if (n1 > kCompStage - 32) comp_stage_flush(a, W, nxt);
}

template <typename OffT, bool kParents>
__device__ __forceinline__ void comp_claim(const CompBfsArgs<OffT>& a, CompStage& W, bool cand, uint32_t x,
                                           uint32_t u, uint32_t next_level, int nxt, uint64_t& acc_deg) {
  if (cand) cand = !((ld_cg(a.vis + (x >> 5)) >> (x & 31)) & 1u);
  if (__ballot_sync(0xFFFFFFFFu, cand) == 0) return;
  bool won = false;
  if (cand) won = !(atomicOr(a.vis + (x >> 5), 1u << (x & 31)) & (1u << (x & 31)));
  if (!__any_sync(0xFFFFFFFFu, won)) return;
  if (won) {
    a.level[x] = next_level;
    if (kParents) a.parent[x] = u;
    acc_deg += (uint64_t)(__ldg(a.off + x + 1) - __ldg(a.off + x));
  }
  comp_stage_add(a, W, won, x, nxt);
}

__device__ __forceinline__ bool comp_in_frontier(const uint32_t* fb, uint32_t u) {
  return (ld_cg(fb + (u >> 5)) >> (u & 31)) & 1u;
}

template <typename OffT, bool kParents>
__global__ void __launch_bounds__(kCompThreads, 4) comp_bfs_kernel(CompBfsArgs<OffT> a) {
  __shared__ unsigned long long red;
  __shared__ CompStage stage[kCompThreads / 32];
  const uint32_t tid = threadIdx.x, lane = lane_id();
  CompStage& W = stage[tid >> 5];
  if (lane == 0) W.n = 0;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + tid;
  const uint64_t gthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint32_t gwarp = (uint32_t)(gtid >> 5), nwarps = (uint32_t)(gthreads >> 5);
  CompCtl* ctl = a.ctl;
  for (uint64_t v = gtid; v < a.n; v += gthreads) {
    a.level[v] = kInf;
    if (kParents) a.parent[v] = kInf;
  }
  for (uint64_t w = gtid; w < a.nw; w += gthreads) a.vis[w] = 0;
  if (tid == 0) red = 0;
  if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
  if (gtid == 0) {
    a.level[a.src] = 0;
    if (kParents) a.parent[a.src] = a.src;
    a.vis[a.src >> 5] = ld_cg(a.vis + (a.src >> 5)) | (1u << (a.src & 31));
    a.queue[0] = a.src;
    ctl->nq[0] = 1;
    ctl->mq[0] = (uint64_t)(__ldg(a.off + a.src + 1) - __ldg(a.off + a.src));
    ctl->nq[1] = 0;
    ctl->mq[1] = 0;
    ctl->nspill[0] = 0;
    ctl->nspill[1] = 0;
  }
  if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
  const uint64_t t0 = globaltimer();
  uint64_t mvis = 0;
  int prev_dir = 1;
  bool fb_valid = false;
  for (uint32_t L = 0;; ++L) {
    const int cur = L & 1, nxt = cur ^ 1;
    const uint64_t nf = ld_cg(&ctl->nq[cur]), mf = ld_cg(&ctl->mq[cur]);
    if (nf == 0) {
      if (gtid == 0) ctl->levels = L;
      break;
    }
    if (L > a.n || globaltimer() - t0 > a.limit_ns) {
      if (tid == 0) atomicCAS(&ctl->err, 0u, (uint32_t)BYO_ERR_TIMEOUT);
      return;
    }
    // the Beamer rule (every CTA computes the same decision from the same counts)
    const uint64_t mu = a.m - mvis - mf;
    int dir = prev_dir;
    if (prev_dir == 1 && (double)mf > (double)mu / (double)a.alpha) dir = 0;
    else if (prev_dir == 0 && (double)nf < (double)a.n / (double)a.beta) dir = 1;
    if (gtid == 0) {  // the level after next starts from zero
      ctl->nq[nxt] = 0;
      ctl->mq[nxt] = 0;
      ctl->nspill[nxt] = 0;
    }
    const uint32_t* q = a.queue + (size_t)cur * a.n;
    uint64_t acc = 0;
    // the counters of the next level are zeroed before any appends to them
    if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
    if (dir == 1) {
      // push: a warp per frontier vertex, decoding its list 32 bytes at a
      // time, the first kCkptValues values only; the rest of a longer list
      // becomes chunk tasks (one per checkpoint) that warps take after a grid
      // barrier, each decoding from its checkpoint, so that a hub's list is
      // shared by many warps
      for (uint64_t j = gwarp; j < nf; j += nwarps) {
        const uint32_t u = ld_cg(q + j);
        uint64_t p = __ldg(a.boff + u), ci = 0;
        const uint64_t end = __ldg(a.boff + u + 1);
        const uint64_t d = (uint64_t)(__ldg(a.off + u + 1) - __ldg(a.off + u));
        const uint64_t lim = d < kCkptValues ? d : kCkptValues;
        uint32_t prev = 0, x = 0;
        while (ci < lim) {
          const uint64_t c0 = ci;
          const uint32_t T = warp_decode_window(a.bytes, &p, end, u, &ci, &prev, &x);
          if (T == 0) break;
          const bool in = ((T >> lane) & 1u) && c0 + __popc(T & lanemask_lt()) < lim;
          comp_claim<OffT, kParents>(a, W, in, x, u, L + 1, nxt, acc);
        }
        if (d > kCkptValues && lane == 0) {
          const uint32_t nch = (uint32_t)((d - 1) / kCkptValues);
          const unsigned long long base = atomicAdd(&ctl->nspill[cur], (unsigned long long)nch);
          for (uint32_t ch = 1; ch <= nch; ++ch) a.spill[base + ch - 1] = make_uint2(u, ch);
        }
      }
      if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
      const uint64_t nsp = ld_cg(&ctl->nspill[cur]);
      for (uint64_t t = gwarp; t < nsp; t += nwarps) {
        const uint2 e = __ldcg(a.spill + t);
        const uint32_t u = e.x;
        const Ckpt k = a.ck[ckpt_index(a.ckv, a.ckfirst, a.nckv, u, e.y)];
        uint64_t p = k.byte, ci = (uint64_t)e.y * kCkptValues;
        const uint64_t end = __ldg(a.boff + u + 1);
        const uint64_t d = (uint64_t)(__ldg(a.off + u + 1) - __ldg(a.off + u));
        const uint64_t lim = d < ci + kCkptValues ? d : ci + kCkptValues;
        uint32_t prev = k.prev, x = 0;
        while (ci < lim) {
          const uint64_t c0 = ci;
          const uint32_t T = warp_decode_window(a.bytes, &p, end, u, &ci, &prev, &x);
          if (T == 0) break;
          const bool in = ((T >> lane) & 1u) && c0 + __popc(T & lanemask_lt()) < lim;
          comp_claim<OffT, kParents>(a, W, in, x, u, L + 1, nxt, acc);
        }
      }
      if (W.n) comp_stage_flush(a, W, nxt);
      fb_valid = false;
    } else {
      uint32_t* fbc = a.fb + (size_t)cur * a.nw;
      uint32_t* fbn = a.fb + (size_t)nxt * a.nw;
      if (!fb_valid) {  // the frontier as bits, from the queue
        for (uint64_t w = gtid; w < a.nw; w += gthreads) fbc[w] = 0;
        if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
        for (uint64_t j = gtid; j < nf; j += gthreads) {
          const uint32_t x = ld_cg(q + j);
          atomicOr(fbc + (x >> 5), 1u << (x & 31));
        }
      }
      for (uint64_t w = gtid; w < a.nw; w += gthreads) fbn[w] = 0;
      if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
      // pull: a lane per unvisited vertex, 32 vertices (one word) per warp step;
      // each lane decodes its list value by value, four values per round,
      // until the first frontier neighbour or 16 values; the warp finishes the
      // lists left over, 32 bytes at a time
      for (uint32_t w = gwarp; w < a.nw; w += nwarps) {
        const uint32_t vw = ld_cg(a.vis + w);
        const uint32_t x = w * 32 + lane;
        const bool todo = x < a.n && !((vw >> lane) & 1u);
        uint64_t p = 0, end = 0, d = 0, ci = 0;
        uint32_t prev = 0, par = kInf;
        if (todo) {
          p = __ldg(a.boff + x);
          end = __ldg(a.boff + x + 1);
          d = (uint64_t)(__ldg(a.off + x + 1) - __ldg(a.off + x));
        }
        bool found = false;
        for (int round = 0; round < 4 && __any_sync(0xFFFFFFFFu, todo && !found && ci < d); ++round) {
          uint32_t id0 = 0, id1 = 0, id2 = 0, id3 = 0;
          uint32_t got = 0;
          if (todo && !found && ci < d) got = lane_decode4(a.bytes, &p, x, &ci, d, &prev, &id0, &id1, &id2, &id3);
          const bool h0 = got > 0 && comp_in_frontier(fbc, id0);
          const bool h1 = got > 1 && comp_in_frontier(fbc, id1);
          const bool h2 = got > 2 && comp_in_frontier(fbc, id2);
          const bool h3 = got > 3 && comp_in_frontier(fbc, id3);
          if (h0 | h1 | h2 | h3) {  // the lowest hit is the parent
            found = true;
            par = h0 ? id0 : (h1 ? id1 : (h2 ? id2 : id3));
          }
        }
        // lists still open: the whole warp, one list at a time
        uint32_t open = __ballot_sync(0xFFFFFFFFu, todo && !found && ci < d);
        while (open) {
          const int l = __ffs(open) - 1;
          open &= open - 1;
          uint64_t pl = __shfl_sync(0xFFFFFFFFu, p, l), cl = __shfl_sync(0xFFFFFFFFu, ci, l);
          const uint64_t el = __shfl_sync(0xFFFFFFFFu, end, l), dl = __shfl_sync(0xFFFFFFFFu, d, l);
          uint32_t pv = __shfl_sync(0xFFFFFFFFu, prev, l), xid = 0, got = kInf;
          const uint32_t xl = w * 32 + (uint32_t)l;
          while (cl < dl) {
            const uint32_t T = warp_decode_window(a.bytes, &pl, el, xl, &cl, &pv, &xid);
            if (T == 0) break;
            const uint32_t hm = __ballot_sync(0xFFFFFFFFu, ((T >> lane) & 1u) && comp_in_frontier(fbc, xid));
            if (hm) {
              got = __shfl_sync(0xFFFFFFFFu, xid, __ffs(hm) - 1);
              break;
            }
          }
          if (lane == (uint32_t)l && got != kInf) {
            found = true;
            par = got;
          }
        }
        const uint32_t fm = __ballot_sync(0xFFFFFFFFu, found);
        if (fm == 0) continue;
        if (lane == 0) {
          a.vis[w] = vw | fm;
          fbn[w] = fm;
        }
        if (found) {
          a.level[x] = L + 1;
          if (kParents) a.parent[x] = par;
          acc += d;
        }
        comp_stage_add(a, W, found, x, nxt);
      }
      if (W.n) comp_stage_flush(a, W, nxt);
      fb_valid = true;
    }
    // the next level's edge count: one atomic per CTA
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0 && acc) atomicAdd(&red, acc);
    __syncthreads();
    if (tid == 0 && red) {
      atomicAdd(&ctl->mq[nxt], red);
      red = 0;
    }
    mvis += mf;
    prev_dir = dir;
    if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
  }
}

template <typename OffT>
byo_status comp_encode(byo_graph* g, CompStore* c, cudaStream_t s) {
  const CsrView<OffT> view{g->n, g->m, static_cast<const OffT*>(g->off), g->col};
  uint32_t* size = nullptr;
  BYO_RETURN_IF(dev_alloc_t(&c->boff, g->n + 1ull, "compressed byte offsets"));
  BYO_RETURN_IF(tmp_alloc_t(&size, g->n + 1ull, s, "compressed sizes"));
  comp_size_kernel<OffT><<<grid_for((uint64_t)g->n * 32, kCompThreads), kCompThreads, 0, s>>>(view, size);
  note_launch();
  byo_status st = scan_u32_to_u64(size, c->boff, g->n, &c->nbytes, s);
  tmp_free(size, s);
  BYO_RETURN_IF(st);
  // 32 bytes of padding: a lane's 32-byte window may start 15 bytes below the last code
  BYO_RETURN_IF(dev_alloc_t(&c->bytes, c->nbytes + 48, "compressed bytes"));
  BYO_CUDA(cudaMemcpyAsync(c->boff + g->n, &c->nbytes, sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  BYO_CUDA(cudaMemsetAsync(c->bytes + c->nbytes, 0, 48, s));
  // checkpoints of the long lists
  uint32_t *ckc = nullptr, *ckh = nullptr;
  uint64_t *ckoff = nullptr, *ckpos = nullptr;
  st = tmp_alloc_t(&ckc, g->n + 1ull, s, "compressed checkpoint counts");
  if (st == BYO_OK) st = tmp_alloc_t(&ckh, g->n + 1ull, s, "compressed checkpoint flags");
  if (st == BYO_OK) st = tmp_alloc_t(&ckoff, g->n + 1ull, s, "compressed checkpoint offsets");
  if (st == BYO_OK) st = tmp_alloc_t(&ckpos, g->n + 1ull, s, "compressed checkpoint list positions");
  if (st == BYO_OK) {
    comp_ckcount_kernel<OffT><<<grid_for(g->n, 256), 256, 0, s>>>(view, ckc, ckh);
    note_launch();
    cudaMemsetAsync(ckc + g->n, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(ckh + g->n, 0, sizeof(uint32_t), s);
    st = scan_u32_to_u64(ckc, ckoff, g->n + 1ull, &c->nck, s);
  }
  if (st == BYO_OK) st = scan_u32_to_u64(ckh, ckpos, g->n + 1ull, &c->nckv, s);
  if (st == BYO_OK) st = dev_alloc_t(&c->ck, c->nck + 1, "compressed checkpoints");
  if (st == BYO_OK) st = dev_alloc_t(&c->ckv, c->nckv + 1, "compressed checkpointed vertices");
  if (st == BYO_OK) st = dev_alloc_t(&c->ckfirst, c->nckv + 1, "compressed first checkpoints");
  if (st == BYO_OK) {
    comp_cklist_kernel<<<grid_for(g->n, 256), 256, 0, s>>>(g->n, ckh, ckpos, ckoff, c->ckv, c->ckfirst);
    comp_write_kernel<OffT><<<grid_for((uint64_t)g->n * 32, kCompThreads), kCompThreads, 0, s>>>(view, c->boff,
                                                                                                  c->bytes, ckoff,
                                                                                                  c->ck);
    note_launch(2);
  }
  tmp_free(ckc, s);
  tmp_free(ckh, s);
  tmp_free(ckoff, s);
  tmp_free(ckpos, s);
  BYO_RETURN_IF(st);
  note_launch();
  BYO_CHECK_LAUNCH("comp_write_kernel");
  BYO_CUDA(cudaStreamSynchronize(s));
  return BYO_OK;
}

template <typename OffT, bool kParents>
byo_status comp_bfs_launch(CompBfsArgs<OffT>& args, cudaStream_t s) {
  auto fn = comp_bfs_kernel<OffT, kParents>;
  int per_sm = 0;
  BYO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCompThreads, 0));
  if (per_sm < 1) {
    set_error("comp_bfs_kernel cannot be resident");
    return BYO_ERR_CUDA;
  }
  void* kargs[] = {&args};
  BYO_CUDA(reset_barrier(&args.ctl->bar, s));
  ProfScope ps("comp_bfs", s);
  BYO_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3(per_sm * sm_count()), dim3(kCompThreads), kargs, 0, s));
  note_launch();
  return BYO_OK;
}

}  // namespace

byo_status comp_from_csr(byo_graph* g, cudaStream_t s) {
  CompStore* c = new (std::nothrow) CompStore();
  if (!c) {
    set_error("host allocation failed");
    return BYO_ERR_OUT_OF_MEMORY;
  }
  byo_status st = g->off64 ? comp_encode<uint64_t>(g, c, s) : comp_encode<uint32_t>(g, c, s);
  if (st != BYO_OK) {
    comp_free(c);
    return st;
  }
  g->comp = c;
  dev_free(g->col);  // the lists live in the codes now; the offsets stay for the degrees
  g->col = nullptr;
  return BYO_OK;
}

// code bytes plus the checkpoints (16 bytes each) and their vertex list (12 bytes per vertex)
uint64_t comp_bytes(const byo_graph* g) {
  return g->comp ? g->comp->nbytes + 16 * g->comp->nck + 12 * g->comp->nckv : 0;
}

byo_status comp_export(const byo_graph* g, const uint64_t* offsets, uint32_t* col, cudaStream_t s) {
  const unsigned grid = grid_for((uint64_t)g->n * 32, kCompThreads);
  if (g->off64)
    comp_decode_kernel<uint64_t><<<grid, kCompThreads, 0, s>>>(static_cast<const uint64_t*>(g->off), g->n,
                                                              g->comp->boff, g->comp->bytes, offsets, col);
  else
    comp_decode_kernel<uint32_t><<<grid, kCompThreads, 0, s>>>(static_cast<const uint32_t*>(g->off), g->n,
                                                              g->comp->boff, g->comp->bytes, offsets, col);
  note_launch();
  BYO_CHECK_LAUNCH("comp_decode_kernel");
  return BYO_OK;
}

byo_status comp_bfs(const byo_graph* gc, const uint32_t* sources, uint32_t ns, uint32_t* levels, uint32_t* parents,
                    const SchedParams& sp, cudaStream_t s) {
  byo_graph* g = const_cast<byo_graph*>(gc);
  CompStore* c = g->comp;
  const uint32_t nw = (g->n + 31) / 32;
  if (!c->vis) {
    byo_status st = dev_alloc_t(&c->vis, nw, "compressed BFS visited bits");
    if (st == BYO_OK) st = dev_alloc_t(&c->fb, 2ull * nw, "compressed BFS frontier bits");
    if (st == BYO_OK) st = dev_alloc_t(&c->queue, 2ull * g->n, "compressed BFS queues");
    if (st == BYO_OK) st = dev_alloc_t(&c->spill, c->nck + 1, "compressed BFS chunk tasks");
    if (st == BYO_OK) st = dev_alloc(&c->ctl, sizeof(CompCtl), "compressed BFS control");
    if (st == BYO_OK) {
      cudaError_t e = cudaMemset(c->ctl, 0, sizeof(CompCtl));
      if (e != cudaSuccess) st = cuda_status(e, "cudaMemset");
    }
    if (st != BYO_OK) {
      dev_free(c->vis);
      dev_free(c->fb);
      dev_free(c->queue);
      dev_free(c->spill);
      dev_free(c->ctl);
      c->vis = c->fb = c->queue = nullptr;
      c->spill = nullptr;
      c->ctl = nullptr;
      return st;
    }
  }
  CompCtl* ctl = static_cast<CompCtl*>(c->ctl);
  for (uint32_t i = 0; i < ns; ++i) {
    auto run = [&](auto off_tag) -> byo_status {
      using OffT = decltype(off_tag);
      CompBfsArgs<OffT> a;
      a.off = static_cast<const OffT*>(g->off);
      a.boff = c->boff;
      a.bytes = c->bytes;
      a.n = g->n;
      a.m = g->m;
      a.src = sources[i];
      a.level = levels + (size_t)i * g->n;
      a.parent = parents ? parents + (size_t)i * g->n : nullptr;
      a.vis = c->vis;
      a.fb = c->fb;
      a.queue = c->queue;
      a.ctl = ctl;
      a.ckv = c->ckv;
      a.ckfirst = c->ckfirst;
      a.nckv = c->nckv;
      a.ck = c->ck;
      a.spill = c->spill;
      a.alpha = sp.alpha;
      a.beta = sp.beta;
      a.limit_ns = timeout_ns();
      a.nw = nw;
      return parents ? comp_bfs_launch<OffT, true>(a, s) : comp_bfs_launch<OffT, false>(a, s);
    };
    BYO_RETURN_IF(g->off64 ? run(uint64_t{}) : run(uint32_t{}));
  }
  uint32_t err = 0;
  BYO_CUDA(cudaMemcpyAsync(&err, &ctl->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  BYO_CUDA(cudaStreamSynchronize(s));
  if (err) {
    cudaMemsetAsync(ctl, 0, sizeof(CompCtl), s);
    cudaStreamSynchronize(s);
    set_error("byo_bfs (compressed): a device-side wait exceeded BYO_TIMEOUT_MS");
    return BYO_ERR_TIMEOUT;
  }
  return BYO_OK;
}

}  // namespace byo

using namespace byo;

extern "C" byo_status byo_export_codes(const byo_graph* g, uint64_t* boff, uint8_t* bytes, uint64_t* host_nbytes,
                                       void* stream) {
  clear_error();
  BYO_RETURN_IF(check_graph(g));
  if (!g->comp) {
    set_error("byo_export_codes: not a compressed container");
    return BYO_ERR_UNSUPPORTED;
  }
  if (!boff || !host_nbytes) {
    set_error("byo_export_codes: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BYO_CUDA(cudaMemcpyAsync(boff, g->comp->boff, sizeof(uint64_t) * (g->n + 1ull), cudaMemcpyDeviceToDevice, s));
  if (bytes && g->comp->nbytes)
    BYO_CUDA(cudaMemcpyAsync(bytes, g->comp->bytes, g->comp->nbytes, cudaMemcpyDeviceToDevice, s));
  BYO_CUDA(cudaStreamSynchronize(s));
  *host_nbytes = g->comp->nbytes;
  return BYO_OK;
}
