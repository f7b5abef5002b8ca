// bfs.cu -- breadth-first search by edgeMap over a vertexSubset (Section 3.2),
// direction-optimising between the sparse (push) and dense (pull) forms with a
// cutoff that uses degree and num_edges (Section 6.3), in ONE persistent
// cooperative launch per source.
//
// Frontier representations (the vertexSubset of Section 3.2):
//   sparse: the queue.  One array of n ids split into per-degree-bucket
//           regions (bucket b >= 1 = degrees [2^(b-1), 2^b)); every vertex
//           enters the frontier at most once, so each region is append-only
//           across levels and level l's entries of bucket b are a contiguous
//           run.  Binning by degree is therefore free, and a push iteration
//           can pick its thread/warp/CTA split per iteration.
//   dense:  a bit-vector (1 bit per vertex; Section 4.4 reports the bit array
//           beating a bool array), double-buffered by level parity.
// Push (sparse edgeMap): degree-binned.  Small-degree vertices: a warp takes
//   32 of them and walks their concatenated edges 32 at a time (edge-balanced
//   inside the warp); mid-degree: one warp per vertex; high degree: CTA-wide
//   chunks of at most kChunk edges.  On small levels a warp takes fewer of the
//   small-degree vertices, so that every warp has about one round of 32 edges.
//   A neighbour is claimed in the visited bit array with one atomicOr per
//   candidate (on large levels after a plain read of its bit).
// Pull (dense edgeMap): a warp owns a contiguous range of words of the visited
//   bit array; its lanes take the unvisited vertices one each and scan their
//   sorted neighbour lists until the first neighbour in the frontier
//   bit-vector (map_neighbors_early_exit, Section 4.2); lists with no hit in
//   their first ids are finished by the whole warp, 128 ids per step.  The
//   warp sets its own visited and next-frontier bits, and appends the
//   discovered vertices to the queue, so both representations of the next
//   frontier exist after a pull.
#include <math.h>

#include <mutex>

#include "byo_internal.cuh"
#include "container.cuh"
#include "prof.cuh"
#include "sched.cuh"

namespace byo {

constexpr int kBfsThreads = 256;
constexpr int kPullThreadMax = 32;  // pull: each lane scans this many ids of its own vertex; the rest, by the warp
constexpr uint32_t kChunk = 2048;   // push: edges per CTA work item in the CTA bin
static_assert(kChunk == 1u << 11, "bucket b >= 12 splits into 2^(b - 11) CTA work items");
constexpr uint32_t kTraceCap = 1u << 16;
constexpr int kPushK = 4;  // push: candidates per lane in flight at once
constexpr uint64_t kPrecheckMinEdges = 1u << 15;  // push levels with fewer frontier edges claim directly

// A counter alone in its 128-byte line: the queue counters take one atomic
// per warp and bucket from every CTA, and counters that share lines (and so
// L2 slices) serialise each other.
struct LineCounter {
  unsigned long long v;
  unsigned long long pad[15];
};

struct BfsCtl {
  GridBar bar;
  uint32_t err;
  uint32_t levels;
  LineCounter cnt[3][kBuckets];  // appends per bucket, by level mod 3
  LineCounter pull_next[3];      // pull: next batch of 32 words to hand out, by level mod 3
  unsigned long long sdeg[3];           // sum of degrees of the frontier being built
  unsigned long long scanned[3];        // neighbour ids read while building it
  // hand-over from a solo run of block 0 to the grid
  uint32_t solo_L, solo_done, solo_prev, pad;
  unsigned long long solo_nvis, solo_mvis;
  unsigned long long solo_base[kBuckets];
};

struct BfsWork {
  uint32_t n = 0;
  uint32_t nw = 0;
  uint32_t* vis = nullptr;
  uint32_t* zmask = nullptr;        // bit per degree-0 vertex (never reached, never scanned)
  uint64_t zmask_version = ~0ull;   // graph version zmask was computed for
  uint32_t* fb = nullptr;  // 2 * nw words
  uint32_t* queue = nullptr;
  BfsCtl* ctl = nullptr;
  byo_bfs_iter* trace = nullptr;
};

void bfs_free(BfsWork* w) {
  if (!w) return;
  dev_free(w->vis);
  dev_free(w->zmask);
  dev_free(w->fb);
  dev_free(w->queue);
  dev_free(w->ctl);
  dev_free(w->trace);
  delete w;
}

template <typename G>
struct BfsArgs {
  G g;
  uint32_t src;
  uint32_t* level;
  uint32_t* parent;
  uint32_t* vis;
  const uint32_t* zmask;  // nullable: the visited bits start as these (degree-0 vertices)
  uint32_t* fb;
  uint32_t* queue;
  const uint64_t* bstart;
  BfsCtl* ctl;
  byo_bfs_iter* trace;
  SchedParams sp;
  uint64_t limit_ns;
  uint32_t nw;
};

namespace {

// Winners of a warp waiting for their queue slots.  Reserving slots costs
// one global atomicAdd per degree bucket, and the counter of a popular
// bucket takes every warp's atomics (a single address sustains about 1.5 G
// atomics/s), so a warp stages its winners and reserves for at least
// kStage - 31 of them at a time.
constexpr uint32_t kStage = 128;
struct WarpStage {
  uint32_t v[kStage];
  uint32_t cur[kBuckets];             // per-bucket counts, then cursors
  unsigned long long base[kBuckets];  // reserved start of each bucket's run
  uint8_t b[kStage];
  uint32_t n;  // entries staged
};

struct BfsShared {
  uint64_t bstart[kBuckets + 1];
  uint64_t base[kBuckets];   // start of the current level's run inside each bucket region
  uint64_t pre[kBuckets + 1];   // prefix of current counts over buckets
  uint64_t preC[kBuckets + 1];  // prefix of CTA-bin work items (counts * chunks)
  uint32_t cnt[kBuckets];
  uint64_t nvis, mvis;
  uint32_t nf;
  uint64_t mf;
  int dir, action, bt, bw, prev_dir;
  int fb_valid;
  uint64_t t_top;
  uint32_t t_level;  // level whose start time t_top is
  uint64_t scan_prev;  // ids read during the level before (trace)
  int precheck;        // push reads the visited bit before claiming
  uint32_t tg_min;     // smallest thread-bin group: 32 / (lower bound of the bin's mean degree)
  uint32_t err_seen;   // the control block's error word at the start of the level
  WarpStage* stage;    // per-warp stages (shared memory, overlaid on the solo lists)
  unsigned long long red[2];  // this CTA's share of the next frontier's degree sum and ids read
};

__device__ __forceinline__ int find_bucket(const uint64_t* pre, int lo, int hi, uint64_t i) {
  // largest b in [lo, hi] with pre[b] <= i
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Writes the calling warp's staged winners to the next level's queue: a
// per-bucket count in shared memory, one global atomicAdd per bucket present
// (issued by different lanes at once), then every entry takes its slot from
// the bucket's shared cursor.  Warp-collective.
template <typename G>
__device__ __noinline__ void stage_flush(const BfsArgs<G>& a, BfsShared& S, int nxt) {
  WarpStage& W = S.stage[threadIdx.x >> 5];
  const uint32_t lane = lane_id();
  const uint32_t ns = W.n;
  for (uint32_t i = lane; i < (uint32_t)kBuckets; i += 32) W.cur[i] = 0;
  __syncwarp();
  for (uint32_t i = lane; i < ns; i += 32) atomicAdd(&W.cur[W.b[i]], 1u);
  __syncwarp();
  for (uint32_t i = lane; i < (uint32_t)kBuckets; i += 32) {
    const uint32_t c = W.cur[i];
    W.base[i] = c ? atomicAdd(&a.ctl->cnt[nxt][i].v, (unsigned long long)c) : 0ull;
    W.cur[i] = 0;
  }
  __syncwarp();
  for (uint32_t i = lane; i < ns; i += 32) {
    const uint32_t b = W.b[i];
    const uint32_t r = atomicAdd(&W.cur[b], 1u);
    const uint64_t at = S.bstart[b] + S.base[b] + S.cnt[b] + W.base[b] + r;
    if (at < S.bstart[b + 1]) a.queue[at] = W.v[i];
    else atomicCAS(&a.ctl->err, 0u, (uint32_t)BYO_ERR_CUDA);  // cannot happen: each vertex is claimed once
  }
  __syncwarp();
  if (lane == 0) W.n = 0;
  __syncwarp();
}

// Stages the calling warp's winners (lanes with `won`: vertex v of degree
// bucket b) and flushes once fewer than 32 free entries remain.  Warp-collective.
template <typename G>
__device__ __forceinline__ void stage_add(const BfsArgs<G>& a, BfsShared& S, bool won, uint32_t v, uint32_t b,
                                          int nxt) {
  const uint32_t m = __ballot_sync(0xFFFFFFFFu, won);
  if (m == 0) return;
  WarpStage& W = S.stage[threadIdx.x >> 5];
  const uint32_t n0 = W.n;
  if (won) {
    const uint32_t slot = n0 + __popc(m & lanemask_lt());
    W.v[slot] = v;
    W.b[slot] = (uint8_t)b;
  }
  __syncwarp();
  const uint32_t n1 = n0 + __popc(m);
  if (lane_id() == 0) W.n = n1;
  __syncwarp();
  if (n1 > kStage - 32) stage_flush(a, S, nxt);
}

// The rest of the calling warp's stage, at the end of a phase.  Warp-collective.
template <typename G>
__device__ __forceinline__ void stage_drain(const BfsArgs<G>& a, BfsShared& S, int nxt) {
  if (S.stage[threadIdx.x >> 5].n) stage_flush(a, S, nxt);
}

// Warp-collective: claim v for every lane with `cand`, then record the
// winners and append them to the next level's queue.  All 32 lanes call it.
// Each candidate lane claims with its own atomicOr on the visited bits: the
// word it returns decides the one winner of each vertex, also between lanes
// of this warp that hold the same vertex.
template <typename G, bool kParents>
__device__ __forceinline__ void claim_emit(const BfsArgs<G>& a, BfsShared& S, bool cand, uint32_t v, uint32_t u,
                                           uint32_t next_level, int nxt, uint64_t& acc_deg) {
  // the plain read of the visited bit spares atomics where many neighbours are
  // already visited; on small levels it is one more round trip and is skipped
  if (cand && S.precheck) cand = !((ld_cg(a.vis + (v >> 5)) >> (v & 31)) & 1u);
  if (__ballot_sync(0xFFFFFFFFu, cand) == 0) return;
  const uint32_t bit = 1u << (v & 31);
  const uint32_t d = cand ? a.g.degree(v) : 0u;  // read while the claim is in flight
  const bool won = cand && !(atomicOr(a.vis + (v >> 5), bit) & bit);
  if (!__any_sync(0xFFFFFFFFu, won)) return;
  uint32_t b = 0xFFFFFFFFu;
  if (won) {
    a.level[v] = next_level;
    if (kParents) a.parent[v] = u;
    acc_deg += d;
    b = (uint32_t)degree_bucket(d);
  }
  stage_add(a, S, won, v, b, nxt);
}

// claim_emit for K candidates per lane (v[k], parent u[k]), with the K
// visited reads, the K degree reads, the K claims and the K queue
// reservations each issued together, so that one warp keeps K chains of
// memory operations in flight instead of one.  Warp-collective.
template <typename G, bool kParents, int K>
__device__ __forceinline__ void claim_emit_k(const BfsArgs<G>& a, BfsShared& S, const bool (&cand_in)[K],
                                             const uint32_t (&v)[K], const uint32_t (&u)[K], uint32_t next_level,
                                             int nxt, uint64_t& acc_deg) {
  bool cand[K];
  bool any = false;
  if (S.precheck) {
    uint32_t w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = cand_in[k] ? ld_cg(a.vis + (v[k] >> 5)) : 0u;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      cand[k] = cand_in[k] && !((w[k] >> (v[k] & 31)) & 1u);
      any |= cand[k];
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      cand[k] = cand_in[k];
      any |= cand[k];
    }
  }
  if (!__any_sync(0xFFFFFFFFu, any)) return;
  uint32_t d[K], old[K];
#pragma unroll
  for (int k = 0; k < K; ++k) d[k] = cand[k] ? a.g.degree(v[k]) : 0u;
#pragma unroll
  for (int k = 0; k < K; ++k) old[k] = cand[k] ? atomicOr(a.vis + (v[k] >> 5), 1u << (v[k] & 31)) : ~0u;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const bool won = cand[k] && !(old[k] & (1u << (v[k] & 31)));
    uint32_t b = 0xFFFFFFFFu;
    if (won) {
      a.level[v[k]] = next_level;
      if (kParents) a.parent[v[k]] = u[k];
      acc_deg += d[k];
      b = (uint32_t)degree_bucket(d[k]);
    }
    stage_add(a, S, won, v[k], b, nxt);
  }
}

template <typename G>
__device__ __forceinline__ uint32_t frontier_vertex(const BfsArgs<G>& a, const BfsShared& S, int b, uint64_t i) {
  return ld_cg(a.queue + S.bstart[b] + S.base[b] + i);
}

// ---------------------------------------------------------------- push
// Who shares a push iteration: the whole grid, or one CTA alone (solo levels).
struct Workers {
  uint32_t cta, ctas;    // this CTA's rank and the number of CTAs
  uint32_t warp, warps;  // this warp's rank and the number of warps
};

template <typename G, bool kParents>
__device__ void push_phase(const BfsArgs<G>& a, BfsShared& S, const Workers& wk, uint32_t L, int nxt,
                           uint64_t& acc_deg, uint64_t& acc_scan) {
  const uint32_t lane = lane_id();
  const uint32_t gwarp = wk.warp;
  const uint32_t nwarps = wk.warps;
  const int bt = S.bt, bw = S.bw;

  // CTA bin: chunks of high-degree vertices
  const uint64_t totC = S.preC[kBuckets] - S.preC[bw + 1];
  for (uint64_t j = wk.cta; j < totC; j += wk.ctas) {
    uint64_t jj = j + S.preC[bw + 1];
    int b = find_bucket(S.preC, bw + 1, kBuckets - 1, jj);
    uint64_t K = (b >= 12) ? (1ull << (b - 11)) : 1ull;  // chunks per vertex: 2^b / kChunk
    uint64_t r = jj - S.preC[b];
    uint32_t u = frontier_vertex(a, S, b, r / K);
    uint32_t chunk = (uint32_t)(r % K);
    Seg s = a.g.seg(u);
    uint32_t per = (uint32_t)((s.len + K - 1) / K);
    uint32_t lo = chunk * per, hi = min(s.len, lo + per);
    for (uint32_t base = lo; base < hi; base += blockDim.x * kPushK) {
      bool ok[kPushK];
      uint32_t v[kPushK], uu[kPushK];
#pragma unroll
      for (int k = 0; k < kPushK; ++k) {
        const uint32_t e = base + k * blockDim.x + threadIdx.x;
        ok[k] = e < hi;
        v[k] = ok[k] ? __ldg(s.p + e) : 0u;
        uu[k] = u;
        acc_scan += ok[k];
      }
      claim_emit_k<G, kParents, kPushK>(a, S, ok, v, uu, L + 1, nxt, acc_deg);
    }
  }
  // warp bin: one warp per vertex
  const uint64_t w0 = S.pre[bt + 1], w1 = S.pre[bw + 1];
  for (uint64_t j = w0 + gwarp; j < w1; j += nwarps) {
    int b = find_bucket(S.pre, bt + 1, bw, j);
    uint32_t u = frontier_vertex(a, S, b, j - S.pre[b]);
    Seg s = a.g.seg(u);
    for (uint32_t base = 0; base < s.len; base += 32 * kPushK) {
      bool ok[kPushK];
      uint32_t v[kPushK], uu[kPushK];
#pragma unroll
      for (int k = 0; k < kPushK; ++k) {
        const uint32_t e = base + k * 32 + lane;
        ok[k] = e < s.len;
        v[k] = ok[k] ? __ldg(s.p + e) : 0u;
        uu[k] = u;
        acc_scan += ok[k];
      }
      claim_emit_k<G, kParents, kPushK>(a, S, ok, v, uu, L + 1, nxt, acc_deg);
    }
  }
  // thread bin: 32 vertices per warp, their edges walked 32 at a time
  const uint64_t t1 = S.pre[bt + 1];
  if (a.sp.flags & BYO_SCHED_SEQUENTIAL_MAPS) {
    // ablation: every lane walks its own vertex's list, one id per step
    for (uint64_t jb = (uint64_t)gwarp * 32; jb < t1; jb += (uint64_t)nwarps * 32) {
      const uint64_t j = jb + lane;
      uint32_t u = 0;
      Seg s{nullptr, 0};
      if (j < t1) {
        const int b = find_bucket(S.pre, 0, bt, j);
        u = frontier_vertex(a, S, b, j - S.pre[b]);
        s = a.g.seg(u);
      }
      const uint32_t kmax = __reduce_max_sync(0xFFFFFFFFu, s.len);
      for (uint32_t k = 0; k < kmax; ++k) {
        const bool ok = k < s.len;
        const uint32_t v = ok ? __ldg(s.p + k) : 0u;
        if (ok) ++acc_scan;
        claim_emit<G, kParents>(a, S, ok, v, u, L + 1, nxt, acc_deg);
      }
    }
    stage_drain(a, S, nxt);
    return;
  }
  // Vertices per warp: 32 once every warp has a group of its own, fewer on
  // smaller levels (down to about one round of 32 edges per warp), because the
  // rounds of one warp run one after another, each a chain of dependent memory
  // operations.
  const uint64_t spread = (t1 + nwarps - 1) / nwarps;
  const uint32_t sp1 = spread >= 32 ? 32u : (spread ? (uint32_t)spread : 1u);
  const uint32_t g = sp1 >= 32 ? 32u : max(S.tg_min, 1u << (31 - __clz(sp1 * 2 - 1)));  // pow2 >= sp1
  for (uint64_t jb = (uint64_t)gwarp * g; jb < t1; jb += (uint64_t)nwarps * g) {
    uint64_t j = jb + lane;
    uint32_t u = 0;
    Seg s{nullptr, 0};
    if (lane < g && j < t1) {
      int b = find_bucket(S.pre, 0, bt, j);
      u = frontier_vertex(a, S, b, j - S.pre[b]);
      s = a.g.seg(u);
    }
    uint32_t incl = s.len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if ((int)lane >= o) incl += y;
    }
    uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t excl = incl - s.len;
    for (uint32_t e0 = 0; e0 < total; e0 += 32) {
      uint32_t e = e0 + lane;
      // owner: the largest lane l with excl_l <= e
      int owner = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        int probe = owner + step;
        uint32_t ex = __shfl_sync(0xFFFFFFFFu, excl, probe & 31);
        if (probe < 32 && ex <= e) owner = probe;
      }
      uint32_t oex = __shfl_sync(0xFFFFFFFFu, excl, owner);
      uint32_t ou = __shfl_sync(0xFFFFFFFFu, u, owner);
      const uint32_t* op = reinterpret_cast<const uint32_t*>(
          __shfl_sync(0xFFFFFFFFu, reinterpret_cast<unsigned long long>(s.p), owner));
      bool ok = e < total;
      uint32_t v = ok ? __ldg(op + (e - oex)) : 0;
      if (ok) ++acc_scan;
      claim_emit<G, kParents>(a, S, ok, v, ou, L + 1, nxt, acc_deg);
    }
  }
  stage_drain(a, S, nxt);
}

// ---------------------------------------------------------------- pull
__device__ __forceinline__ bool in_frontier(const uint32_t* fb, uint32_t u) {
  return (ld_cg(fb + (u >> 5)) >> (u & 31)) & 1u;
}

// The outputs of the vertices a warp found in one pull step (`found` lanes,
// vertex v with parent par and degree len): level and parent, their visited
// and next-frontier bits (grouped by word: one read-modify-write per word,
// the words being the calling warp's own) and their queue slots (one atomic
// per degree bucket).  Warp-collective.
template <typename G, bool kParents>
__device__ __forceinline__ void pull_emit(const BfsArgs<G>& a, BfsShared& S, uint32_t* fbn, bool found,
                                          uint32_t v, uint32_t par, uint32_t len, uint32_t L, int nxt,
                                          uint64_t& acc_deg) {
  if (!__any_sync(0xFFFFFFFFu, found)) return;
  uint32_t b = 0xFFFFFFFFu;
  if (found) {
    a.level[v] = L + 1;
    if (kParents) a.parent[v] = par;
    acc_deg += len;
    b = (uint32_t)degree_bucket(len);
    // the warp's own words (no other warp writes them in this level): plain
    // reductions, nothing to wait for
    atomicOr(a.vis + (v >> 5), 1u << (v & 31));
    atomicOr(fbn + (v >> 5), 1u << (v & 31));
  }
  stage_add(a, S, found, v, b, nxt);
  __syncwarp();  // the word updates are seen by the warp's later readers
}

// Position of the r-th (0-based, from the least significant) set bit of m,
// r < popc(m): the largest p with fewer than r + 1 set bits below p, by a
// binary search over p.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t r) {
  uint32_t p = 0;
#pragma unroll
  for (uint32_t s = 16; s > 0; s >>= 1)
    if ((uint32_t)__popc(m & ((1u << (p + s)) - 1u)) <= r) p += s;
  return p;
}

// Deferred long scans of one warp: vertices whose first kPullThreadMax ids
// hold no frontier neighbour; the whole warp continues each from there.
constexpr uint32_t kPullDefer = 32;

struct PullDefer {
  uint32_t v[kPullDefer];
  uint32_t from[kPullDefer];  // first id (index in the list) not scanned yet
  uint32_t par[kPullDefer];   // no early exit: the first frontier neighbour already found, else INF
};

template <typename G, bool kParents>
__device__ void pull_long(const BfsArgs<G>& a, BfsShared& S, uint32_t* fbn, const uint32_t* fb,
                          PullDefer& D, uint32_t cnt, uint32_t L, int nxt, bool no_exit, uint64_t& acc_deg,
                          uint64_t& acc_scan) {
  const uint32_t lane = lane_id();
  uint32_t sink = 0;
  for (uint32_t d = 0; d < cnt; ++d) {
    const uint32_t v = D.v[d];
    const Seg sg = a.g.seg(v);
    const uint32_t* al = align16_down(sg.p);
    const uint32_t head = (uint32_t)(sg.p - al);
    const uint32_t end = head + sg.len;
    const uint32_t from = head + D.from[d];
    uint32_t got = D.par[d];
    for (uint32_t i0 = from & ~3u; i0 < end; i0 += 128) {
      const uint32_t i = i0 + lane * 4;
      uint32_t hit = kInf;
      if (i < end) {
        const uint4 q = ld_nc_v4(al + i);
        const uint32_t x[4] = {q.x, q.y, q.z, q.w};
        sink ^= q.x ^ q.w;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t idx = i + c;
          if (hit == kInf && got == kInf && idx >= from && idx < end && in_frontier(fb, x[c])) hit = x[c];
        }
      }
      const uint32_t hm = __ballot_sync(0xFFFFFFFFu, hit != kInf);
      if (lane == 0) acc_scan += min(end, i0 + 128) - max(from, i0);  // upper bound of ids read
      if (hm) got = __shfl_sync(0xFFFFFFFFu, hit, __ffs(hm) - 1);
      if (got != kInf && !no_exit) break;  // without the ablation: stop at the first frontier neighbour
    }
    pull_emit<G, kParents>(a, S, fbn, lane == 0 && got != kInf, v, got, sg.len, L, nxt, acc_deg);
  }
  asm volatile("" ::"r"(sink));
}

template <typename G, bool kParents>
__device__ bool pull_phase(const BfsArgs<G>& a, BfsShared& S, PullDefer* defer, uint32_t L, int nxt,
                           uint64_t& acc_deg, uint64_t& acc_scan) {
  // Warps take batches of 32 words (1,024 vertices) from a per-level counter
  // as they finish the previous batch, so a warp that meets long lists does
  // not hold up the level; the visited and next-frontier bits are set with
  // atomic ORs.  The next frontier's words are cleared first, each warp a
  // fixed range, and a grid barrier separates that from the first emits.
  // A warp's lanes work as a pool: a lane scans one unvisited vertex at a time,
  // eight ids per step, and takes the next pending vertex of the warp's range
  // as soon as it is done, so a long scan in one lane does not hold the
  // others (no warp-wide wait on the slowest vertex of a word).  A vertex
  // still without a frontier neighbour after kPullThreadMax ids is deferred
  // and later scanned by the whole warp, 128 ids per step.
  const uint32_t lane = lane_id();
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  PullDefer& D = defer[threadIdx.x >> 5];
  const uint32_t* fb = a.fb + (size_t)(L & 1) * a.nw;
  uint32_t* fbn = a.fb + (size_t)((L + 1) & 1) * a.nw;
  const uint32_t n = a.g.num_vertices();
  const uint32_t per = (a.nw + nwarps - 1) / nwarps;
  const uint32_t w_lo = min(a.nw, gwarp * per), w_hi = min(a.nw, w_lo + per);
  for (uint32_t w = w_lo + lane; w < w_hi; w += 32) fbn[w] = 0;
  if (!grid_barrier(&a.ctl->bar, gridDim.x, &a.ctl->err, a.limit_ns)) return false;
  unsigned long long* next_batch = &a.ctl->pull_next[L % 3].v;
  // 32 words of pending (unvisited) bits are loaded at a time, one per lane
  uint32_t batch = 0;           // first word of the loaded batch
  bool drained = false;         // the level's words are all handed out
  uint32_t pend_lane = 0;       // pending bits of word batch + lane not taken yet
  uint32_t ndef = 0;            // deferred vertices
  uint32_t v = kInf;            // this lane's vertex
  const uint32_t* al = nullptr;
  uint32_t head = 0, end = 0, i = 0, len = 0;
  bool fresh = false;           // v was just taken: its list location is not loaded yet
  const bool no_exit = (a.sp.flags & BYO_SCHED_NO_EARLY_EXIT) != 0;
  const bool seq = (a.sp.flags & BYO_SCHED_SEQUENTIAL_MAPS) != 0;
  uint32_t hit_par = kInf;      // no early exit: the first frontier neighbour found so far
  uint32_t sink = 0;
  while (true) {
    // free lanes take pending vertices, opening words as needed
    // free lanes take the batch's first pending vertices, in word order, all
    // at once: a warp scan of the words' pending counts (one word per lane),
    // then each taking lane finds its word by a 5-step search over the scan
    uint32_t freeL = __ballot_sync(0xFFFFFFFFu, v == kInf);
    while (freeL) {
      if (__ballot_sync(0xFFFFFFFFu, pend_lane != 0) == 0) {  // the batch is used up
        if (drained) break;
        unsigned long long nb = 0;
        if (lane == 0) nb = atomicAdd(next_batch, 32ull);
        nb = __shfl_sync(0xFFFFFFFFu, nb, 0);
        if (nb >= a.nw) {
          drained = true;
          break;
        }
        batch = (uint32_t)nb;
        const uint32_t w = batch + lane;
        uint32_t vw = w < a.nw ? ld_cg(a.vis + w) : ~0u;
        if (w == a.nw - 1 && (n & 31)) vw |= ~0u << (n & 31);  // past n: not a vertex
        pend_lane = ~vw;
        continue;
      }
      const uint32_t c = __popc(pend_lane);
      uint32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
      const uint32_t take = min((uint32_t)__popc(freeL), total);
      const uint32_t r = __popc(freeL & lanemask_lt());
      const uint32_t rr = min(r, total - 1);
      uint32_t j = 0;  // the first word whose inclusive count exceeds rr
#pragma unroll
      for (uint32_t step = 16; step > 0; step >>= 1)
        if (__shfl_sync(0xFFFFFFFFu, incl, j + step - 1) <= rr) j += step;
      const uint32_t wbits = __shfl_sync(0xFFFFFFFFu, pend_lane, j);
      const uint32_t wex = __shfl_sync(0xFFFFFFFFu, incl - c, j);
      if (v == kInf && r < take) {
        v = (batch + j) * 32 + nth_set_bit(wbits, rr - wex);
        fresh = true;
      }
      // the first `take` pending vertices of the batch are gone
      const uint32_t excl = incl - c;
      if (incl <= take) pend_lane = 0u;
      else if (excl < take) pend_lane &= ~((1u << nth_set_bit(pend_lane, take - excl)) - 1u);
      freeL = __ballot_sync(0xFFFFFFFFu, v == kInf);
    }
    const bool active = v != kInf;
    if (__ballot_sync(0xFFFFFFFFu, active) == 0) break;
    if (fresh) {
      const Seg sg = a.g.seg(v);
      al = align16_down(sg.p);
      head = (uint32_t)(sg.p - al);
      len = sg.len;
      end = head + sg.len;
      i = 0;
      fresh = false;
    }
    // one step: eight ids and their eight frontier words in flight; the
    // lowest hit is the parent (the first frontier neighbour in ascending order)
    bool found = false, done = false, defer_it = false;
    uint32_t par = kInf;
    if (active) {
      if (i < end && !(no_exit && hit_par != kInf)) {
        const uint4 q0 = ld_nc_v4(al + i);
        const uint4 q1 = i + 4 < end ? ld_nc_v4(al + i + 4) : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t x[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        uint32_t hf = 8;
#pragma unroll
        for (int c = 7; c >= 0; --c) {
          const uint32_t idx = i + c;
          if (idx >= head && idx < end && in_frontier(fb, x[c])) {
            par = x[c];
            hf = (uint32_t)c;
          }
        }
        const uint32_t lo = head > i ? head : i;
        if (hf < 8) {
          found = true;
          acc_scan += i + hf + 1 - lo;  // ids up to and including the hit
        } else {
          acc_scan += (end < i + 8 ? end : i + 8) - lo;
        }
        i += 8;
      } else if (i < end) {
        // no early exit (ablation): the rest of the list is read all the same
        const uint4 q0 = ld_nc_v4(al + i);
        const uint4 q1 = i + 4 < end ? ld_nc_v4(al + i + 4) : make_uint4(0u, 0u, 0u, 0u);
        sink ^= q0.x ^ q0.y ^ q0.z ^ q0.w ^ q1.x ^ q1.y ^ q1.z ^ q1.w;
        acc_scan += (end < i + 8 ? end : i + 8) - (head > i ? head : i);
        i += 8;
      }
      if (no_exit) {
        if (found && hit_par == kInf) hit_par = par;
        found = false;
        done = i >= end;
        if (done && hit_par != kInf) {
          found = true;
          par = hit_par;
        }
      } else {
        done = found || i >= end;
      }
      defer_it = !done && !seq && i >= head + kPullThreadMax;
    }
    pull_emit<G, kParents>(a, S, fbn, found, v, par, len, L, nxt, acc_deg);
    // long scans go to the warp's deferred list (scanned when it fills up,
    // and at the end)
    const uint32_t dm = __ballot_sync(0xFFFFFFFFu, defer_it);
    if (dm) {
      if (ndef + __popc(dm) > kPullDefer) {
        __syncwarp();
        pull_long<G, kParents>(a, S, fbn, fb, D, ndef, L, nxt, no_exit, acc_deg, acc_scan);
        ndef = 0;
        __syncwarp();
      }
      if (defer_it) {
        const uint32_t slot = ndef + __popc(dm & lanemask_lt());
        D.v[slot] = v;
        D.from[slot] = i - head;
        D.par[slot] = hit_par;
      }
      ndef += __popc(dm);
      __syncwarp();
    }
    if (done || defer_it) {
      v = kInf;
      hit_par = kInf;
    }
  }
  if (ndef) pull_long<G, kParents>(a, S, fbn, fb, D, ndef, L, nxt, no_exit, acc_deg, acc_scan);
  stage_drain(a, S, nxt);
  asm volatile("" ::"r"(sink));  // the ablation's reads are kept
  return true;
}

// warp sum of v into a shared-memory accumulator of the CTA
__device__ __forceinline__ void flush_acc(unsigned long long* dst, uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  if (lane_id() == 0 && v) atomicAdd(dst, (unsigned long long)v);
}

// Start of level L for the calling CTA: frontier counts and prefixes, the
// trace, the schedule decision and the push bins.  `owner` (block 0) also
// zeroes the counters of level L+2 and writes the trace.  Returns |F|.
// The counters come in one round of loads; warp 0 then forms both bucket
// prefixes with shuffle scans (lane b holds bucket b, the last bucket is added
// on top) and decides, while other threads clear the counters of level L-1,
// which no CTA reads any more (all passed the barrier that ended it) and
// which level L+1 fills next.
template <typename G>
__device__ uint32_t level_top(const BfsArgs<G>& a, BfsShared& S, uint32_t L, bool owner) {
  static_assert(kBuckets == 33, "warp 0 scans buckets 0..31 and adds bucket 32");
  const uint32_t tid = threadIdx.x;
  const uint32_t n = a.g.num_vertices();
  const uint64_t m = a.g.num_edges();
  BfsCtl* ctl = a.ctl;
  const int cur = L % 3, old = (L + 2) % 3;
  if (tid < (uint32_t)kBuckets) S.cnt[tid] = (uint32_t)ld_cg(&ctl->cnt[cur][tid].v);
  else if (tid == kBuckets) S.mf = ld_cg(&ctl->sdeg[cur]);
  else if (tid == kBuckets + 1 && owner) S.scan_prev = ld_cg(&ctl->scanned[cur]);
  else if (tid == kBuckets + 2) S.err_seen = ld_cg(&ctl->err);
  __syncthreads();
  if (S.err_seen != 0) return 0;  // another CTA failed: the caller stops
  if (tid < 32) {
    const uint32_t lane = tid;
    uint64_t inc = S.cnt[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if ((int)lane >= o) inc += y;
    }
    const uint64_t nf = __shfl_sync(0xFFFFFFFFu, inc, 31) + S.cnt[32];
    S.pre[lane + 1] = inc;
    if (lane == 0) {
      S.pre[0] = 0;
      S.pre[kBuckets] = nf;
      S.nf = (uint32_t)nf;
      const uint64_t now = globaltimer();
      if (owner && L > 0 && L - 1 < kTraceCap && S.t_level == L - 1) {
        byo_bfs_iter* r = a.trace + (L - 1);
        r->t_ns = now - S.t_top;
        r->edges_examined = S.scan_prev;
      }
      if (S.t_level != L) {
        S.t_top = now;
        S.t_level = L;
      }
    }
    if (nf != 0) {
      SchedFeatures f;
      f.nf = (uint32_t)nf;
      f.mf = S.mf;
      f.nu = (uint64_t)n - S.nvis - nf;
      f.mu = m - S.mvis - S.mf;
      f.n = n;
      f.m = m;
      const uint64_t p3 = __shfl_sync(0xFFFFFFFFu, inc, 2), p6 = __shfl_sync(0xFFFFFFFFu, inc, 5),
                     p9 = __shfl_sync(0xFFFFFFFFu, inc, 8);
      f.h[0] = (uint32_t)p3;
      f.h[1] = (uint32_t)(p6 - p3);
      f.h[2] = (uint32_t)(p9 - p6);
      f.h[3] = (uint32_t)(nf - p9);
      const int action = sched_decide(a.sp, f, S.prev_dir);  // warp-collective
      int bt, bw;
      sched_bins(a.sp, action, &bt, &bw);
      // CTA-bin work items: vertices * chunks per vertex, for buckets above bw
      auto items = [&](int b) -> uint64_t {
        return b > bw ? (uint64_t)S.cnt[b] * ((b >= 12) ? (1ull << (b - 11)) : 1ull) : 0ull;
      };
      uint64_t c = items((int)lane);
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, c, o);
        if ((int)lane >= o) c += y;
      }
      S.preC[lane + 1] = c;
      const uint64_t totC = __shfl_sync(0xFFFFFFFFu, c, 31) + items(32);
      // thread bin (buckets 1..bt; bucket b holds degrees >= 2^(b-1)): vertices
      // and a lower bound of their degree sum
      uint64_t tv = (lane >= 1 && (int)lane <= bt) ? S.cnt[lane] : 0ull;
      uint64_t te = tv << (lane >= 1 ? lane - 1 : 0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        tv += __shfl_xor_sync(0xFFFFFFFFu, tv, o);
        te += __shfl_xor_sync(0xFFFFFFFFu, te, o);
      }
      const uint64_t mean = tv ? (te + tv - 1) / tv : 1;  // >= 1
      const uint32_t tg = mean >= 32 ? 1u : 1u << (31 - __clz((uint32_t)(32 / mean)));
      if (lane == 0) {
        S.preC[0] = 0;
        S.preC[kBuckets] = totC;
        S.action = action;
        S.dir = action == 0 ? 0 : 1;
        S.bt = bt;
        S.bw = bw;
        S.precheck = f.mf >= kPrecheckMinEdges;
        S.tg_min = tg;
        if (owner && L < kTraceCap) {
          byo_bfs_iter* r = a.trace + L;
          r->level = L;
          r->direction = (uint32_t)S.dir;
          r->action = (uint32_t)action;
          r->frontier = (uint32_t)nf;
          r->frontier_edges = f.mf;
          r->unvisited = (uint32_t)f.nu;
          r->unvisited_edges = f.mu;
          for (int k = 0; k < 4; ++k) r->hist[k] = f.h[k];
          r->reserved = 0;
          r->edges_examined = 0;
          r->t_ns = 0;
        }
      }
    }
  } else if (owner && tid >= 64 && tid < 64 + (uint32_t)kBuckets) {
    ctl->cnt[old][tid - 64].v = 0;
  } else if (owner && tid == 64 + (uint32_t)kBuckets) {
    ctl->sdeg[old] = 0;
    ctl->scanned[old] = 0;
    ctl->pull_next[old].v = 0;
  }
  __syncthreads();
  return S.nf;
}

// End of a level for the calling CTA: its share of the next frontier's edge
// and scan counts, then the level-local state moves on.
template <typename G>
__device__ __forceinline__ void level_end(const BfsArgs<G>& a, BfsShared& S, int nxt, uint64_t acc_deg,
                                          uint64_t acc_scan) {
  // warps add into the CTA's accumulators, the CTA into the control block
  // (one global atomic per counter and CTA)
  flush_acc(&S.red[0], acc_deg);
  flush_acc(&S.red[1], acc_scan);
  __syncthreads();
  if (threadIdx.x < (uint32_t)kBuckets) S.base[threadIdx.x] += S.cnt[threadIdx.x];
  if (threadIdx.x == 0) {
    if (S.red[0]) atomicAdd(&a.ctl->sdeg[nxt], S.red[0]);
    if (S.red[1]) atomicAdd(&a.ctl->scanned[nxt], S.red[1]);
    S.red[0] = 0;
    S.red[1] = 0;
    S.nvis += S.nf;
    S.mvis += S.mf;
    S.prev_dir = S.dir;
    S.fb_valid = S.dir == 0;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- solo levels
// While the frontier stays small, block 0 keeps it in shared memory as
// (list pointer, id, degree) entries and runs level after level without
// touching the global queue or counters: per level it walks the frontier's
// concatenated lists, claims neighbours with one atomicOr each on the visited
// bits, writes level/parent and appends the winners (with their own list
// location, fetched once) to the next shared-memory list.  That leaves about
// three dependent memory round trips per level.  If a level's winners do not
// fit, the excess spills to the global queue and the grid takes over.
constexpr uint32_t kSoloCap = 1024;

struct SoloEntry {
  const uint32_t* p;
  uint32_t v, len;
};

struct SoloShared {
  SoloEntry list[2][kSoloCap];
  uint32_t pre[kSoloCap + 1];
  uint32_t wsum[kBfsThreads / 32];
  uint32_t n_next, spilled;
  unsigned long long mf_next;
  uint32_t h_next[4];
  uint32_t h_cur[4];
};

__device__ __forceinline__ int deg_class(uint32_t d) { return d < 4 ? 0 : (d < 32 ? 1 : (d < 256 ? 2 : 3)); }

// Q.pre[0..cnt] = exclusive prefix of list[i].len (cnt <= kSoloCap); CTA-wide.
__device__ void solo_prefix(SoloShared& Q, const SoloEntry* list, uint32_t cnt) {
  constexpr uint32_t kPer = kSoloCap / kBfsThreads;  // 4 entries per thread
  const uint32_t tid = threadIdx.x, lane = lane_id();
  uint32_t v[kPer], sum = 0;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) {
    uint32_t i = tid * kPer + j;
    v[j] = i < cnt ? list[i].len : 0;
    sum += v[j];
  }
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if ((int)lane >= o) inc += y;
  }
  if (lane == 31) Q.wsum[tid >> 5] = inc;
  __syncthreads();
  uint32_t off = 0;
  for (uint32_t w = 0; w < (tid >> 5); ++w) off += Q.wsum[w];
  uint32_t run = off + inc - sum;
#pragma unroll
  for (uint32_t j = 0; j < kPer; ++j) {
    uint32_t i = tid * kPer + j;
    if (i < cnt) Q.pre[i] = run;
    run += v[j];
  }
  if (tid == blockDim.x - 1) {
    uint32_t tot = 0;
    for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) tot += Q.wsum[w];
    Q.pre[cnt] = tot;
  }
  __syncthreads();
}

// Block 0 only.  Entry: level L's frontier (|F| <= kSoloCap) is in the global
// queue described by S.  Exit: the frontier of the returned level is in the
// global queue again (or the traversal is done), S.base/nvis/mvis describe it.
template <typename G, bool kParents>
__device__ void fast_solo(const BfsArgs<G>& a, BfsShared& S, SoloShared& Q, uint32_t& L, bool& done,
                          uint64_t t_begin) {
  const uint32_t tid = threadIdx.x;
  const uint32_t n = a.g.num_vertices();
  const uint64_t m = a.g.num_edges();
  BfsCtl* ctl = a.ctl;
  uint32_t cur = 0;
  uint32_t nA = S.nf;
  unsigned long long mfA = S.mf;
  for (uint32_t i = tid; i < nA; i += blockDim.x) {
    int b = find_bucket(S.pre, 0, kBuckets - 1, i);
    uint32_t v = frontier_vertex(a, S, b, i - S.pre[b]);
    Seg sg = a.g.seg(v);
    Q.list[0][i] = SoloEntry{sg.p, v, sg.len};
  }
  __syncthreads();
  // level L's global entries are consumed: later appends start after them
  if (tid < (uint32_t)kBuckets) S.base[tid] += S.cnt[tid];
  if (tid == 0) {
    Q.h_cur[0] = (uint32_t)S.pre[3];
    Q.h_cur[1] = (uint32_t)(S.pre[6] - S.pre[3]);
    Q.h_cur[2] = (uint32_t)(S.pre[9] - S.pre[6]);
    Q.h_cur[3] = (uint32_t)(S.pre[kBuckets] - S.pre[9]);
  }
  done = false;
  while (true) {
    const int nx = (L + 1) % 3;
    const SoloEntry* A = Q.list[cur];
    SoloEntry* B = Q.list[cur ^ 1];
    solo_prefix(Q, A, nA);
    const uint32_t TE = Q.pre[nA];
    if (tid < (uint32_t)kBuckets) ctl->cnt[nx][tid].v = 0;
    if (tid == 0) {
      Q.n_next = 0;
      Q.spilled = 0;
      Q.mf_next = 0;
      for (int k = 0; k < 4; ++k) Q.h_next[k] = 0;
    }
    __syncthreads();
    // four edges per thread per step: their id loads, then their claims, are
    // independent, so four memory round trips overlap
    constexpr uint32_t kU = 4;
    for (uint32_t e0 = 0; e0 < TE; e0 += kU * blockDim.x) {
      uint32_t wv[kU], uv[kU];
      bool ok[kU];
#pragma unroll
      for (uint32_t j = 0; j < kU; ++j) {
        const uint32_t e = e0 + j * blockDim.x + tid;
        ok[j] = e < TE;
        wv[j] = 0;
        uv[j] = 0;
        if (ok[j]) {
          uint32_t lo = 0, hi = nA - 1;  // owner: largest i with pre[i] <= e
          while (lo < hi) {
            uint32_t mid = (lo + hi + 1) >> 1;
            if (Q.pre[mid] <= e) lo = mid;
            else hi = mid - 1;
          }
          const SoloEntry u = A[lo];
          uv[j] = u.v;
          wv[j] = __ldg(u.p + (e - Q.pre[lo]));
        }
      }
      uint32_t old[kU];
#pragma unroll
      for (uint32_t j = 0; j < kU; ++j) old[j] = ok[j] ? atomicOr(a.vis + (wv[j] >> 5), 1u << (wv[j] & 31)) : ~0u;
#pragma unroll
      for (uint32_t j = 0; j < kU; ++j) {
        const uint32_t w = wv[j];
        if (!ok[j] || (old[j] & (1u << (w & 31)))) continue;
        a.level[w] = L + 1;
        if (kParents) a.parent[w] = uv[j];
        const Seg sg = a.g.seg(w);
        const uint32_t slot = atomicAdd(&Q.n_next, 1u);
        if (slot < kSoloCap) {
          B[slot] = SoloEntry{sg.p, w, sg.len};
        } else {
          const int b = degree_bucket(sg.len);
          const unsigned long long pos = atomicAdd(&ctl->cnt[nx][b].v, 1ull);
          const uint64_t at = S.bstart[b] + S.base[b] + pos;
          if (at < S.bstart[b + 1]) a.queue[at] = w;
          else atomicCAS(&ctl->err, 0u, (uint32_t)BYO_ERR_CUDA);  // cannot happen: each vertex is claimed once
          Q.spilled = 1;
        }
        atomicAdd(&Q.mf_next, (unsigned long long)sg.len);
        atomicAdd(&Q.h_next[deg_class(sg.len)], 1u);
      }
    }
    __syncthreads();
    const uint32_t nB = Q.n_next;
    const unsigned long long mfB = Q.mf_next;
    if (tid == 0) {
      uint64_t now = globaltimer();
      if (L < kTraceCap) {
        byo_bfs_iter* r = a.trace + L;
        r->level = L;
        r->direction = 1;
        r->action = (uint32_t)kActionSolo;
        r->frontier = nA;
        r->frontier_edges = mfA;
        r->edges_examined = TE;
        r->unvisited = (uint32_t)((uint64_t)n - S.nvis - nA);
        r->unvisited_edges = m - S.mvis - mfA;
        for (int k = 0; k < 4; ++k) r->hist[k] = Q.h_cur[k];
        r->reserved = 0;
        r->t_ns = now - S.t_top;
      }
      S.t_top = now;
      S.nvis += nA;
      S.mvis += mfA;
      S.prev_dir = 1;
      S.dir = 1;
    }
    __syncthreads();
    ++L;
    S.t_level = L;
    if (nB == 0) {
      done = true;
      return;
    }
    bool stay = !Q.spilled && L <= n && globaltimer() - t_begin <= a.limit_ns;
    if (stay && tid < 32) {
      SchedFeatures f;
      f.nf = nB;
      f.mf = mfB;
      f.nu = (uint64_t)n - S.nvis - nB;
      f.mu = m - S.mvis - mfB;
      f.n = n;
      f.m = m;
      for (int k = 0; k < 4; ++k) f.h[k] = Q.h_next[k];
      int act = sched_decide(a.sp, f, 1);  // warp-collective
      if (tid == 0) S.action = act;
    }
    __syncthreads();
    if (stay && S.action == kActionSolo) {
      if (tid < 4) Q.h_cur[tid] = Q.h_next[tid];
      cur ^= 1;
      nA = nB;
      mfA = mfB;
      continue;
    }
    // hand the new frontier (level L) back to the global queue
    const uint32_t kept = nB < kSoloCap ? nB : kSoloCap;
    for (uint32_t i = tid; i < kept; i += blockDim.x) {
      const SoloEntry e = B[i];
      const int b = degree_bucket(e.len);
      const unsigned long long pos = atomicAdd(&ctl->cnt[L % 3][b].v, 1ull);
      const uint64_t at = S.bstart[b] + S.base[b] + pos;
      if (at < S.bstart[b + 1]) a.queue[at] = e.v;
      else atomicCAS(&ctl->err, 0u, (uint32_t)BYO_ERR_CUDA);
    }
    if (tid == 0) {
      ctl->sdeg[L % 3] = mfB;
      ctl->scanned[L % 3] = TE;
    }
    // the counters of the next two levels start from zero
    if (tid < (uint32_t)kBuckets) {
      ctl->cnt[(L + 1) % 3][tid].v = 0;
      ctl->cnt[(L + 2) % 3][tid].v = 0;
    }
    if (tid == 0) {
      ctl->sdeg[(L + 1) % 3] = 0;
      ctl->scanned[(L + 1) % 3] = 0;
      ctl->sdeg[(L + 2) % 3] = 0;
      ctl->scanned[(L + 2) % 3] = 0;
    }
    __syncthreads();
    return;
  }
}

template <typename G, bool kParents>
__global__ void __launch_bounds__(kBfsThreads, 4) bfs_kernel(BfsArgs<G> a) {
  __shared__ BfsShared S;
  // the solo lists and the warp stages are never in use at the same time
  // (every phase drains its stage before the level ends)
  __shared__ union SoloOrStage {
    SoloShared solo;
    WarpStage stage[kBfsThreads / 32];
  } U;
  SoloShared& Q = U.solo;
  __shared__ PullDefer defer[kBfsThreads / 32];
  sched_stage_weights(a.sp);
  const uint32_t tid = threadIdx.x;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + tid;
  const uint64_t gthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint32_t n = a.g.num_vertices();
  BfsCtl* ctl = a.ctl;
  const bool owner = blockIdx.x == 0;
  // an earlier source of the same call failed: its status stands, nothing runs
  if (ld_cg(&ctl->err) != 0) return;
  const Workers grid_wk{blockIdx.x, gridDim.x, (uint32_t)(gtid >> 5), (uint32_t)(gthreads >> 5)};
  const Workers solo_wk{0, 1, tid >> 5, blockDim.x >> 5};

  // ---- init: levels, parents, visited bits, counters
  for (uint64_t v = gtid; v < n; v += gthreads) {
    a.level[v] = kInf;
    if (kParents) a.parent[v] = kInf;
  }
  // a vertex without neighbours is never reached (unless it is the source) and
  // has nothing to scan: it starts as visited, so that pulls skip it
  for (uint64_t w = gtid; w < a.nw; w += gthreads) a.vis[w] = a.zmask ? __ldg(a.zmask + w) : 0u;
  if (owner) {
    for (int i = tid; i < 3 * kBuckets; i += blockDim.x) ctl->cnt[i / kBuckets][i % kBuckets].v = 0;
    if (tid < 3) {
      ctl->sdeg[tid] = 0;
      ctl->scanned[tid] = 0;
      ctl->pull_next[tid].v = 0;
    }
  }
  if (tid < kBfsThreads / 32) U.stage[tid].n = 0;
  if (tid == 0) S.stage = U.stage;
  if (tid <= (uint32_t)kBuckets) S.bstart[tid] = a.bstart[tid];
  if (tid < (uint32_t)kBuckets) S.base[tid] = 0;
  if (tid == 0) {
    S.nvis = 0;
    S.red[0] = 0;
    S.red[1] = 0;
    S.mvis = 0;
    S.prev_dir = 1;
    S.fb_valid = 0;
    S.t_level = kInf;
  }
  if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
  if (owner && tid == 0) {
    uint32_t s = a.src;
    uint32_t d = a.g.degree(s);
    int b = degree_bucket(d);
    a.level[s] = 0;
    if (kParents) a.parent[s] = s;
    a.vis[s >> 5] = ld_cg(a.vis + (s >> 5)) | (1u << (s & 31));
    a.queue[S.bstart[b]] = s;
    ctl->cnt[0][b].v = 1;
    ctl->sdeg[0] = d;
  }
  if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;

  const uint64_t t_begin = globaltimer();
  uint32_t L = 0;
  while (true) {
    // a BFS has at most n levels; the whole traversal is also time-bounded
    if (L > n || globaltimer() - t_begin > a.limit_ns) {
      if (tid == 0) atomicCAS(&ctl->err, 0u, (uint32_t)BYO_ERR_TIMEOUT);
      return;
    }
    const uint32_t nf_top = level_top(a, S, L, owner);
    if (S.err_seen != 0) return;  // the error another CTA set stands
    if (nf_top == 0) {
      if (owner && tid == 0) ctl->levels = L;
      break;
    }
    const int nxt = (L + 1) % 3;
    uint64_t acc_deg = 0, acc_scan = 0;
    if (S.action == kActionSolo) {
      // Levels with tiny frontiers: block 0 runs them alone with CTA barriers
      // only, while the other CTAs wait at the grid barrier; it stops when the
      // schedule asks for another action or the traversal ends, and hands the
      // level-local state over through the control block.
      if (owner && S.nf <= kSoloCap) {
        uint32_t Ls = L;
        bool done = false;
        fast_solo<G, kParents>(a, S, Q, Ls, done, t_begin);
        __syncthreads();
        if (tid < kBfsThreads / 32) U.stage[tid].n = 0;  // the solo lists overlaid the stages
        if (tid == 0) {
          ctl->solo_L = Ls;
          ctl->solo_done = done ? 1u : 0u;
          ctl->solo_nvis = S.nvis;
          ctl->solo_mvis = S.mvis;
          ctl->solo_prev = 1u;
          if (done) ctl->levels = Ls;
        }
        if (tid < (uint32_t)kBuckets) ctl->solo_base[tid] = S.base[tid];
      } else if (owner) {
        uint32_t Ls = L;
        bool done = false;
        while (true) {
          const int nx = (Ls + 1) % 3;
          uint64_t ad = 0, as = 0;
          push_phase<G, kParents>(a, S, solo_wk, Ls, nx, ad, as);
          level_end(a, S, nx, ad, as);
          ++Ls;
          if (Ls > n || globaltimer() - t_begin > a.limit_ns) {
            if (tid == 0) atomicCAS(&ctl->err, 0u, (uint32_t)BYO_ERR_TIMEOUT);
            break;
          }
          if (level_top(a, S, Ls, true) == 0) {
            done = true;
            break;
          }
          if (S.action != kActionSolo) break;
        }
        if (tid == 0) {
          ctl->solo_L = Ls;
          ctl->solo_done = done ? 1u : 0u;
          ctl->solo_nvis = S.nvis;
          ctl->solo_mvis = S.mvis;
          ctl->solo_prev = (uint32_t)S.prev_dir;
          if (done) ctl->levels = Ls;
        }
        if (tid < (uint32_t)kBuckets) ctl->solo_base[tid] = S.base[tid];
      }
      if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
      if (ld_cg(&ctl->solo_done)) break;
      L = ld_cg(&ctl->solo_L);
      if (tid < (uint32_t)kBuckets) S.base[tid] = ld_cg(&ctl->solo_base[tid]);
      if (tid == 0) {
        S.nvis = ld_cg(&ctl->solo_nvis);
        S.mvis = ld_cg(&ctl->solo_mvis);
        S.prev_dir = (int)ld_cg(&ctl->solo_prev);
        S.fb_valid = 0;
      }
      __syncthreads();
      continue;
    }
    if (S.dir == 0) {
      if (!S.fb_valid) {
        // queue -> bit-vector for this level
        uint32_t* fb = a.fb + (size_t)(L & 1) * a.nw;
        for (uint64_t w = gtid; w < a.nw; w += gthreads) fb[w] = 0;
        if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
        for (uint64_t i = gtid; i < S.nf; i += gthreads) {
          int b = find_bucket(S.pre, 0, kBuckets - 1, i);
          uint32_t v = frontier_vertex(a, S, b, i - S.pre[b]);
          atomicOr(fb + (v >> 5), 1u << (v & 31));
        }
        if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
      }
      if (!pull_phase<G, kParents>(a, S, defer, L, nxt, acc_deg, acc_scan)) return;
    } else {
      push_phase<G, kParents>(a, S, grid_wk, L, nxt, acc_deg, acc_scan);
    }
    level_end(a, S, nxt, acc_deg, acc_scan);
    ++L;
    if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
  }
}

template <typename G>
__global__ void bfs_zmask_kernel(G g, uint32_t* zmask) {
  const uint32_t n = g.num_vertices();
  const uint64_t nw = ((uint64_t)n + 31) / 32;
  for (uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w0 < nw;
       w0 += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
    const uint64_t v = w0 * 32 + lane_id();
    const uint32_t z = __ballot_sync(0xFFFFFFFFu, v < n && g.degree((uint32_t)v) == 0);
    if (lane_id() == 0) zmask[w0] = z;
  }
}

template <typename G, bool kParents>
byo_status launch_bfs(BfsArgs<G>& args, cudaStream_t s) {
  auto fn = bfs_kernel<G, kParents>;
  int per_sm = 0;
  BYO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBfsThreads, 0));
  if (per_sm < 1) {
    set_error("bfs_kernel cannot be resident");
    return BYO_ERR_CUDA;
  }
  int grid = per_sm * sm_count();
  void* kargs[] = {&args};
  BYO_CUDA(reset_barrier(&args.ctl->bar, s));
  ProfScope ps("bfs_persistent", s);
  BYO_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(kBfsThreads), kargs, 0, s));
  note_launch();
  return BYO_OK;
}

template <typename G>
byo_status run_bfs(const byo_graph* g, G view, const uint32_t* sources, uint32_t ns, uint32_t* levels, uint32_t* parents,
                   const SchedParams& sp, cudaStream_t s) {
  BfsWork* w = g->bfs;
  if (w->zmask_version != g->version) {
    bfs_zmask_kernel<G><<<grid_for(g->n, 256), 256, 0, s>>>(view, w->zmask);
    note_launch();
    BYO_CHECK_LAUNCH("bfs_zmask_kernel");
    w->zmask_version = g->version;
  }
  BfsArgs<G> args;
  args.g = view;
  args.vis = w->vis;
  args.zmask = w->zmask;
  args.fb = w->fb;
  args.queue = w->queue;
  args.bstart = g->d_bstart;
  args.ctl = w->ctl;
  args.trace = w->trace;
  args.sp = sp;
  args.limit_ns = timeout_ns();
  args.nw = w->nw;
  for (uint32_t i = 0; i < ns; ++i) {
    args.src = sources[i];
    args.level = levels + (size_t)i * g->n;
    args.parent = parents ? parents + (size_t)i * g->n : nullptr;
    if (parents) BYO_RETURN_IF((launch_bfs<G, true>(args, s)));
    else BYO_RETURN_IF((launch_bfs<G, false>(args, s)));
  }
  return BYO_OK;
}

byo_status ensure_bfs_work(byo_graph* g) {
  if (g->bfs) return BYO_OK;
  BfsWork* w = new (std::nothrow) BfsWork();
  if (!w) {
    set_error("host allocation failed");
    return BYO_ERR_OUT_OF_MEMORY;
  }
  w->n = g->n;
  w->nw = (g->n + 31) / 32;
  byo_status st = dev_alloc_t(&w->vis, w->nw, "BFS visited bits");
  if (st == BYO_OK) st = dev_alloc_t(&w->zmask, w->nw, "BFS degree-0 bits");
  if (st == BYO_OK) st = dev_alloc_t(&w->fb, 2ull * w->nw, "BFS frontier bits");
  if (st == BYO_OK) st = dev_alloc_t(&w->queue, g->n, "BFS queue");
  if (st == BYO_OK) st = dev_alloc_t(&w->ctl, 1, "BFS control");
  if (st == BYO_OK) st = dev_alloc_t(&w->trace, kTraceCap, "BFS trace");
  if (st == BYO_OK) {
    cudaError_t e = cudaMemset(w->ctl, 0, sizeof(BfsCtl));
    if (e != cudaSuccess) st = cuda_status(e, "cudaMemset");
  }
  if (st != BYO_OK) {
    bfs_free(w);
    return st;
  }
  g->bfs = w;
  return BYO_OK;
}

// The status a BFS launch left in its control block, as the call's result.
byo_status bfs_device_status(uint32_t err, const char* who) {
  if (err == (uint32_t)BYO_ERR_TIMEOUT) {
    set_error("%s: a device-side wait exceeded BYO_TIMEOUT_MS", who);
    return BYO_ERR_TIMEOUT;
  }
  set_error("%s: the kernel reported status %u (a frontier queue region overflowed)", who, err);
  return err <= (uint32_t)BYO_ERR_NOT_SYMMETRIC ? (byo_status)err : BYO_ERR_CUDA;
}

}  // namespace
}  // namespace byo

using namespace byo;

extern "C" byo_status byo_bfs(const byo_graph* gc, const uint32_t* host_sources, uint32_t num_sources,
                              uint32_t* levels, uint32_t* parents, const byo_sched* sched, void* stream) {
  clear_error();
  if (gc && gc->comp) {  // the compressed container has its own traversal
    if (num_sources == 0) return BYO_OK;
    if (!host_sources || !levels) {
      set_error("byo_bfs: NULL sources or levels");
      return BYO_ERR_INVALID_ARG;
    }
    for (uint32_t i = 0; i < num_sources; ++i) {
      if (host_sources[i] >= gc->n) {
        set_error("byo_bfs: source %u is >= n (%u)", host_sources[i], gc->n);
        return BYO_ERR_INVALID_ARG;
      }
    }
    SchedParams sp;
    BYO_RETURN_IF(sched_params(sched, &sp));
    return comp_bfs(gc, host_sources, num_sources, levels, parents, sp, static_cast<cudaStream_t>(stream));
  }
  BYO_RETURN_IF(ready_graph(gc, static_cast<cudaStream_t>(stream)));
  byo_graph* g = const_cast<byo_graph*>(gc);
  if (num_sources == 0) return BYO_OK;
  if (!host_sources || !levels) {
    set_error("byo_bfs: NULL sources or levels");
    return BYO_ERR_INVALID_ARG;
  }
  for (uint32_t i = 0; i < num_sources; ++i) {
    if (host_sources[i] >= g->n) {
      set_error("byo_bfs: source %u is >= n (%u)", host_sources[i], g->n);
      return BYO_ERR_INVALID_ARG;
    }
  }
  SchedParams sp;
  BYO_RETURN_IF(sched_params(sched, &sp));
  BYO_RETURN_IF(ensure_bfs_work(g));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  byo_status st = with_view(g, [&](auto view) {
    return run_bfs(g, view, host_sources, num_sources, levels, parents, sp, s);
  });
  BYO_RETURN_IF(st);
  uint32_t err = 0;
  BYO_CUDA(cudaMemcpyAsync(&err, &g->bfs->ctl->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  BYO_CUDA(cudaStreamSynchronize(s));
  if (err) {
    // the next call starts from a clean control block
    cudaMemsetAsync(&g->bfs->ctl->err, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(&g->bfs->ctl->bar, 0, sizeof(GridBar), s);
    cudaStreamSynchronize(s);
    return bfs_device_status(err, "byo_bfs");
  }
  return BYO_OK;
}

extern "C" byo_status byo_bfs_trace(const byo_graph* g, byo_bfs_iter* host_records, uint32_t cap,
                                    uint32_t* host_count, void* stream) {
  clear_error();
  BYO_RETURN_IF(check_graph(g));
  if (!host_count || (cap && !host_records)) {
    set_error("byo_bfs_trace: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  *host_count = 0;
  if (!g->bfs) return BYO_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t levels = 0;
  BYO_CUDA(cudaMemcpyAsync(&levels, &g->bfs->ctl->levels, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  BYO_CUDA(cudaStreamSynchronize(s));
  *host_count = levels;
  uint32_t c = levels < cap ? levels : cap;
  if (c > kTraceCap) c = kTraceCap;
  if (c) {
    BYO_CUDA(cudaMemcpyAsync(host_records, g->bfs->trace, sizeof(byo_bfs_iter) * c, cudaMemcpyDeviceToHost, s));
    BYO_CUDA(cudaStreamSynchronize(s));
  }
  return BYO_OK;
}

// ============================================================================
// BFS without any device allocation, for callers that cannot allocate device
// memory themselves or through this library.  The caller passes the CSR and
// the outputs; every piece of scratch the persistent BFS kernel needs (control
// block, bucket starts, visited and frontier bits, the bucketed queue, the
// iteration trace) lives in one file-scope __device__ array of fixed size,
// shared by every call on a device and kept until the process exits.

namespace byo {
namespace {

constexpr uint32_t kNoallocMaxVertices = 1u << 20;
constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kNaWords = (kNoallocMaxVertices + 31) / 32;
constexpr size_t kNaCtl = 0;
constexpr size_t kNaBstart = kNaCtl + na_align(sizeof(BfsCtl));
constexpr size_t kNaHist = kNaBstart + na_align(sizeof(uint64_t) * (kBuckets + 1));
constexpr size_t kNaVis = kNaHist + na_align(sizeof(unsigned long long) * kBuckets);
constexpr size_t kNaFb = kNaVis + na_align(4 * kNaWords);
constexpr size_t kNaQueue = kNaFb + na_align(8 * kNaWords);
constexpr size_t kNaTrace = kNaQueue + na_align(4ull * kNoallocMaxVertices);
constexpr size_t kNaBytes = kNaTrace + na_align(sizeof(byo_bfs_iter) * kTraceCap);

// 9,324,800 bytes (8.9 MiB).  In host code this name is only a host-side stand-in for the
// array; kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

std::mutex g_na_mu;
void* g_na_addr[256] = {nullptr};

// Device address of the array on the current device, looked up once per device.
byo_status noalloc_scratch(void** out) {
  int dev = 0;
  BYO_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    set_error("byo_bfs_noalloc: device index %d out of range", dev);
    return BYO_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
    g_na_addr[dev] = p;
  }
  *out = g_na_addr[dev];
  return BYO_OK;
}

__global__ void noalloc_hist_kernel(const uint64_t* __restrict__ off, uint32_t n, unsigned long long* hist) {
  __shared__ unsigned long long h[kBuckets];
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[degree_bucket((uint32_t)(off[v + 1] - off[v]))], 1ull);
  __syncthreads();
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void noalloc_bstart_kernel(const unsigned long long* hist, uint64_t* bstart) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    bstart[0] = 0;
    for (int b = 0; b < kBuckets; ++b) bstart[b + 1] = bstart[b] + hist[b];
  }
}

}  // namespace
}  // namespace byo

extern "C" byo_status byo_bfs_noalloc(uint32_t n, uint64_t m, const uint64_t* offsets, const uint32_t* col,
                                      uint32_t source, uint32_t* levels, uint32_t* parents, const byo_sched* sched,
                                      void* stream) {
  clear_error();
  if (n == 0 || n > kNoallocMaxVertices) {
    set_error("byo_bfs_noalloc: n = %u is outside [1, %u], the size of the built-in scratch", n,
              kNoallocMaxVertices);
    return BYO_ERR_INVALID_ARG;
  }
  if (!offsets || !levels || (m && !col) || source >= n) {
    set_error("byo_bfs_noalloc: NULL offsets/levels/col or source >= n");
    return BYO_ERR_INVALID_ARG;
  }
  if (m && (reinterpret_cast<uintptr_t>(col) & 15)) {
    set_error("byo_bfs_noalloc: col must start on a 16-byte boundary");
    return BYO_ERR_INVALID_ARG;
  }
  SchedParams sp;
  BYO_RETURN_IF(sched_params(sched, &sp));
  void* base = nullptr;
  BYO_RETURN_IF(noalloc_scratch(&base));
  unsigned char* b = static_cast<unsigned char*>(base);
  BfsCtl* ctl = reinterpret_cast<BfsCtl*>(b + kNaCtl);
  uint64_t* bstart = reinterpret_cast<uint64_t*>(b + kNaBstart);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(b + kNaHist);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: clear what must start at zero
  BYO_CUDA(cudaMemsetAsync(ctl, 0, sizeof(BfsCtl), s));
  BYO_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kBuckets, s));
  noalloc_hist_kernel<<<(unsigned)sm_count() * 2, 256, 0, s>>>(offsets, n, hist);
  note_launch();
  BYO_CHECK_LAUNCH("noalloc_hist_kernel");
  noalloc_bstart_kernel<<<1, 32, 0, s>>>(hist, bstart);
  note_launch();
  BYO_CHECK_LAUNCH("noalloc_bstart_kernel");
  BfsArgs<CsrView<uint64_t>> args;
  args.g = CsrView<uint64_t>{n, m, offsets, col};
  args.src = source;
  args.level = levels;
  args.parent = parents;
  args.vis = reinterpret_cast<uint32_t*>(b + kNaVis);
  args.zmask = nullptr;
  args.fb = reinterpret_cast<uint32_t*>(b + kNaFb);
  args.queue = reinterpret_cast<uint32_t*>(b + kNaQueue);
  args.bstart = bstart;
  args.ctl = ctl;
  args.trace = reinterpret_cast<byo_bfs_iter*>(b + kNaTrace);
  args.sp = sp;
  args.limit_ns = timeout_ns();
  args.nw = (n + 31) / 32;
  if (parents) BYO_RETURN_IF((launch_bfs<CsrView<uint64_t>, true>(args, s)));
  else BYO_RETURN_IF((launch_bfs<CsrView<uint64_t>, false>(args, s)));
  uint32_t err = 0;
  BYO_CUDA(cudaMemcpyAsync(&err, &ctl->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  BYO_CUDA(cudaStreamSynchronize(s));
  if (err) return bfs_device_status(err, "byo_bfs_noalloc");
  return BYO_OK;
}
