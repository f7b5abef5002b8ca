// msbfs.cu -- many graphs and many BFS sources in one persistent launch.
//
// A batch of graphs is stored as ONE container over the disjoint union of the
// members (member i owns vertex ids [base_i, base_i + n_i)), so every kernel of
// the library runs on all members at once and CC labels come out per member.
// Multi-source BFS runs up to 64 sources per member together with one bit per
// source (the edgeMap of Section 3.2 over 64 frontiers at once): bit j of a
// vertex's word means "reached from source j of this vertex's member".
//   top-down (sparse): for v with a non-empty frontier word, OR it into the
//                      unseen bits of every neighbour (atomicOr);
//   bottom-up (dense): every vertex with unseen bits ORs its neighbours'
//                      frontier words and stops early once all bits are set.
// The direction is chosen per level on the device (Beamer-style, from the
// frontier's edge count), and the whole traversal is one cooperative launch
// with bounded grid barriers.
#include <vector>

#include "byo_internal.cuh"
#include "container.cuh"
#include "prof.cuh"

namespace byo {

struct MsCtl {
  GridBar bar;
  uint32_t err;
  uint32_t levels;
  unsigned long long nf[2];  // vertices with a non-empty frontier word, by level parity
  unsigned long long mf[2];  // their degree sum
};

namespace {

constexpr int kMsThreads = 256;
constexpr uint32_t kMsWarpDeg = 128;  // bottom-up: vertices of at least this degree get a warp

template <typename G>
struct MsArgs {
  G g;
  const uint32_t* sources;  // global ids, S per member, member-major
  const uint32_t* member_base;
  uint32_t members, S;
  uint32_t* levels;         // S x n
  unsigned long long* seen;
  unsigned long long* visit;
  unsigned long long* next;
  MsCtl* ctl;
  uint64_t limit_ns;
  float alpha;
};

template <typename G>
__global__ void __launch_bounds__(kMsThreads) msbfs_kernel(MsArgs<G> a) {
  const uint32_t n = a.g.num_vertices();
  const uint64_t m = a.g.num_edges();
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t gthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint32_t lane = lane_id();
  const uint64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
  const unsigned long long full = a.S >= 64 ? ~0ull : ((1ull << a.S) - 1);
  MsCtl* ctl = a.ctl;
  for (uint64_t v = gtid; v < n; v += gthreads) {
    a.seen[v] = 0;
    a.visit[v] = 0;
    a.next[v] = 0;
  }
  for (uint64_t i = gtid; i < (uint64_t)a.S * n; i += gthreads) a.levels[i] = kInf;
  if (blockIdx.x == 0 && threadIdx.x < 2) {
    ctl->nf[threadIdx.x] = 0;
    ctl->mf[threadIdx.x] = 0;
  }
  if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
  for (uint64_t i = gtid; i < (uint64_t)a.members * a.S; i += gthreads) {
    uint32_t v = a.sources[i];
    uint32_t j = (uint32_t)(i % a.S);
    atomicOr(a.seen + v, 1ull << j);
    atomicOr(a.visit + v, 1ull << j);
    a.levels[(uint64_t)j * n + v] = 0;
  }
  if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
  // frontier statistics of level 0
  {
    unsigned long long cnt = 0, deg = 0;
    for (uint64_t v = gtid; v < n; v += gthreads)
      if (ld_cg(a.visit + v)) {
        ++cnt;
        deg += a.g.degree((uint32_t)v);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
      deg += __shfl_down_sync(0xFFFFFFFFu, deg, o);
    }
    if (lane == 0 && cnt) {
      atomicAdd(&ctl->nf[0], cnt);
      atomicAdd(&ctl->mf[0], deg);
    }
  }
  if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
  unsigned long long mseen = 0;  // edges of vertices that were frontier at some level
  const uint64_t t_begin = globaltimer();
  for (uint32_t L = 0;; ++L) {
    const int cur = L & 1;
    const unsigned long long nf = ld_cg(&ctl->nf[cur]), mf = ld_cg(&ctl->mf[cur]);
    if (nf == 0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->levels = L;
      break;
    }
    if (L > n || globaltimer() - t_begin > a.limit_ns) {
      if (threadIdx.x == 0) atomicCAS(&ctl->err, 0u, (uint32_t)BYO_ERR_TIMEOUT);
      return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->nf[cur ^ 1] = 0;
      ctl->mf[cur ^ 1] = 0;
    }
    mseen += mf;
    const bool top_down = (double)mf * (double)a.alpha < (double)(m > mseen ? m - mseen : 0) || L == 0;
    if (top_down) {
      // warps look at 32 vertices at a time for non-empty frontier words; each
      // frontier vertex then gets the whole warp, lanes over its neighbours
      for (uint64_t v0 = gwarp * 32; v0 < n; v0 += nwarps * 32) {
        const uint64_t v = v0 + lane;
        const unsigned long long f = v < n ? ld_cg(a.visit + v) : 0ull;
        uint32_t fm = __ballot_sync(0xFFFFFFFFu, f != 0);
        while (fm) {
          const int l = __ffs(fm) - 1;
          fm &= fm - 1;
          const unsigned long long fu = __shfl_sync(0xFFFFFFFFu, f, l);
          const Seg s = a.g.seg((uint32_t)(v0 + l));
          for (uint32_t k = lane; k < s.len; k += 32) {
            const uint32_t u = __ldg(s.p + k);
            const unsigned long long d = fu & ~ld_cg(a.seen + u);
            if (d) atomicOr(a.next + u, d);
          }
        }
      }
    } else {
      // a thread per vertex of degree < kMsWarpDeg with unseen bits, eight
      // neighbours' frontier words in flight per step; early exit once every
      // source has reached it
      for (uint64_t v = gtid; v < n; v += gthreads) {
        const unsigned long long sv = ld_cg(a.seen + v);
        if (sv == full) continue;
        const Seg s = a.g.seg((uint32_t)v);
        if (s.len >= kMsWarpDeg) continue;  // a warp takes it below
        unsigned long long acc = 0;
        for (uint32_t k = 0; k < s.len && (acc | sv) != full; k += 8) {
          unsigned long long w[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) w[j] = k + j < s.len ? ld_cg(a.visit + __ldg(s.p + k + j)) : 0ull;
#pragma unroll
          for (int j = 0; j < 8; ++j) acc |= w[j];
        }
        acc &= ~sv;
        if (acc) a.next[v] = acc;
      }
      // a warp per vertex of degree >= kMsWarpDeg (found 32 at a time): 128
      // neighbours per step, the words OR-ed across the warp
      for (uint64_t v0 = gwarp * 32; v0 < n; v0 += nwarps * 32) {
        const uint64_t v = v0 + lane;
        unsigned long long sv = 0;
        bool heavy = false;
        if (v < n && a.g.degree((uint32_t)v) >= kMsWarpDeg) {
          sv = ld_cg(a.seen + v);
          heavy = sv != full;
        }
        uint32_t hm = __ballot_sync(0xFFFFFFFFu, heavy);
        while (hm) {
          const int l = __ffs(hm) - 1;
          hm &= hm - 1;
          const uint32_t x = (uint32_t)(v0 + l);
          const unsigned long long sx = __shfl_sync(0xFFFFFFFFu, sv, l);
          const Seg s = a.g.seg(x);
          unsigned long long acc = 0;
          for (uint32_t k = 0; k < s.len; k += 128) {
            unsigned long long w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const uint32_t idx = k + 32 * j + lane;
              w[j] = idx < s.len ? ld_cg(a.visit + __ldg(s.p + idx)) : 0ull;
            }
            acc |= (w[0] | w[1]) | (w[2] | w[3]);
            const uint32_t lo = __reduce_or_sync(0xFFFFFFFFu, (uint32_t)acc);
            const uint32_t hi = __reduce_or_sync(0xFFFFFFFFu, (uint32_t)(acc >> 32));
            acc = ((unsigned long long)hi << 32) | lo;
            if ((acc | sx) == full) break;  // warp-uniform
          }
          acc &= ~sx;
          if (lane == 0 && acc) a.next[x] = acc;
        }
      }
    }
    if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
    // finalise: new frontier words, levels of newly reached (vertex, source) pairs
    // (the levels are written one source at a time across the warp, so that
    // the lanes' stores to a source's row of levels are consecutive)
    unsigned long long cnt = 0, deg = 0;
    for (uint64_t vb = gtid - lane; vb < n; vb += gthreads) {
      const uint64_t v = vb + lane;
      unsigned long long x = 0;
      if (v < n) {
        x = ld_cg(a.next + v);
        const unsigned long long sv = ld_cg(a.seen + v);
        x &= ~sv;
        a.visit[v] = x;
        if (x) {
          a.seen[v] = sv | x;
          a.next[v] = 0;
          ++cnt;
          deg += a.g.degree((uint32_t)v);
        }
      }
      unsigned long long any = ((unsigned long long)__reduce_or_sync(0xFFFFFFFFu, (uint32_t)(x >> 32)) << 32) |
                               __reduce_or_sync(0xFFFFFFFFu, (uint32_t)x);
      while (any) {
        const int j = __ffsll((long long)any) - 1;
        any &= any - 1;
        if ((x >> j) & 1ull) a.levels[(uint64_t)j * n + v] = L + 1;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
      deg += __shfl_down_sync(0xFFFFFFFFu, deg, o);
    }
    if (lane == 0 && cnt) {
      atomicAdd(&ctl->nf[cur ^ 1], cnt);
      atomicAdd(&ctl->mf[cur ^ 1], deg);
    }
    if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->err, a.limit_ns)) return;
  }
}

__global__ void shift_ids_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst, uint64_t k,
                                 const uint64_t* __restrict__ kpre, const uint32_t* __restrict__ base,
                                 const uint32_t* __restrict__ nmem, uint32_t members, uint32_t* gsrc, uint32_t* gdst,
                                 uint32_t* bad) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = members - 1;  // member of pair i: largest g with kpre[g] <= i
    while (lo < hi) {
      uint32_t mid = (lo + hi + 1) >> 1;
      if (kpre[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    uint32_t u = src[i], v = dst[i];
    if (u >= nmem[lo] || v >= nmem[lo]) {
      atomicOr(bad, 1u);
      u = v = 0;
    }
    gsrc[i] = base[lo] + u;
    gdst[i] = base[lo] + v;
  }
}

}  // namespace
}  // namespace byo

using namespace byo;

extern "C" byo_status byo_batch_build(uint32_t num_graphs, const uint32_t* host_n, const uint64_t* host_k,
                                      const uint32_t* src, const uint32_t* dst, uint32_t flags, void* stream,
                                      byo_graph** out) {
  clear_error();
  if (!out || !host_n || !host_k || num_graphs == 0) {
    set_error("byo_batch_build: NULL arguments or no graphs");
    return BYO_ERR_INVALID_ARG;
  }
  *out = nullptr;
  std::vector<uint32_t> base(num_graphs);
  std::vector<uint64_t> kpre(num_graphs + 1, 0);
  uint64_t ntot = 0;
  for (uint32_t i = 0; i < num_graphs; ++i) {
    base[i] = (uint32_t)ntot;
    ntot += host_n[i];
    kpre[i + 1] = kpre[i] + host_k[i];
  }
  if (ntot >= 0xFFFFFFFFull) {
    set_error("byo_batch_build: the members have 2^32 - 1 vertices or more in total");
    return BYO_ERR_INVALID_ARG;
  }
  const uint64_t k = kpre[num_graphs];
  if (k && (!src || !dst)) {
    set_error("byo_batch_build: NULL pair arrays");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t *gsrc = nullptr, *gdst = nullptr, *d_base = nullptr, *d_n = nullptr, *bad = nullptr;
  uint64_t* d_kpre = nullptr;
  byo_status st = tmp_alloc_t(&gsrc, k + 1, s, "batch pairs");
  if (st == BYO_OK) st = tmp_alloc_t(&gdst, k + 1, s, "batch pairs");
  if (st == BYO_OK) st = tmp_alloc_t(&d_base, num_graphs, s, "member bases");
  if (st == BYO_OK) st = tmp_alloc_t(&d_n, num_graphs, s, "member sizes");
  if (st == BYO_OK) st = tmp_alloc_t(&d_kpre, num_graphs + 1ull, s, "member pair offsets");
  if (st == BYO_OK) st = tmp_alloc_t(&bad, 1, s, "flag");
  uint32_t hbad = 0;
  if (st == BYO_OK) {
    cudaMemcpyAsync(d_base, base.data(), 4ull * num_graphs, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_n, host_n, 4ull * num_graphs, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_kpre, kpre.data(), 8ull * (num_graphs + 1), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(bad, 0, 4, s);
    if (k) {
      shift_ids_kernel<<<grid_for(k, 256), 256, 0, s>>>(src, dst, k, d_kpre, d_base, d_n, num_graphs, gsrc, gdst,
                                                         bad);
      note_launch();
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_status(e, "shift_ids_kernel");
    else if (hbad) {
      set_error("byo_batch_build: a member's vertex id is >= its n");
      st = BYO_ERR_INVALID_ARG;
    }
  }
  byo_graph* g = nullptr;
  if (st == BYO_OK) st = byo_graph_build((uint32_t)ntot, gsrc, gdst, k, flags, stream, &g);
  tmp_free(gsrc, s);
  tmp_free(gdst, s);
  tmp_free(d_n, s);
  tmp_free(d_kpre, s);
  tmp_free(bad, s);
  if (st == BYO_OK) {
    g->members = num_graphs;
    g->member_base = d_base;  // owned by the graph from now on (stream-ordered allocation)
    g->member_base_host = new (std::nothrow) uint32_t[num_graphs];
    if (!g->member_base_host) {
      byo_graph_destroy(g);
      set_error("host allocation failed");
      return BYO_ERR_OUT_OF_MEMORY;
    }
    for (uint32_t i = 0; i < num_graphs; ++i) g->member_base_host[i] = base[i];
    *out = g;
  } else {
    tmp_free(d_base, s);
  }
  return st;
}

extern "C" byo_status byo_batch_member_base(const byo_graph* g, uint32_t i, uint32_t* host_base) {
  clear_error();
  BYO_RETURN_IF(check_graph(g));
  if (!host_base) {
    set_error("byo_batch_member_base: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  uint32_t members = g->members ? g->members : 1;
  if (i >= members) {
    set_error("byo_batch_member_base: member %u of %u", i, members);
    return BYO_ERR_INVALID_ARG;
  }
  *host_base = g->members ? g->member_base_host[i] : 0;
  return BYO_OK;
}

extern "C" byo_status byo_msbfs(const byo_graph* gc, const uint32_t* host_sources, uint32_t num_sources,
                                uint32_t* levels, const byo_sched* sched, void* stream) {
  clear_error();
  BYO_RETURN_IF(ready_graph(gc, static_cast<cudaStream_t>(stream)));
  byo_graph* g = const_cast<byo_graph*>(gc);
  const uint32_t members = g->members ? g->members : 1;
  if (num_sources == 0 || num_sources > 64 || !host_sources || !levels) {
    set_error("byo_msbfs: need 1..64 sources per member, host sources and device levels");
    return BYO_ERR_INVALID_ARG;
  }
  std::vector<uint32_t> gs((size_t)members * num_sources);
  for (uint32_t i = 0; i < members; ++i) {
    uint32_t base = g->members ? g->member_base_host[i] : 0;
    uint32_t lim = g->members ? ((i + 1 < members ? g->member_base_host[i + 1] : g->n) - base) : g->n;
    for (uint32_t j = 0; j < num_sources; ++j) {
      uint32_t v = host_sources[(size_t)i * num_sources + j];
      if (v >= lim) {
        set_error("byo_msbfs: source %u of member %u is outside it", v, i);
        return BYO_ERR_INVALID_ARG;
      }
      gs[(size_t)i * num_sources + j] = base + v;
    }
  }
  const float alpha = sched ? sched->alpha : 15.0f;
  if (!(alpha > 0.0f)) {
    set_error("byo_msbfs: alpha must be positive");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!g->ms_seen) {
    BYO_RETURN_IF(dev_alloc_t(&g->ms_seen, 3ull * g->n + 1, "MS-BFS words"));
    BYO_RETURN_IF(dev_alloc(&g->ms_ctl, sizeof(MsCtl), "MS-BFS control"));
    BYO_CUDA(cudaMemset(g->ms_ctl, 0, sizeof(MsCtl)));
  }
  if (g->ms_src_cap < gs.size()) {
    dev_free(g->ms_src);
    g->ms_src = nullptr;
    g->ms_src_cap = 0;
    BYO_RETURN_IF(dev_alloc_t(&g->ms_src, gs.size(), "MS-BFS sources"));
    g->ms_src_cap = gs.size();
  }
  BYO_CUDA(cudaMemcpyAsync(g->ms_src, gs.data(), 4 * gs.size(), cudaMemcpyHostToDevice, s));
  MsCtl* ctl = static_cast<MsCtl*>(g->ms_ctl);
  byo_status st = with_view(g, [&](auto view) -> byo_status {
    using G = decltype(view);
    MsArgs<G> a;
    a.g = view;
    a.sources = g->ms_src;
    a.member_base = g->member_base;
    a.members = members;
    a.S = num_sources;
    a.levels = levels;
    a.seen = g->ms_seen;
    a.visit = g->ms_seen + g->n;
    a.next = g->ms_seen + 2ull * g->n;
    a.ctl = ctl;
    a.limit_ns = timeout_ns();
    a.alpha = alpha;
    auto fn = msbfs_kernel<G>;
    int per_sm = 0;
    BYO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMsThreads, 0));
    if (per_sm < 1) {
      set_error("msbfs_kernel cannot be resident");
      return BYO_ERR_CUDA;
    }
    void* kargs[] = {&a};
    BYO_CUDA(reset_barrier(&a.ctl->bar, s));
    ProfScope ps("msbfs_persistent", s);
    BYO_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3(per_sm * sm_count()), dim3(kMsThreads), kargs, 0, s));
    note_launch();
    return BYO_OK;
  });
  BYO_RETURN_IF(st);
  uint32_t err = 0;
  BYO_CUDA(cudaMemcpyAsync(&err, &ctl->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  BYO_CUDA(cudaStreamSynchronize(s));
  if (err) {
    cudaMemsetAsync(ctl, 0, sizeof(MsCtl), s);
    cudaStreamSynchronize(s);
    set_error("byo_msbfs: a device-side wait exceeded BYO_TIMEOUT_MS");
    return BYO_ERR_TIMEOUT;
  }
  return BYO_OK;
}
