// sched.cuh -- per-iteration edgeMap schedule: direction (sparse/push vs
// dense/pull, Section 3.2; the cutoff uses degree and num_edges, Section 6.3)
// and the push iteration's degree bins.  Three deciders share one action set:
//   HEURISTIC  Beamer-style switch: push -> pull when the frontier's edges
//              exceed the unvisited edges / alpha; pull -> push when the
//              frontier has fewer than n / beta vertices.
//   LEARNED    a 12 -> 32 -> 32 -> 5 ReLU network over the frontier
//              features picks the action (evaluated by one warp of every CTA
//              inside the persistent loop) among those the level allows: any
//              push variant; pull only where the Beamer tests would pull
//              (frontier edges > unvisited edges / alpha, or |F| >= n / beta),
//              so that a misprediction never pulls a small frontier; the
//              single-CTA push only for small frontiers.
//   PUSH/PULL  fixed.
// Schedules never change results, only which kernel path runs.
#pragma once

#include "byo_internal.cuh"

namespace byo {

constexpr int kFeatures = 12;
constexpr int kHidden = 32;
// 0 pull; 1 push (thr_thread, thr_warp); 2 push (4, 128); 3 push (64, 4096);
// 4 push run by one CTA alone for as many consecutive levels as the schedule
// keeps choosing it (no grid barrier between those levels)
constexpr int kActions = 5;
constexpr int kActionSolo = 4;
// The network may choose the single-CTA action only for frontiers this small
// (in edges); beyond it one CTA cannot beat the grid whatever the network says.
constexpr uint64_t kSoloMaxEdges = 16384;
constexpr uint32_t kSoloMaxVertices = 1024;  // the shared-memory frontier of a solo run
constexpr int kMlpParams = kHidden * kFeatures + kHidden + kHidden * kHidden + kHidden + kActions * kHidden + kActions;

struct SchedParams {
  int mode;
  int fixed_action;
  int bt, bw;  // log2 of thr_thread / thr_warp
  float alpha, beta;
  uint32_t alpha_i, beta_i;  // alpha and beta when they are whole numbers (<= 2^20), else 0
  const float* w;  // MLP parameters (LEARNED): global on the host side, the CTA's staged copy in kernels
  uint32_t flags;  // BYO_SCHED_NO_EARLY_EXIT | BYO_SCHED_SEQUENTIAL_MAPS
};

// A CTA's shared-memory copy of the network, read once per launch so that
// the per-level inference costs shared-memory latency.  The weight matrices
// are stored transposed (input-major: element [i][j] of W at i * rows + j),
// so that the 32 lanes, one per hidden unit, read 32 consecutive words
// (no bank conflicts).  Every caller of sched_decide in LEARNED mode stages
// the network first.
__shared__ float g_sched_w[kMlpParams];

__device__ __forceinline__ void sched_stage_weights(SchedParams& sp) {
  if (sp.mode != BYO_SCHED_LEARNED || sp.w == nullptr) return;
  constexpr int o1 = kHidden * kFeatures, o2 = o1 + kHidden, o3 = o2 + kHidden * kHidden;
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    int d = i;
    if (i < o1) d = (i % kFeatures) * kHidden + i / kFeatures;                  // W1 [32 x 12]
    else if (i >= o2 && i < o3) d = o2 + ((i - o2) % kHidden) * kHidden + (i - o2) / kHidden;  // W2 [32 x 32]
    g_sched_w[d] = __ldg(sp.w + i);
  }
  __syncthreads();
  sp.w = g_sched_w;
}

struct SchedFeatures {
  uint32_t nf;
  uint64_t mf;
  uint64_t nu;
  uint64_t mu;
  uint64_t n;
  uint64_t m;
  uint32_t h[4];
};

// Host: validate a byo_sched and turn it into kernel parameters.
byo_status sched_params(const byo_sched* s, SchedParams* out);
// Host: device pointer of a network's FP32 parameters (packed as in the oracle).
const float* mlp_device_params(const byo_mlp* m);

__device__ __forceinline__ float u64_to_float(uint64_t v) {
  return fmaf((float)(uint32_t)(v >> 32), 4294967296.0f, (float)(uint32_t)v);
}

// The 12 network inputs, all in [0, ~1]: log-scaled sizes, ratios and the
// degree histogram of the frontier.  Host code that builds training samples
// from byo_bfs_iter records computes the same quantities (in double
// precision; the network does not depend on the last bits).  On the device
// they are on the critical path of every level, so they use the hardware's
// approximate base-2 logarithm and division (each accurate to a few ulp).
__device__ __forceinline__ void sched_feature_vector(const SchedFeatures& f, float* x) {
  x[0] = __log2f(1.0f + (float)f.nf) * (1.0f / 32.0f);
  x[1] = __log2f(1.0f + u64_to_float(f.mf)) * (1.0f / 40.0f);
  x[2] = __log2f(1.0f + u64_to_float(f.nu)) * (1.0f / 32.0f);
  x[3] = __log2f(1.0f + u64_to_float(f.mu)) * (1.0f / 40.0f);
  x[4] = __log2f(1.0f + u64_to_float(f.n)) * (1.0f / 32.0f);
  x[5] = __log2f(1.0f + u64_to_float(f.m)) * (1.0f / 40.0f);
  x[6] = __fdividef((float)f.nf, u64_to_float(f.n ? f.n : 1));
  x[7] = __fdividef(u64_to_float(f.mf), u64_to_float(f.mf + f.mu + 1));
  const float inv = __fdividef(1.0f, (float)(f.nf ? f.nf : 1));
  for (int k = 0; k < 4; ++k) x[8 + k] = (float)f.h[k] * inv;
}

__device__ __forceinline__ void sched_bins(const SchedParams& sp, int action, int* bt, int* bw) {
  if (sp.flags & BYO_SCHED_SEQUENTIAL_MAPS) {  // every frontier vertex in the thread bin
    *bt = kBuckets - 1;
    *bw = kBuckets - 1;
    return;
  }
  switch (action) {
    case 2: *bt = 2; *bw = 7; break;
    case 3: *bt = 6; *bw = 12; break;
    default: *bt = sp.bt; *bw = sp.bw; break;
  }
}

// Warp-collective (all 32 lanes of one warp); returns the action on every lane.
__device__ __forceinline__ int sched_decide(const SchedParams& sp, const SchedFeatures& f, int prev_dir) {
  if (sp.mode == BYO_SCHED_FIXED) return sp.fixed_action;
  if (sp.mode == BYO_SCHED_PUSH) return 1;
  if (sp.mode == BYO_SCHED_PULL) return 0;
  // The decision sits on the critical path of every level, and this part's
  // FP64 pipe is narrow: the two Beamer tests (as products, alpha and beta >
  // 0) run on lane 0 alone and reach the other lanes by a shuffle.
  const uint32_t lane = lane_id();
  uint32_t tests = 0;
  if (lane == 0) {
    // push -> pull: mf * alpha > mu; pull -> push: nf * beta < n (exact in
    // 128-bit integers for whole-number constants)
    const bool p2p = sp.alpha_i ? (unsigned __int128)f.mf * sp.alpha_i > (unsigned __int128)f.mu
                                : (double)f.mf * (double)sp.alpha > (double)f.mu;
    const bool small = sp.beta_i ? (uint64_t)f.nf * sp.beta_i < f.n : (double)f.nf * (double)sp.beta < (double)f.n;
    tests = (p2p ? 1u : 0u) | (small ? 2u : 0u);
  }
  tests = __shfl_sync(0xFFFFFFFFu, tests, 0);
  const int beamer = prev_dir == 1 ? ((tests & 1u) ? 0 : 1) : ((tests & 2u) ? 1 : 0);
  if (sp.mode == BYO_SCHED_HEURISTIC || sp.w == nullptr) return beamer;
  // LEARNED: lane j owns hidden unit j of both layers
  float x[kFeatures];
  sched_feature_vector(f, x);
  // the staged copy, named directly so that its reads are shared-memory loads
  const float* W1 = g_sched_w;
  const float* b1 = W1 + kHidden * kFeatures;
  const float* W2 = b1 + kHidden;
  const float* b2 = W2 + kHidden * kHidden;
  const float* W3 = b2 + kHidden;
  const float* b3 = W3 + kActions * kHidden;
  // four independent partial sums per layer keep the FMA chains short (this
  // runs on the critical path of every BFS level)
  float a1[4] = {b1[lane], 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int i = 0; i < kFeatures; ++i) a1[i & 3] = fmaf(W1[i * kHidden + lane], x[i], a1[i & 3]);  // staged transposed
  const float h1 = fmaxf((a1[0] + a1[1]) + (a1[2] + a1[3]), 0.0f);
  float a2[4] = {b2[lane], 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < kHidden; ++k)
    a2[k & 3] = fmaf(W2[k * kHidden + lane], __shfl_sync(0xFFFFFFFFu, h1, k), a2[k & 3]);
  const float h2 = fmaxf((a2[0] + a2[1]) + (a2[2] + a2[3]), 0.0f);
  const bool solo_ok = f.mf <= kSoloMaxEdges && f.nf <= kSoloMaxVertices && !(sp.flags & BYO_SCHED_SEQUENTIAL_MAPS);
  // pull only where either Beamer test would pull
  const bool pull_ok = (tests & 1u) || !(tests & 2u);
  int best = -1;  // action 1 is always allowed
  float bestz = 0.0f;
#pragma unroll
  for (int c = 0; c < kActions; ++c) {
    float t = W3[c * kHidden + lane] * h2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
    const float z = t + b3[c];
    const bool ok = c == 0 ? pull_ok : (c == kActionSolo ? solo_ok : true);
    if (ok && (best < 0 || z > bestz)) {
      bestz = z;
      best = c;
    }
  }
  return best;
}

}  // namespace byo
