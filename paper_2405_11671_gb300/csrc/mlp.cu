// mlp.cu -- the schedule network: a 12 -> 32 -> 32 -> 5 ReLU MLP that maps the
// frontier features of one edgeMap iteration to a schedule action (not in the
// paper; it only chooses between equivalent execution paths).  Forward and
// backward passes, the weighted softmax cross-entropy loss and the Adam update
// are hand-written kernels; inference runs inside the BFS persistent loop
// (sched.cuh).
//
// Training kernel layout: one warp per strided subset of samples, lane j owning
// hidden unit j of both layers.  Each warp keeps its partial gradient in
// registers (row j of W1 and W2, column j of W3, the biases) and writes it once;
// a second kernel sums the per-warp partials in a fixed order, so the gradient
// is deterministic.
#include <math.h>
#include <string.h>

#include <vector>

#include "byo_internal.cuh"
#include "prof.cuh"
#include "sched.cuh"

struct byo_mlp {
  float* d_params = nullptr;  // kMlpParams
  float* d_grad = nullptr;    // kMlpParams
  float* d_m = nullptr;       // Adam first moment
  float* d_v = nullptr;       // Adam second moment
  float* d_partials = nullptr;
  int partial_warps = 0;
  uint64_t steps = 0;
};

namespace byo {

namespace {

constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHidden * kFeatures;
constexpr int kOffW2 = kOffB1 + kHidden;
constexpr int kOffB2 = kOffW2 + kHidden * kHidden;
constexpr int kOffW3 = kOffB2 + kHidden;
constexpr int kOffB3 = kOffW3 + kActions * kHidden;
constexpr int kTrainWarps = 256;  // warps of the gradient kernel
constexpr int kPartial = kMlpParams + 2;  // + loss numerator + weight sum

__global__ void mlp_grad_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                const int32_t* __restrict__ y, const float* __restrict__ wts, uint32_t B,
                                float* __restrict__ partials) {
  const uint32_t lane = lane_id();
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  float gW1[kFeatures], gW2[kHidden], gW3[kActions], gb3[kActions];
  float gb1 = 0.f, gb2 = 0.f, lsum = 0.f, wsum = 0.f;
#pragma unroll
  for (int i = 0; i < kFeatures; ++i) gW1[i] = 0.f;
#pragma unroll
  for (int i = 0; i < kHidden; ++i) gW2[i] = 0.f;
#pragma unroll
  for (int c = 0; c < kActions; ++c) gW3[c] = gb3[c] = 0.f;
  const float* W1 = P + kOffW1;
  const float* b1 = P + kOffB1;
  const float* W2 = P + kOffW2;
  const float* b2 = P + kOffB2;
  const float* W3 = P + kOffW3;
  const float* b3 = P + kOffB3;
  for (uint32_t i = gw; i < B; i += nwarps) {
    float x[kFeatures];
#pragma unroll
    for (int f = 0; f < kFeatures; ++f) x[f] = X[(size_t)i * kFeatures + f];
    float wi = wts ? wts[i] : 1.0f;
    int yi = y[i];
    float a1 = b1[lane];
#pragma unroll
    for (int f = 0; f < kFeatures; ++f) a1 = fmaf(W1[lane * kFeatures + f], x[f], a1);
    float h1 = fmaxf(a1, 0.f);
    float a2 = b2[lane];
#pragma unroll
    for (int k = 0; k < kHidden; ++k) a2 = fmaf(W2[lane * kHidden + k], __shfl_sync(0xFFFFFFFFu, h1, k), a2);
    float h2 = fmaxf(a2, 0.f);
    float z[kActions];
    float zmax = -INFINITY;
#pragma unroll
    for (int c = 0; c < kActions; ++c) {
      float t = W3[c * kHidden + lane] * h2;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
      z[c] = t + b3[c];
      zmax = fmaxf(zmax, z[c]);
    }
    float se = 0.f;
#pragma unroll
    for (int c = 0; c < kActions; ++c) se += expf(z[c] - zmax);
    float lse = zmax + logf(se);
    float dz[kActions];
#pragma unroll
    for (int c = 0; c < kActions; ++c) dz[c] = wi * (expf(z[c] - lse) - (c == yi ? 1.f : 0.f));
    if (lane == 0) {
      lsum += wi * (lse - z[yi]);
      wsum += wi;
    }
    float d2 = 0.f;
#pragma unroll
    for (int c = 0; c < kActions; ++c) {
      gW3[c] = fmaf(dz[c], h2, gW3[c]);
      gb3[c] += dz[c];
      d2 = fmaf(W3[c * kHidden + lane], dz[c], d2);
    }
    if (a2 <= 0.f) d2 = 0.f;
    gb2 += d2;
    float d1 = 0.f;
#pragma unroll
    for (int k = 0; k < kHidden; ++k) {
      float h1k = __shfl_sync(0xFFFFFFFFu, h1, k);
      float d2k = __shfl_sync(0xFFFFFFFFu, d2, k);
      gW2[k] = fmaf(d2, h1k, gW2[k]);
      d1 = fmaf(W2[k * kHidden + lane], d2k, d1);
    }
    if (a1 <= 0.f) d1 = 0.f;
    gb1 += d1;
#pragma unroll
    for (int f = 0; f < kFeatures; ++f) gW1[f] = fmaf(d1, x[f], gW1[f]);
  }
  float* out = partials + (size_t)gw * kPartial;
#pragma unroll
  for (int f = 0; f < kFeatures; ++f) out[kOffW1 + lane * kFeatures + f] = gW1[f];
  out[kOffB1 + lane] = gb1;
#pragma unroll
  for (int k = 0; k < kHidden; ++k) out[kOffW2 + lane * kHidden + k] = gW2[k];
  out[kOffB2 + lane] = gb2;
#pragma unroll
  for (int c = 0; c < kActions; ++c) out[kOffW3 + c * kHidden + lane] = gW3[c];
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < kActions; ++c) out[kOffB3 + c] = gb3[c];
    out[kMlpParams] = lsum;
    out[kMlpParams + 1] = wsum;
  }
}

// grad[p] = sum over warps of partials[w][p] / sum of weights (fixed order).
__global__ void mlp_reduce_kernel(const float* __restrict__ partials, int nwarps, float* __restrict__ grad,
                                  float* __restrict__ loss) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kPartial) return;
  double s = 0.0, ws = 0.0;
  for (int w = 0; w < nwarps; ++w) {
    s += (double)partials[(size_t)w * kPartial + p];
    ws += (double)partials[(size_t)w * kPartial + kMlpParams + 1];
  }
  if (ws <= 0.0) ws = 1.0;
  if (p < kMlpParams) grad[p] = (float)(s / ws);
  else if (p == kMlpParams) *loss = (float)(s / ws);
}

__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  float gi = g[p];
  float mi = b1 * m[p] + (1.f - b1) * gi;
  float vi = b2 * v[p] + (1.f - b2) * gi * gi;
  m[p] = mi;
  v[p] = vi;
  P[p] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void mlp_predict_kernel(const float* __restrict__ P, const float* __restrict__ X, uint32_t B,
                                   int32_t* __restrict__ out) {
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t lane = lane_id();
  for (uint32_t i = gw; i < B; i += nwarps) {
    float x[kFeatures];
#pragma unroll
    for (int f = 0; f < kFeatures; ++f) x[f] = X[(size_t)i * kFeatures + f];
    float h1 = P[kOffB1 + lane];
#pragma unroll
    for (int f = 0; f < kFeatures; ++f) h1 = fmaf(P[kOffW1 + lane * kFeatures + f], x[f], h1);
    h1 = fmaxf(h1, 0.f);
    float h2 = P[kOffB2 + lane];
#pragma unroll
    for (int k = 0; k < kHidden; ++k) h2 = fmaf(P[kOffW2 + lane * kHidden + k], __shfl_sync(0xFFFFFFFFu, h1, k), h2);
    h2 = fmaxf(h2, 0.f);
    int best = 0;
    float bz = 0.f;
#pragma unroll
    for (int c = 0; c < kActions; ++c) {
      float t = P[kOffW3 + c * kHidden + lane] * h2;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
      float z = t + P[kOffB3 + c];
      if (c == 0 || z > bz) {
        bz = z;
        best = c;
      }
    }
    if (lane == 0) out[i] = best;
  }
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

byo_status mlp_gradient(byo_mlp* m, const float* X, const int32_t* y, const float* w, uint32_t B, float* d_loss,
                        cudaStream_t s) {
  const int threads = 256;
  const int blocks = kTrainWarps * 32 / threads;
  mlp_grad_kernel<<<blocks, threads, 0, s>>>(m->d_params, X, y, w, B, m->d_partials); ::byo::note_launch();
  BYO_CHECK_LAUNCH("mlp_grad_kernel");
  mlp_reduce_kernel<<<(kPartial + 127) / 128, 128, 0, s>>>(m->d_partials, kTrainWarps, m->d_grad, d_loss); ::byo::note_launch();
  BYO_CHECK_LAUNCH("mlp_reduce_kernel");
  return BYO_OK;
}

byo_status check_mlp(const byo_mlp* m) {
  if (!m) {
    set_error("network handle is NULL");
    return BYO_ERR_INVALID_ARG;
  }
  return BYO_OK;
}

}  // namespace

const float* mlp_device_params(const byo_mlp* m) { return m ? m->d_params : nullptr; }

byo_status sched_params(const byo_sched* s, SchedParams* out) {
  byo_sched d = s ? *s : byo_sched_default();
  if (d.mode > BYO_SCHED_FIXED || (d.mode == BYO_SCHED_FIXED && d.action >= (uint32_t)kActions)) {
    set_error("byo_sched: unknown mode %u", d.mode);
    return BYO_ERR_INVALID_ARG;
  }
  auto log2_pow2 = [](uint32_t x, int* out) -> bool {
    if (x == 0 || (x & (x - 1))) return false;
    int l = 0;
    while ((1u << l) < x) ++l;
    *out = l;
    return true;
  };
  int bt = 0, bw = 0;
  if (!log2_pow2(d.thr_thread, &bt) || !log2_pow2(d.thr_warp, &bw) || bw < bt || bw > 31) {
    set_error("byo_sched: thr_thread and thr_warp must be powers of two with thr_thread <= thr_warp < 2^32");
    return BYO_ERR_INVALID_ARG;
  }
  if (!(d.alpha > 0.f) || !(d.beta > 0.f)) {
    set_error("byo_sched: alpha and beta must be positive");
    return BYO_ERR_INVALID_ARG;
  }
  if (d.mode == BYO_SCHED_LEARNED && !d.mlp) {
    set_error("byo_sched: LEARNED needs a network");
    return BYO_ERR_INVALID_ARG;
  }
  if (d.flags & ~(BYO_SCHED_NO_EARLY_EXIT | BYO_SCHED_SEQUENTIAL_MAPS)) {
    set_error("byo_sched: unknown flags 0x%x", d.flags);
    return BYO_ERR_INVALID_ARG;
  }
  if ((d.flags & BYO_SCHED_SEQUENTIAL_MAPS) && d.mode == BYO_SCHED_FIXED && d.action == (uint32_t)kActionSolo) {
    set_error("byo_sched: the single-CTA action maps lists with many threads (BYO_SCHED_SEQUENTIAL_MAPS)");
    return BYO_ERR_INVALID_ARG;
  }
  out->mode = (int)d.mode;
  out->fixed_action = (int)d.action;
  out->bt = bt;
  out->bw = bw;
  out->alpha = d.alpha;
  out->beta = d.beta;
  // whole-number constants (the usual case) let the device test in integers
  auto whole = [](float x) -> uint32_t { return (x >= 1.0f && x <= 1048576.0f && x == floorf(x)) ? (uint32_t)x : 0u; };
  out->alpha_i = whole(d.alpha);
  out->beta_i = whole(d.beta);
  out->w = d.mode == BYO_SCHED_LEARNED ? mlp_device_params(d.mlp) : nullptr;
  out->flags = d.flags;
  return BYO_OK;
}

}  // namespace byo

using namespace byo;

extern "C" {

uint32_t byo_mlp_num_params(void) { return (uint32_t)kMlpParams; }

byo_status byo_mlp_create(uint64_t seed, byo_mlp** out) {
  clear_error();
  if (!out) {
    set_error("byo_mlp_create: out is NULL");
    return BYO_ERR_INVALID_ARG;
  }
  *out = nullptr;
  byo_mlp* m = new (std::nothrow) byo_mlp();
  if (!m) {
    set_error("host allocation failed");
    return BYO_ERR_OUT_OF_MEMORY;
  }
  m->partial_warps = kTrainWarps;
  byo_status st = dev_alloc_t(&m->d_params, kMlpParams, "network parameters");
  if (st == BYO_OK) st = dev_alloc_t(&m->d_grad, kMlpParams, "network gradient");
  if (st == BYO_OK) st = dev_alloc_t(&m->d_m, kMlpParams, "Adam moment");
  if (st == BYO_OK) st = dev_alloc_t(&m->d_v, kMlpParams, "Adam moment");
  if (st == BYO_OK) st = dev_alloc_t(&m->d_partials, (size_t)kTrainWarps * kPartial + 4, "gradient partials");
  if (st != BYO_OK) {
    byo_mlp_destroy(m);
    return st;
  }
  // He-uniform initialisation from a SplitMix64 stream; biases zero
  std::vector<float> h(kMlpParams, 0.f);
  uint64_t state = seed;
  auto fill = [&](int off, int count, int fan_in) {
    float lim = sqrtf(6.0f / (float)fan_in);
    for (int i = 0; i < count; ++i) {
      double u = (double)(splitmix(state) >> 11) * (1.0 / 9007199254740992.0);
      h[off + i] = (float)((2.0 * u - 1.0) * lim);
    }
  };
  fill(kOffW1, kHidden * kFeatures, kFeatures);
  fill(kOffW2, kHidden * kHidden, kHidden);
  fill(kOffW3, kActions * kHidden, kHidden);
  cudaError_t e = cudaMemcpy(m->d_params, h.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, sizeof(float) * kMlpParams);
  if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, sizeof(float) * kMlpParams);
  if (e != cudaSuccess) {
    byo_mlp_destroy(m);
    return cuda_status(e, "byo_mlp_create");
  }
  *out = m;
  return BYO_OK;
}

byo_status byo_mlp_destroy(byo_mlp* m) {
  if (!m) return BYO_OK;
  dev_free(m->d_params);
  dev_free(m->d_grad);
  dev_free(m->d_m);
  dev_free(m->d_v);
  dev_free(m->d_partials);
  delete m;
  return BYO_OK;
}

byo_status byo_mlp_get_params(const byo_mlp* m, float* host_params) {
  clear_error();
  BYO_RETURN_IF(check_mlp(m));
  if (!host_params) {
    set_error("byo_mlp_get_params: NULL output");
    return BYO_ERR_INVALID_ARG;
  }
  BYO_CUDA(cudaMemcpy(host_params, m->d_params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  return BYO_OK;
}

byo_status byo_mlp_set_params(byo_mlp* m, const float* host_params) {
  clear_error();
  BYO_RETURN_IF(check_mlp(m));
  if (!host_params) {
    set_error("byo_mlp_set_params: NULL input");
    return BYO_ERR_INVALID_ARG;
  }
  BYO_CUDA(cudaMemcpy(m->d_params, host_params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
  BYO_CUDA(cudaMemset(m->d_m, 0, sizeof(float) * kMlpParams));
  BYO_CUDA(cudaMemset(m->d_v, 0, sizeof(float) * kMlpParams));
  m->steps = 0;
  return BYO_OK;
}

byo_status byo_mlp_loss_grad(byo_mlp* m, const float* X, const int32_t* y, const float* w, uint32_t B,
                             float* grad, float* host_loss, void* stream) {
  clear_error();
  BYO_RETURN_IF(check_mlp(m));
  if (B == 0 || !X || !y) {
    set_error("byo_mlp_loss_grad: empty batch or NULL inputs");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* d_loss = m->d_partials + (size_t)kTrainWarps * kPartial;
  BYO_RETURN_IF(mlp_gradient(m, X, y, w, B, d_loss, s));
  if (grad) BYO_CUDA(cudaMemcpyAsync(grad, m->d_grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice, s));
  if (host_loss) {
    BYO_CUDA(cudaMemcpyAsync(host_loss, d_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    BYO_CUDA(cudaStreamSynchronize(s));
  }
  return BYO_OK;
}

byo_status byo_mlp_train(byo_mlp* m, const float* X, const int32_t* y, const float* w, uint32_t B, uint32_t epochs,
                         float lr, float* host_loss, void* stream) {
  clear_error();
  BYO_RETURN_IF(check_mlp(m));
  if (B == 0 || !X || !y || !(lr > 0.f)) {
    set_error("byo_mlp_train: empty batch, NULL inputs or lr <= 0");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* d_loss = m->d_partials + (size_t)kTrainWarps * kPartial;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (uint32_t e = 0; e < epochs; ++e) {
    BYO_RETURN_IF(mlp_gradient(m, X, y, w, B, d_loss, s));
    ++m->steps;
    float c1 = 1.f - powf(b1, (float)m->steps), c2 = 1.f - powf(b2, (float)m->steps);
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(m->d_params, m->d_grad, m->d_m, m->d_v, lr, b1, b2,
                                                           eps, c1, c2); ::byo::note_launch();
    BYO_CHECK_LAUNCH("mlp_adam_kernel");
  }
  if (host_loss) {
    BYO_RETURN_IF(mlp_gradient(m, X, y, w, B, d_loss, s));
    BYO_CUDA(cudaMemcpyAsync(host_loss, d_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    BYO_CUDA(cudaStreamSynchronize(s));
  }
  return BYO_OK;
}

byo_status byo_mlp_predict(const byo_mlp* m, const float* X, uint32_t B, int32_t* actions, void* stream) {
  clear_error();
  BYO_RETURN_IF(check_mlp(m));
  if (B == 0) return BYO_OK;
  if (!X || !actions) {
    set_error("byo_mlp_predict: NULL inputs");
    return BYO_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mlp_predict_kernel<<<64, 256, 0, s>>>(m->d_params, X, B, actions); ::byo::note_launch();
  BYO_CHECK_LAUNCH("mlp_predict_kernel");
  return BYO_OK;
}

}  // extern "C"
