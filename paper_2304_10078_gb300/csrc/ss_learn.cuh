// Learned splitters for the semisort_< top level: a monotone CDF model
// trained on the GPU from the sorted top-level sample, inverted into integer
// splitter keys.  Bucketing itself stays exact key comparison, so the model
// only moves load balance, never the result.
//
// Model: a 1-32-32-1 perceptron in FP32 with positive weights (softplus of
// free parameters) and logistic hidden units, so f is non-decreasing:
//   h1 = sig(w1 x + c1), h2 = sig(W2 h1 + c2), f(x) = w3 . h2 + c3.
// Input x = (k - kmin) / (kmax - kmin); target = rank / |S|.  Loss: mean
// squared error over 1024 quantile points of the 2^16-key sample; full-batch
// Adam.  Parameter layout (1153 floats): v1[32] | c1[32] | v2[32*32] (row j
// holds the weights into h2_j) | c2[32] | v3[32] | c3.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ss_common.cuh"
#include "ss_plan.h"

namespace ss {

constexpr int kH = 32;
constexpr int kMlpParams = 4 * kH + kH * kH + 1;  // 1153
constexpr int kOffV1 = 0, kOffC1 = kH, kOffV2 = 2 * kH, kOffC2 = 2 * kH + kH * kH, kOffV3 = 3 * kH + kH * kH,
              kOffC3 = 4 * kH + kH * kH;
constexpr int kGradThreads = 64;   // points per CTA of a gradient step
constexpr int kGradCTAsMax = 64;   // at most 4096 points
constexpr int kLearnPts = 1024;    // training points drawn from the sorted sample
constexpr int kLearnSteps = 800;
constexpr float kLearnLr = 0.01f;

struct LearnState {
  float p[kMlpParams];  // parameters
  float m[kMlpParams];  // Adam first moment
  float v[kMlpParams];  // Adam second moment
  float partial[kGradCTAsMax][kMlpParams + 1];  // per-CTA gradient and squared-error sum
  float grad[kMlpParams + 1];                   // last summed gradient and loss
  float x[kGradCTAsMax * kGradThreads];
  float t[kGradCTAsMax * kGradThreads];
  uint64_t kmin, kmax;   // key range of the normalization
  uint32_t npts;
  uint32_t done;         // CTAs finished in the current step (reset by the last one)
  uint32_t usable;       // 0 when the sample holds a single key
  uint32_t pad;
  uint64_t splitters[1u << kLessTopLog2];  // inverted splitters (key type of the call)
};

__device__ __forceinline__ float softplusf(float v) { return log1pf(expf(-fabsf(v))) + fmaxf(v, 0.0f); }
__device__ __forceinline__ float sigmf(float z) { return 1.0f / (1.0f + expf(-z)); }

// Model weights with the positivity transform applied, in shared memory.
struct MlpSmem {
  float w1[kH], c1[kH], w2[kH * kH], c2[kH], w3[kH], c3;
};

__device__ __forceinline__ void mlp_load(MlpSmem& s, const float* p) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    const float q = p[i];
    if (i < kOffC1)
      s.w1[i] = softplusf(q);
    else if (i < kOffV2)
      s.c1[i - kOffC1] = q;
    else if (i < kOffC2)
      s.w2[i - kOffV2] = softplusf(q);
    else if (i < kOffV3)
      s.c2[i - kOffC2] = q;
    else if (i < kOffC3)
      s.w3[i - kOffV3] = softplusf(q);
    else
      s.c3 = q;
  }
}

__device__ __forceinline__ float mlp_eval(const MlpSmem& s, float x) {
  float h1[kH];
#pragma unroll
  for (int i = 0; i < kH; ++i) h1[i] = sigmf(fmaf(s.w1[i], x, s.c1[i]));
  float y = s.c3;
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float z = s.c2[j];
#pragma unroll
    for (int i = 0; i < kH; ++i) z = fmaf(s.w2[j * kH + i], h1[i], z);
    y = fmaf(s.w3[j], sigmf(z), y);
  }
  return y;
}

// One full-batch gradient step over L->npts points.  Each CTA handles 64
// points (one per thread) and writes its gradient sums; the last CTA to
// finish adds the partial sums in CTA order (a fixed order, so the result is
// deterministic) and, when step > 0, applies Adam step `step`.  No CTA waits
// for another.
struct GradSmem {
  MlpSmem mw;
  float h1[kGradThreads][kH + 1];
  float h2[kGradThreads][kH + 1];
  float d1[kGradThreads][kH + 1];
  float d2[kGradThreads][kH + 1];
  float e[kGradThreads];
  float x[kGradThreads];
  float se[kGradThreads];
  uint32_t last;
};

static __global__ void __launch_bounds__(kGradThreads) k_learn_step(LearnState* L, int step, float lr) {
  __shared__ GradSmem gs;
  const int tid = threadIdx.x;
  const uint32_t npts = L->npts;
  mlp_load(gs.mw, L->p);
  __syncthreads();
  const uint32_t pt = blockIdx.x * kGradThreads + tid;
  const bool live = pt < npts;
  const float x = live ? L->x[pt] : 0.0f;
  const float t = live ? L->t[pt] : 0.0f;
  // forward
  float h1[kH];
#pragma unroll
  for (int i = 0; i < kH; ++i) h1[i] = sigmf(fmaf(gs.mw.w1[i], x, gs.mw.c1[i]));
  float y = gs.mw.c3;
  for (int j = 0; j < kH; ++j) {
    float z = gs.mw.c2[j];
#pragma unroll
    for (int i = 0; i < kH; ++i) z = fmaf(gs.mw.w2[j * kH + i], h1[i], z);
    const float h = sigmf(z);
    gs.h2[tid][j] = h;
    y = fmaf(gs.mw.w3[j], h, y);
  }
  // backward: e = dL/dy, d2 = dL/dz2, d1 = dL/dz1
  const float r = y - t;
  const float e = live ? 2.0f * r / (float)npts : 0.0f;
  gs.e[tid] = e;
  gs.x[tid] = x;
  gs.se[tid] = live ? r * r : 0.0f;
  float acc[kH];
#pragma unroll
  for (int i = 0; i < kH; ++i) acc[i] = 0.0f;
  for (int j = 0; j < kH; ++j) {
    const float h = gs.h2[tid][j];
    const float d = e * gs.mw.w3[j] * h * (1.0f - h);
    gs.d2[tid][j] = d;
#pragma unroll
    for (int i = 0; i < kH; ++i) acc[i] = fmaf(d, gs.mw.w2[j * kH + i], acc[i]);
  }
#pragma unroll
  for (int i = 0; i < kH; ++i) {
    gs.h1[tid][i] = h1[i];
    gs.d1[tid][i] = acc[i] * h1[i] * (1.0f - h1[i]);
  }
  __syncthreads();
  // per-CTA gradient sums over its points, in point order
  float* out = L->partial[blockIdx.x];
  for (int k = tid; k < kMlpParams + 1; k += kGradThreads) {
    float g = 0.0f;
    if (k < kOffC1) {
      for (int q = 0; q < kGradThreads; ++q) g = fmaf(gs.d1[q][k], gs.x[q], g);
    } else if (k < kOffV2) {
      for (int q = 0; q < kGradThreads; ++q) g += gs.d1[q][k - kOffC1];
    } else if (k < kOffC2) {
      const int j = (k - kOffV2) / kH, i = (k - kOffV2) % kH;
      for (int q = 0; q < kGradThreads; ++q) g = fmaf(gs.d2[q][j], gs.h1[q][i], g);
    } else if (k < kOffV3) {
      for (int q = 0; q < kGradThreads; ++q) g += gs.d2[q][k - kOffC2];
    } else if (k < kOffC3) {
      for (int q = 0; q < kGradThreads; ++q) g = fmaf(gs.e[q], gs.h2[q][k - kOffV3], g);
    } else if (k == kOffC3) {
      for (int q = 0; q < kGradThreads; ++q) g += gs.e[q];
    } else {
      for (int q = 0; q < kGradThreads; ++q) g += gs.se[q];
    }
    out[k] = g;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) gs.last = atomicAdd(&L->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!gs.last) return;
  __threadfence();
  for (int k = tid; k < kMlpParams + 1; k += kGradThreads) {
    float g = 0.0f;
    for (uint32_t c = 0; c < gridDim.x; ++c) g += reinterpret_cast<volatile float*>(L->partial[c])[k];
    if (k == kMlpParams) {
      L->grad[k] = g / (float)npts;  // mean squared error
      continue;
    }
    const float q = L->p[k];
    // chain rule through the positivity transform: softplus' = sigmoid
    if (k < kOffC1 || (k >= kOffV2 && k < kOffC2) || (k >= kOffV3 && k < kOffC3)) g *= sigmf(q);
    L->grad[k] = g;
    if (step > 0) {
      const float m = 0.9f * L->m[k] + 0.1f * g;
      const float v = 0.999f * L->v[k] + 0.001f * g * g;
      L->m[k] = m;
      L->v[k] = v;
      const float mh = m / (1.0f - powf(0.9f, (float)step));
      const float vh = v / (1.0f - powf(0.999f, (float)step));
      L->p[k] = q - lr * mh / (sqrtf(vh) + 1e-8f);
    }
  }
  if (tid == 0) L->done = 0;
}

// Training data and initial parameters from the sorted top-level sample S:
// x_m = (S[64 m + 32] - kmin) / (kmax - kmin), t_m = (64 m + 32.5) / 2^16 for
// m < 1024.  The initial first-layer units spread their centres evenly over
// [0, 1]; the rest is seeded.  One CTA.
template <class K>
__global__ void __launch_bounds__(1024) k_learn_prep(const K* S, LearnState* L, uint64_t seed) {
  const uint64_t kmin = (uint64_t)S[0], kmax = (uint64_t)S[kBigSample - 1];
  const float inv = kmax > kmin ? 1.0f / (float)(kmax - kmin) : 0.0f;
  constexpr uint32_t stride = kBigSample / kLearnPts;
  for (uint32_t m = threadIdx.x; m < kLearnPts; m += blockDim.x) {
    const uint32_t r = m * stride + stride / 2;
    L->x[m] = (float)((uint64_t)S[r] - kmin) * inv;
    L->t[m] = ((float)r + 0.5f) / (float)kBigSample;
  }
  for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) {
    const float u = (float)(mix64(seed ^ (0xC0FFEEull + (uint64_t)k)) >> 40) * (1.0f / 16777216.0f);
    float q;
    if (k < kOffC1)
      q = 16.0f;
    else if (k < kOffV2)
      q = -16.0f * ((float)(k - kOffC1) + 0.5f) / (float)kH;
    else if (k < kOffC2)
      q = -2.0f + 0.2f * (u - 0.5f);
    else if (k < kOffV3)
      q = -0.5f * (float)kH * 0.127f + ((float)(k - kOffC2) - 15.5f) / 4.0f;  // 0.127 ~ softplus(-2)
    else if (k < kOffC3)
      q = -2.74f;  // softplus ~ 2 / kH
    else
      q = -0.5f;
    L->p[k] = q;
    L->m[k] = 0.0f;
    L->v[k] = 0.0f;
  }
  if (threadIdx.x == 0) {
    L->kmin = kmin;
    L->kmax = kmax;
    L->npts = kLearnPts;
    L->done = 0;
    L->usable = kmax > kmin;
  }
}

// Splitter j (1 <= j < n_L): the smallest key k in [kmin, kmax] with
// f((k - kmin) / (kmax - kmin)) >= j / n_L, by bisection on the integer key
// domain (the model is evaluated in FP32; a non-monotone rounding step can
// only move a splitter, k_less_split makes the list non-decreasing).
template <class K>
__global__ void __launch_bounds__(256) k_learn_invert(LearnState* L, const Seg* top, uint32_t lbits) {
  __shared__ MlpSmem mw;
  mlp_load(mw, L->p);
  __syncthreads();
  if (top) lbits = top->lbits;  // the top segment's n_L (set by k_plan)
  if (lbits == 0) return;
  const uint32_t nl = 1u << lbits;
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (j >= nl) return;
  const uint64_t kmin = L->kmin, kmax = L->kmax;
  const float inv = kmax > kmin ? 1.0f / (float)(kmax - kmin) : 0.0f;
  const float tau = (float)j / (float)nl;
  uint64_t lo = kmin, hi = kmax;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (mlp_eval(mw, (float)(mid - kmin) * inv) < tau)
      lo = mid + 1;
    else
      hi = mid;
  }
  reinterpret_cast<K*>(L->splitters)[j - 1] = (K)lo;
}

// Key range of the normalization (for a model trained outside the pipeline).
static __global__ void k_learn_range(LearnState* L, uint64_t kmin, uint64_t kmax, uint32_t npts) {
  if (threadIdx.x == 0) {
    L->kmin = kmin;
    L->kmax = kmax;
    L->npts = npts;
    L->done = 0;
    L->usable = kmax > kmin;
  }
}

}  // namespace ss
