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
constexpr int kGradCTAsMax = 64;   // at most 64 x 64 = 4096 points
constexpr int kLearnPts = 1024;    // training points drawn from the sorted sample
constexpr int kLearnSteps = 800;
constexpr float kLearnLr = 0.01f;

struct LearnState {
  float p[kMlpParams];  // parameters
  float m[kMlpParams];  // Adam first moment
  float v[kMlpParams];  // Adam second moment
  float partial[kGradCTAsMax][kMlpParams + 1];  // per-CTA gradient and squared-error sum
  float grad[kMlpParams + 1];                   // last summed gradient and loss
  float x[kGradCTAsMax * 64];
  float t[kGradCTAsMax * 64];
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
// points with 256 threads: four threads per point, each owning 8 of the 32
// units of a layer (h1, h2 and the backward terms go through shared memory).
// The CTA writes its gradient sums; the last CTA to finish adds the partial
// sums in CTA order (a fixed order, so the result is deterministic) and, when
// step > 0, applies Adam step `step`.  No CTA waits for another.
constexpr int kGradThreads = 256;  // threads per CTA of a gradient step
constexpr int kGradPts = 64;       // points per CTA
struct GradSmem {
  MlpSmem mw;
  float h1[kGradPts][kH + 1];
  float h2[kGradPts][kH + 1];
  float d1[kGradPts][kH + 1];
  float d2[kGradPts][kH + 1];
  float e[kGradPts];
  float x[kGradPts];
  float se[kGradPts];
  uint32_t last;
};

static __global__ void __launch_bounds__(kGradThreads) k_learn_step(LearnState* L, int step, float lr) {
  __shared__ GradSmem gs;
  const int tid = threadIdx.x;
  const uint32_t npts = L->npts;
  mlp_load(gs.mw, L->p);
  const int q = tid >> 2;         // point within the CTA
  const int part = tid & 3;       // which 8 units this thread owns
  const int u0 = part * 8;
  const uint32_t pt = blockIdx.x * kGradPts + q;
  const bool live = pt < npts;
  const float x = live ? L->x[pt] : 0.0f;
  const float t = live ? L->t[pt] : 0.0f;
  __syncthreads();
  // forward
#pragma unroll
  for (int i = 0; i < 8; ++i) gs.h1[q][u0 + i] = sigmf(fmaf(gs.mw.w1[u0 + i], x, gs.mw.c1[u0 + i]));
  __syncthreads();
  float h1[kH];
#pragma unroll
  for (int i = 0; i < kH; ++i) h1[i] = gs.h1[q][i];
  float yp = 0.0f, h2v[8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int j = u0 + jj;
    float z = gs.mw.c2[j];
#pragma unroll
    for (int i = 0; i < kH; ++i) z = fmaf(gs.mw.w2[j * kH + i], h1[i], z);
    h2v[jj] = sigmf(z);
    gs.h2[q][j] = h2v[jj];
    yp = fmaf(gs.mw.w3[j], h2v[jj], yp);
  }
  // the four threads of a point are adjacent lanes
  yp += __shfl_xor_sync(kFull, yp, 1);
  yp += __shfl_xor_sync(kFull, yp, 2);
  const float r = yp + gs.mw.c3 - t;
  const float e = live ? 2.0f * r / (float)npts : 0.0f;
  if (part == 0) {
    gs.e[q] = e;
    gs.x[q] = x;
    gs.se[q] = live ? r * r : 0.0f;
  }
  // backward: d2 = dL/dz2 for this thread's units, then d1 = dL/dz1
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int j = u0 + jj;
    gs.d2[q][j] = e * gs.mw.w3[j] * h2v[jj] * (1.0f - h2v[jj]);
  }
  __syncthreads();
#pragma unroll
  for (int ii = 0; ii < 8; ++ii) {
    const int i = u0 + ii;
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kH; ++j) acc = fmaf(gs.d2[q][j], gs.mw.w2[j * kH + i], acc);
    const float h = gs.h1[q][i];
    gs.d1[q][i] = acc * h * (1.0f - h);
  }
  __syncthreads();
  // per-CTA gradient sums over its points, in point order
  float* out = L->partial[blockIdx.x];
  for (int k = tid; k < kMlpParams + 1; k += kGradThreads) {
    float g = 0.0f;
    if (k < kOffC1) {
      for (int p = 0; p < kGradPts; ++p) g = fmaf(gs.d1[p][k], gs.x[p], g);
    } else if (k < kOffV2) {
      for (int p = 0; p < kGradPts; ++p) g += gs.d1[p][k - kOffC1];
    } else if (k < kOffC2) {
      const int j = (k - kOffV2) / kH, i = (k - kOffV2) % kH;
      for (int p = 0; p < kGradPts; ++p) g = fmaf(gs.d2[p][j], gs.h1[p][i], g);
    } else if (k < kOffV3) {
      for (int p = 0; p < kGradPts; ++p) g += gs.d2[p][k - kOffC2];
    } else if (k < kOffC3) {
      for (int p = 0; p < kGradPts; ++p) g = fmaf(gs.e[p], gs.h2[p][k - kOffV3], g);
    } else if (k == kOffC3) {
      for (int p = 0; p < kGradPts; ++p) g += gs.e[p];
    } else {
      for (int p = 0; p < kGradPts; ++p) g += gs.se[p];
    }
    out[k] = g;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) gs.last = atomicAdd(&L->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!gs.last) return;
  __threadfence();
  const uint32_t nc = gridDim.x;
  for (int k = tid; k < kMlpParams + 1; k += kGradThreads) {
    // L2 loads of the CTAs' sums, eight in flight at a time, added in CTA order
    float g = 0.0f;
    for (uint32_t c0 = 0; c0 < nc; c0 += 8) {
      float v[8];
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) v[u] = c0 + u < nc ? __ldcg(&L->partial[c0 + u][k]) : 0.0f;
#pragma unroll
      for (uint32_t u = 0; u < 8; ++u) g += v[u];
    }
    if (k == kMlpParams) {
      L->grad[k] = g / (float)npts;  // mean squared error
      continue;
    }
    const float pk = L->p[k];
    // chain rule through the positivity transform: softplus' = sigmoid
    if (k < kOffC1 || (k >= kOffV2 && k < kOffC2) || (k >= kOffV3 && k < kOffC3)) g *= sigmf(pk);
    L->grad[k] = g;
    if (step > 0) {
      const float m = 0.9f * L->m[k] + 0.1f * g;
      const float vv = 0.999f * L->v[k] + 0.001f * g * g;
      L->m[k] = m;
      L->v[k] = vv;
      const float mh = m / (1.0f - powf(0.9f, (float)step));
      const float vh = vv / (1.0f - powf(0.999f, (float)step));
      L->p[k] = pk - lr * mh / (sqrtf(vh) + 1e-8f);
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
