// Learned splitters for the semisort_< top level: a monotone CDF model
// trained on the GPU from the sorted top-level sample, inverted into integer
// splitter keys.  Bucketing itself stays exact key comparison, so the model
// only moves load balance, never the result.
//
// Model: a 1-32-32-1 perceptron in FP32 with positive weights (softplus of
// free parameters) and logistic hidden units, so f is non-decreasing:
//   h1 = sig(w1 x + c1), h2 = sig(W2 h1 + c2), f(x) = w3 . h2 + c3.
// Input x = (k - kmin) / (kmax - kmin); target = rank among the sample's
// light keys / their number.  Loss: mean squared error over 256 quantile
// points of the light keys of the 2^16-key sample; full-batch Adam.  Parameter layout (1153 floats): v1[32] | c1[32] | v2[32*32] (row j
// holds the weights into h2_j) | c2[32] | v3[32] | c3.
#pragma once
#include <cooperative_groups.h>
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
constexpr int kLearnPts = 256;     // training points drawn from the sorted sample
constexpr int kLearnSteps = 300;
constexpr float kLearnLr = 0.02f;

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
  uint32_t usable;       // 0 when the sample holds too few non-heavy keys to fit
  uint32_t steps_done;   // Adam steps the last training ran
  uint32_t light;        // non-heavy keys of the sample (the model's training population)
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

// Gradient contribution of the points [p0, p0 + NP) (those below npts),
// with 4 NP threads: four per point, each owning 8 of the 32 units of a layer
// (h1, h2 and the backward terms go through shared memory).  The sums over
// the block's points, in point order, are added to acc[0 .. kMlpParams)
// (gradient with respect to the weights w = softplus(v), before the chain
// rule through softplus) and acc[kMlpParams] (squared-error sum); `first`
// starts the sums from zero.  mw must hold the transformed weights.
template <int NP>
struct GradBufs {
  float h1[NP][kH + 1];
  float h2[NP][kH + 1];
  float d1[NP][kH + 1];
  float d2[NP][kH + 1];
  float e[NP];
  float x[NP];
  float se[NP];
};

template <int NP>
__device__ __forceinline__ void grad_block(const MlpSmem& mw, GradBufs<NP>& gs, const float* X, const float* T,
                                           uint32_t p0, uint32_t npts, float* acc, bool first) {
  const int tid = threadIdx.x;
  const int q = tid >> 2;    // point within the block
  const int part = tid & 3;  // which 8 units this thread owns
  const int u0 = part * 8;
  const uint32_t pt = p0 + q;
  const bool live = pt < npts;
  const float x = live ? X[pt] : 0.0f;
  const float t = live ? T[pt] : 0.0f;
  // forward
#pragma unroll
  for (int i = 0; i < 8; ++i) gs.h1[q][u0 + i] = sigmf(fmaf(mw.w1[u0 + i], x, mw.c1[u0 + i]));
  __syncthreads();
  float h1[kH];
#pragma unroll
  for (int i = 0; i < kH; ++i) h1[i] = gs.h1[q][i];
  float yp = 0.0f, h2v[8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const int j = u0 + jj;
    float z = mw.c2[j];
#pragma unroll
    for (int i = 0; i < kH; ++i) z = fmaf(mw.w2[j * kH + i], h1[i], z);
    h2v[jj] = sigmf(z);
    gs.h2[q][j] = h2v[jj];
    yp = fmaf(mw.w3[j], h2v[jj], yp);
  }
  // the four threads of a point are adjacent lanes
  yp += __shfl_xor_sync(kFull, yp, 1);
  yp += __shfl_xor_sync(kFull, yp, 2);
  const float r = yp + mw.c3 - t;
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
    gs.d2[q][j] = e * mw.w3[j] * h2v[jj] * (1.0f - h2v[jj]);
  }
  __syncthreads();
#pragma unroll
  for (int ii = 0; ii < 8; ++ii) {
    const int i = u0 + ii;
    float a = 0.0f;
#pragma unroll
    for (int j = 0; j < kH; ++j) a = fmaf(gs.d2[q][j], mw.w2[j * kH + i], a);
    const float h = gs.h1[q][i];
    gs.d1[q][i] = a * h * (1.0f - h);
  }
  __syncthreads();
  // sums over the block's points, in point order
  for (int k = tid; k < kMlpParams + 1; k += 4 * NP) {
    float g = first ? 0.0f : acc[k];
    if (k < kOffC1) {
      for (int p = 0; p < NP; ++p) g = fmaf(gs.d1[p][k], gs.x[p], g);
    } else if (k < kOffV2) {
      for (int p = 0; p < NP; ++p) g += gs.d1[p][k - kOffC1];
    } else if (k < kOffC2) {
      const int j = (k - kOffV2) / kH, i = (k - kOffV2) % kH;
      for (int p = 0; p < NP; ++p) g = fmaf(gs.d2[p][j], gs.h1[p][i], g);
    } else if (k < kOffV3) {
      for (int p = 0; p < NP; ++p) g += gs.d2[p][k - kOffC2];
    } else if (k < kOffC3) {
      for (int p = 0; p < NP; ++p) g = fmaf(gs.e[p], gs.h2[p][k - kOffV3], g);
    } else if (k == kOffC3) {
      for (int p = 0; p < NP; ++p) g += gs.e[p];
    } else {
      for (int p = 0; p < NP; ++p) g += gs.se[p];
    }
    acc[k] = g;
  }
  __syncthreads();
}

// Whether parameter k is a weight (softplus-transformed) rather than a bias.
__device__ __forceinline__ bool is_weight(int k) {
  return k < kOffC1 || (k >= kOffV2 && k < kOffC2) || (k >= kOffV3 && k < kOffC3);
}

// One Adam update (Kingma and Ba 2015) of parameter value pk with gradient g
// at step `step` (from 1); m and v are updated in place.
__device__ __forceinline__ float adam_update(float pk, float g, float& m, float& v, int step, float lr) {
  m = 0.9f * m + 0.1f * g;
  v = 0.999f * v + 0.001f * g * g;
  const float mh = m / (1.0f - powf(0.9f, (float)step));
  const float vh = v / (1.0f - powf(0.999f, (float)step));
  return pk - lr * mh / (sqrtf(vh) + 1e-8f);
}

// One full-batch gradient (step 0) or Adam step over L->npts points, one
// launch per step (the entry point for a single gradient).  Each CTA handles
// 64 points with 256 threads and writes its sums; the last CTA to finish adds
// the partial sums in CTA order (a fixed order, so the result is
// deterministic) and, when step > 0, applies Adam step `step`.  No CTA waits
// for another.
constexpr int kGradThreads = 256;  // threads per CTA of a gradient step
constexpr int kGradPts = 64;       // points per CTA
struct GradSmem {
  MlpSmem mw;
  GradBufs<kGradPts> gb;
  float acc[kMlpParams + 1];
  uint32_t last;
};

static __global__ void __launch_bounds__(kGradThreads) k_learn_step(LearnState* L, int step, float lr) {
  __shared__ GradSmem gs;
  const int tid = threadIdx.x;
  const uint32_t npts = L->npts;
  mlp_load(gs.mw, L->p);
  __syncthreads();
  grad_block<kGradPts>(gs.mw, gs.gb, L->x, L->t, blockIdx.x * kGradPts, npts, gs.acc, true);
  float* out = L->partial[blockIdx.x];
  for (int k = tid; k < kMlpParams + 1; k += kGradThreads) out[k] = gs.acc[k];
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
    if (is_weight(k)) g *= sigmf(pk);
    L->grad[k] = g;
    if (step > 0) L->p[k] = adam_update(pk, g, L->m[k], L->v[k], step, lr);
  }
  if (tid == 0) L->done = 0;
}

// Every Adam step in one launch: one thread-block cluster of kTrainCTAs CTAs.
// Each CTA keeps the parameters and Adam moments in shared memory and sums
// the gradient over its share of the points (blocks of kTrainPts points, CTA
// c taking blocks c, c + kTrainCTAs, ...) into one of two buffers (by step
// parity).  After one cluster barrier every CTA adds the kTrainCTAs partial
// sums in CTA order through distributed shared memory and applies the same
// Adam update to all parameters, so the copies stay identical without being
// exchanged; the other buffer is what the next step writes, and no CTA can
// reach the step after that before every CTA has passed the next barrier,
// so one barrier per step suffices.  The loss of a step (at the parameters
// it started from) is known to every CTA the same way, so an optional
// plateau stop -- every 25 steps, stop when the loss fell by less than 1% --
// is taken by all CTAs together.  Cluster barriers are hardware barriers of
// co-scheduled CTAs: no CTA spins on memory.
constexpr int kTrainCTAs = 8;
constexpr int kTrainPts = 32;
constexpr int kTrainThreads = 4 * kTrainPts;
constexpr int kPlateauEvery = 25;
struct TrainSmem {
  MlpSmem mw;
  GradBufs<kTrainPts> gb;
  float p[kMlpParams];
  float m[kMlpParams];
  float v[kMlpParams];
  float acc[2][kMlpParams + 1];
  float loss;
};

static __global__ void __cluster_dims__(kTrainCTAs, 1, 1) __launch_bounds__(kTrainThreads)
    k_learn_train(LearnState* L, uint32_t steps, float lr, uint32_t plateau) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& ts = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const uint32_t rank = cl.block_rank();
  const uint32_t npts = L->npts;
  for (int k = tid; k < kMlpParams; k += kTrainThreads) {
    ts.p[k] = L->p[k];
    ts.m[k] = L->m[k];
    ts.v[k] = L->v[k];
  }
  __syncthreads();
  float ref = 3.0e38f;
  uint32_t s = 1;
  for (; s <= steps; ++s) {
    float* acc = ts.acc[s & 1];
    mlp_load(ts.mw, ts.p);
    __syncthreads();
    bool first = true;
    for (uint32_t b = rank * kTrainPts; b < npts; b += kTrainCTAs * kTrainPts) {
      grad_block<kTrainPts>(ts.mw, ts.gb, L->x, L->t, b, npts, acc, first);
      first = false;
    }
    if (first) {  // no points for this CTA: it contributes zeros
      for (int k = tid; k < kMlpParams + 1; k += kTrainThreads) acc[k] = 0.0f;
    }
    cl.sync();
    // bias corrections of step s
    const float bc1 = 1.0f / (1.0f - powf(0.9f, (float)s));
    const float bc2 = 1.0f / (1.0f - powf(0.999f, (float)s));
    for (int k = tid; k < kMlpParams + 1; k += kTrainThreads) {
      float part[kTrainCTAs];
#pragma unroll
      for (int r = 0; r < kTrainCTAs; ++r) part[r] = cl.map_shared_rank(acc, (unsigned)r)[k];
      float g = 0.0f;
#pragma unroll
      for (int r = 0; r < kTrainCTAs; ++r) g += part[r];
      if (k == kMlpParams) {
        ts.loss = g / (float)npts;
        continue;
      }
      const float pk = ts.p[k];
      if (is_weight(k)) g *= sigmf(pk);
      const float mk = 0.9f * ts.m[k] + 0.1f * g;
      const float vk = 0.999f * ts.v[k] + 0.001f * g * g;
      ts.m[k] = mk;
      ts.v[k] = vk;
      ts.p[k] = pk - lr * (mk * bc1) / (sqrtf(vk * bc2) + 1e-8f);
    }
    __syncthreads();
    if (plateau && s % kPlateauEvery == 0) {
      const float cur = ts.loss;  // identical in every CTA
      if (cur > 0.99f * ref) {
        ++s;
        break;
      }
      ref = cur;
    }
  }
  // every CTA holds the same parameters; CTA 0 writes them back
  if (rank == 0) {
    for (int k = tid; k < kMlpParams; k += kTrainThreads) {
      L->p[k] = ts.p[k];
      L->m[k] = ts.m[k];
      L->v[k] = ts.v[k];
    }
    if (tid == 0) L->steps_done = s - 1;
  }
  cl.sync();  // no CTA leaves while another may still read its buffers
}

// Exclusive maximum over the block's threads (-1 for thread 0); wtmp holds at
// least 33 ints of shared memory.  Contains __syncthreads.
__device__ __forceinline__ int block_exclusive_max(int v, int* wtmp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc = t > inc ? t : inc;
  }
  if (lane == 31) wtmp[w] = inc;
  __syncthreads();
  int before = -1;
  for (int j = 0; j < w; ++j) before = wtmp[j] > before ? wtmp[j] : before;
  const int up = __shfl_up_sync(kFull, inc, 1);
  if (lane > 0) before = up > before ? up : before;
  (void)nw;
  __syncthreads();
  return before;
}

// Training data and initial parameters from the sorted top-level sample S
// (kBigSample keys).  Heavy keys -- keys whose sample run reaches
// tau = kBigSample / n_L, the first min(n_L, 512) of them in key order, which
// the splitter step turns into equality buckets (Sec. 3.1) -- are left out,
// so the model fits the distribution of the light keys, whose mass the range
// buckets share.  With the m' light sample keys compacted in order into tmp,
// point m < kLearnPts (256) is x_m = (tmp[r_m] - kmin) / (kmax - kmin) and
// t_m = (r_m + 0.5) / m' with r_m = floor((m + 1/2) m' / kLearnPts); kmin and
// kmax are the whole sample's extremes.  With fewer than 2 kLearnPts light
// sample keys the model is not used (usable = 0).  The initial first-layer units spread
// their centres evenly over [0, 1]; the rest is seeded.  n_L is the top
// segment's, or lbits_fixed when nonzero.  One CTA of 1024 threads, 64
// consecutive sample positions each.
template <class K>
__global__ void __launch_bounds__(1024) k_learn_prep(const K* S, LearnState* L, uint64_t seed, const Seg* top,
                                                     K* tmp, uint32_t lbits_fixed) {
  __shared__ uint32_t excl[kBigSample / 32];  // bit per position: start of a run left out of the training data
  __shared__ uint32_t scan_tmp[33];
  __shared__ int max_tmp[33];
  constexpr uint32_t PER = kBigSample / 1024;
  const uint32_t tid = threadIdx.x;
  // n_L of the top segment, or a fixed one (batched calls: one model for all instances)
  const uint32_t lbits = lbits_fixed ? lbits_fixed : (top->lbits ? top->lbits : 1);
  const uint32_t nl = 1u << lbits;
  const uint32_t tau = kBigSample / nl > 2 ? kBigSample / nl : 2;
  const uint32_t hcap = hcap_of(lbits);
  const uint32_t i0 = tid * PER;
  auto run_start = [&](uint32_t i) { return i == 0 || !KeyT<K>::eq(S[i], S[i - 1]); };
  auto heavy_start = [&](uint32_t i) { return i + tau - 1 < kBigSample && KeyT<K>::eq(S[i + tau - 1], S[i]); };
  for (uint32_t j = tid; j < kBigSample / 32; j += blockDim.x) excl[j] = 0;
  uint32_t nhs = 0;
  int last = -1;
  for (uint32_t j = 0; j < PER; ++j) {
    const uint32_t i = i0 + j;
    if (run_start(i)) {
      last = (int)i;
      if (heavy_start(i)) ++nhs;
    }
  }
  uint32_t htot;
  uint32_t hidx = block_exclusive_scan(nhs, scan_tmp, &htot);  // its barriers order the bitmap reset
  for (uint32_t j = 0; j < PER; ++j) {
    const uint32_t i = i0 + j;
    if (run_start(i) && heavy_start(i)) {
      if (hidx < hcap) atomicOr(&excl[i >> 5], 1u << (i & 31));
      ++hidx;
    }
  }
  const int prev = block_exclusive_max(last, max_tmp);  // run start governing this range's first positions
  __syncthreads();
  auto light_at = [&](uint32_t i, int& cur) {
    if (run_start(i)) cur = (int)i;
    return !(cur >= 0 && ((excl[cur >> 5] >> (cur & 31)) & 1u));
  };
  uint32_t nlight = 0;
  {
    int cur = prev;
    for (uint32_t j = 0; j < PER; ++j) nlight += light_at(i0 + j, cur) ? 1u : 0u;
  }
  uint32_t ltot;
  uint32_t lpos = block_exclusive_scan(nlight, scan_tmp, &ltot);
  {
    int cur = prev;
    for (uint32_t j = 0; j < PER; ++j)
      if (light_at(i0 + j, cur)) tmp[lpos++] = S[i0 + j];
  }
  __syncthreads();  // tmp is global memory written by this block only
  const uint64_t kmin = (uint64_t)S[0], kmax = (uint64_t)S[kBigSample - 1];
  const float inv = kmax > kmin ? 1.0f / (float)(kmax - kmin) : 0.0f;
  const bool usable = kmax > kmin && ltot >= 2 * (uint32_t)kLearnPts;
  if (usable) {
    for (uint32_t m = tid; m < (uint32_t)kLearnPts; m += blockDim.x) {
      const uint32_t r = (uint32_t)(((uint64_t)(2 * m + 1) * ltot) / (2 * (uint64_t)kLearnPts));
      L->x[m] = (float)((uint64_t)tmp[r] - kmin) * inv;
      L->t[m] = ((float)r + 0.5f) / (float)ltot;
    }
  }
  for (int k = tid; k < kMlpParams; k += blockDim.x) {
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
  if (tid == 0) {
    L->kmin = kmin;
    L->kmax = kmax;
    L->npts = kLearnPts;
    L->done = 0;
    L->light = ltot;
    L->steps_done = 0;
    L->usable = usable ? 1u : 0u;
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
