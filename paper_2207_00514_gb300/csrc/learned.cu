// learned.cu -- the learned search radius (no counterpart in the paper: a
// proposal that only tightens each query's cutoff; a certification pass
// reruns every query whose cutoff fell below its component's found minimum,
// so the tree is exactly the plain method's).
//
//   features   8 per point and round (curve position, curve-neighbourhood
//              density, component size, the point's lower bound and its
//              component's cutoff), all from arrays the round already has;
//   network    8 -> 64 -> 64 -> 64 -> 1, ReLU, predicting the normalised log2
//              of the point's nearest other-component weight; inference with
//              BF16 weights and activations on the tensor cores (warp-level
//              mma m16n8k16, FP32 accumulation), training in FP32 (fused
//              forward + backward per 64-sample tile, Adam);
//   logging    (features, exact target) pairs from plain runs.
#include <cuda_bf16.h>

#include <cmath>

#include "traverse.cuh"

namespace emst {

constexpr int kIn = EMST_MLP_FEATURES;
constexpr int kHid = 64;
constexpr int kFeatureWindow = 4;  // curve neighbours on each side in features 3 and 4
constexpr int kOffMu = 0, kOffSigma = 8, kOffOutMu = 16, kOffOutSigma = 17, kOffMargin = 18;
constexpr int kOffW1 = 20;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid * kHid;
constexpr int kOffW4 = kOffB3 + kHid;
constexpr int kOffB4 = kOffW4 + kHid;
static_assert(kOffB4 + 1 == EMST_MLP_PARAMS, "parameter layout");

// ---------------------------------------------------------------------------
// Component sizes of the current labels (one atomic per run of equal labels
// within a warp).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_comp_sizes(const uint32_t *__restrict__ labels, int64_t n,
                                                    uint32_t *__restrict__ size) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t lab = labels[i];
  const unsigned mask = __match_any_sync(__activemask(), lab);
  if ((int)(threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(&size[lab], (uint32_t)__popc(mask));
}

// ---------------------------------------------------------------------------
// Features of point i (curve order) for the current round.
// ---------------------------------------------------------------------------
struct FeatArgs {
  const float4 *pts;
  const uint32_t *labels;
  const uint32_t *bound;
  const CompBest *comp;
  const uint2 *res;
  const uint32_t *comp_size;
  const uint32_t *box;  // ordered scene box
  const uint32_t *inst_of;
  const int64_t *offsets;
  int dim;
  int64_t n;
  int carried;  // res holds the previous round's lower bounds
};

__device__ __forceinline__ float safe_log2(float x) {
  return log2f(fminf(fmaxf(x, 1e-30f), 1e30f));
}

// Writes the 8 features; returns the component-level cutoff U and the point's
// lower bound (used to decide whether the query is skipped anyway).
__device__ __forceinline__ void point_features(const FeatArgs &A, int64_t i, float *f, float &U,
                                               float &lb) {
  const float4 p = A.pts[i];
  const float pc[3] = {p.x, p.y, p.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    f[d] = 0.f;
    if (d < A.dim) {
      const float lo = ordered_to_float(A.box[d]), hi = ordered_to_float(A.box[3 + d]);
      const float ext = hi - lo;
      f[d] = ext > 0.f ? (pc[d] - lo) / ext : 0.f;
    }
  }
  int64_t wlo = 0, whi = A.n;
  if (A.inst_of) {
    const uint32_t I = __ldg(A.inst_of + i);
    wlo = __ldg(A.offsets + I);
    whi = __ldg(A.offsets + I + 1);
  }
  float wmin = 1e30f, wsum = 0.f;
  int cnt = 0;
#pragma unroll
  for (int o = -kFeatureWindow; o <= kFeatureWindow; ++o) {
    const int64_t j = i + o;
    if (o == 0 || j < wlo || j >= whi) continue;
    const float4 c = __ldg(A.pts + j);
    const float w = sq_dist(p.x, p.y, p.z, c.x, c.y, c.z);
    wmin = fminf(wmin, w);
    wsum += w;
    ++cnt;
  }
  const uint32_t me = A.labels[i];
  U = bound_to_radius(A.bound[me]);
  const uint32_t cw =
      (uint32_t)(__ldcg(reinterpret_cast<const unsigned long long *>(&A.comp[me].key)) >> 32);
  U = fminf(U, bound_to_radius(cw));
  lb = A.carried ? __uint_as_float(A.res[i].x) : 0.f;
  f[3] = safe_log2(wmin);
  f[4] = safe_log2(cnt ? wsum / cnt : 1e30f);
  f[5] = log2f((float)__ldg(A.comp_size + me));
  f[6] = safe_log2(lb);
  f[7] = safe_log2(U);
}

// ---------------------------------------------------------------------------
// Tensor-core inference: one warp evaluates 32 points (two m16 row tiles).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float *c, const uint32_t *a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kW1Words = 12;  // row stride (32-bit words) of W1 in shared memory: 8 used
constexpr int kW2Words = 36;  // of W2 / W3: 32 used, padded against bank conflicts

struct MlpSmem {
  uint32_t w1[kHid * kW1Words];
  uint32_t w2[kHid * kW2Words];
  uint32_t w3[kHid * kW2Words];
  float b1[kHid], b2[kHid], b3[kHid], w4[kHid];
  float b4, mu[kIn], inv_sigma[kIn], omu, osig, margin;
  uint32_t x[8][32][4];  // per warp: 32 points x 8 BF16 features
  float y[8][32];
};

// Cooperative load of the network into shared memory (BF16 weights).
__device__ void load_mlp(MlpSmem &S, const float *__restrict__ P) {
  for (int t = threadIdx.x; t < kHid * kW1Words; t += blockDim.x) {
    const int r = t / kW1Words, w = t % kW1Words;
    S.w1[t] = w < kIn / 2 ? pack_bf16(P[kOffW1 + r * kIn + 2 * w], P[kOffW1 + r * kIn + 2 * w + 1]) : 0u;
  }
  for (int t = threadIdx.x; t < kHid * kW2Words; t += blockDim.x) {
    const int r = t / kW2Words, w = t % kW2Words;
    const bool used = w < kHid / 2;
    S.w2[t] = used ? pack_bf16(P[kOffW2 + r * kHid + 2 * w], P[kOffW2 + r * kHid + 2 * w + 1]) : 0u;
    S.w3[t] = used ? pack_bf16(P[kOffW3 + r * kHid + 2 * w], P[kOffW3 + r * kHid + 2 * w + 1]) : 0u;
  }
  for (int t = threadIdx.x; t < kHid; t += blockDim.x) {
    S.b1[t] = P[kOffB1 + t];
    S.b2[t] = P[kOffB2 + t];
    S.b3[t] = P[kOffB3 + t];
    S.w4[t] = P[kOffW4 + t];
  }
  if (threadIdx.x < kIn) {
    S.mu[threadIdx.x] = P[kOffMu + threadIdx.x];
    S.inv_sigma[threadIdx.x] = 1.0f / P[kOffSigma + threadIdx.x];
  }
  if (threadIdx.x == 0) {
    S.b4 = P[kOffB4];
    S.omu = P[kOffOutMu];
    S.osig = P[kOffOutSigma];
    S.margin = P[kOffMargin];
  }
}

// Stores this lane's normalised features (BF16) into the warp's input tile.
__device__ __forceinline__ void put_features(MlpSmem &S, int warp, int lane, const float *f) {
  float x[kIn];
#pragma unroll
  for (int k = 0; k < kIn; ++k) x[k] = (f[k] - S.mu[k]) * S.inv_sigma[k];
#pragma unroll
  for (int w = 0; w < kIn / 2; ++w) S.x[warp][lane][w] = pack_bf16(x[2 * w], x[2 * w + 1]);
}

// Bias + ReLU on the accumulators of n-tile nt (columns nt*8 + 2t, +1).
__device__ __forceinline__ void bias_relu(float *c, const float *bias, int nt, int t) {
  const float b0 = bias[nt * 8 + 2 * t], b1 = bias[nt * 8 + 2 * t + 1];
  c[0] = fmaxf(c[0] + b0, 0.f);
  c[1] = fmaxf(c[1] + b1, 0.f);
  c[2] = fmaxf(c[2] + b0, 0.f);
  c[3] = fmaxf(c[3] + b1, 0.f);
}

// The warp's 32 outputs (normalised prediction y) into S.y[warp].
__device__ void mlp_warp(MlpSmem &S, int warp, int lane) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
  for (int rt = 0; rt < 2; ++rt) {
    float c[8][4];
    {
      const uint32_t a[4] = {S.x[warp][16 * rt + g][t], S.x[warp][16 * rt + g + 8][t], 0u, 0u};
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
        mma_bf16(c[nt], a, S.w1[(nt * 8 + g) * kW1Words + t], 0u);
        bias_relu(c[nt], S.b1, nt, t);
      }
    }
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {
      const uint32_t *W = layer == 0 ? S.w2 : S.w3;
      const float *bias = layer == 0 ? S.b2 : S.b3;
      uint32_t a[4][4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {  // accumulators of n-tiles 2s, 2s+1 = A fragment of k-step s
        a[s][0] = pack_bf16(c[2 * s][0], c[2 * s][1]);
        a[s][1] = pack_bf16(c[2 * s][2], c[2 * s][3]);
        a[s][2] = pack_bf16(c[2 * s + 1][0], c[2 * s + 1][1]);
        a[s][3] = pack_bf16(c[2 * s + 1][2], c[2 * s + 1][3]);
      }
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t *row = W + (nt * 8 + g) * kW2Words;
#pragma unroll
        for (int s = 0; s < 4; ++s) mma_bf16(d, a[s], row[8 * s + t], row[8 * s + 4 + t]);
        bias_relu(d, bias, nt, t);
        c[nt][0] = d[0];
        c[nt][1] = d[1];
        c[nt][2] = d[2];
        c[nt][3] = d[3];
      }
    }
    // last layer (64 -> 1) in FP32 on the CUDA cores
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float w0 = S.w4[nt * 8 + 2 * t], w1 = S.w4[nt * 8 + 2 * t + 1];
      p0 = fmaf(c[nt][0], w0, fmaf(c[nt][1], w1, p0));
      p1 = fmaf(c[nt][2], w0, fmaf(c[nt][3], w1, p1));
    }
    p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
    p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
    if (t == 0) {
      S.y[warp][16 * rt + g] = p0 + S.b4;
      S.y[warp][16 * rt + g + 8] = p1 + S.b4;
    }
  }
}

// Inference on given features: out = predicted log2 weight (with the margin).
__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ feat, int64_t m,
                                                     const float *__restrict__ params,
                                                     float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem_raw);
  load_mlp(S, params);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles = (m + 31) / 32;
  for (int64_t tile = (int64_t)blockIdx.x * 8 + warp; tile < tiles; tile += (int64_t)gridDim.x * 8) {
    const int64_t i = tile * 32 + lane;
    float f[kIn];
#pragma unroll
    for (int k = 0; k < kIn; ++k) f[k] = i < m ? feat[i * kIn + k] : S.mu[k];
    put_features(S, warp, lane, f);
    __syncwarp();
    mlp_warp(S, warp, lane);
    __syncwarp();
    if (i < m) out[i] = S.y[warp][lane] * S.osig + S.omu + S.margin;
    __syncwarp();
  }
}

// Proposed cutoff of every point this round: 2^(predicted log2 weight).
__global__ void __launch_bounds__(256) k_predict(FeatArgs A, const float *__restrict__ params,
                                                 float *__restrict__ pred_r) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem_raw);
  load_mlp(S, params);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles = (A.n + 31) / 32;
  for (int64_t tile = (int64_t)blockIdx.x * 8 + warp; tile < tiles; tile += (int64_t)gridDim.x * 8) {
    const int64_t i = tile * 32 + lane;
    // a query whose lower bound exceeds its component's cutoff is skipped by
    // the search anyway: a warp whose 32 points are all skipped does no work
    bool skip = i >= A.n;
    if (!skip && A.carried) {
      const uint32_t me = A.labels[i];
      float U = bound_to_radius(A.bound[me]);
      const uint32_t cw =
          (uint32_t)(__ldcg(reinterpret_cast<const unsigned long long *>(&A.comp[me].key)) >> 32);
      U = fminf(U, bound_to_radius(cw));
      skip = __uint_as_float(A.res[i].x) > U;
    }
    if (__all_sync(0xffffffffu, skip)) continue;
    float f[kIn];
    float U = 0.f, lb = 0.f;
    if (i < A.n) point_features(A, i, f, U, lb);
    else {
#pragma unroll
      for (int k = 0; k < kIn; ++k) f[k] = S.mu[k];
    }
    put_features(S, warp, lane, f);
    __syncwarp();
    mlp_warp(S, warp, lane);
    __syncwarp();
    if (i < A.n) pred_r[i] = exp2f(S.y[warp][lane] * S.osig + S.omu + S.margin);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Training: loss and gradient of a batch (mean squared error on the
// normalised target), one 64-sample tile per CTA, accumulated with atomics.
// ---------------------------------------------------------------------------
constexpr int kTrainTile = 64;
constexpr int kPad = kHid + 1;

struct TrainSmem {
  float W1[kHid * kIn], b1[kHid], W2[kHid * kHid], b2[kHid], W3[kHid * kHid], b3[kHid], w4[kHid];
  float b4, mu[kIn], sigma[kIn], omu, osig;
  float x[kTrainTile][kIn];
  float h1[kTrainTile][kPad], h2[kTrainTile][kPad], h3[kTrainTile][kPad];
  float d1[kTrainTile][kPad], d2[kTrainTile][kPad], d3[kTrainTile][kPad];
  float dy[kTrainTile];
  float loss;
};

__global__ void __launch_bounds__(256) k_mlp_grad(const float *__restrict__ feat,
                                                  const float *__restrict__ target, int64_t m,
                                                  const float *__restrict__ P, float *grad,
                                                  float *loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
  const int tid = threadIdx.x;
  for (int t = tid; t < kHid * kHid; t += blockDim.x) {
    S.W2[t] = P[kOffW2 + t];
    S.W3[t] = P[kOffW3 + t];
  }
  for (int t = tid; t < kHid * kIn; t += blockDim.x) S.W1[t] = P[kOffW1 + t];
  for (int t = tid; t < kHid; t += blockDim.x) {
    S.b1[t] = P[kOffB1 + t];
    S.b2[t] = P[kOffB2 + t];
    S.b3[t] = P[kOffB3 + t];
    S.w4[t] = P[kOffW4 + t];
  }
  if (tid < kIn) {
    S.mu[tid] = P[kOffMu + tid];
    S.sigma[tid] = P[kOffSigma + tid];
  }
  if (tid == 0) {
    S.b4 = P[kOffB4];
    S.omu = P[kOffOutMu];
    S.osig = P[kOffOutSigma];
    S.loss = 0.f;
  }
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTrainTile;
  const int cnt = (int)(m - base < kTrainTile ? m - base : kTrainTile);
  const float inv_m = 1.0f / (float)m;
  for (int t = tid; t < kTrainTile * kIn; t += blockDim.x) {
    const int s = t / kIn, k = t % kIn;
    S.x[s][k] = s < cnt ? (feat[(base + s) * kIn + k] - S.mu[k]) / S.sigma[k] : 0.f;
  }
  __syncthreads();
  // forward
  for (int t = tid; t < kTrainTile * kHid; t += blockDim.x) {
    const int s = t / kHid, j = t % kHid;
    float z = S.b1[j];
    for (int k = 0; k < kIn; ++k) z = fmaf(S.W1[j * kIn + k], S.x[s][k], z);
    S.h1[s][j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  for (int t = tid; t < kTrainTile * kHid; t += blockDim.x) {
    const int s = t / kHid, j = t % kHid;
    float z = S.b2[j];
    for (int k = 0; k < kHid; ++k) z = fmaf(S.W2[j * kHid + k], S.h1[s][k], z);
    S.h2[s][j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  for (int t = tid; t < kTrainTile * kHid; t += blockDim.x) {
    const int s = t / kHid, j = t % kHid;
    float z = S.b3[j];
    for (int k = 0; k < kHid; ++k) z = fmaf(S.W3[j * kHid + k], S.h2[s][k], z);
    S.h3[s][j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  if (tid < kTrainTile) {
    const int s = tid;
    float y = S.b4;
    for (int j = 0; j < kHid; ++j) y = fmaf(S.w4[j], S.h3[s][j], y);
    float e = 0.f;
    if (s < cnt) e = y - (target[base + s] - S.omu) / S.osig;
    S.dy[s] = 2.0f * e * inv_m;
    atomicAdd(&S.loss, e * e * inv_m);
  }
  __syncthreads();
  // backward: dL/dz of each layer
  for (int t = tid; t < kTrainTile * kHid; t += blockDim.x) {
    const int s = t / kHid, j = t % kHid;
    S.d3[s][j] = S.h3[s][j] > 0.f ? S.dy[s] * S.w4[j] : 0.f;
  }
  __syncthreads();
  for (int t = tid; t < kTrainTile * kHid; t += blockDim.x) {
    const int s = t / kHid, k = t % kHid;
    float a = 0.f;
    for (int j = 0; j < kHid; ++j) a = fmaf(S.d3[s][j], S.W3[j * kHid + k], a);
    S.d2[s][k] = S.h2[s][k] > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int t = tid; t < kTrainTile * kHid; t += blockDim.x) {
    const int s = t / kHid, k = t % kHid;
    float a = 0.f;
    for (int j = 0; j < kHid; ++j) a = fmaf(S.d2[s][j], S.W2[j * kHid + k], a);
    S.d1[s][k] = S.h1[s][k] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // weight gradients, summed over the tile
  for (int t = tid; t < kHid * kHid; t += blockDim.x) {
    const int j = t / kHid, k = t % kHid;
    float g3 = 0.f, g2 = 0.f;
    for (int s = 0; s < kTrainTile; ++s) {
      g3 = fmaf(S.d3[s][j], S.h2[s][k], g3);
      g2 = fmaf(S.d2[s][j], S.h1[s][k], g2);
    }
    atomicAdd(grad + kOffW3 + t, g3);
    atomicAdd(grad + kOffW2 + t, g2);
  }
  for (int t = tid; t < kHid * kIn; t += blockDim.x) {
    const int j = t / kIn, k = t % kIn;
    float g1 = 0.f;
    for (int s = 0; s < kTrainTile; ++s) g1 = fmaf(S.d1[s][j], S.x[s][k], g1);
    atomicAdd(grad + kOffW1 + t, g1);
  }
  for (int j = tid; j < kHid; j += blockDim.x) {
    float gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, gw4 = 0.f;
    for (int s = 0; s < kTrainTile; ++s) {
      gb1 += S.d1[s][j];
      gb2 += S.d2[s][j];
      gb3 += S.d3[s][j];
      gw4 = fmaf(S.dy[s], S.h3[s][j], gw4);
    }
    atomicAdd(grad + kOffB1 + j, gb1);
    atomicAdd(grad + kOffB2 + j, gb2);
    atomicAdd(grad + kOffB3 + j, gb3);
    atomicAdd(grad + kOffW4 + j, gw4);
  }
  if (tid == 0) {
    float gb4 = 0.f;
    for (int s = 0; s < kTrainTile; ++s) gb4 += S.dy[s];
    atomicAdd(grad + kOffB4, gb4);
    atomicAdd(loss, S.loss);
  }
}

// Adam on the trainable parameters (from W1 on); clears the gradient.
__global__ void k_mlp_adam(float *__restrict__ P, float *__restrict__ grad, float *__restrict__ m1,
                           float *__restrict__ m2, int step, float lr, float beta1, float beta2,
                           float eps) {
  const int t = kOffW1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= EMST_MLP_PARAMS) return;
  const float g = grad[t];
  const float a = beta1 * m1[t] + (1.f - beta1) * g;
  const float b = beta2 * m2[t] + (1.f - beta2) * g * g;
  m1[t] = a;
  m2[t] = b;
  const float ah = a / (1.f - powf(beta1, (float)step));
  const float bh = b / (1.f - powf(beta2, (float)step));
  P[t] -= lr * ah / (sqrtf(bh) + eps);
  grad[t] = 0.f;
}

// ---------------------------------------------------------------------------
// Logging of training pairs during a plain run: for a sample of the points of
// each round (hash of position and round), the features and the exact log2
// weight of the nearest point in another component (an unbounded search).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mix32(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return (uint32_t)x;
}

__global__ void __launch_bounds__(128) k_log_samples(FeatArgs F, TravArgs T, int round, int every,
                                                     float *__restrict__ out_feat,
                                                     float *__restrict__ out_target,
                                                     int64_t capacity,
                                                     unsigned long long *count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F.n) return;
  if (mix32(((uint64_t)round << 40) ^ (uint64_t)i) % (uint32_t)every != 0u) return;
  uint32_t start = 0u;
  if (T.inst_of) {
    start = __ldg(T.inst_root + __ldg(T.inst_of + i));
    if (start == kInvalid) return;
  }
  float f[kIn], U, lb;
  point_features(F, i, f, U, lb);
  Query q;
  const float4 p = T.pts[i];
  q.px = p.x;
  q.py = p.y;
  q.pz = p.z;
  q.me = T.labels[i];
  q.radius = __int_as_float(0x7f800000);
  q.best = q.radius;
  q.bj = kInvalid;
  q.bid = kInvalid;
  uint32_t st_node[kStackDepth];
  float st_dist[kStackDepth];
  unsigned long long nv = 0;
  if (!explore<false, false, false>(q, start, T.nodes, T.nlabels, T.pts, T.labels, 1, F.n, st_node, st_dist, nv)) {
    atomicOr(T.status, kErrStack);
    return;
  }
  if (q.bj == kInvalid) return;  // the point's component is its whole instance
  const unsigned long long slot = atomicAdd(count, 1ull);
  if ((int64_t)slot >= capacity) return;
  for (int k = 0; k < kIn; ++k) out_feat[slot * kIn + k] = f[k];
  out_target[slot] = log2f(fmaxf(q.best, 1e-30f));
}

// ---------------------------------------------------------------------------
// Certification: a query that used cutoff r is exact for its component iff
// r >= the component's found minimum weight (every candidate it could still
// contribute is then covered); the others are listed for a rerun with the
// plain cutoff, which includes that minimum.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rerun_mark(const float *__restrict__ r_used,
                                                    const uint32_t *__restrict__ labels,
                                                    const CompBest *__restrict__ comp,
                                                    int64_t n, uint32_t *__restrict__ list,
                                                    uint32_t *counters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float r = r_used[i];
  if (r == __int_as_float(0x7f800000)) return;  // skipped or unbounded: nothing to certify
  const uint32_t wc = (uint32_t)(__ldcg(reinterpret_cast<const unsigned long long *>(&comp[labels[i]].key)) >> 32);
  const bool rerun = r < bound_to_radius(wc);
  const unsigned mask = __ballot_sync(__activemask(), true);
  const unsigned mine = __ballot_sync(mask, rerun);
  const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane == leader) {
    if (mine) base = atomicAdd(&counters[13], (uint32_t)__popc(mine));
    atomicAdd(&counters[15], (uint32_t)__popc(mask));
  }
  base = __shfl_sync(mask, base, leader);
  if (rerun) list[base + __popc(mine & ((1u << lane) - 1u))] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static FeatArgs feat_args(Problem &P, bool carried) {
  FeatArgs F;
  F.pts = P.pts;
  F.labels = P.labels;
  F.bound = P.bound;
  F.comp = P.comp;
  F.res = P.res;
  F.comp_size = P.comp_size;
  F.box = P.counters + 4;
  F.inst_of = P.inst_of;
  F.offsets = P.offsets;
  F.dim = P.dim;
  F.n = P.n;
  F.carried = carried ? 1 : 0;
  return F;
}

static bool g_mlp_attr_set[64] = {false};

static void set_mlp_attrs() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || g_mlp_attr_set[dev]) return;
  cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
  cudaFuncSetAttribute(k_predict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
  cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem));
  g_mlp_attr_set[dev] = true;
}

void launch_comp_sizes(Problem &P) {
  cudaMemsetAsync(P.comp_size, 0, sizeof(uint32_t) * (size_t)P.n, P.stream);
  k_comp_sizes<<<grid_for(P.n, 256), 256, 0, P.stream>>>(P.labels, P.n, P.comp_size);
  P.launches += 1;
}

void launch_predict(Problem &P, bool carried) {
  set_mlp_attrs();
  const int64_t tiles = (P.n + 31) / 32;
  int64_t g = (tiles + 7) / 8;
  if (g > sm_count() * 8) g = sm_count() * 8;
  k_predict<<<(unsigned)g, 256, sizeof(MlpSmem), P.stream>>>(feat_args(P, carried), P.mlp, P.pred_r);
  P.launches += 1;
}

void launch_rerun_mark(Problem &P) {
  k_rerun_mark<<<grid_for(P.n, 256), 256, 0, P.stream>>>(P.r_used, P.labels, P.comp, P.n,
                                                          P.rerun_list, P.counters);
  P.launches += 1;
}

void launch_log_samples(Problem &P, int round, bool carried) {
  if (!P.log_feat) return;
  TravArgs T;
  T.pts = P.pts;
  T.nodes = P.nodes;
  T.nlabels = P.nlabels;
  T.core2 = nullptr;
  T.ties = P.ties;
  T.labels = P.labels;
  T.bound = P.bound;
  T.radius_in = nullptr;
  T.leaf = P.leaf;
  T.inst_of = P.inst_of;
  T.inst_root = P.inst_root;
  T.offsets = P.offsets;
  T.res = P.res;
  T.comp = P.comp;
  T.n = P.n;
  T.status = P.counters + 1;
  T.queue = nullptr;
  T.visits = nullptr;
  T.queries = nullptr;
  T.seen = nullptr;
  T.pred_r = nullptr;
  T.r_used = nullptr;
  k_log_samples<<<grid_for(P.n, 128), 128, 0, P.stream>>>(feat_args(P, carried), T, round,
                                                           P.log_every, P.log_feat, P.log_target,
                                                           P.log_capacity, P.log_count);
  P.launches += 1;
}

}  // namespace emst

using namespace emst;

extern "C" {

int emst_mlp_forward(const float *features, int64_t m, const float *params, float *out_log2w,
                     void *stream) {
  if (m < 0 || (m > 0 && (!features || !params || !out_log2w))) return EMST_ERR_INVALID_ARG;
  if (m == 0) return EMST_OK;
  set_mlp_attrs();
  const int64_t tiles = (m + 31) / 32;
  int64_t g = (tiles + 7) / 8;
  if (g > sm_count() * 8) g = sm_count() * 8;
  k_mlp_forward<<<(unsigned)g, 256, sizeof(MlpSmem), (cudaStream_t)stream>>>(features, m, params,
                                                                            out_log2w);
  return cudaGetLastError() == cudaSuccess ? EMST_OK : EMST_ERR_CUDA;
}

int emst_mlp_grad(const float *features, const float *targets, int64_t m, const float *params,
                  float *grad, float *loss, void *stream) {
  if (m <= 0 || !features || !targets || !params || !grad || !loss) return EMST_ERR_INVALID_ARG;
  set_mlp_attrs();
  const int64_t tiles = (m + kTrainTile - 1) / kTrainTile;
  k_mlp_grad<<<(unsigned)tiles, 256, sizeof(TrainSmem), (cudaStream_t)stream>>>(features, targets,
                                                                               m, params, grad, loss);
  return cudaGetLastError() == cudaSuccess ? EMST_OK : EMST_ERR_CUDA;
}

int emst_mlp_adam(float *params, float *grad, float *m1, float *m2, int step, float lr,
                  float beta1, float beta2, float eps, void *stream) {
  if (!params || !grad || !m1 || !m2 || step < 1) return EMST_ERR_INVALID_ARG;
  const int count = EMST_MLP_PARAMS - kOffW1;
  k_mlp_adam<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m1, m2, step, lr,
                                                                    beta1, beta2, eps);
  return cudaGetLastError() == cudaSuccess ? EMST_OK : EMST_ERR_CUDA;
}

}  // extern "C"
