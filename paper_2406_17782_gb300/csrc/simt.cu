// simt.cu -- FP32 SIMT kernels: the decoder used as the accuracy anchor, the
// training forward/backward passes of decoder and encoder (Sec. 4.2-4.3,
// loss of Eq. 9-11), Adam, and FP64 image-wide error reductions.
//
// All reductions run in a fixed order (owner-computes partial sums per CTA,
// then a fixed-order sum over CTAs), so repeated runs are bitwise identical.
#include <cmath>

#include "fabric_internal.h"
#include "train_common.cuh"

namespace fab {
namespace {

constexpr float kLeaky = 0.01f;       // encoder residual-block activation slope

// Writes the 71 decoder inputs of point p into x[i * stride + r].
__device__ __forceinline__ void build_inputs(const fabric_gbuffer &g, int64_t p, const float *lat, float *x,
                                             int stride, int r) {
  for (int i = 0; i < kLatent; ++i) x[i * stride + r] = lat[i];
  float f[16];
  octaves_accurate(g.u[p], f);
  for (int i = 0; i < 16; ++i) x[(32 + i) * stride + r] = f[i];
  octaves_accurate(g.v[p], f);
  for (int i = 0; i < 16; ++i) x[(48 + i) * stride + r] = f[i];
  x[64 * stride + r] = (logf(fmaxf(g.radius[p], kRFloor)) - kLogRC0) * kLogRInvC1;
  for (int i = 0; i < 3; ++i) {
    x[(65 + i) * stride + r] = g.wi[3 * p + i];
    x[(68 + i) * stride + r] = g.wo[3 * p + i];
  }
}

// ---------------------------------------------------------------------------
// FP32 decoder forward: one point per thread, weights in shared memory,
// activations feature-major in shared memory (each thread owns a column).
// ---------------------------------------------------------------------------
constexpr int kFwdThreads = 64;

struct FwdArgs {
  fabric_gbuffer g;
  const DevMaterial *mats;
  int n_mat;
  const float *latents;
  int n_lat;
  const float *dec;
  float *rgb, *comps, *y_raw;
  int *status;
};

__device__ __forceinline__ void dense_col(const float *W, const float *b, int n_out, int n_in, const float *in,
                                          float *out, int t, bool relu) {
  for (int o = 0; o < n_out; ++o) {
    float acc = b[o];
    const float *w = W + o * n_in;
#pragma unroll 8
    for (int i = 0; i < n_in; ++i) acc = fmaf(w[i], in[i * kFwdThreads + t], acc);
    out[o * kFwdThreads + t] = relu ? fmaxf(acc, 0.0f) : acc;
  }
}

__global__ void __launch_bounds__(kFwdThreads) decoder_fp32_kernel(const FwdArgs a) {
  extern __shared__ float sm[];
  float *W = sm;
  float *bufA = W + ((kDecParams + 3) & ~3);
  float *bufB = bufA + kDecIn * kFwdThreads;
  for (int i = threadIdx.x; i < kDecParams; i += blockDim.x) W[i] = a.dec[i];
  __syncthreads();
  const int t = threadIdx.x;
  const int64_t p = (int64_t)blockIdx.x * kFwdThreads + t;
  if (p >= a.g.n) return;
  const int mat = a.g.material[p];
  const bool need_mat = a.rgb != nullptr;
  if (mat >= a.n_lat || (need_mat && mat >= a.n_mat)) {
    atomicOr(a.status, kStatusBadMaterial);
    const float nan = __int_as_float(0x7FC00000);
    if (a.y_raw) reinterpret_cast<float4 *>(a.y_raw)[p] = make_float4(nan, nan, nan, nan);
    if (a.comps) reinterpret_cast<float4 *>(a.comps)[p] = make_float4(nan, nan, nan, nan);
    if (a.rgb)
      for (int ch = 0; ch < 3; ++ch) a.rgb[3 * p + ch] = nan;
    return;
  }
  build_inputs(a.g, p, a.latents + (int64_t)mat * kLatent, bufA, kFwdThreads, t);
  dense_col(W + kOffW1, W + kOffB1, kHidden, kDecIn, bufA, bufB, t, true);
  dense_col(W + kOffW2, W + kOffB2, kHidden, kHidden, bufB, bufA, t, true);
  dense_col(W + kOffW3, W + kOffB3, kHidden, kHidden, bufA, bufB, t, true);
  float y[4];
  for (int k = 0; k < kOut; ++k) {
    float acc = W[kOffB4 + k];
    for (int i = 0; i < kHidden; ++i) acc = fmaf(W[kOffW4 + k * kHidden + i], bufB[i * kFwdThreads + t], acc);
    y[k] = acc;
  }
  if (a.y_raw) reinterpret_cast<float4 *>(a.y_raw)[p] = make_float4(y[0], y[1], y[2], y[3]);
  const float c0 = fmaxf(0.0f, y[0]), c1 = fmaxf(0.0f, y[1]);
  const float s0 = fmaxf(0.0f, expm1f(y[2]) / kSpecK), s1 = fmaxf(0.0f, expm1f(y[3]) / kSpecK);
  if (a.comps) reinterpret_cast<float4 *>(a.comps)[p] = make_float4(c0, c1, s0, s1);
  if (a.rgb) {
    const DevMaterial &m = a.mats[mat];
    for (int ch = 0; ch < 3; ++ch)
      a.rgb[3 * p + ch] = m.kd[0][ch] * c0 + m.kd[1][ch] * c1 + m.ks[0][ch] * s0 + m.ks[1][ch] * s1;
  }
}

// ---------------------------------------------------------------------------
// Decoder forward + backward over tiles of kTR rows (kBwdThreads per CTA).
// Either dy is given, or it comes from the Eq. 11 loss against `target`.
// Per-CTA parameter-gradient partials stay in shared memory and are written
// out once; dlat_rows receives each row's gradient w.r.t. its latent.
// ---------------------------------------------------------------------------
constexpr int kTR = 32;
constexpr int kBwdThreads = 256;
constexpr int kBwdWarps = kBwdThreads / 32;
constexpr int kRS = kTR + 1;   // row stride (bank-conflict padding)

struct BwdArgs {
  fabric_gbuffer g;
  const float *latents;
  int n_lat;
  const float *dec;
  const float *dy;       // [n][4] or null
  const float *target;   // [n][4] or null
  int loss_mode;         // FABRIC_LOSS_EQ11 or FABRIC_LOSS_RENDERED
  float inv_batch;       // 1/B for the loss
  float *partial;        // [grid][kDecParams]
  double *loss_partial;  // [grid]
  float *dlat_rows;      // [n][32]
  int *status;
};

__device__ __forceinline__ void layer_fwd(const float *W, const float *b, int n_out, int n_in, const float *in,
                                          bool relu_in, float *out) {
  // thread -> (output group, row): row r = lane, outputs o = og, og + kBwdWarps, ...
  const int r = threadIdx.x & 31, og = threadIdx.x >> 5;
  for (int o = og; o < n_out; o += kBwdWarps) {
    float acc = b[o];
    const float *w = W + o * n_in;
    for (int i = 0; i < n_in; ++i) {
      float v = in[i * kRS + r];
      if (relu_in) v = fmaxf(v, 0.0f);
      acc = fmaf(w[i], v, acc);
    }
    out[o * kRS + r] = acc;
  }
}

// din[i][r] = (sum_o W[o][i] dout[o][r]) * (mask ? (pre[i][r] > 0) : 1)
__device__ __forceinline__ void layer_bwd_input(const float *W, int n_out, int n_in, const float *dout,
                                                const float *pre, float *din, int i_limit) {
  const int r = threadIdx.x & 31, ig = threadIdx.x >> 5;
  for (int i = ig; i < i_limit; i += kBwdWarps) {
    float acc = 0.0f;
    for (int o = 0; o < n_out; ++o) acc = fmaf(W[o * n_in + i], dout[o * kRS + r], acc);
    if (pre) acc = pre[i * kRS + r] > 0.0f ? acc : 0.0f;
    din[i * kRS + r] = acc;
  }
}

// dW[o][i] += sum_r dout[o][r] * act(in[i][r]); db[o] += sum_r dout[o][r].
// Owner computes: thread t owns 4x4 blocks (o0..o0+3, i0..i0+3).
__device__ __forceinline__ void layer_bwd_weights(float *dW, float *db, int n_out, int n_in, const float *dout,
                                                  const float *in, bool relu_in) {
  const int ob = (n_out + 3) / 4, ib = (n_in + 3) / 4;
  for (int blk = threadIdx.x; blk < ob * ib; blk += kBwdThreads) {
    const int o0 = (blk / ib) * 4, i0 = (blk % ib) * 4;
    float acc[4][4] = {};
    for (int r = 0; r < kTR; ++r) {
      float d[4], x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        d[q] = (o0 + q < n_out) ? dout[(o0 + q) * kRS + r] : 0.0f;
        float v = (i0 + q < n_in) ? in[(i0 + q) * kRS + r] : 0.0f;
        x[q] = relu_in ? fmaxf(v, 0.0f) : v;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[q][s] = fmaf(d[q], x[s], acc[q][s]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (o0 + q < n_out && i0 + s < n_in) dW[(o0 + q) * n_in + i0 + s] += acc[q][s];
  }
  for (int o = threadIdx.x; o < n_out; o += kBwdThreads) {
    float acc = 0.0f;
    for (int r = 0; r < kTR; ++r) acc += dout[o * kRS + r];
    db[o] += acc;
  }
}

__global__ void __launch_bounds__(kBwdThreads) decoder_bwd_kernel(const BwdArgs a) {
  extern __shared__ float sm[];
  float *W = sm;
  float *dW = W + ((kDecParams + 3) & ~3);
  float *X = dW + ((kDecParams + 3) & ~3);   // [72][kRS]
  float *A1 = X + 72 * kRS;                   // pre-activations [64][kRS]
  float *A2 = A1 + 64 * kRS;
  float *A3 = A2 + 64 * kRS;
  float *Y = A3 + 64 * kRS;                   // [4][kRS] head, then dy
  float *D1 = Y + 4 * kRS;                    // [64][kRS]
  float *D2 = D1 + 64 * kRS;
  __shared__ double loss_red[kBwdThreads];
  for (int i = threadIdx.x; i < kDecParams; i += blockDim.x) {
    W[i] = a.dec[i];
    dW[i] = 0.0f;
  }
  double loss_acc = 0.0;
  const int64_t n_tiles = (a.g.n + kTR - 1) / kTR;
  const int t = threadIdx.x;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    __syncthreads();
    // ---- inputs
    if (t < kTR) {
      const int64_t p = tile * kTR + t;
      int mat = p < a.g.n ? (int)a.g.material[p] : -1;
      if (mat >= a.n_lat) {
        atomicOr(a.status, kStatusBadMaterial);
        mat = -1;
      }
      if (mat >= 0) {
        build_inputs(a.g, p, a.latents + (int64_t)mat * kLatent, X, kRS, t);
      } else {
        for (int i = 0; i < kDecIn; ++i) X[i * kRS + t] = 0.0f;
      }
      X[kDecIn * kRS + t] = mat >= 0 ? 1.0f : 0.0f;   // row-valid flag
    }
    __syncthreads();
    layer_fwd(W + kOffW1, W + kOffB1, kHidden, kDecIn, X, false, A1);
    __syncthreads();
    layer_fwd(W + kOffW2, W + kOffB2, kHidden, kHidden, A1, true, A2);
    __syncthreads();
    layer_fwd(W + kOffW3, W + kOffB3, kHidden, kHidden, A2, true, A3);
    __syncthreads();
    layer_fwd(W + kOffW4, W + kOffB4, kOut, kHidden, A3, true, Y);
    __syncthreads();
    // ---- output gradient
    if (t < kTR * kOut) {
      const int r = t % kTR, k = t / kTR;
      const int64_t p = tile * kTR + r;
      const bool valid = X[kDecIn * kRS + r] > 0.0f;
      float d = 0.0f;
      if (valid) {
        if (a.target) {
          d = loss_grad(k, Y[k * kRS + r], a.target[4 * p + k], a.g.wi[3 * p + 2], a.loss_mode, a.inv_batch,
                        &loss_acc);
        } else {
          d = a.dy[4 * p + k];
        }
      }
      Y[k * kRS + r] = d;
    }
    __syncthreads();
    // ---- backward
    layer_bwd_weights(dW + kOffW4, dW + kOffB4, kOut, kHidden, Y, A3, true);
    layer_bwd_input(W + kOffW4, kOut, kHidden, Y, A3, D1, kHidden);        // dA3
    __syncthreads();
    layer_bwd_weights(dW + kOffW3, dW + kOffB3, kHidden, kHidden, D1, A2, true);
    layer_bwd_input(W + kOffW3, kHidden, kHidden, D1, A2, D2, kHidden);    // dA2
    __syncthreads();
    layer_bwd_weights(dW + kOffW2, dW + kOffB2, kHidden, kHidden, D2, A1, true);
    layer_bwd_input(W + kOffW2, kHidden, kHidden, D2, A1, D1, kHidden);    // dA1
    __syncthreads();
    layer_bwd_weights(dW + kOffW1, dW + kOffB1, kHidden, kDecIn, D1, X, false);
    if (a.dlat_rows) {
      // d x[0:32] = W1[:, 0:32]^T dA1
      layer_bwd_input(W + kOffW1, kHidden, kDecIn, D1, nullptr, D2, kLatent);
      __syncthreads();
      for (int e = t; e < kTR * kLatent; e += kBwdThreads) {
        const int r = e / kLatent, i = e % kLatent;
        const int64_t p = tile * kTR + r;
        if (p < a.g.n) a.dlat_rows[p * kLatent + i] = D2[i * kRS + r];
      }
    }
  }
  __syncthreads();
  float *out = a.partial + (int64_t)blockIdx.x * kDecParams;
  for (int i = t; i < kDecParams; i += blockDim.x) out[i] = dW[i];
  loss_red[t] = loss_acc;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int k = 0; k < kBwdThreads; ++k) s += loss_red[k];
    a.loss_partial[blockIdx.x] = s;
  }
}

// Sum per-CTA partials in CTA order: out[j] = sum_c partial[c][j].
__global__ void reduce_partials_kernel(const float *__restrict__ partial, int n_part, int width,
                                       float *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= width) return;
  float s = 0.0f;
  for (int c = 0; c < n_part; ++c) s += partial[(int64_t)c * width + j];
  out[j] = s;
}

// 32 threads sum fixed strided subsets, then thread 0 sums the 32 in order.
__global__ void reduce_loss_kernel(const double *__restrict__ part, int n, double *__restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int c = threadIdx.x; c < n; c += 32) s += part[c];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 32; ++k) t += red[k];
    *out = t;
  }
}

// dlat[m][i] = sum over rows with material m (row order) of dlat_rows[row][i].
__global__ void __launch_bounds__(256) latent_segment_kernel(const uint16_t *__restrict__ mat, int64_t n,
                                                             const float *__restrict__ rows,
                                                             float *__restrict__ dlat) {
  const int m = blockIdx.x;
  __shared__ float red[256][kLatent + 1];
  float acc[kLatent];
#pragma unroll
  for (int i = 0; i < kLatent; ++i) acc[i] = 0.0f;
  // thread t takes rows t, t + 256, ... in order (coalesced across the
  // block), reading eight material ids ahead so that their loads overlap
  const int64_t step = blockDim.x;
  for (int64_t r = threadIdx.x; r < n; r += 8 * step) {
    int ids[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ids[q] = r + q * step < n ? (int)mat[r + q * step] : -1;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (ids[q] != m) continue;
      const float4 *src = reinterpret_cast<const float4 *>(rows + (r + q * step) * kLatent);
#pragma unroll
      for (int k = 0; k < kLatent / 4; ++k) {
        const float4 v = src[k];
        acc[4 * k] += v.x;
        acc[4 * k + 1] += v.y;
        acc[4 * k + 2] += v.z;
        acc[4 * k + 3] += v.w;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kLatent; ++i) red[threadIdx.x][i] = acc[i];
  __syncthreads();
  if (threadIdx.x < kLatent) {
    float s = 0.0f;
    for (int k = 0; k < 256; ++k) s += red[k][threadIdx.x];
    dlat[m * kLatent + threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Encoder (parameters -> latent), one material per CTA of 128 threads.
// acts (optional) [n][2][128] = pre-activations a1, a2 for the backward pass.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float lrelu(float x) { return x > 0.0f ? x : kLeaky * x; }

__device__ void material_features(const fabric_material &m, float *f) {
  for (int k = 0; k < kPatternSlots; ++k) f[k] = (m.pattern_id == k) ? 1.0f : 0.0f;
  f[kPatternSlots + 0] = m.twist_deg / 30.0f;
  f[kPatternSlots + 1] = m.incl_deg / 45.0f;
  f[kPatternSlots + 2] = m.alpha[0];
  f[kPatternSlots + 3] = m.beta[0];
  f[kPatternSlots + 4] = m.alpha[1];
  f[kPatternSlots + 5] = m.beta[1];
}

__global__ void material_features_kernel(const fabric_material *__restrict__ raw, int n, float *__restrict__ f) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n) material_features(raw[m], f + m * kEncIn);
}

__global__ void __launch_bounds__(kEncHidden) encoder_fwd_kernel(const float *__restrict__ feats,
                                                                 const float *__restrict__ enc,
                                                                 float *__restrict__ z, float *__restrict__ acts) {
  __shared__ float f[kEncIn], h1[kEncHidden], h2[kEncHidden];
  const int m = blockIdx.x, j = threadIdx.x;
  if (j < kEncIn) f[j] = feats[m * kEncIn + j];
  __syncthreads();
  float a1 = enc[kOffEb1 + j];
  for (int i = 0; i < kEncIn; ++i) a1 = fmaf(enc[kOffE1 + j * kEncIn + i], f[i], a1);
  h1[j] = lrelu(a1);
  __syncthreads();
  float a2 = enc[kOffEb2 + j] + h1[j];   // skip connection before the last activation
  for (int i = 0; i < kEncHidden; ++i) a2 = fmaf(enc[kOffE2 + j * kEncHidden + i], h1[i], a2);
  h2[j] = lrelu(a2);
  if (acts) {
    acts[(int64_t)m * 2 * kEncHidden + j] = a1;
    acts[(int64_t)m * 2 * kEncHidden + kEncHidden + j] = a2;
  }
  __syncthreads();
  if (j < kLatent) {
    float acc = enc[kOffEb3 + j];
    for (int i = 0; i < kEncHidden; ++i) acc = fmaf(enc[kOffE3 + j * kEncHidden + i], h2[i], acc);
    z[m * kLatent + j] = acc;
  }
}

// Per material: back-propagated pre-activation gradients da1, da2 and the
// activations h1, h2 into work [n][4][128].
__global__ void __launch_bounds__(kEncHidden) encoder_bwd_vec_kernel(const float *__restrict__ enc,
                                                                     const float *__restrict__ acts,
                                                                     const float *__restrict__ dz,
                                                                     float *__restrict__ work) {
  __shared__ float sdz[kLatent], da2s[kEncHidden];
  const int m = blockIdx.x, j = threadIdx.x;
  if (j < kLatent) sdz[j] = dz[m * kLatent + j];
  const float a1 = acts[(int64_t)m * 2 * kEncHidden + j];
  const float a2 = acts[(int64_t)m * 2 * kEncHidden + kEncHidden + j];
  __syncthreads();
  float dh2 = 0.0f;
  for (int k = 0; k < kLatent; ++k) dh2 = fmaf(enc[kOffE3 + k * kEncHidden + j], sdz[k], dh2);
  const float da2 = dh2 * (a2 > 0.0f ? 1.0f : kLeaky);
  da2s[j] = da2;
  __syncthreads();
  float dh1 = da2;   // through the skip
  for (int o = 0; o < kEncHidden; ++o) dh1 = fmaf(enc[kOffE2 + o * kEncHidden + j], da2s[o], dh1);
  const float da1 = dh1 * (a1 > 0.0f ? 1.0f : kLeaky);
  float *w = work + (int64_t)m * 4 * kEncHidden;
  w[j] = da1;
  w[kEncHidden + j] = da2;
  w[2 * kEncHidden + j] = lrelu(a1);
  w[3 * kEncHidden + j] = lrelu(a2);
}

// One thread per encoder parameter, materials summed in order.
__global__ void encoder_grad_kernel(const float *__restrict__ feats, int n, const float *__restrict__ dz,
                                    const float *__restrict__ work, float *__restrict__ denc) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kEncParams) return;
  float s = 0.0f;
  if (e < kOffEb1) {                       // E1[j][i]
    const int j = e / kEncIn, i = e % kEncIn;
    for (int m = 0; m < n; ++m) s += work[(int64_t)m * 512 + j] * feats[m * kEncIn + i];
  } else if (e < kOffE2) {                 // e1[j]
    const int j = e - kOffEb1;
    for (int m = 0; m < n; ++m) s += work[(int64_t)m * 512 + j];
  } else if (e < kOffEb2) {                // E2[j][i]
    const int j = (e - kOffE2) / kEncHidden, i = (e - kOffE2) % kEncHidden;
    for (int m = 0; m < n; ++m) s += work[(int64_t)m * 512 + 128 + j] * work[(int64_t)m * 512 + 256 + i];
  } else if (e < kOffE3) {                 // e2[j]
    const int j = e - kOffEb2;
    for (int m = 0; m < n; ++m) s += work[(int64_t)m * 512 + 128 + j];
  } else if (e < kOffEb3) {                // E3[k][i]
    const int k = (e - kOffE3) / kEncHidden, i = (e - kOffE3) % kEncHidden;
    for (int m = 0; m < n; ++m) s += dz[m * kLatent + k] * work[(int64_t)m * 512 + 384 + i];
  } else {                                 // e3[k]
    const int k = e - kOffEb3;
    for (int m = 0; m < n; ++m) s += dz[m * kLatent + k];
  }
  denc[e] = s;
}

// ---------------------------------------------------------------------------
// Adam (Kingma and Ba 2015) with bias correction.
// ---------------------------------------------------------------------------
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float bc1, float bc2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

// ---------------------------------------------------------------------------
// FP64 error statistics: fixed grid of partial sums, then one fixed-order sum.
// ---------------------------------------------------------------------------
constexpr int kErrBlocks = 512;
constexpr int kErrThreads = 256;

__global__ void __launch_bounds__(kErrThreads) err_partial_kernel(const float *__restrict__ a,
                                                                  const float *__restrict__ b, int64_t n,
                                                                  const float *__restrict__ w, int group,
                                                                  int w_stride, double *__restrict__ part) {
  __shared__ double s0[kErrThreads], s1[kErrThreads], s2[kErrThreads];
  double e2 = 0.0, b2 = 0.0, mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kErrThreads + threadIdx.x; i < n; i += (int64_t)kErrBlocks * kErrThreads) {
    const double wi = w ? (double)w[(i / group) * w_stride] : 1.0;
    const double d = ((double)a[i] - (double)b[i]) * wi;
    const double bb = (double)b[i] * wi;
    e2 += d * d;
    b2 += bb * bb;
    mx = fmax(mx, fabs(d));
  }
  s0[threadIdx.x] = e2;
  s1[threadIdx.x] = b2;
  s2[threadIdx.x] = mx;
  __syncthreads();
  for (int off = kErrThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      s0[threadIdx.x] += s0[threadIdx.x + off];
      s1[threadIdx.x] += s1[threadIdx.x + off];
      s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + off]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = s0[0];
    part[3 * blockIdx.x + 1] = s1[0];
    part[3 * blockIdx.x + 2] = s2[0];
  }
}

__global__ void err_final_kernel(const double *__restrict__ part, double *__restrict__ out) {
  if (threadIdx.x != 0) return;
  double e2 = 0.0, b2 = 0.0, mx = 0.0;
  for (int k = 0; k < kErrBlocks; ++k) {
    e2 += part[3 * k];
    b2 += part[3 * k + 1];
    mx = fmax(mx, part[3 * k + 2]);
  }
  out[0] = e2;
  out[1] = b2;
  out[2] = mx;
}

size_t fwd_smem_bytes() { return (((kDecParams + 3) & ~3) + (size_t)(kDecIn + kHidden) * kFwdThreads) * 4; }
size_t bwd_smem_bytes() {
  return (2 * (size_t)((kDecParams + 3) & ~3) + (size_t)(72 + 64 * 3 + 4 + 64 * 2) * kRS) * 4;
}

}  // namespace

cudaError_t launch_decoder_fp32(const fabric_gbuffer &g, const DevMaterial *mats, int n_mat, const float *latents,
                                const float *dec, float *rgb, float *comps, float *y_raw, int *status,
                                cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(decoder_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fwd_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  FwdArgs a;
  a.g = g;
  a.mats = mats;
  a.n_mat = n_mat;
  a.latents = latents;
  a.n_lat = mats ? n_mat : 0;
  a.dec = dec;
  a.rgb = rgb;
  a.comps = comps;
  a.y_raw = y_raw;
  a.status = status;
  const unsigned blocks = (unsigned)((g.n + kFwdThreads - 1) / kFwdThreads);
  decoder_fp32_kernel<<<blocks, kFwdThreads, fwd_smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_decoder_raw(const fabric_gbuffer &g, const float *latents, int n_lat, const float *dec,
                               float *y_raw, int *status, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(decoder_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fwd_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  FwdArgs a;
  a.g = g;
  a.mats = nullptr;
  a.n_mat = 0;
  a.latents = latents;
  a.n_lat = n_lat;
  a.dec = dec;
  a.rgb = nullptr;
  a.comps = nullptr;
  a.y_raw = y_raw;
  a.status = status;
  const unsigned blocks = (unsigned)((g.n + kFwdThreads - 1) / kFwdThreads);
  decoder_fp32_kernel<<<blocks, kFwdThreads, fwd_smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

// Work layout: [grid][kDecParams] floats | [grid] doubles | [n][32] floats.
static int bwd_grid(int64_t n, int sm_count) {
  const int64_t tiles = (n + kTR - 1) / kTR;
  int64_t g = sm_count > 0 ? sm_count : 148;
  if (g > tiles) g = tiles;
  return (int)(g < 1 ? 1 : g);
}

size_t decoder_backward_work_bytes(int64_t n, int sm_count) {
  const int grid = bwd_grid(n, sm_count);
  size_t bytes = (size_t)grid * kDecParams * 4;
  bytes = (bytes + 15) & ~size_t(15);
  bytes += (size_t)grid * 8;
  bytes = (bytes + 15) & ~size_t(15);
  bytes += (size_t)n * kLatent * 4;
  return bytes + 64;
}

cudaError_t launch_decoder_backward(const fabric_gbuffer &g, const float *latents, int n_lat, const float *dec,
                                    const float *dy, const float *target, int loss_mode, float *ddec, float *dlat,
                                    double *loss, void *work, int sm_count, int *status, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(decoder_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bwd_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int grid = bwd_grid(g.n, sm_count);
  uint8_t *w = static_cast<uint8_t *>(work);
  float *partial = reinterpret_cast<float *>(w);
  size_t off = ((size_t)grid * kDecParams * 4 + 15) & ~size_t(15);
  double *loss_part = reinterpret_cast<double *>(w + off);
  off = (off + (size_t)grid * 8 + 15) & ~size_t(15);
  float *rows = reinterpret_cast<float *>(w + off);
  BwdArgs a;
  a.g = g;
  a.latents = latents;
  a.n_lat = n_lat;
  a.dec = dec;
  a.dy = dy;
  a.target = target;
  a.loss_mode = loss_mode;
  a.inv_batch = 1.0f / (float)(g.n > 0 ? g.n : 1);
  a.partial = partial;
  a.loss_partial = loss_part;
  a.dlat_rows = dlat ? rows : nullptr;
  a.status = status;
  decoder_bwd_kernel<<<grid, kBwdThreads, bwd_smem_bytes(), s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_partials_kernel<<<(kDecParams + 255) / 256, 256, 0, s>>>(partial, grid, kDecParams, ddec);
  if (loss) reduce_loss_kernel<<<1, 32, 0, s>>>(loss_part, grid, loss);
  if (dlat) latent_segment_kernel<<<n_lat, 256, 0, s>>>(g.material, g.n, rows, dlat);
  return cudaGetLastError();
}

cudaError_t launch_decoder_grad_finish(const fabric_gbuffer &g, int n_lat, const float *partial, int grid,
                                      const double *loss_part, const float *rows, float *ddec, double *loss,
                                      float *dlat, cudaStream_t s) {
  reduce_partials_kernel<<<(kDecParams + 255) / 256, 256, 0, s>>>(partial, grid, kDecParams, ddec);
  if (loss) reduce_loss_kernel<<<1, 32, 0, s>>>(loss_part, grid, loss);
  if (dlat) latent_segment_kernel<<<n_lat, 256, 0, s>>>(g.material, g.n, rows, dlat);
  return cudaGetLastError();
}

cudaError_t launch_material_features(const fabric_material *raw, int n, float *feats, cudaStream_t s) {
  material_features_kernel<<<(n + 127) / 128, 128, 0, s>>>(raw, n, feats);
  return cudaGetLastError();
}

cudaError_t launch_encoder_feats(const float *feats, int n, const float *enc, float *z, float *acts,
                                 cudaStream_t s) {
  encoder_fwd_kernel<<<n, kEncHidden, 0, s>>>(feats, enc, z, acts);
  return cudaGetLastError();
}

size_t encoder_backward_work_floats(int n) { return (size_t)n * 2 * kEncHidden + (size_t)n * 4 * kEncHidden; }

cudaError_t launch_encoder_backward(const float *feats, int n, const float *enc, const float *acts_in,
                                    const float *dz, float *denc, float *work, cudaStream_t s) {
  // work: [n][2][128] activations (recomputed when acts_in is null) | [n][4][128]
  float *acts = work;
  float *vec = work + (size_t)n * 2 * kEncHidden;
  if (!acts_in) {
    // recompute the forward pass to obtain the pre-activations (z discarded into vec)
    encoder_fwd_kernel<<<n, kEncHidden, 0, s>>>(feats, enc, vec, acts);
    acts_in = acts;
  }
  encoder_bwd_vec_kernel<<<n, kEncHidden, 0, s>>>(enc, acts_in, dz, vec);
  encoder_grad_kernel<<<(kEncParams + 255) / 256, 256, 0, s>>>(feats, n, dz, vec, denc);
  return cudaGetLastError();
}

cudaError_t launch_adam(float *params, const float *grad, float *m, float *v, int64_t n, float lr, int64_t step,
                        cudaStream_t s) {
  const float bc1 = (float)(1.0 - std::pow(0.9, (double)step));
  const float bc2 = (float)(1.0 - std::pow(0.999, (double)step));
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(params, grad, m, v, n, lr, bc1, bc2);
  return cudaGetLastError();
}

size_t error_stats_work_bytes(int64_t) { return (size_t)kErrBlocks * 3 * sizeof(double); }

cudaError_t launch_error_stats(const float *a, const float *b, int64_t n, const float *w, int group, int w_stride,
                               double *out, void *work, cudaStream_t s) {
  double *part = static_cast<double *>(work);
  err_partial_kernel<<<kErrBlocks, kErrThreads, 0, s>>>(a, b, n, w, group, w_stride, part);
  err_final_kernel<<<1, 32, 0, s>>>(part, out);
  return cudaGetLastError();
}

}  // namespace fab
