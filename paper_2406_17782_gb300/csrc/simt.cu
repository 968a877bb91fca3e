// simt.cu -- FP32 SIMT kernels: the decoder used as the accuracy anchor, the
// training forward/backward passes of decoder and encoder (Sec. 4.2-4.3,
// loss of Eq. 9-11), Adam, and FP64 image-wide error reductions.
//
// All reductions run in a fixed order (owner-computes partial sums per CTA,
// then a fixed-order sum over CTAs), so repeated runs are bitwise identical.
#include <cmath>

#include <algorithm>

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
    if (a.y_raw) store_row4(a.y_raw, p, nan, nan, nan, nan);
    if (a.comps) store_row4(a.comps, p, nan, nan, nan, nan);
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
  if (a.y_raw) store_row4(a.y_raw, p, y[0], y[1], y[2], y[3]);
  const float c0 = fmaxf(0.0f, y[0]), c1 = fmaxf(0.0f, y[1]);
  const float s0 = fmaxf(0.0f, expm1f(y[2]) / kSpecK), s1 = fmaxf(0.0f, expm1f(y[3]) / kSpecK);
  if (a.comps) store_row4(a.comps, p, c0, c1, s0, s1);
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

// Column sums out[j] = sum_c partial[c][j].  A CTA takes 32 consecutive
// columns; its kSumSegs warps sum consecutive ranges of rows (in row order),
// then the range sums are added in range order: a fixed order, so the
// result does not change from run to run.
constexpr int kSumSegs = 8;
constexpr int kSumBatch = 24;   // one batch for up to 192 partials

__device__ void reduce_loss_warp(const double *__restrict__ part, int n, double *__restrict__ out);

// Columns [0, w0) go to out0, columns [w0, width) to out1.  One CTA past the
// column blocks (when loss_out is set) sums the loss partials instead, so
// that both reductions take one launch.
__global__ void __launch_bounds__(32 * kSumSegs) reduce_partials_kernel(const float *__restrict__ partial,
                                                                        int n_part, int stride, int width, int w0,
                                                                        float *__restrict__ out0,
                                                                        float *__restrict__ out1,
                                                                        const double *__restrict__ loss_part,
                                                                        double *__restrict__ loss_out) {
  grid_dependency_wait();
  grid_dependents_launch();
  __shared__ float seg_sum[kSumSegs][32];
  if (loss_out && blockIdx.x == gridDim.x - 1) {
    if (threadIdx.x < 32) reduce_loss_warp(loss_part, n_part, loss_out);
    return;
  }
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const int per = (n_part + kSumSegs - 1) / kSumSegs;
  const int c0 = min(n_part, seg * per), c1 = min(n_part, c0 + per);
  float s = 0.0f;
  if (j < width) {
    // kSumBatch loads in flight, then their sum in order
    for (int c = c0; c < c1; c += kSumBatch) {
      float t[kSumBatch];
#pragma unroll
      for (int q = 0; q < kSumBatch; ++q) t[q] = c + q < c1 ? partial[(int64_t)(c + q) * stride + j] : 0.0f;
#pragma unroll
      for (int q = 0; q < kSumBatch; ++q)
        if (c + q < c1) s += t[q];
    }
  }
  seg_sum[seg][lane] = s;
  __syncthreads();
  if (seg == 0 && j < width) {
    float tot = seg_sum[0][lane];
#pragma unroll
    for (int k = 1; k < kSumSegs; ++k) tot += seg_sum[k][lane];
    if (j < w0) out0[j] = tot;
    else out1[j - w0] = tot;
  }
}

// 32 threads (one warp) sum fixed strided subsets, then lane 0 sums the 32
// in order.
__device__ void reduce_loss_warp(const double *__restrict__ part, int n, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += part[c];
  double t = 0.0;
  for (int k = 0; k < 32; ++k) t += __shfl_sync(0xFFFFFFFFu, s, k);
  if (lane == 0) *out = t;
}

// dlat[m][i] = sum over rows with material m of dlat_rows[row][i]; one CTA
// per material scans every id.  Thread t takes the rows of id groups t,
// t + 256, ... in row order (V: groups of eight ids read as one 16-byte
// load, four groups in flight; otherwise single ids), then the 256 thread
// sums are added in thread order, so the result is the same on every run.
__device__ __forceinline__ void add_row(float *acc, const float *__restrict__ rows, int64_t r) {
  const float4 *src = reinterpret_cast<const float4 *>(rows + r * kLatent);
#pragma unroll
  for (int k = 0; k < kLatent / 4; ++k) {
    const float4 v = src[k];
    acc[4 * k] += v.x;
    acc[4 * k + 1] += v.y;
    acc[4 * k + 2] += v.z;
    acc[4 * k + 3] += v.w;
  }
}

template <bool V>
__global__ void __launch_bounds__(256) latent_segment_kernel(const uint16_t *__restrict__ mat, int64_t n,
                                                             const float *__restrict__ rows,
                                                             float *__restrict__ dlat) {
  grid_dependency_wait();
  grid_dependents_launch();
  const int m = blockIdx.x;
  __shared__ float red[256][kLatent + 1];
  float acc[kLatent];
#pragma unroll
  for (int i = 0; i < kLatent; ++i) acc[i] = 0.0f;
  const int64_t step = blockDim.x;
  int64_t tail = 0;
  if (V) {
    const uint4 *ids8 = reinterpret_cast<const uint4 *>(mat);
    const int64_t groups = n / 8;
    tail = groups * 8;
    for (int64_t g = threadIdx.x; g < groups; g += 4 * step) {
      uint4 w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] = g + q * step < groups ? ids8[g + q * step] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (g + q * step >= groups) break;
        const uint32_t word[4] = {w[q].x, w[q].y, w[q].z, w[q].w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if ((int)((word[k >> 1] >> (16 * (k & 1))) & 0xFFFFu) == m) add_row(acc, rows, 8 * (g + q * step) + k);
        }
      }
    }
  }
  // single ids: every row (V = false), or the last n % 8 rows
  for (int64_t r = tail + threadIdx.x; r < n; r += 8 * step) {
    int ids[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ids[q] = r + q * step < n ? (int)mat[r + q * step] : -1;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (ids[q] == m) add_row(acc, rows, r + q * step);
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
// Encoder (parameters -> latent), kEncGroup materials per CTA of 128 threads.
// acts (optional) [n][2][128] = pre-activations a1, a2 for the backward pass.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float lrelu(float x) { return x > 0.0f ? x : kLeaky * x; }

__device__ __forceinline__ void material_features(const fabric_material &m, float *f) {
#pragma unroll
  for (int k = 0; k < kPatternSlots; ++k) f[k] = (m.pattern_id == k) ? 1.0f : 0.0f;
  f[kPatternSlots + 0] = m.twist_deg / 30.0f;
  f[kPatternSlots + 1] = m.incl_deg / 45.0f;
  f[kPatternSlots + 2] = m.alpha[0];
  f[kPatternSlots + 3] = m.beta[0];
  f[kPatternSlots + 4] = m.alpha[1];
  f[kPatternSlots + 5] = m.beta[1];
}

// Materials per encoder CTA: thread j reads its weight row once for all of
// them and keeps one accumulator per material (each sum still runs over the
// inputs in order, as for a single material).
constexpr int kEncGroup = 4;

// The encoder kernels stage the weights they read in shared memory with
// asynchronous copies issued at once, so that all of them are one round trip
// rather than one dependent round trip per few elements.  Rows read by one
// thread each (thread j: row j) are padded so that a warp's reads fall into
// distinct banks: E1 rows of kEncIn floats at a stride of kE1Ld (odd),
// E2 and E3 rows of 128 floats at a stride of 132 (read as float4: eight
// lanes of a quarter-warp cover the 32 banks).
constexpr int kE1Ld = kEncIn | 1;
constexpr int kERowLd = kEncHidden + 4;
constexpr size_t kEncFwdSmem = (size_t)(kEncHidden * kE1Ld + kEncHidden * kERowLd + kLatent * kERowLd) * 4;
constexpr size_t kEncBwdSmem = (size_t)(kEncHidden * kEncHidden + kLatent * kEncHidden) * 4;

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// rows x cols floats at src (row stride cols) into dst (row stride ld), by
// all threads of the CTA; 16-byte copies when V (src, cols and ld multiples
// of four floats, src 16-byte aligned), else 4-byte ones
template <bool V>
__device__ __forceinline__ void stage_rows(float *dst, int ld, const float *src, int rows, int cols) {
  if (V) {
    const int c4 = cols / 4;
    for (int e = threadIdx.x; e < rows * c4; e += blockDim.x)
      cp_async16(dst + (e / c4) * ld + 4 * (e % c4), src + (e / c4) * cols + 4 * (e % c4));
  } else {
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x)
      cp_async4(dst + (e / cols) * ld + e % cols, src + e);
  }
}

// dot of a shared-memory weight row w (LEN floats; 16-byte aligned) with the
// group's vectors x[g][0..LEN), one accumulator per material, inputs in order
template <int LEN, int LD>
__device__ __forceinline__ void enc_dot_s(const float *w, const float (*x)[LD], float *acc) {
#pragma unroll 8
  for (int i4 = 0; i4 < LEN / 4; ++i4) {
    const float4 c = reinterpret_cast<const float4 *>(w)[i4];
#pragma unroll
    for (int g = 0; g < kEncGroup; ++g) {
      acc[g] = fmaf(c.x, x[g][4 * i4], acc[g]);
      acc[g] = fmaf(c.y, x[g][4 * i4 + 1], acc[g]);
      acc[g] = fmaf(c.z, x[g][4 * i4 + 2], acc[g]);
      acc[g] = fmaf(c.w, x[g][4 * i4 + 3], acc[g]);
    }
  }
}

template <bool V>
__global__ void __launch_bounds__(kEncHidden) encoder_fwd_kernel(const float *__restrict__ feats,
                                                                 const fabric_material *__restrict__ raw,
                                                                 float *__restrict__ feats_out, int n,
                                                                 const float *__restrict__ enc,
                                                                 float *__restrict__ z, float *__restrict__ acts) {
  grid_dependency_wait();
  grid_dependents_launch();
  extern __shared__ __align__(16) float enc_smem[];
  float *e1 = enc_smem;                             // [128][kE1Ld]
  float *e2 = e1 + kEncHidden * kE1Ld;              // [128][kERowLd]
  float *e3 = e2 + kEncHidden * kERowLd;            // [32][kERowLd]
  static_assert((kEncHidden * kE1Ld) % 4 == 0, "E2 rows 16-byte aligned in shared memory");
  stage_rows<false>(e1, kE1Ld, enc + kOffE1, kEncHidden, kEncIn);
  stage_rows<V>(e2, kERowLd, enc + kOffE2, kEncHidden, kEncHidden);
  stage_rows<V>(e3, kERowLd, enc + kOffE3, kLatent, kEncHidden);
  __shared__ float f[kEncGroup][kEncIn];
  __shared__ __align__(16) float h1[kEncGroup][kEncHidden];
  __shared__ __align__(16) float h2[kEncGroup][kEncHidden];
  const int m0 = blockIdx.x * kEncGroup, j = threadIdx.x;
  const int nm = min(kEncGroup, n - m0);
  if (raw) {
    if (j < kEncGroup) {
      float t[kEncIn];
      if (j < nm) {
        material_features(raw[m0 + j], t);
      } else {
#pragma unroll
        for (int i = 0; i < kEncIn; ++i) t[i] = 0.0f;
      }
#pragma unroll
      for (int i = 0; i < kEncIn; ++i) {
        f[j][i] = t[i];
        if (j < nm && feats_out) feats_out[(int64_t)(m0 + j) * kEncIn + i] = t[i];
      }
    }
  } else {
    for (int t = j; t < kEncGroup * kEncIn; t += kEncHidden) {
      const int g = t / kEncIn, i = t % kEncIn;
      f[g][i] = g < nm ? feats[(int64_t)(m0 + g) * kEncIn + i] : 0.0f;
    }
  }
  const float b1 = enc[kOffEb1 + j], b2 = enc[kOffEb2 + j], b3 = enc[kOffEb3 + j % kLatent];
  cp_async_wait_all();
  __syncthreads();
  float a1[kEncGroup], a2[kEncGroup];
#pragma unroll
  for (int g = 0; g < kEncGroup; ++g) a1[g] = b1;
#pragma unroll
  for (int i = 0; i < kEncIn; ++i) {
    const float c = e1[j * kE1Ld + i];
#pragma unroll
    for (int g = 0; g < kEncGroup; ++g) a1[g] = fmaf(c, f[g][i], a1[g]);
  }
#pragma unroll
  for (int g = 0; g < kEncGroup; ++g) h1[g][j] = lrelu(a1[g]);
  __syncthreads();
#pragma unroll
  for (int g = 0; g < kEncGroup; ++g) a2[g] = b2 + h1[g][j];   // skip connection before the last activation
  enc_dot_s<kEncHidden, kEncHidden>(e2 + j * kERowLd, h1, a2);
#pragma unroll
  for (int g = 0; g < kEncGroup; ++g) {
    h2[g][j] = lrelu(a2[g]);
    if (acts && g < nm) {
      acts[(int64_t)(m0 + g) * 2 * kEncHidden + j] = a1[g];
      acts[(int64_t)(m0 + g) * 2 * kEncHidden + kEncHidden + j] = a2[g];
    }
  }
  __syncthreads();
  // layer 3: thread j computes latent output k = j % 32 of material j / 32
  static_assert(kEncGroup * kLatent == kEncHidden, "one layer-3 output per thread");
  const int k = j % kLatent, g = j / kLatent;
  float acc = b3;
  const float *w3 = e3 + k * kERowLd;
#pragma unroll 8
  for (int i4 = 0; i4 < kEncHidden / 4; ++i4) {
    const float4 c = reinterpret_cast<const float4 *>(w3)[i4];
    acc = fmaf(c.x, h2[g][4 * i4], acc);
    acc = fmaf(c.y, h2[g][4 * i4 + 1], acc);
    acc = fmaf(c.z, h2[g][4 * i4 + 2], acc);
    acc = fmaf(c.w, h2[g][4 * i4 + 3], acc);
  }
  if (g < nm) z[(int64_t)(m0 + g) * kLatent + k] = acc;
}

// Per material: back-propagated pre-activation gradients da1, da2 and the
// activations h1, h2 into work [n][4][128]; kEncGroup materials per CTA.
template <bool V>
__global__ void __launch_bounds__(kEncHidden) encoder_bwd_vec_kernel(const float *__restrict__ enc, int n,
                                                                     const float *__restrict__ acts,
                                                                     const float *__restrict__ dz,
                                                                     float *__restrict__ work) {
  grid_dependency_wait();
  grid_dependents_launch();
  // E2 and E3 staged as they are (thread j reads their column j: a warp's
  // reads are consecutive words)
  extern __shared__ __align__(16) float enc_smem[];
  float *e2 = enc_smem;                          // [128][128]
  float *e3 = e2 + kEncHidden * kEncHidden;      // [32][128]
  stage_rows<V>(e2, kEncHidden, enc + kOffE2, kEncHidden, kEncHidden);
  stage_rows<V>(e3, kEncHidden, enc + kOffE3, kLatent, kEncHidden);
  __shared__ float sdz[kEncGroup][kLatent], da2s[kEncGroup][kEncHidden];
  const int m0 = blockIdx.x * kEncGroup, j = threadIdx.x;
  const int nm = min(kEncGroup, n - m0);
  float a1[kEncGroup], a2[kEncGroup];
#pragma unroll
  for (int g = 0; g < kEncGroup; ++g) {
    const int64_t m = g < nm ? m0 + g : m0;
    a1[g] = acts[m * 2 * kEncHidden + j];
    a2[g] = acts[m * 2 * kEncHidden + kEncHidden + j];
  }
  {
    const int k = j % kLatent, g = j / kLatent;
    sdz[g][k] = g < nm ? dz[(int64_t)(m0 + g) * kLatent + k] : 0.0f;
  }
  cp_async_wait_all();
  __syncthreads();
  float dh2[kEncGroup], dh1[kEncGroup];
#pragma unroll
  for (int g = 0; g < kEncGroup; ++g) dh2[g] = 0.0f;
#pragma unroll 8
  for (int k = 0; k < kLatent; ++k) {
    const float w3 = e3[k * kEncHidden + j];
#pragma unroll
    for (int g = 0; g < kEncGroup; ++g) dh2[g] = fmaf(w3, sdz[g][k], dh2[g]);
  }
#pragma unroll
  for (int g = 0; g < kEncGroup; ++g) {
    const float da2 = dh2[g] * (a2[g] > 0.0f ? 1.0f : kLeaky);
    da2s[g][j] = da2;
    dh1[g] = da2;   // through the skip
  }
  __syncthreads();
#pragma unroll 8
  for (int o = 0; o < kEncHidden; ++o) {
    const float w2 = e2[o * kEncHidden + j];
#pragma unroll
    for (int g = 0; g < kEncGroup; ++g) dh1[g] = fmaf(w2, da2s[g][o], dh1[g]);
  }
#pragma unroll
  for (int g = 0; g < kEncGroup; ++g) {
    if (g >= nm) break;
    float *w = work + (int64_t)(m0 + g) * 4 * kEncHidden;
    w[j] = dh1[g] * (a1[g] > 0.0f ? 1.0f : kLeaky);
    w[kEncHidden + j] = da2s[g][j];
    w[2 * kEncHidden + j] = lrelu(a1[g]);
    w[3 * kEncHidden + j] = lrelu(a2[g]);
  }
}

// Encoder parameter gradients: every block is a sum over materials of outer
// products, out[r][c] = sum_m L[m][r] R[m][c] (R = 1 for the biases).  A CTA
// takes a 32 x 32 block of one of them with two groups of 256 threads: group
// q sums over the q-th half of the materials, staging 64 materials' rows of L
// and R at a time in shared memory (all of a chunk's loads in flight
// together), thread (w, c) accumulating rows 4w..4w+3 of column c over its
// materials in order; the block is then (first half) + (second half).
constexpr int kGradChunk = 64;

// Adam (Kingma and Ba 2015) with bias correction, one parameter.
__device__ __forceinline__ void adam_update(float *p, float *m, float *v, float g, float lr, float bc1, float bc2) {
  const float mi = 0.9f * *m + 0.1f * g;
  const float vi = 0.999f * *v + 0.001f * g * g;
  *m = mi;
  *v = vi;
  *p -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

// Block cb of the decoder's gradient: columns 32 cb .. 32 cb + 31 summed over
// the partials exactly as reduce_partials_kernel sums them (kSumSegs
// segments of partials in order, then the segments in order), then Adam.
// Run by threads 0..255 of the block.
__device__ void dec_reduce_adam(const DecAdamArgs &d, int cb) {
  __shared__ float seg_sum[kSumSegs][32];
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const int j = cb * 32 + lane;
  const int per = (d.n_part + kSumSegs - 1) / kSumSegs;
  const int c0 = min(d.n_part, seg * per), c1 = min(d.n_part, c0 + per);
  float s = 0.0f;
  if (j < d.n) {
    for (int c = c0; c < c1; c += kSumBatch) {
      float t[kSumBatch];
#pragma unroll
      for (int q = 0; q < kSumBatch; ++q) t[q] = c + q < c1 ? d.partial[(int64_t)(c + q) * d.stride + j] : 0.0f;
#pragma unroll
      for (int q = 0; q < kSumBatch; ++q)
        if (c + q < c1) s += t[q];
    }
  }
  seg_sum[seg][lane] = s;
  asm volatile("bar.sync 1, %0;" ::"n"(32 * kSumSegs) : "memory");
  if (seg == 0 && j < d.n) {
    float tot = seg_sum[0][lane];
#pragma unroll
    for (int k = 1; k < kSumSegs; ++k) tot += seg_sum[k][lane];
    adam_update(d.p + j, d.m + j, d.v + j, tot, d.lr, d.bc1, d.bc2);
  }
}

struct GradBlock {
  int l_off, r_off;        // column offsets of L and R in their per-material rows (r_off < 0: R = 1)
  int l_src, r_src;        // 0: work rows (512 floats), 1: feats rows (kEncIn), 2: dz rows (kLatent)
  int rows, cols;          // extent of the whole parameter block
  int out;                 // offset of the block in the encoder parameters
};

__constant__ GradBlock kGradBlocks[6] = {
    {0, 0, 0, 1, kEncHidden, kEncIn, kOffE1},                              // E1[j][i] = sum da1_j f_i
    {0, -1, 0, 0, kEncHidden, 1, kOffEb1},                                 // e1[j]
    {kEncHidden, 2 * kEncHidden, 0, 0, kEncHidden, kEncHidden, kOffE2},    // E2[j][i] = sum da2_j h1_i
    {kEncHidden, -1, 0, 0, kEncHidden, 1, kOffEb2},                        // e2[j]
    {0, 3 * kEncHidden, 2, 0, kLatent, kEncHidden, kOffE3},                // E3[k][i] = sum dz_k h2_i
    {0, -1, 2, 0, kLatent, 1, kOffEb3},                                    // e3[k]
};

__device__ __forceinline__ const float *grad_src(int src, const float *work, const float *feats, const float *dz,
                                                 int &ld) {
  ld = src == 0 ? 4 * kEncHidden : src == 1 ? kEncIn : kLatent;
  return src == 0 ? work : src == 1 ? feats : dz;
}

// Blocks of 32 x 32 outputs, in the order of kGradBlocks.
__host__ __device__ constexpr int grad_tiles(int rows, int cols) { return ((rows + 31) / 32) * ((cols + 31) / 32); }
constexpr int kGradTiles = grad_tiles(kEncHidden, kEncIn) + grad_tiles(kEncHidden, 1) +
                           grad_tiles(kEncHidden, kEncHidden) + grad_tiles(kEncHidden, 1) +
                           grad_tiles(kLatent, kEncHidden) + grad_tiles(kLatent, 1);

constexpr int kGradThreads = 512;

__global__ void __launch_bounds__(kGradThreads) encoder_grad_kernel(const float *__restrict__ feats, int n,
                                                                    const float *__restrict__ dz,
                                                                    const float *__restrict__ work,
                                                                    float *__restrict__ denc, const DecAdamArgs dec) {
  grid_dependency_wait();
  grid_dependents_launch();
  if (blockIdx.x >= kGradTiles) {   // the decoder's gradient sums and Adam update
    if (threadIdx.x < 32 * kSumSegs) dec_reduce_adam(dec, blockIdx.x - kGradTiles);
    return;
  }
  __shared__ __align__(16) float sl[2][kGradChunk][32];
  __shared__ float sr[2][kGradChunk][32];
  // which block, and which 32 x 32 tile of it
  int t = blockIdx.x, b = 0;
  while (t >= grad_tiles(kGradBlocks[b].rows, kGradBlocks[b].cols)) {
    t -= grad_tiles(kGradBlocks[b].rows, kGradBlocks[b].cols);
    ++b;
  }
  const GradBlock B = kGradBlocks[b];
  const int ct = (B.cols + 31) / 32;
  const int r0 = (t / ct) * 32, c0 = (t % ct) * 32;
  int ldl, ldr;
  const float *L = grad_src(B.l_src, work, feats, dz, ldl);
  const float *R = grad_src(B.r_src, work, feats, dz, ldr);
  const int q = threadIdx.x >> 8, tid = threadIdx.x & 255, c = tid & 31, w = tid >> 5;
  const int half = (n + 1) / 2, m_begin = q == 0 ? 0 : half, m_end = q == 0 ? half : n;
  const int rounds = (half + kGradChunk - 1) / kGradChunk;   // the same for both groups (CTA barriers)
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int k0 = 0; k0 < rounds; ++k0) {
    const int m0 = m_begin + k0 * kGradChunk;
    const int mc = max(0, min(kGradChunk, m_end - m0));
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kGradChunk * 32 / 256; ++u) {
      const int e = tid + 256 * u, mm = e >> 5, k = e & 31;
      const bool in = mm < mc;
      sl[q][mm][k] = in && r0 + k < B.rows ? L[(int64_t)(m0 + mm) * ldl + B.l_off + r0 + k] : 0.0f;
      sr[q][mm][k] = !in ? 0.0f
                         : B.r_off < 0 ? 1.0f
                                       : (c0 + k < B.cols ? R[(int64_t)(m0 + mm) * ldr + B.r_off + c0 + k] : 0.0f);
    }
    __syncthreads();
    for (int mm = 0; mm < mc; ++mm) {
      const float4 a = reinterpret_cast<const float4 *>(sl[q][mm])[w];
      const float x = sr[q][mm][c];
      acc[0] = fmaf(a.x, x, acc[0]);
      acc[1] = fmaf(a.y, x, acc[1]);
      acc[2] = fmaf(a.z, x, acc[2]);
      acc[3] = fmaf(a.w, x, acc[3]);
    }
  }
  // the second half's sums through shared memory, added to the first half's
  __syncthreads();
  float(*part)[32] = sl[1];   // [32 rows][32 columns]: rows 4w..4w+3 of column c
  if (q == 1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) part[4 * w + k][c] = acc[k];
  }
  __syncthreads();
  if (q == 0 && c0 + c < B.cols) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = r0 + 4 * w + k;
      if (r < B.rows) denc[B.out + r * B.cols + c0 + c] = acc[k] + part[4 * w + k][c];
    }
  }
}

// ---------------------------------------------------------------------------
// Adam (Kingma and Ba 2015) with bias correction.
// ---------------------------------------------------------------------------
// Parameters [0, n0) live in p0 and [n0, n0 + n1) in p1; g, m and v hold
// both sets back to back.
__global__ void adam_kernel(float *__restrict__ p0, int64_t n0, float *__restrict__ p1, int64_t n1,
                            const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v, float lr,
                            float bc1, float bc2) {
  grid_dependency_wait();
  grid_dependents_launch();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0 + n1) return;
  float *p = i < n0 ? p0 + i : p1 + (i - n0);
  adam_update(p, m + i, v + i, g[i], lr, bc1, bc2);
}

// ---------------------------------------------------------------------------
// FP64 error statistics: fixed grid of partial sums, then one fixed-order sum.
// ---------------------------------------------------------------------------
constexpr int kErrBlocks = 608;   // one wave: 4 CTAs of 256 threads (64 registers) on each of 152 SMs
constexpr int kErrThreads = 256;

// Per element the kernel needs (w(a-b))^2, (w b)^2 and |w(a-b)| to FP64
// accuracy.  On this GPU FP64 instructions issue at a small fraction of the
// FP32 rate, so the main loop holds no FP64 arithmetic at all: the terms are
// formed with error-free FP32 transformations (Knuth's TwoSum, the FMA
// TwoProduct) as unevaluated sums hi + lo -- a - b is exact as a pair, its
// square exact to about 2^-48 relative -- and each thread adds runs of
// kErrRun terms in renormalised double-float form (error below
// kErrRun * 2^-47 of a run's sum) before adding the run into its FP64 sums.
// The maximum is kept as a pair too: |a - b| = |hi| + sign(hi) lo, compared
// lexicographically, which is exact because FP32 rounding is monotone (with
// weights, the pair carries the product to about 2^-47 relative).  Elements
// whose values fall outside [2^-40, 2^60] in magnitude (where a square could
// overflow or its low part leave the normal range), and non-finite ones,
// are skipped there and handled in FP64 by a second pass over the thread's
// share, which runs only in threads that met one.
constexpr int kErrRun = 32;
constexpr int kErrBatch = 8;   // loads in flight per thread

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// s = h + l (|l| <= ulp(h) / 2) += x + y, with x >= 0 and |y| << x
struct DFloat {
  float h = 0.0f, l = 0.0f;
  __device__ __forceinline__ void add(float x, float y) {
    float t, e;
    two_sum(h, x, t, e);
    e = __fadd_rn(e, __fadd_rn(l, y));
    h = __fadd_rn(t, e);                 // fast two-sum: t >= |e|
    l = __fsub_rn(e, __fsub_rn(h, t));
  }
};

__device__ __forceinline__ bool err_fast(float x) {
  const float ax = fabsf(x);
  return ax == 0.0f || (ax >= 0x1p-40f && ax <= 0x1p60f);
}

// w (a - b) as dh + dl and w b as bh + bl; true when the pairs' range holds
template <bool W>
__device__ __forceinline__ bool err_pairs(float ai, float bi, float wv, float &dh, float &dl, float &bh, float &bl) {
  two_sum(ai, -bi, dh, dl);
  if (W) {
    float th, te;
    two_prod(dh, wv, th, te);
    dl = __fmaf_rn(dl, wv, te);
    dh = th;
    two_prod(bi, wv, bh, bl);
  } else {
    bh = bi;
    bl = 0.0f;
  }
  return err_fast(dh) && err_fast(bh) && (!W || err_fast(wv));
}

// W: weights present; Idx: index type (32-bit when n and the strides fit).
template <bool W, typename Idx>
__global__ void __launch_bounds__(kErrThreads) err_partial_kernel(const float *__restrict__ a,
                                                                  const float *__restrict__ b, int64_t n_,
                                                                  const float *__restrict__ w, int group,
                                                                  int w_stride, double *__restrict__ part) {
  __shared__ double s0[kErrThreads], s1[kErrThreads], s2[kErrThreads];
  const Idx n = (Idx)n_;
  const Idx stride = (Idx)gridDim.x * kErrThreads;
  const Idx start = (Idx)blockIdx.x * kErrThreads + threadIdx.x;
  double e2 = 0.0, b2 = 0.0;
  float mh = -1.0f, ml = 0.0f;   // largest |w(a-b)| so far as mh + ml (mh < 0: none)
  bool slow = false;
  for (Idx i0 = start; i0 < n; i0 += kErrRun * stride) {
    DFloat E, B;
#pragma unroll 1
    for (int r0 = 0; r0 < kErrRun; r0 += kErrBatch) {
      // a batch of loads in flight together; positions past n read as a = b = 0
      float av[kErrBatch], bv[kErrBatch], wv[kErrBatch];
#pragma unroll
      for (int q = 0; q < kErrBatch; ++q) {
        const Idx i = i0 + (Idx)(r0 + q) * stride;
        const bool in = i < n;
        av[q] = in ? a[i] : 0.0f;
        bv[q] = in ? b[i] : 0.0f;
        wv[q] = W && in ? w[(int64_t)(i / group) * w_stride] : 1.0f;
      }
#pragma unroll
      for (int q = 0; q < kErrBatch; ++q) {
        float dh, dl, bh, bl;
        if (!err_pairs<W>(av[q], bv[q], wv[q], dh, dl, bh, bl)) {
          slow = true;
          continue;
        }
        float p, pe, qq, qe;
        two_prod(dh, dh, p, pe);
        two_prod(bh, bh, qq, qe);
        E.add(p, __fmaf_rn(2.0f * dh, dl, pe));   // (dh + dl)^2 without the dl^2 term (below 2^-48)
        B.add(qq, __fmaf_rn(2.0f * bh, bl, qe));
        const float sh = fabsf(dh);
        if (sh >= mh) {   // rare once the running maximum has grown: one compare per element
          const float sl = dh < 0.0f ? -dl : dl;
          if (sh > mh || sl > ml) {
            mh = sh;
            ml = sl;
          }
        }
      }
    }
    e2 += (double)E.h + (double)E.l;
    b2 += (double)B.h + (double)B.l;
  }
  double mx = mh < 0.0f ? 0.0 : (double)mh + (double)ml;
  if (slow) {
    for (Idx i = start; i < n; i += stride) {
      const float ai = a[i], bi = b[i];
      const float wv = W ? w[(int64_t)(i / group) * w_stride] : 1.0f;
      float dh, dl, bh, bl;
      if (err_pairs<W>(ai, bi, wv, dh, dl, bh, bl)) continue;
      const double wi = (double)wv;
      const double d = ((double)ai - (double)bi) * wi;
      const double bb = (double)bi * wi;
      e2 += d * d;
      b2 += bb * bb;
      mx = fmax(mx, fabs(d));
    }
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

// ---- the same reduction on pairs of elements with packed FP32x2
// instructions (add/sub/mul/fma.rn.f32x2: one instruction for two lanes),
// which halves the arithmetic instruction count of the error-free
// transformations; used when a and b are 8-byte aligned.  Lane 0 of every
// packed value carries the even element of a pair, lane 1 the odd one; each
// lane has its own double-float run sums.
// No element is range-checked in the main loop.  Where the FP32 pairs cannot
// carry a term exactly, the thread's results show it: a square or sum that
// overflows (or a non-finite input) makes its FP64 sums non-finite, and a
// square whose low part falls below the normal range loses at most 2^-149
// absolutely, which is below 2^-49 of the thread's sum unless its largest
// |w(a-b)| (or |w b|) is under sqrt(elements) 2^-50.  A thread in either
// case redoes its whole share in FP64 instead; one whose largest value is
// exactly zero does not, since its sums are then exact.
constexpr int kErrRun2 = 16;    // pairs per run
constexpr int kErrBatch2 = 4;   // pair loads in flight per thread (eight without weights)
constexpr int kErrPerSm2 = 4;   // resident CTAs per SM
constexpr int kErrBlocks2 = 152 * kErrPerSm2;   // one wave on 152 SMs

__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
constexpr uint64_t kSign2 = 0x8000000080000000ull;   // both lanes' sign bits

// Packed DFloat: (h, l) += (x, y) per lane, as DFloat::add.
__device__ __forceinline__ void dadd2(uint64_t &h, uint64_t &l, uint64_t x, uint64_t y) {
  const uint64_t t = add2(h, x);
  const uint64_t bv = sub2(t, h);
  const uint64_t av = sub2(t, bv);
  uint64_t e = add2(sub2(h, av), sub2(x, bv));
  e = add2(e, add2(l, y));
  h = add2(t, e);
  l = sub2(e, sub2(h, t));
}

template <bool W, typename Idx>
__global__ void __launch_bounds__(kErrThreads, kErrPerSm2) err_partial2_kernel(const float *__restrict__ a,
                                                                   const float *__restrict__ b, int64_t n_,
                                                                   const float *__restrict__ w, int group,
                                                                   int w_stride, double *__restrict__ part) {
  __shared__ double s0[kErrThreads], s1[kErrThreads], s2[kErrThreads];
  const uint64_t *a2 = reinterpret_cast<const uint64_t *>(a);
  const uint64_t *b2 = reinterpret_cast<const uint64_t *>(b);
  const Idx n = (Idx)n_;
  const Idx np = n / 2;   // pairs; an odd last element is added by the FP64 pass of thread 0
  const Idx stride = (Idx)gridDim.x * kErrThreads;
  const Idx start = (Idx)blockIdx.x * kErrThreads + threadIdx.x;
  const uint64_t two = pk2(2.0f, 2.0f);
  double e2 = 0.0, b2s = 0.0;
  float mh = -1.0f, ml = 0.0f, bmax = 0.0f;
  for (Idx j0 = start; j0 < np; j0 += kErrRun2 * stride) {
    uint64_t EH = 0, EL = 0, BH = 0, BL = 0;
#pragma unroll 1
    constexpr int NB = W ? kErrBatch2 : 2 * kErrBatch2;
    for (int r0 = 0; r0 < kErrRun2; r0 += NB) {
      uint64_t av[NB], bv[NB], wv[NB];
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const Idx j = j0 + (Idx)(r0 + q) * stride;
        const bool in = j < np;
        av[q] = in ? __ldg(a2 + j) : 0ull;
        bv[q] = in ? __ldg(b2 + j) : 0ull;
        if (W) {
          const float w0 = in ? w[(int64_t)((2 * j) / group) * w_stride] : 1.0f;
          const float w1 = in ? w[(int64_t)((2 * j + 1) / group) * w_stride] : 1.0f;
          wv[q] = pk2(w0, w1);
        }
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        // w (a - b) as D + E exactly (TwoSum, then the FMA TwoProduct by w)
        uint64_t D = sub2(av[q], bv[q]);
        const uint64_t BV = sub2(D, av[q]);
        const uint64_t AV = sub2(D, BV);
        uint64_t E = sub2(sub2(av[q], AV), add2(bv[q], BV));
        uint64_t Bh = bv[q], Bl = 0;
        if (W) {
          const uint64_t P = mul2(D, wv[q]);
          const uint64_t PE = fma2(D, wv[q], P ^ kSign2);
          E = fma2(E, wv[q], PE);
          D = P;
          Bh = mul2(bv[q], wv[q]);
          Bl = fma2(bv[q], wv[q], Bh ^ kSign2);
        }
        float dh0, dh1, bh0, bh1;
        upk2(D, dh0, dh1);
        upk2(Bh, bh0, bh1);
        const uint64_t PP = mul2(D, D);
        const uint64_t X = fma2(mul2(D, two), E, fma2(D, D, PP ^ kSign2));
        const uint64_t QQ = mul2(Bh, Bh);
        const uint64_t Y = W ? fma2(mul2(Bh, two), Bl, fma2(Bh, Bh, QQ ^ kSign2)) : fma2(Bh, Bh, QQ ^ kSign2);
        dadd2(EH, EL, PP, X);
        dadd2(BH, BL, QQ, Y);
        bmax = fmaxf(bmax, fmaxf(fabsf(bh0), fabsf(bh1)));
        float dl0, dl1;
        upk2(E, dl0, dl1);
#pragma unroll
        for (int lane = 0; lane < 2; ++lane) {
          const float dh = lane ? dh1 : dh0, dl = lane ? dl1 : dl0;
          const float sh = fabsf(dh);
          if (sh >= mh) {
            const float sl = dh < 0.0f ? -dl : dl;
            if (sh > mh || sl > ml) {
              mh = sh;
              ml = sl;
            }
          }
        }
      }
    }
    float h0, h1, l0, l1;
    upk2(EH, h0, h1);
    upk2(EL, l0, l1);
    e2 += ((double)h0 + (double)l0) + ((double)h1 + (double)l1);
    upk2(BH, h0, h1);
    upk2(BL, l0, l1);
    b2s += ((double)h0 + (double)l0) + ((double)h1 + (double)l1);
  }
  double mx = mh < 0.0f ? 0.0 : (double)mh + (double)ml;
  {
    const double pairs = (double)((np - (start < np ? start : np) + stride - 1) / stride);   // this thread's pairs
    const double floor_v = sqrt(2.0 * pairs) * 0x1p-50;
    const bool slow = !isfinite(e2) || !isfinite(b2s) || (mh > 0.0f && (double)mh < floor_v) ||
                      (bmax > 0.0f && (double)bmax < floor_v);
    if (slow) {   // the thread's whole share again, in FP64
      e2 = 0.0;
      b2s = 0.0;
      mx = 0.0;
    }
    auto fp64 = [&](Idx i) {
      const float ai = a[i], bi = b[i];
      const double wi = W ? (double)w[(int64_t)(i / group) * w_stride] : 1.0;
      const double d = ((double)ai - (double)bi) * wi;
      const double bb = (double)bi * wi;
      e2 += d * d;
      b2s += bb * bb;
      mx = fmax(mx, fabs(d));
    };
    if (slow)
      for (Idx j = start; j < np; j += stride) {
        fp64(2 * j);
        fp64(2 * j + 1);
      }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) fp64(n - 1);   // the odd last element
  }
  s0[threadIdx.x] = e2;
  s1[threadIdx.x] = b2s;
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

// One warp: lane l sums the partials l, l + 32, ... in order, then the 32
// lane sums are added in lane order.
__global__ void err_final_kernel(const double *__restrict__ part, int n_parts, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  double e2 = 0.0, b2 = 0.0, mx = 0.0;
  for (int k = lane; k < n_parts; k += 32) {
    e2 += part[3 * k];
    b2 += part[3 * k + 1];
    mx = fmax(mx, part[3 * k + 2]);
  }
  double t0 = 0.0, t1 = 0.0, t2 = 0.0;
  for (int k = 0; k < 32; ++k) {
    t0 += __shfl_sync(0xFFFFFFFFu, e2, k);
    t1 += __shfl_sync(0xFFFFFFFFu, b2, k);
    t2 = fmax(t2, __shfl_sync(0xFFFFFFFFu, mx, k));
  }
  if (lane == 0) {
    out[0] = t0;
    out[1] = t1;
    out[2] = t2;
  }
}

size_t fwd_smem_bytes() { return (((kDecParams + 3) & ~3) + (size_t)(kDecIn + kHidden) * kFwdThreads) * 4; }
size_t bwd_smem_bytes() {
  return (2 * (size_t)((kDecParams + 3) & ~3) + (size_t)(72 + 64 * 3 + 4 + 64 * 2) * kRS) * 4;
}

}  // namespace

cudaError_t launch_decoder_fp32(const fabric_gbuffer &g, const DevMaterial *mats, int n_mat, const float *latents,
                                const float *dec, float *rgb, float *comps, float *y_raw, int *status,
                                cudaStream_t s) {
  {
    const cudaError_t e = ensure_max_dyn_smem(reinterpret_cast<const void *>(decoder_fp32_kernel),
                                              (int)fwd_smem_bytes());
    if (e != cudaSuccess) return e;
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
  {
    const cudaError_t e = ensure_max_dyn_smem(reinterpret_cast<const void *>(decoder_fp32_kernel),
                                              (int)fwd_smem_bytes());
    if (e != cudaSuccess) return e;
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

namespace {
void latent_sums(const fabric_gbuffer &g, int n_lat, const float *rows, float *dlat, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(g.material) & 15) == 0)
    launch_dependent(latent_segment_kernel<true>, n_lat, 256, 0, s, g.material, g.n, rows, dlat);
  else
    launch_dependent(latent_segment_kernel<false>, n_lat, 256, 0, s, g.material, g.n, rows, dlat);
}
}  // namespace

cudaError_t launch_decoder_backward(const fabric_gbuffer &g, const float *latents, int n_lat, const float *dec,
                                    const float *dy, const float *target, int loss_mode, float *ddec, float *dlat,
                                    double *loss, void *work, int sm_count, int *status, cudaStream_t s) {
  {
    const cudaError_t e = ensure_max_dyn_smem(reinterpret_cast<const void *>(decoder_bwd_kernel),
                                              (int)bwd_smem_bytes());
    if (e != cudaSuccess) return e;
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
  launch_dependent(reduce_partials_kernel, (kDecParams + 31) / 32 + (loss ? 1 : 0), 32 * kSumSegs, 0, s, partial, grid,
                   kDecParams, kDecParams, kDecParams, ddec, nullptr, loss_part, loss);
  if (dlat) latent_sums(g, n_lat, rows, dlat, s);
  return cudaGetLastError();
}

cudaError_t launch_decoder_grad_finish(const fabric_gbuffer &g, int n_lat, const float *partial, int grid, int width,
                                      const double *loss_part, const float *rows, float *ddec, double *loss,
                                      float *dlat, cudaStream_t s) {
  // width > kDecParams: the per-CTA partials already hold the per-material
  // latent-gradient sums after the decoder's columns
  const bool folded = width > kDecParams;
  if (ddec) {
    const int cols = dlat ? width : kDecParams;
    launch_dependent(reduce_partials_kernel, (cols + 31) / 32 + (loss ? 1 : 0), 32 * kSumSegs, 0, s, partial, grid,
                     width, cols, kDecParams, ddec, dlat, loss_part, loss);
  } else {   // only the latent columns (folded) and the loss
    const int cols = dlat && folded ? width - kDecParams : 0;
    if (cols > 0 || loss)
      launch_dependent(reduce_partials_kernel, (cols + 31) / 32 + (loss ? 1 : 0), 32 * kSumSegs, 0, s,
                       partial + kDecParams, grid, width, cols, 0, static_cast<float *>(nullptr), dlat, loss_part,
                       loss);
  }
  if (dlat && !folded) latent_sums(g, n_lat, rows, dlat, s);
  return cudaGetLastError();
}

namespace {
cudaError_t encoder_fwd(const float *feats, const fabric_material *raw, float *feats_out, int n, const float *enc,
                        float *z, float *acts, cudaStream_t s) {
  const int grid = (n + kEncGroup - 1) / kEncGroup;
  const bool v = (reinterpret_cast<uintptr_t>(enc) & 15) == 0;
  const void *k = v ? reinterpret_cast<const void *>(encoder_fwd_kernel<true>)
                    : reinterpret_cast<const void *>(encoder_fwd_kernel<false>);
  const cudaError_t e = ensure_max_dyn_smem(k, (int)kEncFwdSmem);
  if (e != cudaSuccess) return e;
  if (v)
    launch_dependent(encoder_fwd_kernel<true>, grid, kEncHidden, kEncFwdSmem, s, feats, raw, feats_out, n, enc, z,
                     acts);
  else
    launch_dependent(encoder_fwd_kernel<false>, grid, kEncHidden, kEncFwdSmem, s, feats, raw, feats_out, n, enc, z,
                     acts);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_encoder_feats(const float *feats, int n, const float *enc, float *z, float *acts,
                                 cudaStream_t s) {
  return encoder_fwd(feats, nullptr, nullptr, n, enc, z, acts, s);
}

cudaError_t launch_encoder_raw(const fabric_material *raw, int n, const float *enc, float *feats_out, float *z,
                               float *acts, cudaStream_t s) {
  return encoder_fwd(nullptr, raw, feats_out, n, enc, z, acts, s);
}

size_t encoder_backward_work_floats(int n) { return (size_t)n * 2 * kEncHidden + (size_t)n * 4 * kEncHidden; }

cudaError_t launch_encoder_backward(const float *feats, int n, const float *enc, const float *acts_in,
                                    const float *dz, float *denc, float *work, cudaStream_t s,
                                    const DecAdamArgs *dec_adam) {
  // work: [n][2][128] activations (recomputed when acts_in is null) | [n][4][128]
  float *acts = work;
  float *vec = work + (size_t)n * 2 * kEncHidden;
  if (!acts_in) {
    // recompute the forward pass to obtain the pre-activations (z discarded into vec)
    const cudaError_t e = encoder_fwd(feats, nullptr, nullptr, n, enc, vec, acts, s);
    if (e != cudaSuccess) return e;
    acts_in = acts;
  }
  const bool v = (reinterpret_cast<uintptr_t>(enc) & 15) == 0;
  const void *k = v ? reinterpret_cast<const void *>(encoder_bwd_vec_kernel<true>)
                    : reinterpret_cast<const void *>(encoder_bwd_vec_kernel<false>);
  {
    const cudaError_t e = ensure_max_dyn_smem(k, (int)kEncBwdSmem);
    if (e != cudaSuccess) return e;
  }
  const int grid = (n + kEncGroup - 1) / kEncGroup;
  if (v)
    launch_dependent(encoder_bwd_vec_kernel<true>, grid, kEncHidden, kEncBwdSmem, s, enc, n, acts_in, dz, vec);
  else
    launch_dependent(encoder_bwd_vec_kernel<false>, grid, kEncHidden, kEncBwdSmem, s, enc, n, acts_in, dz, vec);
  DecAdamArgs d{};
  int extra = 0;
  if (dec_adam) {
    d = *dec_adam;
    extra = (d.n + 31) / 32;
  }
  launch_dependent(encoder_grad_kernel, kGradTiles + extra, kGradThreads, 0, s, feats, n, dz, vec, denc, d);
  return cudaGetLastError();
}

void adam_bias(int64_t step, float *bc1, float *bc2) {
  *bc1 = (float)(1.0 - std::pow(0.9, (double)step));
  *bc2 = (float)(1.0 - std::pow(0.999, (double)step));
}

cudaError_t launch_adam(float *p0, int64_t n0, float *p1, int64_t n1, const float *grad, float *m, float *v, float lr,
                        int64_t step, cudaStream_t s) {
  float bc1, bc2;
  adam_bias(step, &bc1, &bc2);
  launch_dependent(adam_kernel, (unsigned)((n0 + n1 + 255) / 256), 256, 0, s, p0, n0, p1, n1, grad, m, v, lr, bc1, bc2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dataset shuffle: a pseudo-random permutation of [0, n) from a four-round
// Feistel network on [0, 4^k) (balanced halves of k bits, 4^k >= n) with
// the SplitMix64 finaliser of (seed, round, half) as round function; values
// at or past n are walked along their cycle (the network is a bijection of
// [0, 4^k), so the walk returns to [0, n)).
// ---------------------------------------------------------------------------
namespace {
__device__ __forceinline__ uint64_t shuffle_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t feistel(uint64_t x, int k, uint64_t seed) {
  const uint64_t mask = (1ull << k) - 1ull;
  uint64_t l = x >> k, r = x & mask;
#pragma unroll
  for (int round = 0; round < 4; ++round) {
    const uint64_t f = shuffle_mix(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(round + 1) + r) & mask;
    const uint64_t t = l ^ f;
    l = r;
    r = t;
  }
  return (l << k) | r;
}

__global__ void shuffle_dataset_kernel(const fabric_train_batch src, const fabric_dataset_out dst, int k,
                                       uint64_t seed) {
  const int64_t n = src.queries.n;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    uint64_t j = feistel((uint64_t)p, k, seed);
    while (j >= (uint64_t)n) j = feistel(j, k, seed);
    const fabric_gbuffer &g = src.queries;
    dst.u[p] = g.u[j];
    dst.v[p] = g.v[j];
    dst.radius[p] = g.radius[j];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dst.wi[3 * p + c] = g.wi[3 * j + c];
      dst.wo[3 * p + c] = g.wo[3 * j + c];
    }
    dst.material[p] = g.material[j];
    if (dst.target) {
#pragma unroll
      for (int c = 0; c < 4; ++c) dst.target[4 * p + c] = src.target[4 * j + c];
    }
  }
}
}  // namespace

cudaError_t launch_shuffle_dataset(const fabric_train_batch &src, const fabric_dataset_out &dst, uint64_t seed,
                                   int sm_count, cudaStream_t s) {
  const int64_t n = src.queries.n;
  int k = 1;
  while ((1ll << (2 * k)) < n) ++k;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)(sm_count > 0 ? sm_count : 148) * 8);
  shuffle_dataset_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, k, seed);
  return cudaGetLastError();
}

size_t error_stats_work_bytes(int64_t) { return (size_t)kErrBlocks * 3 * sizeof(double); }

cudaError_t launch_error_stats(const float *a, const float *b, int64_t n, const float *w, int group, int w_stride,
                               double *out, void *work, cudaStream_t s) {
  double *part = static_cast<double *>(work);
  const bool small = n + (int64_t)kErrRun * kErrBlocks * kErrThreads < ((int64_t)1 << 31);
  const bool packed = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 7u) == 0;
  const int blocks = packed ? kErrBlocks2 : kErrBlocks;
  if (packed) {
    if (w && small) err_partial2_kernel<true, int><<<blocks, kErrThreads, 0, s>>>(a, b, n, w, group, w_stride, part);
    else if (w) err_partial2_kernel<true, int64_t><<<blocks, kErrThreads, 0, s>>>(a, b, n, w, group, w_stride, part);
    else if (small) err_partial2_kernel<false, int><<<blocks, kErrThreads, 0, s>>>(a, b, n, w, group, w_stride, part);
    else err_partial2_kernel<false, int64_t><<<blocks, kErrThreads, 0, s>>>(a, b, n, w, group, w_stride, part);
  } else if (w && small) err_partial_kernel<true, int><<<blocks, kErrThreads, 0, s>>>(a, b, n, w, group, w_stride, part);
  else if (w) err_partial_kernel<true, int64_t><<<blocks, kErrThreads, 0, s>>>(a, b, n, w, group, w_stride, part);
  else if (small) err_partial_kernel<false, int><<<blocks, kErrThreads, 0, s>>>(a, b, n, w, group, w_stride, part);
  else err_partial_kernel<false, int64_t><<<blocks, kErrThreads, 0, s>>>(a, b, n, w, group, w_stride, part);
  err_final_kernel<<<1, 32, 0, s>>>(part, blocks, out);
  return cudaGetLastError();
}

}  // namespace fab
