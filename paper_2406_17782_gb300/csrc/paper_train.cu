// paper_train.cu -- FP32 training kernels of the paper's decoder structure
// (Sec. 4.2 "Decoder", Fig. 3; losses of Sec. 4.3, Eq. 9-11) and of its
// 64-wide parameter encoder, for fabric_paper_train_step.
//
// The decoder's layers run over the whole batch as products of row-major
// activation matrices [B][K] (one tiled FP32 kernel, SIMT): the forward pass
// keeps every post-activation matrix (a leaky ReLU keeps the sign, so its
// derivative is read from the output); the backward pass forms the input
// gradients with the same kernel and the weight gradients as partial sums
// over fixed chunks of the batch, summed in chunk order, so every step is
// bitwise repeatable.  The per-material latent gradient sums the first
// layer's gradient over each material's queries (fixed segments, fixed
// order) and multiplies by the latent block of S1.
#include <cmath>

#include "fabric_internal.h"
#include "paper_net.h"
#include "train_common.cuh"

namespace fab {
namespace {

constexpr int kGemmThreads = 256;
constexpr int kBK = 8;             // depth of one shared-memory stage
constexpr int kChunkRows = 256;    // batch rows per weight-gradient partial

// Epilogue of the product: forward (bias, residual, leaky ReLU), input
// gradient (addend, leaky ReLU derivative of the layer's own output), or
// weight-gradient partial (plain store into a chunk's slab).
struct Epi {
  int mode;               // 0 forward, 1 input gradient, 2 partial
  const float *bias;      // [N] (forward)
  const float *res;       // residual / addend [M][ld_res] or null
  int ld_res;
  const float *h;         // post-activation whose derivative multiplies (input gradient) or null
  int ld_h;
  int lrelu;              // forward: apply leaky ReLU
  float *out;
  int ld_out;
  int64_t slab;           // partial: floats per chunk slab
};

__device__ __forceinline__ uint64_t pn_pk2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 pn_upk2(uint64_t r) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(r));
  return f;
}
// d = a * b + c in each 32-bit lane, rounded once (the same as two fmaf)
__device__ __forceinline__ uint64_t pn_fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// C(i, j) = sum_r A(i, r) B(j, r) for i < M, j < N, r in [r0, r1), with
// A(i, r) = A[i a_i + r a_r] and B(j, r) = B[j b_j + r b_r].  AR / BR: the
// operand is contiguous along r (else along i / j).  B_ONES: column j = N - 1
// of B is the constant 1 (the bias gradient as an extra output column); the
// tiles then cover the N - 1 other columns and the first column of tiles
// also keeps the running sums of A's rows for it.
// A BM x BN tile per CTA of 256 threads, each thread BM/16 x BN/16 outputs
// (rows ty*4 + {0..3} of every 64-row band, columns likewise with tx), so
// that one 16-byte shared-memory read feeds four products, and two adjacent
// outputs of a row share one packed FP32x2 fma; operands pass through two
// shared-memory stages of depth 8, the next stage's global loads in
// registers while the current one is multiplied.  Every output is a chain of
// fmaf over r in increasing order (bitwise repeatable).
template <int BM, int BN, bool AR, bool BR, bool B_ONES>
__global__ void __launch_bounds__(kGemmThreads, 2) pn_gemm_kernel(const float *__restrict__ A, int64_t a_i,
                                                                  int64_t a_r, const float *__restrict__ Bm,
                                                                  int64_t b_j, int64_t b_r, int M, int N, int64_t R,
                                                                  int64_t r_chunk, Epi e) {
  constexpr int RM = BM / 16, RN = BN / 16;            // outputs per thread along i and j
  constexpr int LA = BM * kBK / kGemmThreads, LB = BN * kBK / kGemmThreads;   // loads per thread and stage
  __shared__ __align__(16) float As[2][kBK][BM + 4];
  __shared__ __align__(16) float Bs[2][kBK][BN + 4];
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int NB = B_ONES ? N - 1 : N;                   // columns that come from B
  const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
  const int64_t r_begin = (int64_t)blockIdx.z * r_chunk;
  const int64_t r_end = r_begin + r_chunk < R ? r_begin + r_chunk : R;
  float ra[LA], rb[LB];
  auto fetch = [&](int64_t r0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int el = tid + kGemmThreads * q;
      const int rr = AR ? el % kBK : el / BM, ii = AR ? el / kBK : el % BM;
      const int64_t gi = i0 + ii, gr = r0 + rr;
      ra[q] = (gi < M && gr < r_end) ? A[gi * a_i + gr * a_r] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int el = tid + kGemmThreads * q;
      const int rb_ = BR ? el % kBK : el / BN, jj = BR ? el / kBK : el % BN;
      const int64_t gj = j0 + jj, gb = r0 + rb_;
      rb[q] = (gj < NB && gb < r_end) ? Bm[gj * b_j + gb * b_r] : 0.0f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int el = tid + kGemmThreads * q;
      As[buf][AR ? el % kBK : el / BM][AR ? el / kBK : el % BM] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int el = tid + kGemmThreads * q;
      Bs[buf][BR ? el % kBK : el / BN][BR ? el / kBK : el % BN] = rb[q];
    }
  };
  uint64_t acc[RM][RN / 2];   // adjacent output pairs (t, t + 1) of row q
  float rsum[B_ONES ? RM : 1];
#pragma unroll
  for (int q = 0; q < RM; ++q) {
#pragma unroll
    for (int t = 0; t < RN / 2; ++t) acc[q][t] = 0ull;
    if (B_ONES) rsum[q] = 0.0f;
  }
  int buf = 0;
  if (r_begin < r_end) {
    fetch(r_begin);
    stash(0);
  }
  __syncthreads();
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kBK) {
    const bool more = r0 + kBK < r_end;
    if (more) fetch(r0 + kBK);   // next stage's loads in flight during this stage's products
#pragma unroll
    for (int r = 0; r < kBK; ++r) {
      float av[RM];
      uint64_t bv[RN / 2];
#pragma unroll
      for (int q = 0; q < RM / 4; ++q) {
        const float4 t = *reinterpret_cast<const float4 *>(&As[buf][r][64 * q + 4 * ty]);
        av[4 * q] = t.x;
        av[4 * q + 1] = t.y;
        av[4 * q + 2] = t.z;
        av[4 * q + 3] = t.w;
      }
#pragma unroll
      for (int q = 0; q < RN / 4; ++q) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(&Bs[buf][r][64 * q + 4 * tx]);
        bv[2 * q] = t.x;
        bv[2 * q + 1] = t.y;
      }
#pragma unroll
      for (int q = 0; q < RM; ++q) {
        const uint64_t a2 = pn_pk2(av[q], av[q]);
#pragma unroll
        for (int t = 0; t < RN / 2; ++t) acc[q][t] = pn_fma2(a2, bv[t], acc[q][t]);
        if (B_ONES) rsum[q] += av[q];   // = fmaf(av[q], 1, rsum[q])
      }
    }
    if (more) stash(buf ^ 1);   // the other stage: its last readers finished before the previous barrier
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int q = 0; q < RM; ++q) {
    const int64_t i = i0 + 64 * (q / 4) + 4 * ty + (q % 4);
    if (i >= M) continue;
    if (B_ONES && blockIdx.y == 0 && tx == 0) e.out[blockIdx.z * e.slab + i * N + (N - 1)] = rsum[q];
#pragma unroll
    for (int t = 0; t < RN; ++t) {
      const int j = j0 + 64 * (t / 4) + 4 * tx + (t % 4);
      if (j >= NB) continue;
      const float2 pr = pn_upk2(acc[q][t / 2]);
      float v = (t & 1) ? pr.y : pr.x;
      if (e.mode == 0) {
        v += e.bias[j];
        if (e.res) v += e.res[i * e.ld_res + j];
        if (e.lrelu) v = fmaxf(v, kPnSlope * v);
        e.out[i * e.ld_out + j] = v;
      } else if (e.mode == 1) {
        if (e.res) v += e.res[i * e.ld_res + j];
        if (e.h) v *= e.h[i * e.ld_h + j] > 0.0f ? 1.0f : kPnSlope;
        e.out[i * e.ld_out + j] = v;
      } else {
        e.out[blockIdx.z * e.slab + i * N + j] = v;
      }
    }
  }
}

// out_w[i][j] = sum_c part[c][i][j] for j < K, out_b[i] = sum_c part[c][i][K]:
// four lanes per element, lane g summing the g-th quarter of the chunks in
// order, the quarters then added as (q0 + q1) + (q2 + q3).
__global__ void pn_reduce_chunks_kernel(const float *__restrict__ part, int chunks, int M, int K,
                                       float *__restrict__ out_w, float *__restrict__ out_b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int e = (int)(t >> 2), g = (int)(t & 3);
  const int N = K + 1;
  const bool in = e < M * N;
  const int64_t mn = (int64_t)M * N;
  const int per = (chunks + 3) / 4;
  const int c1 = min(chunks, (g + 1) * per);
  float s = 0.0f;
  if (in) {
    int c = g * per;
    for (; c + 8 <= c1; c += 8) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = part[(c + q) * mn + e];   // eight loads in flight, added in order
#pragma unroll
      for (int q = 0; q < 8; ++q) s += v[q];
    }
    for (; c < c1; ++c) s += part[c * mn + e];
  }
  // every lane forms the same (q0 + q1) + (q2 + q3): addition commutes exactly
  const float o1 = __shfl_xor_sync(0xffffffffu, s, 1);
  const float p = (g & 1) ? o1 + s : s + o1;
  const float o2 = __shfl_xor_sync(0xffffffffu, p, 2);
  const float tot = (g & 2) ? o2 + p : p + o2;
  if (!in || g != 0) return;
  const int i = e / N, j = e % N;
  if (j < K)
    out_w[i * K + j] = tot;
  else
    out_b[i] = tot;
}

// One-blob channel k (FP32, accurate exp) of the footprint: k < 8 the
// periodic Gaussians of frac u (nearest image and the one on the far side),
// 8..15 those of frac v, 16..23 the plain ones of the size coordinate.
__device__ __forceinline__ float pn_blob_channel(float u, float v, float r, int k) {
  const float c = ((k & 7) + 0.5f) * 0.125f;
  if (k >= 16) {
    const float t = (logf(fmaxf(r, kRFloor)) - kPnLnRLo) * kPnInvLnSpan;
    const float d = t - c;
    return expf(-32.0f * d * d);
  }
  const float x = k < 8 ? u : v;
  float d = (x - floorf(x)) - c;
  d -= rintf(d);
  const float e = 1.0f - fabsf(d);
  return expf(-32.0f * d * d) + expf(-32.0f * e * e);
}

// X0[b] = [z_mat (64) | spatial channels (24 one-blob, or 3 unencoded)]
// (row stride ld0) and the angular inputs (wi, wo.xy) at columns
// ang0..ang0+4 of the row of A (row stride lda): XA after the fused
// spatial feature, or X0 itself without the fusion.  One warp per row, so
// that every store of a row is coalesced: lanes copy the latent in two
// 32-float halves, lane k < 24 computes spatial channel k, lanes < 5 the
// angular inputs.
__global__ void __launch_bounds__(256) pn_inputs_kernel(fabric_gbuffer g, const float *__restrict__ z, int n_lat,
                                                        int ablation, float *__restrict__ X0, int ld0,
                                                        float *__restrict__ A, int lda, int ang0, int *status) {
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= g.n) return;
  const int m = g.material[b];
  float *x = X0 + b * ld0;
  float *xa = A + b * lda;
  const int ks = paper_spatial_channels(ablation);
  if (m >= n_lat) {
    if (lane == 0) atomicOr(status, kStatusBadMaterial);
    x[lane] = 0.0f;
    x[32 + lane] = 0.0f;
    if (lane < ks) x[kPnLatent + lane] = 0.0f;
    if (lane < kPnAng) xa[ang0 + lane] = 0.0f;
    return;
  }
  x[lane] = z[(int64_t)m * kPnLatent + lane];
  x[32 + lane] = z[(int64_t)m * kPnLatent + 32 + lane];
  const float u = g.u[b], v = g.v[b], r = g.radius[b];
  if (ablation == kPnNoOneBlob) {
    if (lane < 3)
      x[kPnLatent + lane] = lane == 0   ? u - floorf(u)
                            : lane == 1 ? v - floorf(v)
                                        : (logf(fmaxf(r, kRFloor)) - kPnLnRLo) * kPnInvLnSpan;
  } else if (lane < kPnBlob) {
    x[kPnLatent + lane] = pn_blob_channel(u, v, r, lane);
  }
  if (lane < kPnAng) xa[ang0 + lane] = lane < 3 ? g.wi[3 * b + lane] : g.wo[3 * b + lane - 3];
}

// Components (C = max(0, y), S = max(0, expm1(y) / 100), the inverse of
// Eq. 9) and RGB by Eq. 8 from the raw head y [n][4].
__global__ void pn_head_kernel(const float *__restrict__ Y, const uint16_t *__restrict__ mat, int64_t n,
                               const DevMaterial *__restrict__ mats, int n_mat, float *__restrict__ rgb,
                               float *__restrict__ comps) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int m = mat[b];
  float c4[4];
  if (m >= n_mat) {
    c4[0] = c4[1] = c4[2] = c4[3] = __int_as_float(0x7FC00000);
  } else {
    c4[0] = fmaxf(0.0f, Y[4 * b]);
    c4[1] = fmaxf(0.0f, Y[4 * b + 1]);
    c4[2] = fmaxf(0.0f, expm1f(Y[4 * b + 2]) / kSpecK);
    c4[3] = fmaxf(0.0f, expm1f(Y[4 * b + 3]) / kSpecK);
  }
  if (comps) store_row4(comps, b, c4[0], c4[1], c4[2], c4[3]);
  if (rgb) {
    const DevMaterial &M = mats[m < n_mat ? m : 0];
    for (int ch = 0; ch < 3; ++ch)
      rgb[3 * b + ch] = M.kd[0][ch] * c4[0] + M.kd[1][ch] * c4[1] + M.ks[0][ch] * c4[2] + M.ks[1][ch] * c4[3];
  }
}

// d loss / d y and the loss of each query (Eq. 11 or the rendered option);
// one partial per CTA of 256 queries.
__global__ void __launch_bounds__(256) pn_loss_kernel(const float *__restrict__ Y, const float *__restrict__ target,
                                                      const float *__restrict__ wi, int64_t n, int mode,
                                                      float inv_batch, float *__restrict__ DY,
                                                      double *__restrict__ part) {
  __shared__ double red[256];
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double loss = 0.0;
  if (b < n) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      DY[4 * b + k] = loss_grad(k, Y[4 * b + k], target[4 * b + k], wi[3 * b + 2], mode, inv_batch, &loss);
  }
  red[threadIdx.x] = loss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < 256; ++k) s += red[k];
    part[blockIdx.x] = s;
  }
}

// One warp: lane l sums the partials l, l + 32, ... in order, then a fixed
// shuffle tree adds the lanes.
__global__ void pn_loss_final_kernel(const double *__restrict__ part, int n, double *__restrict__ loss) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int k = lane; k < n; k += 32) s += part[k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) *loss = s;
}

// Per batch segment s: the sums of the rows of D [B][W] by material, part
// [s][m][W].  One CTA of 256 threads per segment and 32 columns: the CTA
// sorts the segment's (material, row) keys in shared memory (bitonic) while
// its 512 x 32 slice of D lands in shared memory (all loads in flight
// together), finds each material's run in the sorted keys, and then warp w
// takes materials w, w + 8, ...: each lane adds its column's rows of the
// material in row order in a register (zero for a material the segment
// lacks).  Every sum runs in row order (bitwise repeatable).
constexpr int kSumRows = 512;     // rows per segment
constexpr int kSumThreads = 256;
constexpr int kSumLd = 33;        // shared row stride of the D slice (conflict-free column reads)
constexpr uint32_t kNoMat = 0xFFFFu;
constexpr size_t kSumTileBytes = (size_t)kSumRows * kSumLd * sizeof(float);
// the D slice, then each material's first and end index in the sorted keys
inline size_t sum_smem(int n_mat) { return kSumTileBytes + 2 * sizeof(int) * (size_t)n_mat; }

__global__ void __launch_bounds__(kSumThreads) pn_material_sums_kernel(const uint16_t *__restrict__ mat, int64_t n,
                                                                       const float *__restrict__ D, int W,
                                                                       int n_mat, float *__restrict__ part) {
  extern __shared__ float tile[];          // [kSumRows][kSumLd]
  __shared__ uint32_t key[kSumRows];       // (material << 16) | row
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = blockIdx.y * 32;
  const int64_t b0 = (int64_t)blockIdx.x * kSumRows;
  const int rows = (int)(n - b0 < kSumRows ? n - b0 : kSumRows);
  // the slice: row r, column lane, by warp r % 8
  for (int k0 = 0; k0 < kSumRows / 8; k0 += 16) {   // sixteen loads in flight per thread
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = warp + 8 * (k0 + k);
      v[k] = r < rows && c0 + lane < W ? D[(b0 + r) * W + c0 + lane] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) tile[(warp + 8 * (k0 + k)) * kSumLd + lane] = v[k];
  }
  for (int r = tid; r < kSumRows; r += kSumThreads) {
    uint32_t m = r < rows ? (uint32_t)mat[b0 + r] : kNoMat;
    if (m >= (uint32_t)n_mat) m = kNoMat;   // a bad index (flagged by the inputs kernel) sorts last, unused
    key[r] = (m << 16) | (uint32_t)r;
  }
  __syncthreads();
  for (int k = 2; k <= kSumRows; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < kSumRows; i += kSumThreads) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint32_t x = key[i], y = key[ixj];
          if ((x > y) == ((i & k) == 0)) {
            key[i] = y;
            key[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  // each material's run [first, end) in the sorted keys (first = -1: absent)
  int *first = reinterpret_cast<int *>(tile + kSumRows * kSumLd);
  int *end = first + n_mat;
  for (int m = tid; m < n_mat; m += kSumThreads) first[m] = -1;
  __syncthreads();
  for (int i = tid; i < rows; i += kSumThreads) {
    const uint32_t m = key[i] >> 16;
    if (m == kNoMat) continue;
    if (i == 0 || (key[i - 1] >> 16) != m) first[m] = i;
    if (i == rows - 1 || (key[i + 1] >> 16) != m) end[m] = i + 1;
  }
  __syncthreads();
  // warp w: materials w, w + 8, ...; lane: one column, the material's rows in row order
  const int c = c0 + lane;
  if (c >= W) return;
  float *out = part + (int64_t)blockIdx.x * n_mat * W + c;
  for (int m = warp; m < n_mat; m += kSumThreads / 32) {
    float s = 0.0f;
    const int i0 = first[m];
    if (i0 >= 0) {
      const int i1 = end[m];
      int i = i0;
      for (; i + 4 <= i1; i += 4) {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = tile[(key[i + q] & 0xFFFFu) * kSumLd + lane];
#pragma unroll
        for (int q = 0; q < 4; ++q) s += v[q];
      }
      for (; i < i1; ++i) s += tile[(key[i] & 0xFFFFu) * kSumLd + lane];
    }
    out[(int64_t)m * W] = s;
  }
}

// G[m][d] = sum over segments, in segment order.
__global__ void pn_segment_total_kernel(const float *__restrict__ part, int n_mat, int segs, int W,
                                        float *__restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_mat * W) return;
  const int64_t stride = (int64_t)n_mat * W;
  float s = 0.0f;
  int k = 0;
  for (; k + 8 <= segs; k += 8) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = part[(k + q) * stride + e];   // eight loads in flight, added in order
#pragma unroll
    for (int q = 0; q < 8; ++q) s += v[q];
  }
  for (; k < segs; ++k) s += part[k * stride + e];
  G[e] = s;
}

// ---------------------------------------------------------------- encoder
constexpr int kEH = 128;
constexpr int kEI = kPatternSlots + 6;   // 22 material features
constexpr int oE1 = 0, oe1 = oE1 + kEH * kEI, oE2 = oe1 + kEH, oe2 = oE2 + kEH * kEH, oE3 = oe2 + kEH,
              oe3 = oE3 + kPnLatent * kEH;
static_assert(oe3 + kPnLatent == kPnEncParams, "encoder layout");

__device__ __forceinline__ float elrelu(float x) { return x > 0.0f ? x : kPnSlope * x; }

// Four materials per CTA of 128 threads: features, h1, h2 (post-activation)
// and z; h1, h2 and the features are kept for the backward pass.  Thread j
// loads row j of a layer's weights into registers once (all loads in flight
// together) and applies it to the four materials; every output is a chain
// of fmaf over its inputs in order, from the bias.
constexpr int kEncG = 4;

__global__ void __launch_bounds__(kEH) pn_enc_fwd_kernel(const fabric_material *__restrict__ raw, int n_mat,
                                                         const float *__restrict__ enc, float *__restrict__ F,
                                                         float *__restrict__ H1, float *__restrict__ H2,
                                                         float *__restrict__ z) {
  __shared__ float f[kEncG][kEI];
  __shared__ float h1[kEncG][kEH], h2[kEncG][kEH];
  const int m0 = blockIdx.x * kEncG, j = threadIdx.x;
  const int nm = min(kEncG, n_mat - m0);
  for (int e = j; e < kEncG * kEI; e += kEH) {
    const int g = e / kEI, i = e % kEI;
    float v = 0.0f;
    if (g < nm) {
      const fabric_material &M = raw[m0 + g];
      if (i < kPatternSlots) {
        v = M.pattern_id == i ? 1.0f : 0.0f;
      } else {
        const int q = i - kPatternSlots;
        v = q == 0 ? M.twist_deg / 30.0f : q == 1 ? M.incl_deg / 45.0f : q == 2 ? M.alpha[0] : q == 3 ? M.beta[0]
          : q == 4 ? M.alpha[1] : M.beta[1];
      }
      if (F) F[(int64_t)(m0 + g) * kEI + i] = v;
    }
    f[g][i] = v;
  }
  __syncthreads();
  float a[kEncG];
  {
    float c[kEI];
#pragma unroll
    for (int i = 0; i < kEI; ++i) c[i] = enc[oE1 + j * kEI + i];
    const float b = enc[oe1 + j];
#pragma unroll
    for (int g = 0; g < kEncG; ++g) {
      a[g] = b;
#pragma unroll
      for (int i = 0; i < kEI; ++i) a[g] = fmaf(c[i], f[g][i], a[g]);
      h1[g][j] = elrelu(a[g]);
    }
  }
  __syncthreads();
  {
    float c[kEH];
    const float4 *w4 = reinterpret_cast<const float4 *>(enc + oE2 + j * kEH);
#pragma unroll
    for (int i4 = 0; i4 < kEH / 4; ++i4) {
      const float4 t = w4[i4];
      c[4 * i4] = t.x;
      c[4 * i4 + 1] = t.y;
      c[4 * i4 + 2] = t.z;
      c[4 * i4 + 3] = t.w;
    }
    const float b = enc[oe2 + j];
#pragma unroll
    for (int g = 0; g < kEncG; ++g) {
      a[g] = b + h1[g][j];   // skip before the last activation
#pragma unroll
      for (int i = 0; i < kEH; ++i) a[g] = fmaf(c[i], h1[g][i], a[g]);
      h2[g][j] = elrelu(a[g]);
      if (g < nm) {
        if (H1) H1[(int64_t)(m0 + g) * kEH + j] = h1[g][j];
        if (H2) H2[(int64_t)(m0 + g) * kEH + j] = h2[g][j];
      }
    }
  }
  __syncthreads();
  // z: thread j takes output k = j % 64 of materials g = j / 64 and g + 2
  {
    const int k = j % kPnLatent, g0 = j / kPnLatent;
    float c[kEH];
    const float4 *w4 = reinterpret_cast<const float4 *>(enc + oE3 + k * kEH);
#pragma unroll
    for (int i4 = 0; i4 < kEH / 4; ++i4) {
      const float4 t = w4[i4];
      c[4 * i4] = t.x;
      c[4 * i4 + 1] = t.y;
      c[4 * i4 + 2] = t.z;
      c[4 * i4 + 3] = t.w;
    }
    const float b = enc[oe3 + k];
#pragma unroll
    for (int gg = 0; gg < kEncG / 2; ++gg) {
      const int g = g0 + 2 * gg;
      float acc = b;
#pragma unroll
      for (int i = 0; i < kEH; ++i) acc = fmaf(c[i], h2[g][i], acc);
      if (g < nm) z[(int64_t)(m0 + g) * kPnLatent + k] = acc;
    }
  }
}

// Per material: da2, da1 (pre-activation gradients) from dz.
__global__ void __launch_bounds__(kEH) pn_enc_bwd_kernel(const float *__restrict__ enc, const float *__restrict__ H1,
                                                         const float *__restrict__ H2, const float *__restrict__ dz,
                                                         float *__restrict__ DA1, float *__restrict__ DA2) {
  __shared__ float sdz[kPnLatent], da2[kEH];
  const int m = blockIdx.x, j = threadIdx.x;
  if (j < kPnLatent) sdz[j] = dz[m * kPnLatent + j];
  __syncthreads();
  float g = 0.0f;
  for (int k = 0; k < kPnLatent; ++k) g = fmaf(enc[oE3 + k * kEH + j], sdz[k], g);
  const float d2 = g * (H2[m * kEH + j] > 0.0f ? 1.0f : kPnSlope);
  da2[j] = d2;
  DA2[m * kEH + j] = d2;
  __syncthreads();
  g = d2;   // through the skip
  for (int o = 0; o < kEH; ++o) g = fmaf(enc[oE2 + o * kEH + j], da2[o], g);
  DA1[m * kEH + j] = g * (H1[m * kEH + j] > 0.0f ? 1.0f : kPnSlope);
}

// Encoder parameter gradients as sums over materials of outer products,
// G[o][i] = sum_m L[m][o] R[m][i] (R = 1 for a bias): E1 (da1, features),
// e1, E2 (da2, h1), e2, E3 (dz, h2), e3.  A CTA of 256 threads takes a
// 32 x 32 tile of one block, stages 64 materials' slices of L and R in
// shared memory at a time, and thread (w, c) keeps outputs 4w..4w+3 of
// column c, each a chain of fmaf over the materials in order.
constexpr int kEncGradChunk = 64;

__host__ __device__ constexpr int pn_tiles(int rows, int cols) { return ((rows + 31) / 32) * ((cols + 31) / 32); }
constexpr int kPnEncGradTiles = pn_tiles(kEH, kEI) + pn_tiles(kEH, 1) + pn_tiles(kEH, kEH) + pn_tiles(kEH, 1) +
                                pn_tiles(kPnLatent, kEH) + pn_tiles(kPnLatent, 1);

__global__ void __launch_bounds__(256) pn_enc_grad_kernel(int n_mat, const float *__restrict__ F,
                                                          const float *__restrict__ H1, const float *__restrict__ H2,
                                                          const float *__restrict__ dz,
                                                          const float *__restrict__ DA1,
                                                          const float *__restrict__ DA2, float *__restrict__ genc) {
  __shared__ __align__(16) float sl[kEncGradChunk][32];
  __shared__ float sr[kEncGradChunk][32];
  // which block, and which 32 x 32 tile of it
  const float *L = DA1, *R = F;
  int ldl = kEH, ldr = kEI, rows = kEH, cols = kEI, out = oE1;
  int t = blockIdx.x;
  const int t0 = pn_tiles(kEH, kEI), t1 = t0 + pn_tiles(kEH, 1), t2 = t1 + pn_tiles(kEH, kEH),
            t3 = t2 + pn_tiles(kEH, 1), t4 = t3 + pn_tiles(kPnLatent, kEH);
  if (t >= t4) {
    L = dz; ldl = kPnLatent; R = nullptr; rows = kPnLatent; cols = 1; out = oe3; t -= t4;
  } else if (t >= t3) {
    L = dz; ldl = kPnLatent; R = H2; ldr = kEH; rows = kPnLatent; cols = kEH; out = oE3; t -= t3;
  } else if (t >= t2) {
    L = DA2; R = nullptr; cols = 1; out = oe2; t -= t2;
  } else if (t >= t1) {
    L = DA2; R = H1; ldr = kEH; cols = kEH; out = oE2; t -= t1;
  } else if (t >= t0) {
    R = nullptr; cols = 1; out = oe1; t -= t0;
  }
  const int ct = (cols + 31) / 32;
  const int r0 = (t / ct) * 32, c0 = (t % ct) * 32;
  const int tid = threadIdx.x, c = tid & 31, w = tid >> 5;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int m0 = 0; m0 < n_mat; m0 += kEncGradChunk) {
    const int mc = min(kEncGradChunk, n_mat - m0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kEncGradChunk * 32 / 256; ++q) {
      const int e = tid + 256 * q, mm = e >> 5, k = e & 31;
      const bool in = mm < mc;
      sl[mm][k] = in && r0 + k < rows ? L[(int64_t)(m0 + mm) * ldl + r0 + k] : 0.0f;
      sr[mm][k] = !in ? 0.0f : !R ? 1.0f : (c0 + k < cols ? R[(int64_t)(m0 + mm) * ldr + c0 + k] : 0.0f);
    }
    __syncthreads();
    for (int mm = 0; mm < mc; ++mm) {
      const float4 a = reinterpret_cast<const float4 *>(sl[mm])[w];
      const float x = sr[mm][c];
      acc[0] = fmaf(a.x, x, acc[0]);
      acc[1] = fmaf(a.y, x, acc[1]);
      acc[2] = fmaf(a.z, x, acc[2]);
      acc[3] = fmaf(a.w, x, acc[3]);
    }
  }
  if (c0 + c < cols) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = r0 + 4 * w + k;
      if (r < rows) genc[out + r * cols + c0 + c] = acc[k];
    }
  }
}

template <bool AR, bool BR, bool B_ONES>
cudaError_t gemm(const float *A, int64_t a_i, int64_t a_r, const float *B, int64_t b_j, int64_t b_r, int M, int N,
                 int64_t R, int64_t r_chunk, int chunks, const Epi &e, cudaStream_t s) {
  // 128-wide tiles where the extent fills them, else 64 (and 64-column
  // tiles for 129..192 columns: three instead of two mostly empty ones)
  const int nb = B_ONES ? N - 1 : N;   // columns that come from B
  const bool wm = M > 64, wn = nb > 64 && !(nb > 128 && nb <= 192);
  const int bm = wm ? 128 : 64, bn = wn ? 128 : 64;
  const dim3 grid((M + bm - 1) / bm, (nb + bn - 1) / bn, chunks);
  if (wm && wn)
    pn_gemm_kernel<128, 128, AR, BR, B_ONES><<<grid, kGemmThreads, 0, s>>>(A, a_i, a_r, B, b_j, b_r, M, N, R, r_chunk, e);
  else if (wm)
    pn_gemm_kernel<128, 64, AR, BR, B_ONES><<<grid, kGemmThreads, 0, s>>>(A, a_i, a_r, B, b_j, b_r, M, N, R, r_chunk, e);
  else if (wn)
    pn_gemm_kernel<64, 128, AR, BR, B_ONES><<<grid, kGemmThreads, 0, s>>>(A, a_i, a_r, B, b_j, b_r, M, N, R, r_chunk, e);
  else
    pn_gemm_kernel<64, 64, AR, BR, B_ONES><<<grid, kGemmThreads, 0, s>>>(A, a_i, a_r, B, b_j, b_r, M, N, R, r_chunk, e);
  return cudaGetLastError();
}

// forward layer: out[b][j] = act(sum_k X[b][k] Wt[j][k] + bias[j] (+ res))
cudaError_t fwd(const float *X, int ldx, int K, const float *Wt, const float *bias, int N, int64_t B, float *out,
                int ldo, const float *res, int ldr, bool act, cudaStream_t s) {
  Epi e{};
  e.mode = 0;
  e.bias = bias;
  e.res = res;
  e.ld_res = ldr;
  e.lrelu = act ? 1 : 0;
  e.out = out;
  e.ld_out = ldo;
  return gemm<true, true, false>(X, ldx, 1, Wt, K, 1, (int)B, N, K, K, 1, e, s);
}

// input gradient: dX[b][k] = (sum_j dZ[b][j] Wt[j][k] (+ add)) * lrelu'(h[b][k]), k < Kout
cudaError_t bwd_in(const float *dZ, int ldz, int N, const float *Wt, int ldw, int Kout, int64_t B, float *out,
                   int ldo, const float *add, int lda, const float *h, int ldh, cudaStream_t s) {
  Epi e{};
  e.mode = 1;
  e.res = add;
  e.ld_res = lda;
  e.h = h;
  e.ld_h = ldh;
  e.out = out;
  e.ld_out = ldo;
  return gemm<true, false, false>(dZ, ldz, 1, Wt, 1, ldw, (int)B, Kout, N, N, 1, e, s);
}

// weight and bias gradients: dW[j][k] = sum_b dZ[b][j] X[b][k], db[j] = sum_b dZ[b][j]
cudaError_t wgrad(const float *dZ, int ldz, int N, const float *X, int ldx, int K, int64_t B, float *part,
                  float *dW, float *db, cudaStream_t s) {
  const int chunks = (int)((B + kChunkRows - 1) / kChunkRows);
  Epi e{};
  e.mode = 2;
  e.out = part;
  e.slab = (int64_t)N * (K + 1);
  cudaError_t err = gemm<false, false, true>(dZ, 1, ldz, X, 1, ldx, N, K + 1, B, kChunkRows, chunks, e, s);
  if (err != cudaSuccess) return err;
  const int tot = N * (K + 1);
  pn_reduce_chunks_kernel<<<(unsigned)((4 * (int64_t)tot + 255) / 256), 256, 0, s>>>(part, chunks, N, K, dW, db);
  return cudaGetLastError();
}

}  // namespace

// Largest training material table the step accepts, at any width (the
// latent sums keep n_mat x W partials per 512-row segment in the scratch).
int paper_train_max_materials(int) { return 1600; }

size_t paper_train_work_bytes(int w, int64_t B, int n_mat) {
  const int64_t chunks = (B + kChunkRows - 1) / kChunkRows;
  const int64_t segs = (B + kSumRows - 1) / kSumRows;
  const int kx_max = kPnLatent + kPnBlob + kPnAng;        // widest first layer (no fusion)
  const int k_max = kx_max > w + kPnAng ? kx_max : w + kPnAng;
  size_t f = 0;
  f += (size_t)B * kx_max;                        // X0
  f += (size_t)B * w;                             // H1
  f += (size_t)B * (w + kPnAng);                  // XA
  f += 4 * (size_t)B * w;                         // K1..K4
  f += 2 * (size_t)B * 4;                         // Y, DY
  f += 3 * (size_t)B * w;                         // three gradient buffers
  f += (size_t)chunks * w * (k_max + 1);          // weight-gradient partials (widest layer)
  f += (size_t)n_mat * segs * w + (size_t)n_mat * w + (size_t)n_mat * kPnLatent;   // latent sums, G, dz
  f += (size_t)n_mat * (kEI + 4 * kEH + kPnLatent);                                // encoder
  f += 64 * 32;
  return f * 4 + ((size_t)(B + 255) / 256) * 8 + 8192;
}

namespace {

// Activation buffers of one pass over a batch of B queries: the first
// layer's input X0 [B][KX0], the first layer's output H1, A1's input XA
// [B][KA] (the second layer's output, then the angular inputs with the
// spatial fusion), K1..K4, the raw head Y.
struct PnPass {
  int w, ablation, KX0, KA;
  float *X0, *H1, *XA, *K1, *K2, *K3, *K4, *Y;
};

template <class Take>
PnPass pn_pass_buffers(int w, int ablation, int64_t B, Take take) {
  PnPass P;
  P.w = w;
  P.ablation = ablation;
  P.KX0 = paper_x0_inputs(ablation);
  P.KA = paper_a1_inputs(w, ablation);
  P.X0 = take((size_t)B * P.KX0);
  P.H1 = take((size_t)B * w);
  P.XA = take((size_t)B * P.KA);
  P.K1 = take((size_t)B * w);
  P.K2 = take((size_t)B * w);
  P.K3 = take((size_t)B * w);
  P.K4 = take((size_t)B * w);
  P.Y = take((size_t)B * 4);
  return P;
}

// Inputs and the forward pass of the structure (or its ablation): the raw
// head in P.Y.
cudaError_t pn_forward(const PnPass &P, const fabric_gbuffer &q, const float *z, int n_mat, const float *dec,
                       int *status, cudaStream_t s) {
  const PaperOffsets o = paper_offsets_ablation(P.w, P.ablation);
  const int64_t B = q.n;
  const int w = P.w;
  cudaError_t e;
  const bool fusion = P.ablation != kPnNoFusion;
  pn_inputs_kernel<<<(unsigned)((B + 7) / 8), 256, 0, s>>>(
      q, z, n_mat, P.ablation, P.X0, P.KX0, fusion ? P.XA : P.X0, fusion ? P.KA : P.KX0,
      fusion ? w : kPnLatent + kPnBlob, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = fwd(P.X0, P.KX0, P.KX0, dec + o.S1, dec + o.s1, w, B, P.H1, w, nullptr, 0, true, s)) != cudaSuccess)
    return e;
  if ((e = fwd(P.H1, w, w, dec + o.S2, dec + o.s2, w, B, P.XA, P.KA, nullptr, 0, true, s)) != cudaSuccess) return e;
  if ((e = fwd(P.XA, P.KA, P.KA, dec + o.A1, dec + o.a1, w, B, P.K1, w, nullptr, 0, true, s)) != cudaSuccess) return e;
  if ((e = fwd(P.K1, w, w, dec + o.A2, dec + o.a2, w, B, P.K2, w, nullptr, 0, true, s)) != cudaSuccess) return e;
  if ((e = fwd(P.K2, w, w, dec + o.A3, dec + o.a3, w, B, P.K3, w, P.K1, w, true, s)) != cudaSuccess) return e;   // skip
  if ((e = fwd(P.K3, w, w, dec + o.A4, dec + o.a4, w, B, P.K4, w, nullptr, 0, true, s)) != cudaSuccess) return e;
  return fwd(P.K4, w, w, dec + o.A5, dec + o.a5, 4, B, P.Y, 4, nullptr, 0, false, s);
}

}  // namespace

// One step's forward, loss and backward: grad [decoder | encoder] and the
// batch loss; raw = device copy of the training materials.
cudaError_t launch_paper_train(int w, int ablation, const fabric_gbuffer &q, const float *target, int loss_mode,
                               const fabric_material *raw, int n_mat, const float *dec, const float *enc,
                               float *grad, double *loss, void *work, int *status, cudaStream_t s) {
  const PaperOffsets o = paper_offsets_ablation(w, ablation);
  const int64_t B = q.n;
  const int segs = (int)((B + kSumRows - 1) / kSumRows);
  float *p = static_cast<float *>(work);
  auto take = [&](size_t nfl) {
    float *r = p;
    p += (nfl + 63) & ~size_t(63);
    return r;
  };
  const PnPass P = pn_pass_buffers(w, ablation, B, take);
  const int KX0 = P.KX0, KA = P.KA;
  float *DY = take((size_t)B * 4);
  float *D1 = take((size_t)B * w), *D2 = take((size_t)B * w), *D3 = take((size_t)B * w);
  const int64_t chunks = (B + kChunkRows - 1) / kChunkRows;
  // weight-gradient partials of the widest layer: K = KX0 (first), KA (A1) or W
  const int k_max = KX0 > KA ? (KX0 > w ? KX0 : w) : (KA > w ? KA : w);
  float *part = take((size_t)chunks * w * (k_max + 1));
  float *msum = take((size_t)n_mat * segs * w), *G = take((size_t)n_mat * w), *dz = take((size_t)n_mat * kPnLatent);
  float *F = take((size_t)n_mat * kEI), *EH1 = take((size_t)n_mat * kEH), *EH2 = take((size_t)n_mat * kEH);
  float *DA1 = take((size_t)n_mat * kEH), *DA2 = take((size_t)n_mat * kEH), *z = take((size_t)n_mat * kPnLatent);
  double *lpart = reinterpret_cast<double *>(take((size_t)((B + 255) / 256) * 2));
  float *gd = grad, *ge = grad + o.total;
  cudaError_t e;
#define PN_TRY(x)                     \
  do {                                \
    e = (x);                          \
    if (e != cudaSuccess) return e;   \
  } while (0)
  // ---- encoder, inputs and forward
  pn_enc_fwd_kernel<<<(n_mat + kEncG - 1) / kEncG, kEH, 0, s>>>(raw, n_mat, enc, F, EH1, EH2, z);
  PN_TRY(cudaGetLastError());
  PN_TRY(pn_forward(P, q, z, n_mat, dec, status, s));
  // ---- loss
  const int lblocks = (int)((B + 255) / 256);
  pn_loss_kernel<<<lblocks, 256, 0, s>>>(P.Y, target, q.wi, B, loss_mode, 1.0f / (float)B, DY, lpart);
  PN_TRY(cudaGetLastError());
  pn_loss_final_kernel<<<1, 32, 0, s>>>(lpart, lblocks, loss);
  PN_TRY(cudaGetLastError());
  // ---- backward (D1..D3 rotate as dq4, dq3, dq2, dq1, dg2, dg1)
  PN_TRY(wgrad(DY, 4, 4, P.K4, w, w, B, part, gd + o.A5, gd + o.a5, s));
  PN_TRY(bwd_in(DY, 4, 4, dec + o.A5, w, w, B, D1, w, nullptr, 0, P.K4, w, s));          // dq4
  PN_TRY(wgrad(D1, w, w, P.K3, w, w, B, part, gd + o.A4, gd + o.a4, s));
  PN_TRY(bwd_in(D1, w, w, dec + o.A4, w, w, B, D2, w, nullptr, 0, P.K3, w, s));          // dq3
  PN_TRY(wgrad(D2, w, w, P.K2, w, w, B, part, gd + o.A3, gd + o.a3, s));
  PN_TRY(bwd_in(D2, w, w, dec + o.A3, w, w, B, D3, w, nullptr, 0, P.K2, w, s));          // dq2
  PN_TRY(wgrad(D3, w, w, P.K1, w, w, B, part, gd + o.A2, gd + o.a2, s));
  PN_TRY(bwd_in(D3, w, w, dec + o.A2, w, w, B, D1, w, D2, w, P.K1, w, s));               // dq1 (+ dq3 through the skip)
  PN_TRY(wgrad(D1, w, w, P.XA, KA, KA, B, part, gd + o.A1, gd + o.a1, s));
  PN_TRY(bwd_in(D1, w, w, dec + o.A1, KA, w, B, D2, w, nullptr, 0, P.XA, KA, s));        // dg2
  PN_TRY(wgrad(D2, w, w, P.H1, w, w, B, part, gd + o.S2, gd + o.s2, s));
  PN_TRY(bwd_in(D2, w, w, dec + o.S2, w, w, B, D3, w, nullptr, 0, P.H1, w, s));          // dg1
  PN_TRY(wgrad(D3, w, w, P.X0, KX0, KX0, B, part, gd + o.S1, gd + o.s1, s));
  // ---- latent gradient: per-material sums of dg1 in row order, times S1's latent block
  {
    PN_TRY(ensure_max_dyn_smem(reinterpret_cast<const void *>(pn_material_sums_kernel), (int)sum_smem(1600)));
    pn_material_sums_kernel<<<dim3(segs, (w + 31) / 32), kSumThreads, sum_smem(n_mat), s>>>(q.material, B, D3, w, n_mat,
                                                                                       msum);
    PN_TRY(cudaGetLastError());
    pn_segment_total_kernel<<<(n_mat * w + 255) / 256, 256, 0, s>>>(msum, n_mat, segs, w, G);
    PN_TRY(cudaGetLastError());
    // dz[m][k] = sum_j G[m][j] S1[j][k], k < 64
    Epi ep{};
    ep.mode = 1;
    ep.out = dz;
    ep.ld_out = kPnLatent;
    PN_TRY((gemm<true, false, false>(G, w, 1, dec + o.S1, 1, KX0, n_mat, kPnLatent, w, w, 1, ep, s)));
  }
  // ---- encoder backward
  pn_enc_bwd_kernel<<<n_mat, kEH, 0, s>>>(enc, EH1, EH2, dz, DA1, DA2);
  PN_TRY(cudaGetLastError());
  pn_enc_grad_kernel<<<kPnEncGradTiles, 256, 0, s>>>(n_mat, F, EH1, EH2, dz, DA1, DA2, ge);
  PN_TRY(cudaGetLastError());
#undef PN_TRY
  return cudaSuccess;
}

size_t paper_forward_work_bytes(int w, int64_t B) {
  const int kx_max = kPnLatent + kPnBlob + kPnAng;
  return ((size_t)B * (kx_max + (w + kPnAng) + 5 * (size_t)w + 4) + 64 * 16) * 4 + 4096;
}

// FP32 forward of the structure (or an ablation) over a G-buffer, with
// per-material latents z [n_mat][64]: components and RGB.
cudaError_t launch_paper_forward(int w, int ablation, const fabric_gbuffer &g, const float *z,
                                 const DevMaterial *mats, int n_mat, const float *dec, float *rgb, float *comps,
                                 void *work, int *status, cudaStream_t s) {
  float *p = static_cast<float *>(work);
  auto take = [&](size_t nfl) {
    float *r = p;
    p += (nfl + 63) & ~size_t(63);
    return r;
  };
  const PnPass P = pn_pass_buffers(w, ablation, g.n, take);
  cudaError_t e = pn_forward(P, g, z, n_mat, dec, status, s);
  if (e != cudaSuccess) return e;
  pn_head_kernel<<<(unsigned)((g.n + 255) / 256), 256, 0, s>>>(P.Y, g.material, g.n, mats, n_mat, rgb, comps);
  return cudaGetLastError();
}

cudaError_t launch_paper_encoder(const fabric_material *raw, int n_mat, const float *enc, float *z, cudaStream_t s) {
  pn_enc_fwd_kernel<<<(n_mat + kEncG - 1) / kEncG, kEH, 0, s>>>(raw, n_mat, enc, nullptr, nullptr, nullptr, z);
  return cudaGetLastError();
}

}  // namespace fab
