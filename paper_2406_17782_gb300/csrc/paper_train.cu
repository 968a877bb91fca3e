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

constexpr int TM = 64, TN = 64, TR = 16;
constexpr int kGemmThreads = 256;
constexpr int kChunkRows = 512;    // batch rows per weight-gradient partial

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

// C(i, j) = sum_r A(i, r) B(j, r) for i < M, j < N, r in [r0, r1), with
// A(i, r) = A[i a_i + r a_r] and B(j, r) = B[j b_j + r b_r].  AR / BR: the
// operand is contiguous along r (else along i / j).  B_ONES: column j = N - 1
// of B is the constant 1 (the bias gradient as an extra output column).
template <bool AR, bool BR, bool B_ONES>
__global__ void __launch_bounds__(kGemmThreads) pn_gemm_kernel(const float *__restrict__ A, int64_t a_i, int64_t a_r,
                                                               const float *__restrict__ Bm, int64_t b_j,
                                                               int64_t b_r, int M, int N, int64_t R,
                                                               int64_t r_chunk, Epi e) {
  __shared__ float As[TR][TM + 4];
  __shared__ float Bs[TR][TN + 4];
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int i0 = blockIdx.x * TM, j0 = blockIdx.y * TN;
  const int64_t r_begin = (int64_t)blockIdx.z * r_chunk;
  const int64_t r_end = r_begin + r_chunk < R ? r_begin + r_chunk : R;
  float acc[4][4] = {};
  for (int64_t r0 = r_begin; r0 < r_end; r0 += TR) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int el = tid + kGemmThreads * q;
      const int rr = AR ? el % TR : el / TM, ii = AR ? el / TR : el % TM;
      const int64_t gi = i0 + ii, gr = r0 + rr;
      As[rr][ii] = (gi < M && gr < r_end) ? A[gi * a_i + gr * a_r] : 0.0f;
      const int rb = BR ? el % TR : el / TN, jj = BR ? el / TR : el % TN;
      const int64_t gj = j0 + jj, gb = r0 + rb;
      float bv = 0.0f;
      if (gj < N && gb < r_end) bv = (B_ONES && gj == N - 1) ? 1.0f : Bm[gj * b_j + gb * b_r];
      Bs[rb][jj] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TR; ++r) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[r][ty * 4 + q];
        b[q] = Bs[r][tx * 4 + q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[q][s] = fmaf(a[q], b[s], acc[q][s]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t i = i0 + ty * 4 + q;
    if (i >= M) continue;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int j = j0 + tx * 4 + s;
      if (j >= N) continue;
      float v = acc[q][s];
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

// out_w[i][j] = sum_c part[c][i][j] for j < K, out_b[i] = sum_c part[c][i][K]
// (chunks in order).
__global__ void pn_reduce_chunks_kernel(const float *__restrict__ part, int chunks, int M, int K,
                                       float *__restrict__ out_w, float *__restrict__ out_b) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = K + 1;
  if (e >= M * N) return;
  float s = 0.0f;
  for (int c = 0; c < chunks; ++c) s += part[(int64_t)c * M * N + e];
  const int i = e / N, j = e % N;
  if (j < K)
    out_w[i * K + j] = s;
  else
    out_b[i] = s;
}

// One-blob bins of the footprint (FP32, accurate exp): the periodic
// Gaussians of frac u and frac v (nearest image and the one on the far
// side) and the plain ones of the size coordinate.
__device__ __forceinline__ void pn_blob_fp32(float u, float v, float r, float *o) {
  const float fu = u - floorf(u), fv = v - floorf(v);
  const float t = (logf(fmaxf(r, kRFloor)) - kPnLnRLo) * kPnInvLnSpan;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float c = (i + 0.5f) * 0.125f;
    float d = fu - c;
    d -= rintf(d);
    float e = 1.0f - fabsf(d);
    o[i] = expf(-32.0f * d * d) + expf(-32.0f * e * e);
    d = fv - c;
    d -= rintf(d);
    e = 1.0f - fabsf(d);
    o[8 + i] = expf(-32.0f * d * d) + expf(-32.0f * e * e);
    d = t - c;
    o[16 + i] = expf(-32.0f * d * d);
  }
}

// X0[b] = [z_mat (64) | spatial channels (24 one-blob, or 3 unencoded)]
// (row stride ld0) and the angular inputs (wi, wo.xy) at columns
// ang0..ang0+4 of the row of A (row stride lda): XA after the fused
// spatial feature, or X0 itself without the fusion.
__global__ void pn_inputs_kernel(fabric_gbuffer g, const float *__restrict__ z, int n_lat, int ablation,
                                 float *__restrict__ X0, int ld0, float *__restrict__ A, int lda, int ang0,
                                 int *status) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.n) return;
  int m = g.material[b];
  float *x = X0 + b * ld0;
  float *xa = A + b * lda;
  const int ks = paper_spatial_channels(ablation);
  if (m >= n_lat) {
    atomicOr(status, kStatusBadMaterial);
    for (int k = 0; k < kPnLatent + ks; ++k) x[k] = 0.0f;
    for (int k = 0; k < kPnAng; ++k) xa[ang0 + k] = 0.0f;
    return;
  }
  for (int k = 0; k < kPnLatent; ++k) x[k] = z[(int64_t)m * kPnLatent + k];
  if (ablation == kPnNoOneBlob) {
    const float u = g.u[b], v = g.v[b];
    x[kPnLatent + 0] = u - floorf(u);
    x[kPnLatent + 1] = v - floorf(v);
    x[kPnLatent + 2] = (logf(fmaxf(g.radius[b], kRFloor)) - kPnLnRLo) * kPnInvLnSpan;
  } else {
    pn_blob_fp32(g.u[b], g.v[b], g.radius[b], x + kPnLatent);
  }
  xa[ang0 + 0] = g.wi[3 * b];
  xa[ang0 + 1] = g.wi[3 * b + 1];
  xa[ang0 + 2] = g.wi[3 * b + 2];
  xa[ang0 + 3] = g.wo[3 * b];
  xa[ang0 + 4] = g.wo[3 * b + 1];
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
  if (comps) reinterpret_cast<float4 *>(comps)[b] = make_float4(c4[0], c4[1], c4[2], c4[3]);
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

__global__ void pn_loss_final_kernel(const double *__restrict__ part, int n, double *__restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += part[k];
    *loss = s;
  }
}

// Per batch segment s: the sums of the rows of D [B][W] by material, part
// [s][m][W].  Each thread owns one column and walks the segment's rows in
// order, adding into its column of a shared-memory table of every
// material, so every sum runs in row order (bitwise repeatable).
constexpr int kSumRows = 512;   // rows per segment

__global__ void pn_material_sums_kernel(const uint16_t *__restrict__ mat, int64_t n, const float *__restrict__ D,
                                        int W, int n_mat, float *__restrict__ part) {
  extern __shared__ float acc[];   // [n_mat][W]
  __shared__ uint16_t smat[kSumRows];
  const int d = threadIdx.x;
  const int64_t b0 = (int64_t)blockIdx.x * kSumRows;
  const int rows = (int)(n - b0 < kSumRows ? n - b0 : kSumRows);
  for (int e = d; e < n_mat * W; e += blockDim.x) acc[e] = 0.0f;
  for (int r = d; r < rows; r += blockDim.x) smat[r] = mat[b0 + r];
  __syncthreads();
  const float *col = D + b0 * W + d;
  int r = 0;
  for (; r + 8 <= rows; r += 8) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = col[(int64_t)(r + q) * W];   // eight loads in flight
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (smat[r + q] < n_mat) acc[smat[r + q] * W + d] += v[q];   // a bad index is flagged by the inputs kernel
  }
  for (; r < rows; ++r)
    if (smat[r] < n_mat) acc[smat[r] * W + d] += col[(int64_t)r * W];
  float *out = part + (int64_t)blockIdx.x * n_mat * W;
  for (int m = 0; m < n_mat; ++m) out[m * W + d] = acc[m * W + d];
}

// G[m][d] = sum over segments, in segment order.
__global__ void pn_segment_total_kernel(const float *__restrict__ part, int n_mat, int segs, int W,
                                        float *__restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_mat * W) return;
  float s = 0.0f;
  for (int k = 0; k < segs; ++k) s += part[(int64_t)k * n_mat * W + e];
  G[e] = s;
}

// ---------------------------------------------------------------- encoder
constexpr int kEH = 128;
constexpr int kEI = kPatternSlots + 6;   // 22 material features
constexpr int oE1 = 0, oe1 = oE1 + kEH * kEI, oE2 = oe1 + kEH, oe2 = oE2 + kEH * kEH, oE3 = oe2 + kEH,
              oe3 = oE3 + kPnLatent * kEH;
static_assert(oe3 + kPnLatent == kPnEncParams, "encoder layout");

__device__ __forceinline__ float elrelu(float x) { return x > 0.0f ? x : kPnSlope * x; }

// One material per CTA of 128 threads: features, h1, h2 (post-activation)
// and z; h1, h2 and the features are kept for the backward pass.
__global__ void __launch_bounds__(kEH) pn_enc_fwd_kernel(const fabric_material *__restrict__ raw,
                                                         const float *__restrict__ enc, float *__restrict__ F,
                                                         float *__restrict__ H1, float *__restrict__ H2,
                                                         float *__restrict__ z) {
  __shared__ float f[kEI], h1[kEH], h2[kEH];
  const int m = blockIdx.x, j = threadIdx.x;
  if (j < kEI) {
    const fabric_material &M = raw[m];
    float v;
    if (j < kPatternSlots)
      v = M.pattern_id == j ? 1.0f : 0.0f;
    else {
      const int q = j - kPatternSlots;
      v = q == 0 ? M.twist_deg / 30.0f : q == 1 ? M.incl_deg / 45.0f : q == 2 ? M.alpha[0] : q == 3 ? M.beta[0]
        : q == 4 ? M.alpha[1] : M.beta[1];
    }
    f[j] = v;
    if (F) F[m * kEI + j] = v;
  }
  __syncthreads();
  float a = enc[oe1 + j];
  for (int i = 0; i < kEI; ++i) a = fmaf(enc[oE1 + j * kEI + i], f[i], a);
  h1[j] = elrelu(a);
  __syncthreads();
  a = enc[oe2 + j] + h1[j];   // skip before the last activation
  for (int i = 0; i < kEH; ++i) a = fmaf(enc[oE2 + j * kEH + i], h1[i], a);
  h2[j] = elrelu(a);
  if (H1) H1[m * kEH + j] = h1[j];
  if (H2) H2[m * kEH + j] = h2[j];
  __syncthreads();
  if (j < kPnLatent) {
    a = enc[oe3 + j];
    for (int i = 0; i < kEH; ++i) a = fmaf(enc[oE3 + j * kEH + i], h2[i], a);
    z[m * kPnLatent + j] = a;
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

// One thread per encoder parameter: sums over materials in order.
__global__ void pn_enc_grad_kernel(int n_mat, const float *__restrict__ F, const float *__restrict__ H1,
                                   const float *__restrict__ H2, const float *__restrict__ dz,
                                   const float *__restrict__ DA1, const float *__restrict__ DA2,
                                   float *__restrict__ genc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kPnEncParams) return;
  const float *dv;
  const float *xv = nullptr;
  int ldd, ldx = 0, o, i = -1;
  if (p < oe1) {
    o = p / kEI; i = p % kEI; dv = DA1; ldd = kEH; xv = F; ldx = kEI;
  } else if (p < oE2) {
    o = p - oe1; dv = DA1; ldd = kEH;
  } else if (p < oe2) {
    o = (p - oE2) / kEH; i = (p - oE2) % kEH; dv = DA2; ldd = kEH; xv = H1; ldx = kEH;
  } else if (p < oE3) {
    o = p - oe2; dv = DA2; ldd = kEH;
  } else if (p < oe3) {
    o = (p - oE3) / kEH; i = (p - oE3) % kEH; dv = dz; ldd = kPnLatent; xv = H2; ldx = kEH;
  } else {
    o = p - oe3; dv = dz; ldd = kPnLatent;
  }
  float s = 0.0f;
  for (int m = 0; m < n_mat; ++m) s = fmaf(dv[m * ldd + o], xv ? xv[m * ldx + i] : 1.0f, s);
  genc[p] = s;
}

template <bool AR, bool BR, bool B_ONES>
cudaError_t gemm(const float *A, int64_t a_i, int64_t a_r, const float *B, int64_t b_j, int64_t b_r, int M, int N,
                 int64_t R, int64_t r_chunk, int chunks, const Epi &e, cudaStream_t s) {
  const dim3 grid((M + TM - 1) / TM, (N + TN - 1) / TN, chunks);
  pn_gemm_kernel<AR, BR, B_ONES><<<grid, kGemmThreads, 0, s>>>(A, a_i, a_r, B, b_j, b_r, M, N, R, r_chunk, e);
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
  pn_reduce_chunks_kernel<<<(tot + 255) / 256, 256, 0, s>>>(part, chunks, N, K, dW, db);
  return cudaGetLastError();
}

}  // namespace

// Largest material table whose per-material sums fit the shared memory of
// one CTA (n_mat x W floats); the training call refuses larger tables.
int paper_train_max_materials(int w) { return (int)((200 * 1024) / (w * 4)); }

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
  pn_inputs_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(
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
  pn_enc_fwd_kernel<<<n_mat, kEH, 0, s>>>(raw, enc, F, EH1, EH2, z);
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
    const size_t smem = (size_t)n_mat * w * sizeof(float);
    PN_TRY(ensure_max_dyn_smem(reinterpret_cast<const void *>(pn_material_sums_kernel), 200 * 1024));
    pn_material_sums_kernel<<<segs, w, smem, s>>>(q.material, B, D3, w, n_mat, msum);
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
  pn_enc_grad_kernel<<<(kPnEncParams + 255) / 256, 256, 0, s>>>(n_mat, F, EH1, EH2, dz, DA1, DA2, ge);
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
  pn_enc_fwd_kernel<<<n_mat, kEH, 0, s>>>(raw, enc, nullptr, nullptr, nullptr, z);
  return cudaGetLastError();
}

}  // namespace fab
