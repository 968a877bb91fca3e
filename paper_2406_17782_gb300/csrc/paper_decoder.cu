// paper_decoder.cu -- the paper's own decoder structure (Sec. 4.2, "Decoder";
// Fig. 3) on the 5th-generation tensor cores: the footprint's position and
// size one-blob encoded (3 -> 24 channels), fused with the material latent by
// two fully connected layers (the spatial feature), then, with the angular
// inputs wi (x, y, z) and wo (x, y), an angular decoder of five fully
// connected layers with one skip connection; leaky ReLU throughout; the four
// components of Eq. 7 become RGB by Eq. 8.
//
// Same execution scheme as the workload's decoder (decoder_tc.cu): a
// persistent CTA holds one copy of the packed 16-bit weights in shared memory
// (one bulk copy), and WG tile pipelines of one warpgroup each stream
// 128-point tiles, one point per thread.  Per pipeline, tensor memory holds the
// FP32 accumulator D (W columns) and the 16-bit A operand of the next layer
// (two values per 32-bit column).  Seven MMA chains per tile:
//   L0  S1': [one-blob (24) | one-hot material] -> W     (latent folded: the
//       per-material column holds S1[:, :64] z_m + s1, exact algebra)
//   L1  S2 : h1 -> h                                    (bias in a constant-one column)
//   L2  A1 : [h | wi | wo.xy] -> k1
//   L3  A2 : k1 -> k2
//   L4  A3 : k2 -> k3, with the skip: k3 = lrelu(A3 k2 + a3 + k1), k1 kept
//       in registers as the 16-bit operand values written after L2
//   L5  A4 : k3 -> k4
//   L6  A5 : k4 -> y (N = 16, four used)
// The one-blob bins of the periodic footprint centre are Gaussians wrapped
// around the weave repeat (nearest image plus the one on the far side; the
// others weigh below exp(-32)).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fabric_internal.h"
#include "paper_net.h"
#include "tc_ptx.h"

namespace fab {
namespace {

constexpr int kTile = 128;
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz
constexpr int kPnMaxK1 = 128;                     // layer-0 K: 24 + materials, padded to 16

// Packed operands of width W (bytes; identical in global and shared memory):
// seven K-major weight blocks, then the per-material albedos.
struct PnBlob {
  int k1, kh;
  uint32_t l[7];
  uint32_t alb, total;
};

__host__ __device__ constexpr PnBlob pn_blob(int w, int n_mat) {
  PnBlob b{};
  b.k1 = (kPnBlob + n_mat + 15) / 16 * 16;
  b.kh = w + 16;
  b.l[0] = 0;
  b.l[1] = b.l[0] + (uint32_t)w * b.k1 * 2u;
  for (int i = 2; i <= 6; ++i) b.l[i] = b.l[i - 1] + (uint32_t)w * b.kh * 2u;
  b.alb = b.l[6] + 16u * b.kh * 2u;
  b.total = b.alb + ((uint32_t)(n_mat * 12 * 4) + 15u) / 16u * 16u;
  return b;
}

__host__ __device__ constexpr int pn_cols(int w) { return w == 64 ? 128 : 256; }   // tensor-memory columns per pipeline

template <bool F16>
__device__ __forceinline__ void put_op(uint8_t *base, uint32_t off, float v) {
  if (F16)
    *reinterpret_cast<__half *>(base + off) = __float2half_rn(v);
  else
    *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}

// Fold the latents into layer 0 and pack every layer into the canonical
// K-major layout; layers 1-6 carry their bias in input column W (A1: column
// W + 5, after the angular inputs), the rest of the K padding is zero.  One CTA.
template <int W, bool F16>
__global__ void __launch_bounds__(256) pn_pack_kernel(const float *__restrict__ p, const float *__restrict__ lat,
                                                      const DevMaterial *__restrict__ mats, int n_mat,
                                                      uint8_t *__restrict__ blob) {
  extern __shared__ float fold[];   // [n_mat][W]
  constexpr PaperOffsets o = paper_offsets(W);
  const PnBlob B = pn_blob(W, n_mat);
  for (int e = threadIdx.x; e < n_mat * W; e += blockDim.x) {
    const int m = e / W, r = e % W;
    float acc = p[o.s1 + r];
    for (int j = 0; j < kPnLatent; ++j) acc = fmaf(p[o.S1 + r * (kPnLatent + kPnBlob) + j], lat[m * kPnLatent + j], acc);
    fold[m * W + r] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < W * B.k1; e += blockDim.x) {
    const int r = e / B.k1, c = e % B.k1;
    float v = 0.0f;
    if (c < kPnBlob)
      v = p[o.S1 + r * (kPnLatent + kPnBlob) + kPnLatent + c];
    else if (c < kPnBlob + n_mat)
      v = fold[(c - kPnBlob) * W + r];
    put_op<F16>(blob, B.l[0] + tc::core_offset(r, c, B.k1), v);
  }
  // layers 1..5: [W][kh]; layer 6: [16][kh]
  const int wofs[6] = {o.S2, o.A1, o.A2, o.A3, o.A4, o.A5};
  const int bofs[6] = {o.s2, o.a1, o.a2, o.a3, o.a4, o.a5};
  for (int l = 1; l <= 6; ++l) {
    const int rows = l == 6 ? 16 : W;
    const int rows_used = l == 6 ? 4 : W;
    const int in = l == 2 ? W + kPnAng : W;   // weight columns
    for (int e = threadIdx.x; e < rows * B.kh; e += blockDim.x) {
      const int r = e / B.kh, c = e % B.kh;
      float v = 0.0f;
      if (r < rows_used) {
        if (c < in)
          v = p[wofs[l - 1] + r * in + c];
        else if (c == in)
          v = p[bofs[l - 1] + r];
      }
      put_op<F16>(blob, B.l[l] + tc::core_offset(r, c, B.kh), v);
    }
  }
  float *alb = reinterpret_cast<float *>(blob + B.alb);
  for (int e = threadIdx.x; e < n_mat * 12; e += blockDim.x) {
    const int m = e / 12, q = e % 12;
    const DevMaterial &M = mats[m];
    alb[e] = q < 3 ? M.kd[0][q] : q < 6 ? M.kd[1][q - 3] : q < 9 ? M.ks[0][q - 6] : M.ks[1][q - 9];
  }
}

struct PnArgs {
  const float *u, *v, *radius, *wi, *wo;
  const uint16_t *material;
  int64_t n, n_tiles;
  const uint8_t *blob;
  int n_mat;
  float *rgb, *comps;
  int *status;
};

struct PnPoint {
  float u, v, r, wi0, wi1, wi2, wo0, wo1;
  int mat;   // -1: beyond the end
};

__device__ __forceinline__ PnPoint pn_load(const PnArgs &a, int64_t p) {
  PnPoint q;
  q.u = q.v = q.r = q.wi0 = q.wi1 = q.wi2 = q.wo0 = q.wo1 = 0.0f;
  q.mat = -1;
  if (p < a.n) {
    q.mat = __ldg(a.material + p);
    q.u = __ldg(a.u + p);
    q.v = __ldg(a.v + p);
    q.r = __ldg(a.radius + p);
    q.wi0 = __ldg(a.wi + 3 * p);
    q.wi1 = __ldg(a.wi + 3 * p + 1);
    q.wi2 = __ldg(a.wi + 3 * p + 2);
    q.wo0 = __ldg(a.wo + 3 * p);
    q.wo1 = __ldg(a.wo + 3 * p + 1);
  }
  return q;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// exp(-d^2 / (2 sigma^2)) with sigma = 1/8, i.e. 2^(-32 log2(e) d^2)
constexpr float kGaussK = -46.16624130844683f;

// Eight periodic one-blob bins of x (wrapped Gaussians around the unit
// interval), packed two per word into w[0..3].
template <bool F16>
__device__ __forceinline__ void blob_periodic(float x, uint32_t *w) {
  const float f = x - floorf(x);
  float b[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float d = f - (i + 0.5f) * 0.125f;
    d -= rintf(d);                       // nearest image, |d| <= 1/2
    const float e = 1.0f - fabsf(d);     // the image on the far side
    b[i] = ex2_approx(kGaussK * d * d) + ex2_approx(kGaussK * e * e);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = tc::pack2<F16>(b[2 * k], b[2 * k + 1]);
}

template <bool F16>
__device__ __forceinline__ void blob_plain(float t, uint32_t *w) {
  float b[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float d = t - (i + 0.5f) * 0.125f;
    b[i] = ex2_approx(kGaussK * d * d);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = tc::pack2<F16>(b[2 * k], b[2 * k + 1]);
}

template <int PT>
__device__ __forceinline__ bool pn_bar_or(int wg, bool pred) {
  int r;
  const int id = 1 + wg;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((int)pred), "r"(id), "n"(PT)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ float lrelu(float x) { return fmaxf(x, kPnSlope * x); }

template <bool F16>
__device__ __forceinline__ float2 unpack2(uint32_t w) {
  if (F16) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
  } else {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
  }
}

// W: network width; F16: FP16 (else BF16) operands; WG tile pipelines per CTA;
// LDR: 32-column tensor-memory loads in flight per wait in the epilogues.
template <int W, bool F16, int WG, int LDR>
__global__ void __launch_bounds__(kTile * WG, (W == 64 && WG == 2) ? 2 : 1) pn_decoder_kernel(const PnArgs a) {
  constexpr int PT = kTile;
  constexpr uint32_t COLS = pn_cols(W);
  constexpr uint32_t COL_A = W;
  constexpr int KH = W + 16;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bar_w = reinterpret_cast<uint64_t *>(smem);
  uint64_t *bar_mma = bar_w + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar_w + 1 + WG);
  const PnBlob B = pn_blob(W, a.n_mat);
  uint8_t *wts = smem + 1024;
  const int tid = threadIdx.x;
  const int wg = tid / PT;
  const int row = tid % PT;
  const int warp = tid >> 5;
  const bool lead = row == 0;
  uint64_t *my_bar = bar_mma + wg;

  if (tid == 0) {
    tc::mbar_init(bar_w, 1);
    for (int g = 0; g < WG; ++g) tc::mbar_init(bar_mma + g, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, COLS * WG);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot + COLS * (uint32_t)wg;
  const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t t_d = tmem + lane, t_a = tmem + lane + COL_A;

  if (tid == 0) {
    tc::mbar_arrive_expect_tx(bar_w, B.total);
    tc::bulk_g2s(wts, a.blob, B.total, bar_w);
  }
  const int64_t stride = (int64_t)gridDim.x * WG;
  int64_t tile = (int64_t)blockIdx.x * WG + wg;
  PnPoint pt = pn_load(a, tile * kTile + row);
  bool ok = tc::mbar_wait_sleep(bar_w, 0, kWaitCycles);
  const float *alb = reinterpret_cast<const float *>(wts + B.alb);
  uint32_t wl[7];
#pragma unroll
  for (int l = 0; l < 7; ++l) wl[l] = tc::smem_addr(wts + B.l[l]);
  const uint32_t idW = F16 ? tc::idesc_f16(128, W) : tc::idesc_bf16(128, W);
  const uint32_t id16 = F16 ? tc::idesc_f16(128, 16) : tc::idesc_bf16(128, 16);
  const uint32_t one16 = F16 ? 0x3C00u : 0x3F80u;
  uint32_t phase = 0;

  for (; tile < a.n_tiles; tile += stride) {
    const int64_t p = tile * kTile + row;
    int mat = pt.mat;
    if (mat >= a.n_mat) {
      atomicOr(a.status, kStatusBadMaterial);
      mat = -2;
    }
    const float wi0 = pt.wi0, wi1 = pt.wi1, wi2 = pt.wi2, wo0 = pt.wo0, wo1 = pt.wo1;
    // ---- layer-0 A operand: one-blob (24 channels) and the one-hot material
    {
      uint32_t w[16];
      if (mat >= 0) {
        blob_periodic<F16>(pt.u, w);
        blob_periodic<F16>(pt.v, w + 4);
        const float t = (__logf(fmaxf(pt.r, kRFloor)) - kPnLnRLo) * kPnInvLnSpan;
        blob_plain<F16>(t, w + 8);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) w[k] = 0u;
      }
      const int hot = kPnBlob + mat;   // feature index of the material's bias column
#pragma unroll
      for (int k = 12; k < 16; ++k) w[k] = (hot == 2 * k ? one16 : 0u) | (hot == 2 * k + 1 ? one16 << 16 : 0u);
      tc::tmem_st16(t_a, w);           // features 0..31
      for (int c = 2; c < B.k1 / 16; ++c) {
        uint32_t h8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          h8[k] = (hot == 16 * c + 2 * k ? one16 : 0u) | (hot == 16 * c + 2 * k + 1 ? one16 << 16 : 0u);
        tc::tmem_st8(t_a + 8 * c, h8);
      }
      tc::tmem_st_wait();
    }
    uint32_t skip[W / 2];   // k1 as 16-bit operand pairs, for the residual block
#pragma unroll
    for (int layer = 0; layer < 7; ++layer) {
      tc::tc_fence_before();
      if (pn_bar_or<PT>(wg, !ok)) {
        ok = false;
        goto teardown;
      }
      if (lead) {
        tc::tc_fence_after();
        const int K = layer == 0 ? B.k1 : KH;
        const uint32_t sbo = (uint32_t)K * 16u;
        for (int kk = 0; kk < K / 16; ++kk) {
          const uint64_t bd = tc::smem_desc(wl[layer] + kk * 256u, 128u, sbo);
          tc::mma_f16_ts(tmem, tmem + COL_A + 8u * kk, bd, layer == 6 ? id16 : idW, kk > 0 ? 1u : 0u);
        }
        tc::mma_commit(my_bar);
      }
      if (layer == 0) pt = pn_load(a, (tile + stride) * kTile + row);   // next tile's inputs in flight
      ok = tc::mbar_wait_sleep(my_bar, phase, kWaitCycles) && ok;
      phase ^= 1u;
      tc::tc_fence_after();
      if (layer < 6) {
#pragma unroll
        for (int c0 = 0; c0 < W / 32; c0 += LDR) {
          float acc[32 * LDR];
#pragma unroll
          for (int r = 0; r < LDR; ++r) tc::tmem_ld32(t_d + 32 * (c0 + r), acc + 32 * r);
          tc::tmem_ld_wait();
#pragma unroll
          for (int r = 0; r < LDR; ++r) {
            uint32_t w[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              float x0 = acc[32 * r + 2 * k], x1 = acc[32 * r + 2 * k + 1];
              if (layer == 4) {
                const float2 s = unpack2<F16>(skip[(c0 + r) * 16 + k]);
                x0 += s.x;
                x1 += s.y;
              }
              w[k] = tc::pack2<F16>(lrelu(x0), lrelu(x1));
              if (layer == 2) skip[(c0 + r) * 16 + k] = w[k];
            }
            tc::tmem_st16(t_a + 16 * (c0 + r), w);
          }
        }
        // input columns W..W+15: the angular inputs and the constant one of
        // A1's bias after the spatial fusion, else the constant-one bias column
        uint32_t w8[8] = {one16, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        if (layer == 1) {
          w8[0] = tc::pack2<F16>(wi0, wi1);
          w8[1] = tc::pack2<F16>(wi2, wo0);
          w8[2] = tc::pack2<F16>(wo1, 1.0f);
        }
        tc::tmem_st8(t_a + W / 2, w8);
        tc::tmem_st_wait();
      } else {
        float y[4];
        tc::tmem_ld4(t_d, y);
        tc::tmem_ld_wait();
        if (p < a.n) {
          float c4[4];
          if (mat < 0) {
            c4[0] = c4[1] = c4[2] = c4[3] = __int_as_float(0x7FC00000);
          } else {
            c4[0] = fmaxf(0.0f, y[0]);
            c4[1] = fmaxf(0.0f, y[1]);
            c4[2] = fmaxf(0.0f, (__expf(y[2]) - 1.0f) * (1.0f / kSpecK));
            c4[3] = fmaxf(0.0f, (__expf(y[3]) - 1.0f) * (1.0f / kSpecK));
          }
          if (a.comps) store_row4(a.comps, p, c4[0], c4[1], c4[2], c4[3]);
          const float4 *al = reinterpret_cast<const float4 *>(alb + (mat < 0 ? 0 : mat) * 12);
          const float4 k0 = al[0], k1 = al[1], k2 = al[2];
          a.rgb[3 * p + 0] = k0.x * c4[0] + k0.w * c4[1] + k1.z * c4[2] + k2.y * c4[3];
          a.rgb[3 * p + 1] = k0.y * c4[0] + k1.x * c4[1] + k1.w * c4[2] + k2.z * c4[3];
          a.rgb[3 * p + 2] = k0.z * c4[0] + k1.y * c4[1] + k2.x * c4[2] + k2.w * c4[3];
        }
      }
    }
  }

  ok = !pn_bar_or<PT>(wg, !ok);
teardown:
  if (!ok) {
    if (tid == 0) atomicOr(a.status, kStatusTimeout);
    tc::mbar_wait(bar_w, 0, kWaitCycles);
    tc::mbar_wait(my_bar, phase ^ 1u, kWaitCycles);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(*tmem_slot, COLS * WG);
  }
}

// W = 64: two pipelines of 128 columns per CTA, two CTAs per SM (four CTAs
// of one pipeline would need four copies of the 57 KB of weights); W = 128:
// one CTA of two pipelines of 256 columns.  Either way the SM's 512
// tensor-memory columns are taken.
template <int W, bool F16>
const void *pn_kernel() {
  if (W == 64) return reinterpret_cast<const void *>(pn_decoder_kernel<64, F16, 2, 1>);
  return reinterpret_cast<const void *>(pn_decoder_kernel<128, F16, 2, 2>);
}

}  // namespace

int paper_k1(int n_mat) {
  const int k1 = (kPnBlob + n_mat + 15) / 16 * 16;
  return (n_mat >= 1 && k1 <= kPnMaxK1) ? k1 : -1;
}

size_t paper_blob_bytes(int w, int n_mat) { return pn_blob(w, n_mat).total; }

cudaError_t launch_paper_pack(int w, int precision, const float *params, const float *latents,
                              const DevMaterial *mats, int n_mat, void *blob, cudaStream_t s) {
  if (!paper_width_ok(w) || paper_k1(n_mat) < 0) return cudaErrorInvalidValue;
  const bool f16 = precision == FABRIC_PREC_FP16;
  const size_t smem = (size_t)n_mat * w * sizeof(float);
  uint8_t *out = static_cast<uint8_t *>(blob);
  const void *fn = w == 64 ? (f16 ? reinterpret_cast<const void *>(pn_pack_kernel<64, true>)
                                  : reinterpret_cast<const void *>(pn_pack_kernel<64, false>))
                           : (f16 ? reinterpret_cast<const void *>(pn_pack_kernel<128, true>)
                                  : reinterpret_cast<const void *>(pn_pack_kernel<128, false>));
  cudaError_t e = ensure_max_dyn_smem(fn, 64 * 1024);
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&params, (void *)&latents, (void *)&mats, (void *)&n_mat, (void *)&out};
  return cudaLaunchKernel(fn, dim3(1), dim3(256), args, smem, s);
}

cudaError_t launch_paper_decoder(int w, int precision, const fabric_gbuffer &g, const void *blob, int n_mat,
                                 float *rgb, float *comps, int *status, int sm_count, cudaStream_t s) {
  if (!paper_width_ok(w) || paper_k1(n_mat) < 0) return cudaErrorInvalidValue;
  const bool f16 = precision == FABRIC_PREC_FP16;
  const void *fn = w == 64 ? (f16 ? pn_kernel<64, true>() : pn_kernel<64, false>())
                           : (f16 ? pn_kernel<128, true>() : pn_kernel<128, false>());
  const int wg = 2;
  PnArgs a = {};
  a.u = g.u;
  a.v = g.v;
  a.radius = g.radius;
  a.wi = g.wi;
  a.wo = g.wo;
  a.material = g.material;
  a.n = g.n;
  a.n_tiles = (g.n + kTile - 1) / kTile;
  a.blob = static_cast<const uint8_t *>(blob);
  a.n_mat = n_mat;
  a.rgb = rgb;
  a.comps = comps;
  a.status = status;
  // Shared memory: alignment slack, barriers, the blob; padded so that no
  // CTA beyond the ones whose tensor memory fits (it would wait for it) can
  // share an SM: width 64 two CTAs of two 128-column pipelines (at least
  // 80 KB each), width 128 one CTA of two 256-column pipelines (116 KB).
  const int per_sm = w == 64 ? 2 : 1;
  const size_t floor_smem = (size_t)(w == 64 ? 80 : 116) * 1024;
  size_t smem = 2048 + ((pn_blob(w, n_mat).total + 1023u) & ~1023u);
  if (smem < floor_smem) smem = floor_smem;
  cudaError_t e = ensure_max_dyn_smem(fn, 227 * 1024);
  if (e != cudaSuccess) return e;
  int64_t grid = (int64_t)sm_count * per_sm;
  const int64_t need = (a.n_tiles + wg - 1) / wg;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  void *args[] = {&a};
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kTile * wg), args, smem, s);
}

}  // namespace fab
