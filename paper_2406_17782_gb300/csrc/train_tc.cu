// train_tc.cu -- the decoder's training forward and backward on the tensor
// cores (tcgen05, BF16 operands, FP32 accumulation), one 128-query tile per
// step of a persistent loop; one CTA of one warpgroup per SM.
//
// Per tile, with one query per thread and tile row:
//   forward   x = [z | q | 1] (K = 80) -> h1 -> h2 -> h3 -> y (N = 16, 4 used):
//             A operands in tensor memory, B = the weights in shared memory;
//             every activation also goes, transposed, to shared memory
//             (j-major rows of 128 queries) for the weight gradients, and its
//             ReLU mask stays in registers;
//   loss      dy from Eq. 11 (or the rendered-space option), scaled by 1/B;
//   backward  da_l = dh_l * mask_l; dh_{l-1} = da_l W_l (B = W_l transposed)
//             and dW_l^T += h_{l-1}^T da_l (M = 128 input rows of which 65-72
//             are used, N = 64 outputs, K = 128 queries), accumulated over
//             all of the CTA's tiles in tensor memory; the bias gradients
//             come out as the row of the constant-one input.
//   latent    dz rows = da_1 W1[:, :32] (FP32, for the per-material sums).
// At the end each CTA writes its gradient partials; the fixed-order
// reduction over CTAs, the encoder backward and Adam are shared with the FP32
// path.  Tensor-memory columns: D [0, 64), A [64, 104), dW1^T [128, 192),
// dW2^T [192, 256), dW3^T [256, 320), dW4^T [320, 336).
#include <cuda_bf16.h>

#include "fabric_internal.h"
#include "tc_ptx.h"
#include "train_common.cuh"

namespace fab {
namespace {

constexpr int kRows = 128;
constexpr int kK1 = 80;    // x = z (32) | q (39) | 1 | pad
constexpr int kKH = 80;    // h (64) | 1 | pad
constexpr long long kWaitCycles = 4000000000ll;

// Packed BF16 operands (bytes).
constexpr uint32_t kW1f = 0;                          // [64][80]  forward, K = x
constexpr uint32_t kW2f = kW1f + 64 * kK1 * 2;        // [64][80]
constexpr uint32_t kW3f = kW2f + 64 * kKH * 2;        // [64][80]
constexpr uint32_t kW4f = kW3f + 64 * kKH * 2;        // [16][80]
constexpr uint32_t kW4t = kW4f + 16 * kKH * 2;        // [64][16]  W4^T, K = outputs (4 used)
constexpr uint32_t kW3t = kW4t + 64 * 16 * 2;         // [64][64]  W3^T
constexpr uint32_t kW2t = kW3t + 64 * 64 * 2;         // [64][64]  W2^T
constexpr uint32_t kW1t = kW2t + 64 * 64 * 2;         // [32][64]  W1[:, :32]^T
constexpr uint32_t kBlob = kW1t + 32 * 64 * 2;

// Shared memory after the 1 KB header.
constexpr uint32_t kSmWts = 0;
constexpr uint32_t kSmXT = (kBlob + 1023) / 1024 * 1024;   // [128][128] x^T (rows 0..79 used)
constexpr uint32_t kSmH1T = kSmXT + 128 * 128 * 2;
constexpr uint32_t kSmH2T = kSmH1T + 128 * 128 * 2;
constexpr uint32_t kSmH3T = kSmH2T + 128 * 128 * 2;
constexpr uint32_t kSmDaT = kSmH3T + 128 * 128 * 2;        // [64][128] da^T
constexpr uint32_t kSmTotal = kSmDaT + 64 * 128 * 2;
constexpr size_t kDynSmem = 1024 /* align */ + 1024 /* header */ + kSmTotal;

constexpr uint32_t kColD = 0, kColA = 64, kColW1 = 128, kColW2 = 192, kColW3 = 256, kColW4 = 320;

__device__ __forceinline__ void put(uint8_t *base, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}

__global__ void __launch_bounds__(256) train_pack_kernel(const float *__restrict__ dec, uint8_t *__restrict__ blob) {
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < 64 * 80; e += blockDim.x * gridDim.x) {
    const int o = e / 80, j = e % 80;
    const float w1 = j < kDecIn ? dec[kOffW1 + o * kDecIn + j] : (j == kDecIn ? dec[kOffB1 + o] : 0.0f);
    const float w2 = j < kHidden ? dec[kOffW2 + o * kHidden + j] : (j == kHidden ? dec[kOffB2 + o] : 0.0f);
    const float w3 = j < kHidden ? dec[kOffW3 + o * kHidden + j] : (j == kHidden ? dec[kOffB3 + o] : 0.0f);
    put(blob, kW1f + tc::core_offset(o, j, kK1), w1);
    put(blob, kW2f + tc::core_offset(o, j, kKH), w2);
    put(blob, kW3f + tc::core_offset(o, j, kKH), w3);
    if (o < 16) {
      const float w4 = o >= kOut ? 0.0f
                                 : (j < kHidden ? dec[kOffW4 + o * kHidden + j] : (j == kHidden ? dec[kOffB4 + o] : 0.0f));
      put(blob, kW4f + tc::core_offset(o, j, kKH), w4);
    }
  }
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < 64 * 64; e += blockDim.x * gridDim.x) {
    const int j = e / 64, o = e % 64;   // transposed: row j (input), column o (output)
    put(blob, kW3t + tc::core_offset(j, o, 64), dec[kOffW3 + o * kHidden + j]);
    put(blob, kW2t + tc::core_offset(j, o, 64), dec[kOffW2 + o * kHidden + j]);
    if (j < 32) put(blob, kW1t + tc::core_offset(j, o, 64), dec[kOffW1 + o * kDecIn + j]);
    if (o < 16) put(blob, kW4t + tc::core_offset(j, o, 16), o < kOut ? dec[kOffW4 + o * kHidden + j] : 0.0f);
  }
}

struct TrainTcArgs {
  fabric_gbuffer g;
  const float *latents;   // [n_lat][32]
  int n_lat;
  const uint8_t *blob;
  const float *target;    // [n][4]
  int loss_mode;
  float inv_batch;
  float *partial;         // [grid][kDecParams]
  double *loss_partial;   // [grid]
  float *dlat_rows;       // [n][32]
  int *status;
};

// Element (row, k) of a K-major [rows][K] BF16 tile in shared memory.
__device__ __forceinline__ void st_bf16(uint8_t *base, int row, int k, int K, float v) {
  *reinterpret_cast<__nv_bfloat16 *>(base + tc::core_offset(row, k, K)) = __float2bfloat16_rn(v);
}

// 128-thread barrier of the CTA with tensor-memory ordering on both sides.
__device__ __forceinline__ void sync_all() {
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
}

__global__ void __launch_bounds__(kRows, 1) train_tc_kernel(const TrainTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bar_w = reinterpret_cast<uint64_t *>(smem);
  uint64_t *bar_mma = bar_w + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar_w + 2);
  __shared__ double loss_red[kRows];
  uint8_t *sm = smem + 1024;
  uint8_t *wts = sm + kSmWts, *xT = sm + kSmXT, *h1T = sm + kSmH1T, *h2T = sm + kSmH2T, *h3T = sm + kSmH3T;
  uint8_t *daT = sm + kSmDaT;
  const int r = threadIdx.x;                 // tile row (query) and tensor-memory lane
  const int warp = r >> 5;
  const bool lead = r == 0;

  if (lead) {
    tc::mbar_init(bar_w, 1);
    tc::mbar_init(bar_mma, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
  // unused rows of the transposed buffers stay zero
  for (uint32_t e = r; e < (kSmDaT + 64 * 128 * 2 - kSmXT) / 16; e += kRows)
    reinterpret_cast<uint4 *>(xT)[e] = make_uint4(0u, 0u, 0u, 0u);
  tc::fence_proxy_async_smem();
  sync_all();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane = (uint32_t)(warp * 32) << 16;
  const uint32_t t_d = tmem + lane + kColD, t_a = tmem + lane + kColA;
  if (lead) {
    tc::mbar_arrive_expect_tx(bar_w, kBlob);
    tc::bulk_g2s(wts, a.blob, kBlob, bar_w);
  }
  bool ok = tc::mbar_wait_sleep(bar_w, 0, kWaitCycles);
  const uint32_t s_w = tc::smem_addr(wts), s_xT = tc::smem_addr(xT), s_h1T = tc::smem_addr(h1T);
  const uint32_t s_h2T = tc::smem_addr(h2T), s_h3T = tc::smem_addr(h3T), s_daT = tc::smem_addr(daT);
  uint32_t phase = 0;
  double loss_acc = 0.0;
  const int64_t n_tiles = (a.g.n + kRows - 1) / kRows;
  bool first = true;

  // one MMA chain (K/16 steps) of A in tensor memory by B in shared memory
  auto mma_ts = [&](uint32_t d_col, uint32_t b_addr, int K, int N) {
    for (int kk = 0; kk < K / 16; ++kk) {
      const uint64_t bd = tc::smem_desc(b_addr + kk * 256u, 128u, (uint32_t)K * 16u);
      tc::mma_f16_ts(tmem + d_col, tmem + kColA + 8u * kk, bd, tc::idesc_bf16(128, N), kk > 0 ? 1u : 0u);
    }
  };
  // dW^T (M = 128 input rows, N outputs) += act^T (shared) by da^T (shared), K = 128 queries
  auto mma_dw = [&](uint32_t d_col, uint32_t actT, int N, bool acc) {
    for (int kk = 0; kk < kRows / 16; ++kk) {
      const uint64_t ad = tc::smem_desc(actT + kk * 256u, 128u, kRows * 16u);
      const uint64_t bd = tc::smem_desc(s_daT + kk * 256u, 128u, kRows * 16u);
      tc::mma_bf16(tmem + d_col, ad, bd, tc::idesc_bf16(128, N), (acc || kk > 0) ? 1u : 0u);
    }
  };
  // all threads: make the stores visible, then the lead issues `issue` and
  // everyone waits for the products
  auto round = [&](auto issue) -> bool {
    tc::tmem_st_wait();
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (lead) {
      tc::tc_fence_after();
      issue();
      tc::mma_commit(bar_mma);
    }
    const bool w = tc::mbar_wait_sleep(bar_mma, phase, kWaitCycles);
    phase ^= 1u;
    tc::tc_fence_after();
    return __syncthreads_and(w);
  };

  for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int64_t p = tile * kRows + r;
    int mat = p < a.g.n ? (int)a.g.material[p] : -1;
    if (mat >= a.n_lat) {
      atomicOr(a.status, kStatusBadMaterial);
      mat = -1;
    }
    const bool valid = mat >= 0;
    // ---- x = [z | q | 1 | 0] into the A operand and x^T
    {
      float x[kK1];
#pragma unroll
      for (int i = 0; i < kK1; ++i) x[i] = 0.0f;
      if (valid) {
        for (int i = 0; i < kLatent; ++i) x[i] = a.latents[(int64_t)mat * kLatent + i];
        query_features(a.g, p, x + kLatent);
        x[kDecIn] = 1.0f;
      }
      uint32_t w[8];
#pragma unroll
      for (int c = 0; c < kK1 / 16; ++c) {
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = tc::pack_bf16(x[16 * c + 2 * k], x[16 * c + 2 * k + 1]);
        tc::tmem_st8(t_a + 8 * c, w);
      }
#pragma unroll
      for (int j = 0; j < kK1; ++j) st_bf16(xT, j, r, kRows, x[j]);
    }
    // ---- forward: three hidden layers (ReLU masks in registers) and the head
    uint32_t mask[3][2];
    const uint32_t wf[3] = {s_w + kW1f, s_w + kW2f, s_w + kW3f};
    uint8_t *const hT[3] = {h1T, h2T, h3T};
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      if (!round([&] { mma_ts(kColD, wf[l], l == 0 ? kK1 : kKH, 64); })) { ok = false; break; }
      float acc[64];
      tc::tmem_ld32(t_d, acc);
      tc::tmem_ld32(t_d + 32, acc + 32);
      tc::tmem_ld_wait();
      mask[l][0] = mask[l][1] = 0u;
      float h[kKH];
#pragma unroll
      for (int j = 0; j < 64; ++j) {
        const bool on = valid && acc[j] > 0.0f;
        mask[l][j >> 5] |= on ? (1u << (j & 31)) : 0u;
        h[j] = on ? acc[j] : 0.0f;
      }
#pragma unroll
      for (int j = 64; j < kKH; ++j) h[j] = (j == 64 && valid) ? 1.0f : 0.0f;
      uint32_t w[8];
#pragma unroll
      for (int c = 0; c < kKH / 16; ++c) {
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = tc::pack_bf16(h[16 * c + 2 * k], h[16 * c + 2 * k + 1]);
        tc::tmem_st8(t_a + 8 * c, w);
      }
#pragma unroll
      for (int j = 0; j < 65; ++j) st_bf16(hT[l], j, r, kRows, h[j]);
    }
    if (!ok) break;
    if (!round([&] { mma_ts(kColD, s_w + kW4f, kKH, 16); })) { ok = false; break; }
    // ---- loss and the head's gradient da4 (A operand, K = 16, and da4^T)
    {
      float y[4];
      tc::tmem_ld4(t_d, y);
      tc::tmem_ld_wait();
      float d4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (valid) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          d4[k] = loss_grad(k, y[k], a.target[4 * p + k], a.g.wi[3 * p + 2], a.loss_mode, a.inv_batch, &loss_acc);
      }
      uint32_t w[8] = {tc::pack_bf16(d4[0], d4[1]), tc::pack_bf16(d4[2], d4[3]), 0u, 0u, 0u, 0u, 0u, 0u};
      tc::tmem_st8(t_a, w);
#pragma unroll
      for (int o = 0; o < 16; ++o) st_bf16(daT, o, r, kRows, o < 4 ? d4[o] : 0.0f);
    }
    // ---- backward: dh_{l} = da_{l+1} W_{l+1}; dW_{l+1}^T += h_l^T da_{l+1}
    const uint32_t wt[3] = {s_w + kW2t, s_w + kW3t, s_w + kW4t};   // transposed W2, W3, W4
    const uint32_t hTa[3] = {s_h1T, s_h2T, s_h3T};
    const uint32_t cdw[3] = {kColW2, kColW3, kColW4};
#pragma unroll
    for (int l = 2; l >= 0; --l) {
      // layer l+2 (1-based) produced h_{l+1}: dh_{l+1} = da W_{l+2}, dW_{l+2}^T += h_{l+1}^T da
      const int Kin = l == 2 ? 16 : 64, Nw = l == 2 ? 16 : 64;
      if (!round([&] {
            mma_ts(kColD, wt[l], Kin, 64);
            mma_dw(cdw[l], hTa[l], Nw, !first);
          })) { ok = false; break; }
      float acc[64];
      tc::tmem_ld32(t_d, acc);
      tc::tmem_ld32(t_d + 32, acc + 32);
      tc::tmem_ld_wait();
      float da[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) da[j] = (mask[l][j >> 5] >> (j & 31)) & 1u ? acc[j] : 0.0f;
      uint32_t w[8];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = tc::pack_bf16(da[16 * c + 2 * k], da[16 * c + 2 * k + 1]);
        tc::tmem_st8(t_a + 8 * c, w);
      }
#pragma unroll
      for (int o = 0; o < 64; ++o) st_bf16(daT, o, r, kRows, da[o]);
    }
    if (!ok) break;
    // ---- dz rows = da1 W1[:, :32]; dW1^T += x^T da1
    if (!round([&] {
          mma_ts(kColD, s_w + kW1t, 64, 32);
          mma_dw(kColW1, s_xT, 64, !first);
        })) { ok = false; break; }
    {
      float dz[32];
      tc::tmem_ld32(t_d, dz);
      tc::tmem_ld_wait();
      if (p < a.g.n) {
        float4 *out = reinterpret_cast<float4 *>(a.dlat_rows + p * kLatent);
#pragma unroll
        for (int i = 0; i < 8; ++i) out[i] = make_float4(dz[4 * i], dz[4 * i + 1], dz[4 * i + 2], dz[4 * i + 3]);
      }
    }
    first = false;
  }
  // ---- this CTA's gradient partials: lane j holds row j of every dW^T
  float *out = a.partial + (int64_t)blockIdx.x * kDecParams;
  if (ok) {
    const int j = r;
    const uint32_t t_row = tmem + lane;
    for (int l = 0; l < 4; ++l) {
      const int N = l == 3 ? 16 : 64, in = l == 0 ? kDecIn : kHidden, nout = l == 3 ? kOut : kHidden;
      const int offW = l == 0 ? kOffW1 : l == 1 ? kOffW2 : l == 2 ? kOffW3 : kOffW4;
      const int offB = l == 0 ? kOffB1 : l == 1 ? kOffB2 : l == 2 ? kOffB3 : kOffB4;
      const uint32_t col = l == 0 ? kColW1 : l == 1 ? kColW2 : l == 2 ? kColW3 : kColW4;
      for (int c = 0; c < N; c += 16) {
        float v[16];
        tc::tmem_ld16(t_row + col + c, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int o = c + e;
          if (o >= nout) continue;
          const float g = first ? 0.0f : v[e];   // a CTA without tiles contributes zeros
          if (j < in) out[offW + o * in + j] = g;
          else if (j == in) out[offB + o] = g;
        }
      }
    }
  }
  loss_red[r] = loss_acc;
  __syncthreads();
  if (r == 0) {
    double s = 0.0;
    for (int k = 0; k < kRows; ++k) s += loss_red[k];
    a.loss_partial[blockIdx.x] = s;
    if (!ok) atomicOr(a.status, kStatusTimeout);
  }
  if (!ok) {
    tc::mbar_wait(bar_w, 0, kWaitCycles);
    tc::mbar_wait(bar_mma, phase ^ 1u, kWaitCycles);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

}  // namespace

size_t train_tc_blob_bytes() { return kBlob; }

int train_tc_grid(int64_t n, int sm_count) {
  const int64_t tiles = (n + kRows - 1) / kRows;
  int64_t g = sm_count > 0 ? sm_count : 148;
  if (g > tiles) g = tiles;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_train_tc(const fabric_gbuffer &g, const float *latents, int n_lat, const float *dec,
                            const float *target, int loss_mode, void *blob, float *partial, double *loss_partial,
                            float *dlat_rows, int sm_count, int *status, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  train_pack_kernel<<<8, 256, 0, s>>>(dec, static_cast<uint8_t *>(blob));
  TrainTcArgs a;
  a.g = g;
  a.latents = latents;
  a.n_lat = n_lat;
  a.blob = static_cast<const uint8_t *>(blob);
  a.target = target;
  a.loss_mode = loss_mode;
  a.inv_batch = 1.0f / (float)(g.n > 0 ? g.n : 1);
  a.partial = partial;
  a.loss_partial = loss_partial;
  a.dlat_rows = dlat_rows;
  a.status = status;
  train_tc_kernel<<<train_tc_grid(g.n, sm_count), kRows, kDynSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fab
