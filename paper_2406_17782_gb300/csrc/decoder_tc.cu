// decoder_tc.cu -- fused decoder MLP on the 5th-generation tensor cores
// (tcgen05, tensor memory), the per-shading-point hot path of the neural
// method (Sec. 4.4: only the decoder runs per pixel).
//
// Per CTA (128 threads, one shading point per thread and per tile row):
//   1. one bulk (TMA) copy stages the packed BF16 weights, biases and the
//      per-material albedos in shared memory, once per CTA;
//   2. persistent loop over 128-point tiles: each thread streams its point
//      from the G-buffer, encodes it (sin/cos of 8 octaves of u and v, log
//      footprint, wi, wo) and writes one BF16 row of the A tile;
//   3. layer 1 (the latent part of W1 is folded into one per-material bias
//      column selected by a one-hot of the material: W1 z_m + b1 is exact
//      algebra, computed once per call) and layers 2-4 run as tcgen05.mma
//      chains into tensor memory; the epilogue of each layer reads its row
//      back with tcgen05.ld, adds the bias, applies ReLU, rounds to BF16 and
//      writes the next A tile;
//   4. the head's four outputs become C = max(0, y), S = max(0, expm1(y)/100)
//      and RGB by Eq. 8; only RGB (and optionally the components) is stored.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fabric_internal.h"
#include "tc_ptx.h"

namespace fab {
namespace {

constexpr int kTile = 128;
constexpr int kTmemCols = 64;
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz

// ---- packed-weight blob layout (bytes), identical in global and shared memory
struct BlobLayout {
  int k1;
  uint32_t w1, w2, w3, w4, b2, b3, b4, alb, total;
};

__host__ __device__ inline BlobLayout blob_layout(int n_mat, int k1) {
  BlobLayout L;
  L.k1 = k1;
  L.w1 = 0;
  L.w2 = L.w1 + 64u * k1 * 2u;
  L.w3 = L.w2 + 64u * 64u * 2u;
  L.w4 = L.w3 + 64u * 64u * 2u;
  L.b2 = L.w4 + 16u * 64u * 2u;
  L.b3 = L.b2 + 64u * 4u;
  L.b4 = L.b3 + 64u * 4u;
  L.alb = L.b4 + 16u * 4u;
  L.total = L.alb + ((uint32_t)(n_mat * 12 * 4) + 15u) / 16u * 16u;
  return L;
}

__device__ __forceinline__ void put_bf16(uint8_t *base, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}
template <bool F16>
__device__ __forceinline__ void put_op(uint8_t *base, uint32_t off, float v) {
  if (F16)
    *reinterpret_cast<__half *>(base + off) = __float2half_rn(v);
  else
    put_bf16(base, off, v);
}

// Fold the latents into the first layer and pack every operand into the
// canonical shared-memory layout (FP16 or BF16 operands).  One CTA.
template <bool F16>
__global__ void __launch_bounds__(256) pack_kernel(const float *__restrict__ dec, const float *__restrict__ lat,
                                                   const DevMaterial *__restrict__ mats, int n_mat, int k1,
                                                   uint8_t *__restrict__ blob) {
  extern __shared__ float fold[];   // [n_mat][64]
  const BlobLayout L = blob_layout(n_mat, k1);
  const float *W1 = dec + kOffW1;
  for (int e = threadIdx.x; e < n_mat * kHidden; e += blockDim.x) {
    const int m = e / kHidden, o = e % kHidden;
    float acc = dec[kOffB1 + o];
    for (int j = 0; j < kLatent; ++j) acc = fmaf(W1[o * kDecIn + j], lat[m * kLatent + j], acc);
    fold[m * kHidden + o] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kHidden * k1; e += blockDim.x) {
    const int o = e / k1, c = e % k1;
    float v = 0.0f;
    if (c < kQueryFeat)
      v = W1[o * kDecIn + kLatent + c];
    else if (c < kQueryFeat + n_mat)
      v = fold[(c - kQueryFeat) * kHidden + o];
    put_op<F16>(blob, L.w1 + tc::core_offset(o, c, k1), v);
  }
  for (int e = threadIdx.x; e < kHidden * kHidden; e += blockDim.x) {
    const int o = e / kHidden, c = e % kHidden;
    put_op<F16>(blob, L.w2 + tc::core_offset(o, c, 64), dec[kOffW2 + e]);
    put_op<F16>(blob, L.w3 + tc::core_offset(o, c, 64), dec[kOffW3 + e]);
  }
  for (int e = threadIdx.x; e < 16 * kHidden; e += blockDim.x) {
    const int o = e / kHidden, c = e % kHidden;
    put_op<F16>(blob, L.w4 + tc::core_offset(o, c, 64), o < kOut ? dec[kOffW4 + o * kHidden + c] : 0.0f);
  }
  float *b2 = reinterpret_cast<float *>(blob + L.b2);
  float *b3 = reinterpret_cast<float *>(blob + L.b3);
  float *b4 = reinterpret_cast<float *>(blob + L.b4);
  for (int e = threadIdx.x; e < kHidden; e += blockDim.x) {
    b2[e] = dec[kOffB2 + e];
    b3[e] = dec[kOffB3 + e];
  }
  if (threadIdx.x < 16) b4[threadIdx.x] = threadIdx.x < kOut ? dec[kOffB4 + threadIdx.x] : 0.0f;
  float *alb = reinterpret_cast<float *>(blob + L.alb);
  for (int e = threadIdx.x; e < n_mat * 12; e += blockDim.x) {
    const int m = e / 12, q = e % 12;
    const DevMaterial &M = mats[m];
    alb[e] = q < 3 ? M.kd[0][q] : q < 6 ? M.kd[1][q - 3] : q < 9 ? M.ks[0][q - 6] : M.ks[1][q - 9];
  }
}

struct TcArgs {
  const float *u, *v, *radius, *wi, *wo;
  const uint16_t *material;
  int64_t n;
  int64_t n_tiles;
  const uint8_t *blob;
  int n_mat, k1;
  float *rgb, *comps;
  int *status;
};

template <bool F16>
__device__ __forceinline__ void store_row_chunk(uint8_t *tile, int row, int chunk, int K, const float *f8) {
  tc::st_shared_v4(tile + tc::core_offset(row, chunk * 8, K), tc::pack2<F16>(f8[0], f8[1]),
                   tc::pack2<F16>(f8[2], f8[3]), tc::pack2<F16>(f8[4], f8[5]), tc::pack2<F16>(f8[6], f8[7]));
}

// sin / cos of 2 pi 2^k frac(x) for k = 0..7 by angle doubling from one
// hardware sincos of the reduced angle 2 pi (frac(x) - 1/2) in [-pi, pi).
__device__ __forceinline__ void octave_sincos(float x, float *f16) {
  const float fr = x - floorf(x);
  float s, c;
  __sincosf(6.283185307179586f * (fr - 0.5f), &s, &c);
  s = -s;
  c = -c;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    f16[2 * k] = s;
    f16[2 * k + 1] = c;
    const float s2 = 2.0f * s * c;
    c = (c - s) * (c + s);
    s = s2;
  }
}

template <bool F16>
__global__ void __launch_bounds__(kTile, 1) decoder_tc_kernel(const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bar_w = reinterpret_cast<uint64_t *>(smem);
  uint64_t *bar_mma = bar_w + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar_w + 2);
  const BlobLayout L = blob_layout(a.n_mat, a.k1);
  uint8_t *wts = smem + 1024;
  uint8_t *atile = wts + ((L.total + 1023u) & ~1023u);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;

  if (tid == 0) {
    tc::mbar_init(bar_w, 1);
    tc::mbar_init(bar_mma, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);

  if (tid == 0) {
    tc::mbar_arrive_expect_tx(bar_w, L.total);
    tc::bulk_g2s(wts, a.blob, L.total, bar_w);
  }
  bool ok = tc::mbar_wait(bar_w, 0, kWaitCycles);
  const float *b2 = reinterpret_cast<const float *>(wts + L.b2);
  const float *b3 = reinterpret_cast<const float *>(wts + L.b3);
  const float *b4 = reinterpret_cast<const float *>(wts + L.b4);
  const float *alb = reinterpret_cast<const float *>(wts + L.alb);

  const uint32_t a_addr = tc::smem_addr(atile);
  const uint32_t w1_addr = tc::smem_addr(wts + L.w1), w2_addr = tc::smem_addr(wts + L.w2);
  const uint32_t w3_addr = tc::smem_addr(wts + L.w3), w4_addr = tc::smem_addr(wts + L.w4);
  const uint32_t id64 = F16 ? tc::idesc_f16(128, 64) : tc::idesc_bf16(128, 64);
  const uint32_t id16 = F16 ? tc::idesc_f16(128, 16) : tc::idesc_bf16(128, 16);
  uint32_t phase = 0;

  if (__syncthreads_or(!ok)) goto teardown;

  for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int64_t p = tile * kTile + tid;
    const bool live = p < a.n;
    int mat = -1;
    // ---- encode this thread's point into row `tid` of the layer-1 A tile
    {
      float q[40];
#pragma unroll
      for (int i = 0; i < 40; ++i) q[i] = 0.0f;
      if (live) {
        mat = a.material[p];
        if (mat >= a.n_mat) {
          atomicOr(a.status, kStatusBadMaterial);
          mat = -2;
        } else {
          octave_sincos(a.u[p], q);
          octave_sincos(a.v[p], q + 16);
          q[32] = (__logf(fmaxf(a.radius[p], kRFloor)) - kLogRC0) * kLogRInvC1;
          q[33] = a.wi[3 * p];
          q[34] = a.wi[3 * p + 1];
          q[35] = a.wi[3 * p + 2];
          q[36] = a.wo[3 * p];
          q[37] = a.wo[3 * p + 1];
          q[38] = a.wo[3 * p + 2];
          q[39] = mat == 0 ? 1.0f : 0.0f;
        }
      }
#pragma unroll
      for (int c = 0; c < 5; ++c) store_row_chunk<F16>(atile, tid, c, a.k1, q + 8 * c);
      for (int c = 5; c < a.k1 / 8; ++c) {
        float f[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) f[e] = (8 * c + e == kQueryFeat + mat) ? 1.0f : 0.0f;
        store_row_chunk<F16>(atile, tid, c, a.k1, f);
      }
    }
    // ---- four layers
#pragma unroll 1
    for (int layer = 0; layer < 4; ++layer) {
      tc::fence_proxy_async_smem();
      tc::tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc::tc_fence_after();
        const int K = layer == 0 ? a.k1 : 64;
        const uint32_t w_addr = layer == 0 ? w1_addr : layer == 1 ? w2_addr : layer == 2 ? w3_addr : w4_addr;
        const uint32_t sbo = (uint32_t)K * 16u;
        for (int kk = 0; kk < K / 16; ++kk) {
          const uint64_t ad = tc::smem_desc(a_addr + kk * 256u, 128u, sbo);
          const uint64_t bd = tc::smem_desc(w_addr + kk * 256u, 128u, sbo);
          tc::mma_bf16(tmem, ad, bd, layer == 3 ? id16 : id64, kk > 0 ? 1u : 0u);
        }
        tc::mma_commit(bar_mma);
      }
      ok = tc::mbar_wait(bar_mma, phase, kWaitCycles);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) goto teardown;
      tc::tc_fence_after();
      if (layer < 3) {
        float acc[64];
#pragma unroll
        for (int c = 0; c < 4; ++c) tc::tmem_ld16(tmem_row + 16 * c, acc + 16 * c);
        tc::tmem_ld_wait();
        const float *bias = layer == 1 ? b2 : b3;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          uint32_t w[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int col = 8 * c + 2 * e;
            float lo = acc[col], hi = acc[col + 1];
            if (layer > 0) {
              lo += bias[col];
              hi += bias[col + 1];
            }
            w[e] = tc::pack2_relu<F16>(lo, hi);
          }
          tc::st_shared_v4(atile + tc::core_offset(tid, 8 * c, 64), w[0], w[1], w[2], w[3]);
        }
      } else {
        float y[16];
        tc::tmem_ld16(tmem_row, y);
        tc::tmem_ld_wait();
        if (live) {
          float c4[4];
          if (mat < 0) {
            c4[0] = c4[1] = c4[2] = c4[3] = __int_as_float(0x7FC00000);
          } else {
            c4[0] = fmaxf(0.0f, y[0] + b4[0]);
            c4[1] = fmaxf(0.0f, y[1] + b4[1]);
            c4[2] = fmaxf(0.0f, expm1f(y[2] + b4[2]) * (1.0f / kSpecK));
            c4[3] = fmaxf(0.0f, expm1f(y[3] + b4[3]) * (1.0f / kSpecK));
          }
          if (a.comps) reinterpret_cast<float4 *>(a.comps)[p] = make_float4(c4[0], c4[1], c4[2], c4[3]);
          const float *al = alb + (mat < 0 ? 0 : mat) * 12;
#pragma unroll
          for (int ch = 0; ch < 3; ++ch)
            a.rgb[3 * p + ch] = al[ch] * c4[0] + al[3 + ch] * c4[1] + al[6 + ch] * c4[2] + al[9 + ch] * c4[3];
        }
      }
    }
  }

teardown:
  if (!ok) {
    if (tid == 0) atomicOr(a.status, kStatusTimeout);
    // let any copy or product still in flight land before the memory goes away
    tc::mbar_wait(bar_w, 0, kWaitCycles);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

size_t tc_smem_bytes(int n_mat, int k1) {
  const BlobLayout L = blob_layout(n_mat, k1);
  const int kmax = k1 > 64 ? k1 : 64;
  return 1024 /* alignment slack */ + 1024 /* barriers */ + ((L.total + 1023u) & ~1023u) + (size_t)kTile * kmax * 2;
}

// ---- self-test: one 128 x n x k product through the same layout and path
__global__ void __launch_bounds__(128, 1) selftest_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                          int n, int k, float *__restrict__ D, int *status) {
  __shared__ __align__(1024) uint8_t sa[128 * 64 * 2];
  __shared__ __align__(1024) uint8_t sb[64 * 64 * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < 128 * k; e += 128) {
    const int r = e / k, c = e % k;
    put_bf16(sa, tc::core_offset(r, c, k), A[e]);
  }
  for (int e = tid; e < n * k; e += 128) {
    const int r = e / k, c = e % k;
    put_bf16(sb, tc::core_offset(r, c, k), B[e]);
  }
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&slot, 64);
  tc::fence_proxy_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = slot;
  if (tid == 0) {
    for (int kk = 0; kk < k / 16; ++kk) {
      const uint64_t ad = tc::smem_desc(tc::smem_addr(sa) + kk * 256u, 128u, (uint32_t)k * 16u);
      const uint64_t bd = tc::smem_desc(tc::smem_addr(sb) + kk * 256u, 128u, (uint32_t)k * 16u);
      tc::mma_bf16(tmem, ad, bd, tc::idesc_bf16(128, n), kk > 0 ? 1u : 0u);
    }
    tc::mma_commit(&bar);
  }
  const bool ok = tc::mbar_wait(&bar, 0, kWaitCycles);
  if (!ok && tid == 0) atomicOr(status, kStatusTimeout);
  tc::tc_fence_after();
  if (__syncthreads_and(ok)) {
    for (int c = 0; c < n; c += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int e = 0; e < 16; ++e) D[tid * n + c + e] = v[e];
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 64);
  }
}

}  // namespace

int tc_k1(int n_mat) {
  const int k1 = (kQueryFeat + n_mat + 15) / 16 * 16;
  return (n_mat >= 1 && k1 <= 128) ? k1 : -1;
}

size_t tc_blob_bytes(int n_mat) { return blob_layout(n_mat, tc_k1(n_mat) > 0 ? tc_k1(n_mat) : 128).total; }

cudaError_t launch_tc_pack(const float *dec, const float *latents, const DevMaterial *mats, int n_mat, int precision,
                           void *blob, cudaStream_t s) {
  (void)precision;
  const int k1 = tc_k1(n_mat);
  if (k1 < 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)n_mat * kHidden * sizeof(float);
  if (precision == FABRIC_PREC_FP16)
    pack_kernel<true><<<1, 256, smem, s>>>(dec, latents, mats, n_mat, k1, static_cast<uint8_t *>(blob));
  else
    pack_kernel<false><<<1, 256, smem, s>>>(dec, latents, mats, n_mat, k1, static_cast<uint8_t *>(blob));
  return cudaGetLastError();
}

cudaError_t launch_decoder_tc(const fabric_gbuffer &g, const void *blob, int n_mat, int precision, float *rgb,
                              float *comps, int *status, int sm_count, int ctas_per_sm, cudaStream_t s) {
  const bool f16 = precision == FABRIC_PREC_FP16;
  const int k1 = tc_k1(n_mat);
  if (k1 < 0) return cudaErrorInvalidValue;
  const size_t smem = tc_smem_bytes(n_mat, k1);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(decoder_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(decoder_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TcArgs a;
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
  a.k1 = k1;
  a.rgb = rgb;
  a.comps = comps;
  a.status = status;
  int per_sm = ctas_per_sm;
  if (per_sm <= 0) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f16 ? decoder_tc_kernel<true> : decoder_tc_kernel<false>,
                                                  kTile, smem);
    per_sm = occ < 1 ? 1 : occ;
  }
  if (per_sm > 512 / kTmemCols) per_sm = 512 / kTmemCols;
  int64_t grid = (int64_t)sm_count * per_sm;
  if (grid > a.n_tiles) grid = a.n_tiles;
  if (grid < 1) grid = 1;
  if (f16)
    decoder_tc_kernel<true><<<(unsigned)grid, kTile, smem, s>>>(a);
  else
    decoder_tc_kernel<false><<<(unsigned)grid, kTile, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_selftest_mma(const float *a, const float *b, int n, int k, float *d, int *status,
                                cudaStream_t s) {
  selftest_kernel<<<1, 128, 0, s>>>(a, b, n, k, d, status);
  return cudaGetLastError();
}

}  // namespace fab
