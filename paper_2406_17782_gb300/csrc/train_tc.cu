// train_tc.cu -- the decoder's training forward and backward on the tensor
// cores (tcgen05, BF16 operands, FP32 accumulation), one 128-query tile per
// step of a persistent loop; one CTA of two warpgroups per SM, two threads
// per query row (warps w and w + 4 share lane quadrant w).
//
// Per tile, with one query per thread and tile row:
//   forward   x = [z | q | 1] (K = 80) -> h1 -> h2 -> h3 -> y (N = 16, 4 used):
//             A operands in tensor memory, B = the weights in shared memory;
//             every activation also goes to shared memory, as the query's own
//             row in the MN-major operand layout (16-byte vector stores), for
//             the weight gradients, and its ReLU mask stays in registers;
//   loss      dy from Eq. 11 (or the rendered-space option), scaled by 1/B;
//   backward  da_l = dh_l * mask_l; dh_{l-1} = da_l W_l (B = W_l transposed)
//             and dW_l^T += h_{l-1}^T da_l (M = 128 input rows of which 65-72
//             are used, N = 64 outputs, K = 128 queries), accumulated over
//             all of the CTA's tiles in tensor memory; the bias gradients
//             come out as the row of the constant-one input.
//   latent    dz rows = da_1 W1[:, :32] (FP32, for the per-material sums).
// Thread 0 issues the products an epilogue reads and thread 128 the weight-
// gradient products, which nothing reads until the tile loop ends: each dW
// chain is waited for only before the shared-memory operand it reads is
// rewritten (the da operands alternate between two buffers for this).
// At the end each CTA writes its gradient partials (and, for up to 1588
// materials, its per-material latent sums); fixed-order reductions over the
// CTAs follow in other kernels, the decoder's together with its Adam update
// beside the encoder's gradients.  Tensor-memory columns: D [0, 64),
// A [64, 104), dW1^T [128, 192), dW2^T [192, 256), dW3^T [256, 320),
// dW4^T [320, 336), and the latent-gradient rows of up to five tiles
// [336, 496).
#include <cuda_bf16.h>

#include "fabric_internal.h"
#include "tc_ptx.h"
#include "train_common.cuh"

namespace fab {
namespace {

constexpr int kRows = 128;
constexpr int kThreads = 256;   // two threads per query row: warps w and w + 4 share lane quadrant w
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

// Shared memory after the 1 KB header.  The weight-gradient operands act^T
// (M = 128 inputs, 0..79 used) and da (N = 64 or 16 outputs), both with
// K = the tile's 128 queries, are MN-major: element (j, r) -- input or output
// j of query r -- lives at mn_offset(j, r, width), core matrices of 8 j by 8 r
// (16-byte rows along j), 128 bytes apart along j, width * 16 bytes apart
// along r.
constexpr uint32_t kSmWts = 0;
constexpr uint32_t kSmXT = (kBlob + 1023) / 1024 * 1024;   // x^T: 128 inputs x 128 queries (0..79 used)
constexpr uint32_t kSmH1T = kSmXT + 128 * 128 * 2;
constexpr uint32_t kSmH2T = kSmH1T + 128 * 128 * 2;
constexpr uint32_t kSmH3T = kSmH2T + 128 * 128 * 2;
constexpr uint32_t kSmDaA = kSmH3T + 128 * 128 * 2;        // da: 64 outputs x 128 queries, two buffers
constexpr uint32_t kSmDaB = kSmDaA + 64 * 128 * 2;          // (layers alternate between them)
constexpr uint32_t kSmTotal = kSmDaB + 64 * 128 * 2;
constexpr size_t kDynSmem = 1024 /* align */ + 1024 /* header */ + kSmTotal;

constexpr uint32_t kColD = 0, kColA = 64, kColW1 = 128, kColW2 = 192, kColW3 = 256, kColW4 = 320;
// The latent-gradient rows of up to kDzTiles tiles stay in tensor memory,
// 32 columns per tile from kColDz, for the per-material sums at the end.
constexpr uint32_t kColDz = 336;
constexpr int kDzTiles = 5;
static_assert(kColDz + 32 * kDzTiles <= 512, "latent-gradient rows inside the allocation");

// Thread 0 issues the products the epilogues read; thread 128 (the first
// thread of half 1) issues the weight-gradient products.
constexpr int kDwIssuer = 128;

// Instruction-descriptor bits: A and B read MN-major (transposed).
constexpr uint32_t kTransA = 1u << 15, kTransB = 1u << 16;

// Shared-memory descriptor of an MN-major operand without swizzle: here the
// leading-dimension field is the stride between 8-deep groups along K and the
// stride-dimension field the stride between 8-wide core matrices along M or N
// (the reverse of the K-major roles; checked by fabric_selftest_mma_mn).
__device__ __forceinline__ uint64_t mn_desc(uint32_t saddr, uint32_t k_group_stride) {
  return tc::smem_desc(saddr, k_group_stride, 128u);
}

__host__ __device__ constexpr uint32_t mn_offset(int j, int r, int width) {
  return (uint32_t)((j & 7) * 2 + (r & 7) * 16 + (j >> 3) * 128 + (r >> 3) * width * 16);
}

// Eight consecutive values j0..j0+7 (j0 % 8 == 0) of query r, packed as four
// BF16 pairs, into an MN-major operand of the given width.
__device__ __forceinline__ void st_row8(uint8_t *base, int j0, int r, int width, const uint32_t *w4) {
  *reinterpret_cast<uint4 *>(base + mn_offset(j0, r, width)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
}

// Global loads that stay where they are written: volatile asm keeps the
// compiler from moving them to their first use, so that they are in flight
// during the work in between.
__device__ __forceinline__ float ld_pinned(const float *p) {
  float v;
  asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ float4 ld_pinned4(const float *p) {   // p 16-byte aligned
  float4 v;
  asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}

__device__ __forceinline__ int ld_pinned_u16(const uint16_t *p) {
  unsigned short v;
  asm volatile("ld.global.u16 %0, [%1];" : "=h"(v) : "l"(p));
  return (int)v;
}

__device__ __forceinline__ void put(uint8_t *base, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}

// Launched right after the encoder forward, on which it does not depend: it
// reads the parameters the previous step's Adam wrote, which completed before
// the encoder forward got past its own dependency wait -- the point from
// which this kernel may start.  So it packs at once, overlapping the encoder,
// and waits for the encoder only at its end, so that its completion still
// implies the encoder's for the kernel after it.
__global__ void __launch_bounds__(256) train_pack_kernel(const float *__restrict__ dec, uint8_t *__restrict__ blob) {
  grid_dependents_launch();
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
  grid_dependency_wait();
}

struct TrainTcArgs {
  fabric_gbuffer g;
  const float *latents;   // [n_lat][32], 16-byte aligned
  int n_lat;
  const uint8_t *blob;
  const float *target;    // [n][4]
  int loss_mode;
  float inv_batch;
  float *partial;         // [grid][partial_width]
  int partial_width;      // kDecParams, or kDecParams + 32 n_lat with the latent sums folded in
  double *loss_partial;   // [grid]
  float *dlat_rows;       // [n][32]
  int *status;
};

// 128-thread barrier of the CTA with tensor-memory ordering on both sides.
__device__ __forceinline__ void sync_all() {
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
}

__global__ void __launch_bounds__(kThreads, 1) train_tc_kernel(const TrainTcArgs a) {
  // The set-up and the first tile's G-buffer reads (inputs of the step, which
  // the step's first kernel waited for) overlap the kernels before this one;
  // the wait for them comes before the weights and latents they write.
  grid_dependents_launch();
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bar_w = reinterpret_cast<uint64_t *>(smem);
  uint64_t *bar_mma = bar_w + 1;     // thread 0's products
  uint64_t *bar_dw = bar_w + 2;      // [3]: dW4, dW3 and dW1 (each once per tile)
  uint64_t *bar_drain = bar_w + 5;   // both issuers' products, after a failed wait
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar_w + 6);
  __shared__ double loss_red[4];
  uint8_t *sm = smem + 1024;
  uint8_t *wts = sm + kSmWts, *xT = sm + kSmXT, *h1T = sm + kSmH1T, *h2T = sm + kSmH2T, *h3T = sm + kSmH3T;
  uint8_t *daA = sm + kSmDaA, *daB = sm + kSmDaB;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int hf = warp >> 2;                      // which half of every epilogue's columns
  const int r = ((warp & 3) << 5) | (tid & 31);  // tile row (query) = tensor-memory lane
  const bool lead = tid == 0;

  if (lead) {
    tc::mbar_init(bar_w, 1);
    tc::mbar_init(bar_mma, 1);
    for (int k = 0; k < 3; ++k) tc::mbar_init(bar_dw + k, 1);
    tc::mbar_init(bar_drain, 2);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, 512);
  // unused rows of the gradient operands stay zero
  for (uint32_t e = tid; e < (kSmTotal - kSmXT) / 16; e += kThreads)
    reinterpret_cast<uint4 *>(xT)[e] = make_uint4(0u, 0u, 0u, 0u);
  tc::fence_proxy_async_smem();
  sync_all();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;   // this warp's lane quadrant
  const uint32_t t_d = tmem + lane + kColD, t_a = tmem + lane + kColA;
  bool ok = true;
  const uint32_t s_w = tc::smem_addr(wts), s_xT = tc::smem_addr(xT), s_h1T = tc::smem_addr(h1T);
  const uint32_t s_h2T = tc::smem_addr(h2T), s_h3T = tc::smem_addr(h3T);
  const uint32_t s_daA = tc::smem_addr(daA), s_daB = tc::smem_addr(daB);
  uint32_t phase = 0;    // bar_mma's
  uint32_t dw_par = 0;   // this tile's phase of the bar_dw barriers
  double loss_acc = 0.0;
  const int64_t n_tiles = (a.g.n + kRows - 1) / kRows;
  bool first = true;
  // With the per-material latent sums folded into the partials, a CTA of at
  // most kDzTiles tiles (all staged at once at the end) keeps its rows in
  // tensor memory; otherwise they go to a.dlat_rows.
  const int my_tiles = n_tiles > blockIdx.x ? (int)((n_tiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;
  const int sum_group = (int)max((int64_t)0, ((int64_t)kSmTotal - (int64_t)a.n_lat * kLatent * 4) /
                                                 (int64_t)(kRows * (kLatent * 4 + 4)));   // tiles staged at once
  const bool dz_tmem = a.partial_width > kDecParams && my_tiles <= kDzTiles && my_tiles <= sum_group;
  int ti = 0;   // tiles done

  // one MMA chain (K/16 steps) of A in tensor memory by B in shared memory
  auto mma_ts = [&](uint32_t d_col, uint32_t b_addr, int K, int N) {
    for (int kk = 0; kk < K / 16; ++kk) {
      const uint64_t bd = tc::smem_desc(b_addr + kk * 256u, 128u, (uint32_t)K * 16u);
      tc::mma_f16_ts(tmem + d_col, tmem + kColA + 8u * kk, bd, tc::idesc_bf16(128, N), kk > 0 ? 1u : 0u);
    }
  };
  // dW^T (M = 128 input rows, N outputs) += act^T (shared) by da (shared),
  // K = 128 queries, both operands MN-major: K = 16 spans two 8-query groups
  auto mma_dw = [&](uint32_t d_col, uint32_t actT, uint32_t da, int N, bool acc) {
    const uint32_t kg_a = 128u * 16u, kg_b = (uint32_t)N * 16u;   // bytes per 8-query group
    for (int kk = 0; kk < kRows / 16; ++kk) {
      const uint64_t ad = mn_desc(actT + kk * 2u * kg_a, kg_a);
      const uint64_t bd = mn_desc(da + kk * 2u * kg_b, kg_b);
      tc::mma_bf16(tmem + d_col, ad, bd, tc::idesc_bf16(128, N) | kTransA | kTransB, (acc || kk > 0) ? 1u : 0u);
    }
  };
  // All threads make their stores visible and meet.  Then thread 0 issues
  // `issue` (the products the epilogue reads) and commits it to bar_mma, and
  // thread 128 issues `issue_dw` (weight-gradient products, read only after
  // the tile loop) and commits it to dw_bar where one is given; a dW chain
  // is waited for only before the shared-memory operands it reads are
  // overwritten.  Every thread then runs `overlap` (half 1's share of the
  // next tile's inputs) and waits for bar_mma.  The outcome of each wait
  // travels with the next round's barrier (or the one after the tile loop),
  // so a round costs one CTA barrier; false: some thread's wait expired.
  auto round = [&](auto issue, auto issue_dw, uint64_t *dw_bar, auto overlap) -> bool {
    tc::tmem_st_wait();
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    if (!__syncthreads_and(ok)) return false;
    if (lead) {
      tc::tc_fence_after();
      issue();
      tc::mma_commit(bar_mma);
    } else if (tid == kDwIssuer) {
      tc::tc_fence_after();
      issue_dw();
      if (dw_bar != nullptr) tc::mma_commit(dw_bar);
    }
    overlap();
    ok = tc::mbar_wait(bar_mma, phase, kWaitCycles);   // spin: one CTA per SM, nothing else to run
    phase ^= 1u;
    tc::tc_fence_after();
    return true;
  };
  auto none = [] {};
  // 32 activations of this half (columns c0 .. c0 + 31 of a 64-wide layer)
  // into the next A operand (16 columns) and the MN-major copy
  auto put_half = [&](const float *v, uint8_t *mn, int width, int c0) {
    uint32_t w[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) w[k] = tc::pack_bf16(v[2 * k], v[2 * k + 1]);
    tc::tmem_st16(t_a + c0 / 2, w);
#pragma unroll
    for (int q = 0; q < 4; ++q) st_row8(mn, c0 + 8 * q, r, width, w + 4 * q);
  };

  // A tile's global inputs are loaded ahead, so that no wait for them falls
  // on the tile's critical path.  When a tile starts, every thread issues the
  // load of the next tile's material id, and half 1 those of its G-buffer
  // record.  Half 1 encodes the record in four pieces when it has nothing
  // else to do: during the products of layers 2 and 3 and of the head, and
  // while half 0 evaluates the loss; half 0 then issues the latent row,
  // target and <wi.n_s> loads, in flight during the backward pass.
  int nxt_raw = -1;       // the next tile's raw material id
  int nxt_mat = -1;       // resolved: -1 for no query or a material out of range
  float in_v[kLatent];    // half 0: the latent row; half 1: the G-buffer record (9 used)
  uint32_t in_x[24];      // half 1: inputs 32..79 as BF16 pairs
  float in_tg[4], in_wz = 0.0f;
#pragma unroll
  for (int i = 0; i < kLatent; ++i) in_v[i] = 0.0f;
#pragma unroll
  for (int k = 0; k < 24; ++k) in_x[k] = 0u;
#pragma unroll
  for (int k = 0; k < 4; ++k) in_tg[k] = 0.0f;
  auto load_early = [&](int64_t t) {
    const int64_t q = t * kRows + r;
    nxt_raw = -1;
    if (t < n_tiles && q < a.g.n) {
      nxt_raw = ld_pinned_u16(a.g.material + q);
      if (hf == 1) {
        in_v[0] = ld_pinned(a.g.u + q);
        in_v[1] = ld_pinned(a.g.v + q);
        in_v[2] = ld_pinned(a.g.radius + q);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          in_v[3 + i] = ld_pinned(a.g.wi + 3 * q + i);
          in_v[6 + i] = ld_pinned(a.g.wo + 3 * q + i);
        }
      }
    }
  };
  auto resolve = [&]() {
    nxt_mat = nxt_raw;
    if (nxt_mat >= a.n_lat) {
      if (hf == 0) atomicOr(a.status, kStatusBadMaterial);
      nxt_mat = -1;
    }
  };
  // half 1, step s of encoding the next tile's record into [q | 1 | 0], in
  // pieces that fit the waits they fill: 1 and 2 the octaves 0-3 and 4-7 of
  // u, 3 and 4 those of v, and with 4 also log r, the directions, the
  // constant one and the padding, and all zeros where there is no query.
  // Each octave is the one octaves_accurate() computes.
  auto octave = [&](float x, int k) -> uint32_t {
    const float f0 = x - floorf(x);
    const float sc = f0 * (float)(1 << k);
    const float fk = sc - floorf(sc);
    float sn, cs;
    sincospif(2.0f * fk, &sn, &cs);
    return tc::pack_bf16(sn, cs);
  };
  auto encode_step = [&](int s) {
    if (hf != 1 || s < 1) return;
    const int c = (s - 1) >> 1, k0 = 4 * ((s - 1) & 1);   // coordinate (u, v) and first octave
#pragma unroll
    for (int k = 0; k < 4; ++k) in_x[8 * c + k0 + k] = octave(in_v[c], k0 + k);
    if (s == 4) {
      resolve();
      static_assert(kDecIn - kLatent - 32 == 7, "inputs 32..79: 32 octave values, log r, 6 directions, one");
      float x[16];
      x[0] = (logf(fmaxf(in_v[2], kRFloor)) - kLogRC0) * kLogRInvC1;
#pragma unroll
      for (int i = 0; i < 6; ++i) x[1 + i] = in_v[3 + i];
      x[7] = 1.0f;
#pragma unroll
      for (int i = 8; i < 16; ++i) x[i] = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) in_x[16 + k] = tc::pack_bf16(x[2 * k], x[2 * k + 1]);
      if (nxt_mat < 0) {
#pragma unroll
        for (int k = 0; k < 24; ++k) in_x[k] = 0u;
      }
    }
  };
  // half 0: latent row (16-byte loads: the rows of different queries are
  // different lines, so wider loads mean fewer of them), targets, <wi.n_s>
  const bool target_v4 = (reinterpret_cast<uintptr_t>(a.target) & 15u) == 0;
  auto load_late = [&](int64_t t) {
    const int64_t q = t * kRows + r;
    const int m = nxt_mat;
    if (m >= 0) {
#pragma unroll
      for (int i = 0; i < kLatent / 4; ++i) {
        const float4 z4 = ld_pinned4(a.latents + (int64_t)m * kLatent + 4 * i);
        in_v[4 * i] = z4.x;
        in_v[4 * i + 1] = z4.y;
        in_v[4 * i + 2] = z4.z;
        in_v[4 * i + 3] = z4.w;
      }
      if (target_v4) {
        const float4 t4 = ld_pinned4(a.target + 4 * q);
        in_tg[0] = t4.x;
        in_tg[1] = t4.y;
        in_tg[2] = t4.z;
        in_tg[3] = t4.w;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) in_tg[k] = ld_pinned(a.target + 4 * q + k);
      }
      in_wz = ld_pinned(a.g.wi + 3 * q + 2);
    } else {
#pragma unroll
      for (int i = 0; i < kLatent; ++i) in_v[i] = 0.0f;
#pragma unroll
      for (int k = 0; k < 4; ++k) in_tg[k] = 0.0f;
      in_wz = 0.0f;
    }
  };
  load_early(blockIdx.x);
  resolve();
  if (hf == 1) {
    for (int k = 1; k <= 4; ++k) encode_step(k);
  }
  grid_dependency_wait();
  if (lead) {
    tc::mbar_arrive_expect_tx(bar_w, kBlob);
    tc::bulk_g2s(wts, a.blob, kBlob, bar_w);
  }
  if (hf == 0) load_late(blockIdx.x);
  ok = tc::mbar_wait_sleep(bar_w, 0, kWaitCycles);

  bool fail = false;   // CTA-uniform: a round found an expired wait
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    // the previous tile's dW1 (and with it every earlier dW chain) has read
    // x^T, h^T and the da buffers before they are rewritten
    if (!first) {
      ok = tc::mbar_wait(bar_dw + 2, dw_par ^ 1u, kWaitCycles) && ok;
      tc::tc_fence_after();
    }
    const int64_t p = tile * kRows + r;
    const int mat = nxt_mat;
    const bool valid = mat >= 0;
    float tg[4] = {in_tg[0], in_tg[1], in_tg[2], in_tg[3]};
    const float wz = in_wz;
    // ---- x = [z | q | 1 | 0] into the A operand and the MN-major x^T:
    // half 0 writes the latent (inputs 0..31), half 1 the query features,
    // the constant one and the padding (inputs 32..79)
    if (hf == 0) {
      put_half(in_v, xT, 128, 0);
    } else {
      tc::tmem_st16(t_a + 16, in_x);
#pragma unroll
      for (int q = 0; q < 4; ++q) st_row8(xT, 32 + 8 * q, r, 128, in_x + 4 * q);
      tc::tmem_st8(t_a + 32, in_x + 16);
      st_row8(xT, 64, r, 128, in_x + 16);
      st_row8(xT, 72, r, 128, in_x + 20);
    }
    load_early(tile + gridDim.x);
    // ---- forward: three hidden layers (ReLU masks of this half's columns
    // in registers) and the head; half 1 encodes the next tile's record
    // during the products of layers 2, 3 and the head, and while half 0
    // evaluates the loss
    uint32_t mask[3];
    const uint32_t wf[3] = {s_w + kW1f, s_w + kW2f, s_w + kW3f};
    uint8_t *const hT[3] = {h1T, h2T, h3T};
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      if (!round([&] { mma_ts(kColD, wf[l], l == 0 ? kK1 : kKH, 64); }, none, nullptr,
                 [&] { encode_step(l); })) { fail = true; break; }
      float acc[32];
      tc::tmem_ld32(t_d + 32 * hf, acc);
      tc::tmem_ld_wait();
      mask[l] = 0u;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const bool on = valid && acc[j] > 0.0f;
        mask[l] |= on ? (1u << j) : 0u;
        acc[j] = on ? acc[j] : 0.0f;
      }
      put_half(acc, hT[l], 128, 32 * hf);
      if (hf == 1) {   // constant-one input of the next layer and padding, K = 64..79
        uint32_t w[8] = {valid ? tc::pack_bf16(1.0f, 0.0f) : 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        tc::tmem_st8(t_a + 32, w);
        st_row8(hT[l], 64, r, 128, w);
        st_row8(hT[l], 72, r, 128, w + 4);
      }
    }
    if (fail) break;
    if (!round([&] { mma_ts(kColD, s_w + kW4f, kKH, 16); }, none, nullptr, [&] { encode_step(3); })) {
      fail = true;
      break;
    }
    // ---- loss and the head's gradient da4 (A operand, K = 16, and da4 in buffer A)
    if (hf == 0) {
      resolve();
      float y[4];
      tc::tmem_ld4(t_d, y);
      tc::tmem_ld_wait();
      float d4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (valid) {
        float lq = 0.0f;   // the query's four loss terms in FP32, their total in FP64
#pragma unroll
        for (int k = 0; k < 4; ++k) d4[k] = loss_grad(k, y[k], tg[k], wz, a.loss_mode, a.inv_batch, &lq);
        loss_acc += (double)lq;
      }
      uint32_t w[8] = {tc::pack_bf16(d4[0], d4[1]), tc::pack_bf16(d4[2], d4[3]), 0u, 0u, 0u, 0u, 0u, 0u};
      tc::tmem_st8(t_a, w);
      st_row8(daA, 0, r, 16, w);
      st_row8(daA, 8, r, 16, w + 4);
      load_late(tile + gridDim.x);   // in flight during the backward pass
    } else {
      encode_step(4);
    }
    // ---- backward: dh_{l} = da_{l+1} W_{l+1}; dW_{l+1}^T += h_l^T da_{l+1}.
    // The da of the head, of layer 3, 2 and 1 go to buffers A, B, A, B; an
    // epilogue that rewrites a buffer first waits for the dW chain that read it.
    const uint32_t wt[3] = {s_w + kW2t, s_w + kW3t, s_w + kW4t};   // transposed W2, W3, W4
    const uint32_t hTa[3] = {s_h1T, s_h2T, s_h3T};
    const uint32_t cdw[3] = {kColW2, kColW3, kColW4};
    const uint32_t da_in[3] = {s_daA, s_daB, s_daA};    // by l: the da this round's dW chain reads
    uint8_t *const da_out[3] = {daB, daA, daB};         // by l: where its epilogue writes
    uint64_t *const dw_commit[3] = {nullptr, bar_dw + 1, bar_dw + 0};
    uint64_t *const dw_before[3] = {bar_dw + 1, bar_dw + 0, nullptr};
#pragma unroll
    for (int l = 2; l >= 0; --l) {
      // layer l+2 (1-based) produced h_{l+1}: dh_{l+1} = da W_{l+2}, dW_{l+2}^T += h_{l+1}^T da
      const int Kin = l == 2 ? 16 : 64, Nw = l == 2 ? 16 : 64;
      if (!round([&] { mma_ts(kColD, wt[l], Kin, 64); }, [&] { mma_dw(cdw[l], hTa[l], da_in[l], Nw, !first); },
                 dw_commit[l], none)) { fail = true; break; }
      float acc[32];
      tc::tmem_ld32(t_d + 32 * hf, acc);
      tc::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = (mask[l] >> j) & 1u ? acc[j] : 0.0f;
      if (dw_before[l] != nullptr) ok = tc::mbar_wait(dw_before[l], dw_par, kWaitCycles) && ok;
      put_half(acc, da_out[l], 64, 32 * hf);
    }
    if (fail) break;
    // ---- dz rows = da1 W1[:, :32] (16 columns per half); dW1^T += x^T da1
    const uint32_t dz_col = dz_tmem ? kColDz + 32u * (uint32_t)ti : kColD;
    if (!round([&] { mma_ts(dz_col, s_w + kW1t, 64, 32); }, [&] { mma_dw(kColW1, s_xT, s_daB, 64, !first); },
               bar_dw + 2, none)) { fail = true; break; }
    if (!dz_tmem) {
      float dz[16];
      tc::tmem_ld16(t_d + 16 * hf, dz);
      tc::tmem_ld_wait();
      if (p < a.g.n) {
        float4 *out = reinterpret_cast<float4 *>(a.dlat_rows + p * kLatent + 16 * hf);
#pragma unroll
        for (int i = 0; i < 4; ++i) out[i] = make_float4(dz[4 * i], dz[4 * i + 1], dz[4 * i + 2], dz[4 * i + 3]);
      }
    }
    first = false;
    dw_par ^= 1u;
    ++ti;
  }
  // every dW chain has finished before the accumulators are read
  if (!first && !fail) {
    ok = tc::mbar_wait(bar_dw + 2, dw_par ^ 1u, kWaitCycles) && ok;
    tc::tc_fence_after();
  }
  ok = __syncthreads_and(ok && !fail);   // one outcome for the CTA before the barriers below
  // ---- this CTA's gradient partials: lane j holds row j of every dW^T;
  // the two halves take alternate 16-column chunks, all loaded before one wait
  float *out = a.partial + (int64_t)blockIdx.x * a.partial_width;
  if (ok) {
    const int j = r;
    const uint32_t t_row = tmem + lane;
    float v[4][32];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int N = l == 3 ? 16 : 64;
      const uint32_t col = l == 0 ? kColW1 : l == 1 ? kColW2 : l == 2 ? kColW3 : kColW4;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (16 * hf + 32 * h < N) tc::tmem_ld16(t_row + col + 16 * hf + 32 * h, v[l] + 16 * h);
    }
    tc::tmem_ld_wait();
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int N = l == 3 ? 16 : 64, in = l == 0 ? kDecIn : kHidden, nout = l == 3 ? kOut : kHidden;
      const int offW = l == 0 ? kOffW1 : l == 1 ? kOffW2 : l == 2 ? kOffW3 : kOffW4;
      const int offB = l == 0 ? kOffB1 : l == 1 ? kOffB2 : l == 2 ? kOffB3 : kOffB4;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = 16 * hf + 32 * h;
        if (c >= N) continue;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int o = c + e;
          if (o >= nout) continue;
          const float g = first ? 0.0f : v[l][16 * h + e];   // a CTA without tiles contributes zeros
          if (j < in) out[offW + o * in + j] = g;
          else if (j == in) out[offB + o] = g;
        }
      }
    }
  }
  // ---- per-material sums of this CTA's latent-gradient rows, in row order,
  // into the partials' columns past kDecParams (the operand buffers are free
  // now).  The CTA's tiles are staged in shared memory as many at a time as
  // fit; warp w then walks, in row order, the rows of the materials m with
  // m % 8 == w (found with ballots), so no two warps touch one sum.
  if (ok && a.partial_width > kDecParams) {
    float *acc = reinterpret_cast<float *>(sm);                   // [n_lat][32]
    float *stage = acc + (size_t)a.n_lat * kLatent;                // [group][128][32]
    const int group = sum_group;
    int *ids = reinterpret_cast<int *>(stage + (size_t)group * kRows * kLatent);   // [group][128]
    const int lane32 = tid & 31;
    __syncthreads();
    for (int e = tid; e < a.n_lat * kLatent; e += kThreads) acc[e] = 0.0f;
    for (int64_t t0 = blockIdx.x; t0 < n_tiles; t0 += (int64_t)group * gridDim.x) {
      int nt = 0;   // tiles in this group
      while (nt < group && t0 + (int64_t)nt * gridDim.x < n_tiles) ++nt;
      __syncthreads();
      // the rows: from tensor memory (every tile of the CTA in this one
      // group), or from a.dlat_rows with eight loads in flight per thread
      // before their stores
      const int n4 = dz_tmem ? 0 : nt * kRows * (kLatent / 4);
      if (dz_tmem) {
        tc::tc_fence_after();
        for (int t = 0; t < nt; ++t) {
          float v[16];
          tc::tmem_ld16(tmem + lane + kColDz + 32u * (uint32_t)t + 16u * (uint32_t)hf, v);
          tc::tmem_ld_wait();
          const bool in = (t0 + (int64_t)t * gridDim.x) * kRows + r < a.g.n;
          float4 *dst = reinterpret_cast<float4 *>(stage + ((size_t)t * kRows + r) * kLatent + 16 * hf);
#pragma unroll
          for (int i = 0; i < 4; ++i)
            dst[i] = in ? make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3])
                        : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
      }
      for (int e0 = tid; e0 < n4; e0 += 8 * kThreads) {
        float4 v4[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kThreads;
          const int t = e / (kRows * (kLatent / 4)), rest = e % (kRows * (kLatent / 4));
          const int64_t row = (t0 + (int64_t)t * gridDim.x) * kRows + rest / (kLatent / 4);
          v4[u] = e < n4 && row < a.g.n
                      ? reinterpret_cast<const float4 *>(a.dlat_rows)[row * (kLatent / 4) + rest % (kLatent / 4)]
                      : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (e0 + u * kThreads < n4) reinterpret_cast<float4 *>(stage)[e0 + u * kThreads] = v4[u];
      }
      for (int e0 = tid; e0 < nt * kRows; e0 += 4 * kThreads) {
        int m4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e0 + u * kThreads;
          const int64_t row = (t0 + (int64_t)(e / kRows) * gridDim.x) * kRows + e % kRows;
          m4[u] = e < nt * kRows && row < a.g.n ? (int)a.g.material[row] : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (e0 + u * kThreads < nt * kRows) ids[e0 + u * kThreads] = m4[u] < a.n_lat ? m4[u] : -1;
      }
      __syncthreads();
      for (int t = 0; t < nt; ++t) {
#pragma unroll
        for (int k = 0; k < kRows / 32; ++k) {
          const int q0 = t * kRows + 32 * k;
          const int m_l = ids[q0 + lane32];
          uint32_t hit = __ballot_sync(0xFFFFFFFFu, m_l >= 0 && (m_l & 7) == warp);
          while (hit) {
            const int b = __ffs(hit) - 1;
            hit &= hit - 1;
            const int m = __shfl_sync(0xFFFFFFFFu, m_l, b);
            acc[m * kLatent + lane32] += stage[(size_t)(q0 + b) * kLatent + lane32];
          }
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < a.n_lat * kLatent; e += kThreads) out[kDecParams + e] = first ? 0.0f : acc[e];
  }
  // the loss: a fixed shuffle tree in each of half 0's warps, then their four sums in order
  if (hf == 0) {
    double l = loss_acc;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, d);
    if ((tid & 31) == 0) loss_red[warp] = l;
  }
  __syncthreads();
  if (tid == 0) {
    a.loss_partial[blockIdx.x] = (loss_red[0] + loss_red[1]) + (loss_red[2] + loss_red[3]);
    if (!ok) atomicOr(a.status, kStatusTimeout);
  }
  if (!ok) {   // after an expired wait: let the weights' copy and both issuers' products finish
    tc::mbar_wait(bar_w, 0, kWaitCycles);
    if (lead || tid == kDwIssuer) tc::mma_commit(bar_drain);
    tc::mbar_wait(bar_drain, 0, kWaitCycles);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ---- self-test of the MN-major operands: d[128][n] = a[128][k] b[n][k]^T
// with a and b stored by mn_offset (the weight-gradient layout above).
__global__ void __launch_bounds__(128, 1) selftest_mn_kernel(const float *__restrict__ A,
                                                              const float *__restrict__ B, int n, int k,
                                                              float *__restrict__ D, int *status) {
  __shared__ __align__(1024) uint8_t sa[128 * 64 * 2];
  __shared__ __align__(1024) uint8_t sb[64 * 64 * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < 128 * k; e += 128) put(sa, mn_offset(e / k, e % k, 128), A[e]);
  for (int e = tid; e < n * k; e += 128) put(sb, mn_offset(e / k, e % k, n), B[e]);
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&slot, 64);
  tc::fence_proxy_async_smem();
  sync_all();
  const uint32_t tmem = slot;
  if (tid == 0) {
    const uint32_t kg_a = 128u * 16u, kg_b = (uint32_t)n * 16u;
    for (int kk = 0; kk < k / 16; ++kk)
      tc::mma_bf16(tmem, mn_desc(tc::smem_addr(sa) + kk * 2u * kg_a, kg_a),
                   mn_desc(tc::smem_addr(sb) + kk * 2u * kg_b, kg_b), tc::idesc_bf16(128, n) | kTransA | kTransB,
                   kk > 0 ? 1u : 0u);
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
  sync_all();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

}  // namespace

cudaError_t launch_selftest_mn(const float *a, const float *b, int n, int k, float *d, int *status, cudaStream_t s) {
  selftest_mn_kernel<<<1, 128, 0, s>>>(a, b, n, k, d, status);
  return cudaGetLastError();
}

size_t train_tc_blob_bytes() { return kBlob; }

// Materials up to this count have their latent-gradient sums folded into the
// kernel's per-CTA partials (their sums, one tile of staged rows and its ids
// fit in the operand buffers); more take the separate per-material kernel.
int train_tc_partial_width(int n_lat) {
  const size_t need = (size_t)n_lat * kLatent * 4 + kRows * (kLatent * 4 + 4);   // sums + one staged tile
  return need <= kSmTotal ? kDecParams + kLatent * n_lat : kDecParams;
}

int train_tc_grid(int64_t n, int sm_count) {
  const int64_t tiles = (n + kRows - 1) / kRows;
  int64_t g = sm_count > 0 ? sm_count : 148;
  if (g > tiles) g = tiles;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_train_tc(const fabric_gbuffer &g, const float *latents, int n_lat, const float *dec,
                            const float *target, int loss_mode, void *blob, float *partial, double *loss_partial,
                            float *dlat_rows, int sm_count, int *status, cudaStream_t s) {
  if (reinterpret_cast<uintptr_t>(latents) & 15u) return cudaErrorInvalidValue;   // rows read as float4
  {
    const cudaError_t e = ensure_max_dyn_smem(reinterpret_cast<const void *>(train_tc_kernel), (int)kDynSmem);
    if (e != cudaSuccess) return e;
  }
  launch_dependent(train_pack_kernel, 8, 256, 0, s, dec, static_cast<uint8_t *>(blob));
  TrainTcArgs a;
  a.g = g;
  a.latents = latents;
  a.n_lat = n_lat;
  a.blob = static_cast<const uint8_t *>(blob);
  a.target = target;
  a.loss_mode = loss_mode;
  a.inv_batch = 1.0f / (float)(g.n > 0 ? g.n : 1);
  a.partial = partial;
  a.partial_width = train_tc_partial_width(n_lat);
  a.loss_partial = loss_partial;
  a.dlat_rows = dlat_rows;
  a.status = status;
  return launch_dependent(train_tc_kernel, train_tc_grid(g.n, sm_count), kThreads, kDynSmem, s, a);
}

}  // namespace fab
