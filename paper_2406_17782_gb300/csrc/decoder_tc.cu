// decoder_tc.cu -- fused decoder MLP on the 5th-generation tensor cores
// (tcgen05, tensor memory), the per-shading-point hot path of the neural
// method (Sec. 4.4: only the decoder runs per pixel).
//
// A CTA holds one copy of the packed 16-bit weights in shared memory and WG
// independent tile pipelines (warpgroups of 128 threads, one shading point
// per thread and tile row).  Activations never touch shared memory: each
// warpgroup owns 128 tensor-memory columns, [0, 64) for the FP32
// accumulator D and [64, 128) for the 16-bit A operand of the next layer
// (two values per 32-bit column, row i in lane i).
//   1. one bulk (TMA) copy stages the weights and the per-material albedos
//      in shared memory, once per CTA;
//   2. each warpgroup loops over its 128-point tiles: every thread encodes
//      its point (sin/cos of 8 octaves of u and v, log footprint, wi, wo)
//      from registers loaded during the previous tile and stores its row of
//      the layer-1 A operand into tensor memory (tcgen05.st);
//   3. layer 1 (the latent part of W1 folded into one per-material bias
//      column selected by a one-hot of the material: W1 z_m + b1 is exact
//      algebra, computed once per call) and layers 2-4 (their biases in a
//      constant-one input column) run as tcgen05.mma with A in tensor memory
//      and B in shared memory; each epilogue reads D back (tcgen05.ld),
//      converts it with ReLU (cvt.rn.relu) and stores the next A operand;
//   4. the head's four outputs become C = max(0, y), S = max(0, expm1(y)/100)
//      and RGB by Eq. 8; only RGB (and optionally the components) is stored.
// Operand precisions: FP16 or BF16 throughout, or E4M3 for layers 2-4
// (kind::f8f6f4, K = 64 in two instructions, four values per tensor-memory
// column) with layer 1 in FP16; there the weights of layers 2-4 carry a
// per-layer power-of-two scale, and the unscaling and their biases are one
// FP32 FMA per value in the epilogue instead of a constant-one column.
// While one warpgroup waits for its products the others encode and convert,
// which keeps the tensor pipe and the ALUs busy together.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "decoder_blob.h"
#include "fabric_internal.h"
#include "tc_ptx.h"

namespace fab {
namespace {

constexpr int kTile = 128;
constexpr uint32_t kColsPerTile = 128;             // D [0, 64) | A [64, 128)
constexpr uint32_t kColA = 64;
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz

// Operand precision of a kernel instance.
constexpr int kPrBF16 = 0;   // BF16 everywhere
constexpr int kPrF16 = 1;    // FP16 everywhere
constexpr int kPrE4M3 = 2;   // FP16 layer 1, E4M3 layers 2-4

__host__ __device__ constexpr int prec_code(int fabric_prec) {
  return fabric_prec == FABRIC_PREC_FP16 ? kPrF16 : fabric_prec == FABRIC_PREC_FP8 ? kPrE4M3 : kPrBF16;
}

__host__ __device__ inline uint32_t align1k(uint32_t x) { return (x + 1023u) & ~1023u; }

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

__device__ __forceinline__ uint8_t to_e4m3(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// Fold the latents into the first layer and pack every operand into the
// canonical shared-memory layout.  16-bit layers 2-4 get their biases as an
// extra input column; E4M3 layers 2-4 get the per-layer power-of-two scale
// 2^(8 - E), amax = m 2^E with m in [0.5, 1), and an FP32 epilogue block.
// One CTA.
template <int PR>
__global__ void __launch_bounds__(256) pack_kernel(const float *__restrict__ dec, const float *__restrict__ lat,
                                                   const DevMaterial *__restrict__ mats, int n_mat, int k1,
                                                   uint8_t *__restrict__ blob) {
  constexpr bool H16 = PR != kPrBF16, F8 = PR == kPrE4M3;
  extern __shared__ float fold[];   // [n_mat][64]
  __shared__ unsigned amax_bits[3];
  const BlobLayout L = blob_layout(n_mat, k1, F8);
  const float *W1 = dec + kOffW1;
  if (threadIdx.x < 3) amax_bits[threadIdx.x] = 0u;
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
    put_op<H16>(blob, L.w1 + tc::core_offset(o, c, k1), v);
  }
  if (!F8) {
    for (int e = threadIdx.x; e < kHidden * kKH; e += blockDim.x) {
      const int o = e / kKH, c = e % kKH;
      const float v2 = c < kHidden ? dec[kOffW2 + o * kHidden + c] : (c == kHidden ? dec[kOffB2 + o] : 0.0f);
      const float v3 = c < kHidden ? dec[kOffW3 + o * kHidden + c] : (c == kHidden ? dec[kOffB3 + o] : 0.0f);
      put_op<H16>(blob, L.w2 + tc::core_offset(o, c, kKH), v2);
      put_op<H16>(blob, L.w3 + tc::core_offset(o, c, kKH), v3);
    }
    for (int e = threadIdx.x; e < 16 * kKH; e += blockDim.x) {
      const int o = e / kKH, c = e % kKH;
      float v = 0.0f;
      if (o < kOut) v = c < kHidden ? dec[kOffW4 + o * kHidden + c] : (c == kHidden ? dec[kOffB4 + o] : 0.0f);
      put_op<H16>(blob, L.w4 + tc::core_offset(o, c, kKH), v);
    }
  } else {
    // per-layer amax (non-negative floats order like their bit patterns)
    float m2 = 0.0f, m3 = 0.0f, m4 = 0.0f;
    for (int e = threadIdx.x; e < kHidden * kHidden; e += blockDim.x) {
      m2 = fmaxf(m2, fabsf(dec[kOffW2 + e]));
      m3 = fmaxf(m3, fabsf(dec[kOffW3 + e]));
      if (e < kOut * kHidden) m4 = fmaxf(m4, fabsf(dec[kOffW4 + e]));
    }
    atomicMax(&amax_bits[0], __float_as_uint(m2));
    atomicMax(&amax_bits[1], __float_as_uint(m3));
    atomicMax(&amax_bits[2], __float_as_uint(m4));
    __syncthreads();
    float scale[3];
    float *epi = reinterpret_cast<float *>(blob + L.epi);
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      int ex = 0;
      frexpf(__uint_as_float(amax_bits[l]), &ex);
      scale[l] = ldexpf(1.0f, 8 - ex);
      if (threadIdx.x == 0) epi[kF8Inv + 1 + l] = ldexpf(1.0f, ex - 8);
    }
    if (threadIdx.x == 0) epi[kF8Inv] = 1.0f;
    for (int e = threadIdx.x; e < 4 * 64; e += blockDim.x) {
      const int l = e / 64, o = e % 64;
      epi[kF8Bias + e] = l == 1 ? dec[kOffB2 + o] : l == 2 ? dec[kOffB3 + o] : (l == 3 && o < kOut) ? dec[kOffB4 + o] : 0.0f;
    }
    for (int e = threadIdx.x; e < kHidden * kHidden; e += blockDim.x) {
      const int o = e / kHidden, c = e % kHidden;
      blob[L.w2 + tc::core_offset8(o, c, 64)] = to_e4m3(dec[kOffW2 + e] * scale[0]);
      blob[L.w3 + tc::core_offset8(o, c, 64)] = to_e4m3(dec[kOffW3 + e] * scale[1]);
    }
    for (int e = threadIdx.x; e < 16 * kHidden; e += blockDim.x) {
      const int o = e / kHidden, c = e % kHidden;
      blob[L.w4 + tc::core_offset8(o, c, 64)] = o < kOut ? to_e4m3(dec[kOffW4 + e] * scale[2]) : (uint8_t)0;
    }
  }
  float *alb = reinterpret_cast<float *>(blob + L.alb);
  for (int e = threadIdx.x; e < n_mat * 12; e += blockDim.x) {
    const int m = e / 12, q = e % 12;
    const DevMaterial &M = mats[m];
    alb[e] = q < 3 ? M.kd[0][q] : q < 6 ? M.kd[1][q - 3] : q < 9 ? M.ks[0][q - 6] : M.ks[1][q - 9];
  }
}

// Single G-buffer: the pointers below.  Batched: `segs` / `seg_tile0` list
// the segments (tile t belongs to the segment s with seg_tile0[s] <= t <
// seg_tile0[s + 1]) and the single-buffer fields are unused.
struct TcArgs {
  const float *u, *v, *radius, *wi, *wo;
  const uint16_t *material;
  int64_t n;
  int64_t n_tiles;
  const uint8_t *blob;
  int n_mat, k1;
  float *rgb, *comps;
  int *status;
  const SegDesc *segs;
  const int64_t *seg_tile0;   // read through `seg_t0` below: global, or the CTA's shared copy
  int n_segs;
  int seg_in_smem;            // 1: each CTA copies seg_tile0 into its spare shared memory
};

// Segment holding global tile `tile`: the largest s < n_segs with
// seg_tile0[s] <= tile (seg_tile0[n_segs] = n_tiles > tile).  A pipeline
// visits its tiles in increasing order, so the search starts from the
// segment of its previous tile (`cursor`): one load while the tile stays in
// that segment, otherwise a galloping search then bisection, instead of a
// full bisection of dependent loads for every tile.
__device__ __forceinline__ int find_segment(const TcArgs &a, const int64_t *seg_t0, int64_t tile, int cursor,
                                            int64_t &first_tile) {
  int lo = cursor;   // seg_t0[lo] <= tile
  int64_t lo_t0 = seg_t0[lo];
  if (seg_t0[lo + 1] > tile) {
    first_tile = lo_t0;
    return lo;
  }
  int hi = lo + 1, step = 1;   // seg_tile0[hi] <= tile
  while (true) {
    lo = hi;
    step <<= 1;
    hi = lo + step;
    if (hi >= a.n_segs) {
      hi = a.n_segs;
      break;
    }
    if (seg_t0[hi] > tile) break;
  }
  while (hi - lo > 1) {   // seg_t0[lo] <= tile < seg_t0[hi]
    const int mid = (lo + hi) >> 1;
    if (seg_t0[mid] <= tile) lo = mid; else hi = mid;
  }
  first_tile = seg_t0[lo];
  return lo;
}

// Where tile `tile`'s rows live: point index base and the buffers.
struct TileView {
  const float *u, *v, *radius, *wi, *wo;
  const uint16_t *material;
  float *rgb, *comps;
  int64_t n, first;   // points in the segment, index of the tile's first point in it
};

template <bool MULTI>
__device__ __forceinline__ TileView tile_view(const TcArgs &a, const int64_t *seg_t0, int64_t tile, int &cursor) {
  TileView t;
  if (!MULTI || tile >= a.n_tiles) {
    t.u = a.u; t.v = a.v; t.radius = a.radius; t.wi = a.wi; t.wo = a.wo; t.material = a.material;
    t.rgb = a.rgb; t.comps = a.comps; t.n = MULTI ? 0 : a.n; t.first = tile * 128;
  } else {
    int64_t t0;
    const int s = find_segment(a, seg_t0, tile, cursor, t0);
    cursor = s;
    const SegDesc &d = a.segs[s];
    t.u = d.u; t.v = d.v; t.radius = d.radius; t.wi = d.wi; t.wo = d.wo; t.material = d.material;
    t.rgb = d.rgb; t.comps = d.comps; t.n = d.n; t.first = (tile - t0) * 128;
  }
  return t;
}

// sin / cos of 2 pi 2^k frac(x) for k = 0..7: f_k = frac(2^k frac(x)) is
// exact in FP32 (doubling and dropping the integer part), and each octave
// takes one hardware sincos of the reduced angle 2 pi (f_k - 1/2) in
// [-pi, pi), whose absolute error (~4e-7) does not grow with k as an
// angle-doubling recurrence would; w[k] packs (sin, cos) of octave k.
template <bool F16>
__device__ __forceinline__ void octave_words(float x, uint32_t *w) {
  float f = x - floorf(x);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float s, c;
    __sincosf(6.283185307179586f * (f - 0.5f), &s, &c);
    w[k] = tc::pack2<F16>(-s, -c);
    f = 2.0f * f;
    f -= floorf(f);
  }
}

// One shading point's G-buffer record, held in registers between tiles.
struct Point {
  float u, v, r, wi0, wi1, wi2, wo0, wo1, wo2;
  int mat;   // -1: beyond the end
};

// Load the fields this thread encodes: all of them with one thread per row
// (H = 1); with two threads per row (H = 2) half 0 takes u, the footprint and
// the directions, half 1 takes v; both take the material.
template <int H>
__device__ __forceinline__ Point load_point(const TileView &a, int64_t p, int h) {
  Point q;
  q.u = q.v = q.r = q.wi0 = q.wi1 = q.wi2 = q.wo0 = q.wo1 = q.wo2 = 0.0f;
  q.mat = -1;
  if (p < a.n) {
    q.mat = __ldg(a.material + p);
    if (H == 1 || h == 0) {
      q.u = __ldg(a.u + p);
      q.r = __ldg(a.radius + p);
      q.wi0 = __ldg(a.wi + 3 * p);
      q.wi1 = __ldg(a.wi + 3 * p + 1);
      q.wi2 = __ldg(a.wi + 3 * p + 2);
      q.wo0 = __ldg(a.wo + 3 * p);
      q.wo1 = __ldg(a.wo + 3 * p + 1);
      q.wo2 = __ldg(a.wo + 3 * p + 2);
    }
    if (H == 1 || h == 1) q.v = __ldg(a.v + p);
  }
  return q;
}

// Named barrier ID over the PT threads of one tile pipeline, OR-reducing `pred`.
template <int ID, int PT>
__device__ __forceinline__ bool bar_or(bool pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((int)pred), "n"(ID), "n"(PT)
      : "memory");
  return r != 0;
}
// Pipeline wg synchronises on barrier 1 + wg (barrier 0 is __syncthreads).
template <int PT>
__device__ __forceinline__ bool wg_sync_or(int wg, bool pred) {
  switch (wg) {
    case 0: return bar_or<1, PT>(pred);
    case 1: return bar_or<2, PT>(pred);
    case 2: return bar_or<3, PT>(pred);
    default: return bar_or<4, PT>(pred);
  }
}

// WG tile pipelines per CTA, each of H warpgroups: with H = 2 the two threads
// of a row (warps w and w + 4 share the tensor-memory lane quadrant) split
// the encoding and every epilogue's columns, which halves the serial work per
// thread and doubles the warps that hide the MMA and tcgen05.ld latencies.
template <int PR, int WG, int H, bool MULTI>
__global__ void __launch_bounds__(kTile * H * WG, 4 / WG) decoder_tc_kernel(const TcArgs a) {
  constexpr bool F16 = PR != kPrBF16;   // layer-1 (and, unless E4M3, every) operand type
  constexpr bool F8 = PR == kPrE4M3;
  constexpr int PT = kTile * H;         // threads per tile pipeline
  constexpr int CH = 2 / H;             // 32-column chunks of D per thread
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bar_w = reinterpret_cast<uint64_t *>(smem);
  uint64_t *bar_mma = bar_w + 1;                         // one per pipeline
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar_w + 1 + WG);
  const BlobLayout L = blob_layout(a.n_mat, a.k1, F8);
  uint8_t *wts = smem + 1024;
  const int tid = threadIdx.x;
  const int wg = tid / PT;              // tile pipeline
  const int tp = tid % PT;              // thread within the pipeline
  const int h = H == 1 ? 0 : tp >> 7;   // which half of the row's columns
  const int row = tp & (kTile - 1);     // tile row owned by this thread
  const int warp = tid >> 5;
  const bool lead = tp == 0;            // issues the MMAs
  uint64_t *my_bar = bar_mma + wg;

  if (tid == 0) {
    tc::mbar_init(bar_w, 1);
    for (int g = 0; g < WG; ++g) tc::mbar_init(bar_mma + g, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kColsPerTile * WG);
  // batched launches: the segment table (prefix sums of tile counts) in the
  // shared memory past the weights, when the launch gave room for it
  const int64_t *seg_t0 = a.seg_tile0;
  if (MULTI && a.seg_in_smem) {
    int64_t *s_t0 = reinterpret_cast<int64_t *>(smem + 1024 + align1k(L.total));
    for (int i = tid; i <= a.n_segs; i += blockDim.x) s_t0[i] = a.seg_tile0[i];
    seg_t0 = s_t0;
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot + kColsPerTile * (uint32_t)wg;   // this pipeline's D column 0, lane 0
  const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;          // this warp's lane quadrant
  const uint32_t t_d = tmem + lane, t_a = tmem + lane + kColA;

  if (tid == 0) {
    tc::mbar_arrive_expect_tx(bar_w, L.total);
    tc::bulk_g2s(wts, a.blob, L.total, bar_w);
  }
  // first tile's inputs travel while the weights land
  const int64_t stride = (int64_t)gridDim.x * WG;
  int64_t tile = (int64_t)blockIdx.x * WG + wg;
  int seg_cursor = 0;   // segment of the pipeline's latest tile (batched launches)
  TileView view = tile_view<MULTI>(a, seg_t0, tile, seg_cursor);
  Point pt = load_point<H>(view, view.first + row, h);
  bool ok = tc::mbar_wait_sleep(bar_w, 0, kWaitCycles);
  const float *alb = reinterpret_cast<const float *>(wts + L.alb);
  const float *epi = reinterpret_cast<const float *>(wts + L.epi);   // E4M3 only

  const uint32_t w1_addr = tc::smem_addr(wts + L.w1), w2_addr = tc::smem_addr(wts + L.w2);
  const uint32_t w3_addr = tc::smem_addr(wts + L.w3), w4_addr = tc::smem_addr(wts + L.w4);
  const uint32_t id64 = F16 ? tc::idesc_f16(128, 64) : tc::idesc_bf16(128, 64);
  const uint32_t id16 = F16 ? tc::idesc_f16(128, 16) : tc::idesc_bf16(128, 16);
  const uint32_t id8_64 = tc::idesc_e4m3(128, 64), id8_16 = tc::idesc_e4m3(128, 16);
  const uint32_t one16 = F16 ? 0x3C00u : 0x3F80u;   // 1.0 in the operand type
  uint32_t phase = 0;

  for (; tile < a.n_tiles; tile += stride) {
    // this tile's outputs (the view moves on to the next tile at layer 1)
    float *const out_rgb = view.rgb;
    float *const out_comps = view.comps;
    const int64_t p = view.first + row;
    const int64_t p_end = view.n;
    int mat = pt.mat;
    if (mat >= a.n_mat) {
      if (H == 1 || h == 0) atomicOr(a.status, kStatusBadMaterial);
      mat = -2;
    }
    // ---- encode this thread's share of its row of the layer-1 A operand
    {
      uint32_t w[8];
      if (H == 1 || h == 0) {                        // features 0..15: octaves of u
        if (mat >= 0) {
          octave_words<F16>(pt.u, w);
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) w[k] = 0u;
        }
        tc::tmem_st8(t_a, w);
      }
      if (H == 1 || h == 1) {                        // features 16..31: octaves of v
        if (mat >= 0) {
          octave_words<F16>(pt.v, w);
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) w[k] = 0u;
        }
        tc::tmem_st8(t_a + 8, w);
      }
      if (H == 1 || h == 0) {
        if (mat >= 0) {
          const float l = (__logf(fmaxf(pt.r, kRFloor)) - kLogRC0) * kLogRInvC1;
          w[0] = tc::pack2<F16>(l, pt.wi0);
          w[1] = tc::pack2<F16>(pt.wi1, pt.wi2);
          w[2] = tc::pack2<F16>(pt.wo0, pt.wo1);
          w[3] = tc::pack2<F16>(pt.wo2, mat == 0 ? 1.0f : 0.0f);
        } else {
          w[0] = w[1] = w[2] = w[3] = 0u;
        }
        // features 40.. are the one-hot material columns (39 is in w[3])
        const int hot = kQueryFeat + mat;
#pragma unroll
        for (int k = 4; k < 8; ++k) w[k] = (hot == 2 * (16 + k) ? one16 : 0u) | (hot == 2 * (16 + k) + 1 ? one16 << 16 : 0u);
        tc::tmem_st8(t_a + 16, w);                   // features 32..47
        for (int c = 3; c < a.k1 / 16; ++c) {        // features 48.. (wider one-hot)
#pragma unroll
          for (int k = 0; k < 8; ++k)
            w[k] = (hot == 16 * c + 2 * k ? one16 : 0u) | (hot == 16 * c + 2 * k + 1 ? one16 << 16 : 0u);
          tc::tmem_st8(t_a + 8 * c, w);
        }
      }
      tc::tmem_st_wait();
    }
    // ---- four layers
#pragma unroll
    for (int layer = 0; layer < 4; ++layer) {
      tc::tc_fence_before();
      if (wg_sync_or<PT>(wg, !ok)) {
        ok = false;
        goto teardown;
      }
      if (lead) {
        tc::tc_fence_after();
        const uint32_t w_addr = layer == 0 ? w1_addr : layer == 1 ? w2_addr : layer == 2 ? w3_addr : w4_addr;
        if (F8 && layer > 0) {
          // E4M3: K = 64 in two K = 32 steps (8 columns of A, 2 core matrices of B each)
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t bd = tc::smem_desc(w_addr + kk * 256u, 128u, 64u * 8u);
            tc::mma_f8_ts(tmem, tmem + kColA + 8u * kk, bd, layer == 3 ? id8_16 : id8_64, kk > 0 ? 1u : 0u);
          }
        } else {
          const int K = layer == 0 ? a.k1 : kKH;
          const uint32_t sbo = (uint32_t)K * 16u;
          for (int kk = 0; kk < K / 16; ++kk) {
            const uint64_t bd = tc::smem_desc(w_addr + kk * 256u, 128u, sbo);
            tc::mma_f16_ts(tmem, tmem + kColA + 8u * kk, bd, layer == 3 ? id16 : id64, kk > 0 ? 1u : 0u);
          }
        }
        tc::mma_commit(my_bar);
      }
      if (layer == 0) {   // next tile's inputs, in flight during this tile's layers
        view = tile_view<MULTI>(a, seg_t0, tile + stride, seg_cursor);
        pt = load_point<H>(view, view.first + row, h);
      }
      // every warp sleeps on the mbarrier until the products land (no
      // further barrier hop); an expired wait is OR-reduced at the next
      // named barrier, where the whole pipeline leaves together
      ok = tc::mbar_wait_sleep(my_bar, phase, kWaitCycles) && ok;
      phase ^= 1u;
      tc::tc_fence_after();
      if (layer < 3) {
        const float inv = F8 ? epi[kF8Inv + layer] : 1.0f;
        const float4 *bl = reinterpret_cast<const float4 *>(epi + kF8Bias + 64 * layer);
#pragma unroll
        for (int cc = 0; cc < CH; ++cc) {
          const int chunk = h * CH + cc;             // D columns [32 chunk, 32 chunk + 32)
          if (F8) {
            // y = acc * 2^-s_l + b_l (exactly acc for layer 1), ReLU, E4M3;
            // 16 columns of D become 4 columns of A
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              float acc[16];
              tc::tmem_ld16(t_d + 32 * chunk + 16 * q, acc);
              tc::tmem_ld_wait();
              uint32_t w[4];
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const float4 b = bl[8 * chunk + 4 * q + k];
                w[k] = tc::pack4_e4m3_relu(fmaf(acc[4 * k], inv, b.x), fmaf(acc[4 * k + 1], inv, b.y),
                                           fmaf(acc[4 * k + 2], inv, b.z), fmaf(acc[4 * k + 3], inv, b.w));
              }
              tc::tmem_st4(t_a + 8 * chunk + 4 * q, w);
            }
          }
        }
        if (!F8) {
          // all of this thread's D columns in flight at once (32 columns per
          // tcgen05.ld), one wait, 16 columns of A per tcgen05.st
          float acc[32 * CH];
#pragma unroll
          for (int cc = 0; cc < CH; ++cc) tc::tmem_ld32(t_d + 32 * (h * CH + cc), acc + 32 * cc);
          tc::tmem_ld_wait();
#pragma unroll
          for (int cc = 0; cc < CH; ++cc) {
            const int chunk = h * CH + cc;
            uint32_t w[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) w[k] = tc::pack2_relu<F16>(acc[32 * cc + 2 * k], acc[32 * cc + 2 * k + 1]);
            tc::tmem_st16(t_a + 16 * chunk, w);
          }
        }
        if (!F8 && (H == 1 || h == H - 1)) {
          // constant-one column (bias of layers 2-4) and zero padding, K = 64..79
          uint32_t w[8] = {one16, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
          tc::tmem_st8(t_a + 32, w);
        }
        tc::tmem_st_wait();
      } else if (H == 1 || h == 0) {
        float y[4];
        tc::tmem_ld4(t_d, y);
        tc::tmem_ld_wait();
        if (F8) {
          const float inv = epi[kF8Inv + 3];
#pragma unroll
          for (int c = 0; c < 4; ++c) y[c] = fmaf(y[c], inv, epi[kF8Bias + 64 * 3 + c]);
        }
        if (p < p_end) {
          float c4[4];
          if (mat < 0) {
            c4[0] = c4[1] = c4[2] = c4[3] = __int_as_float(0x7FC00000);
          } else {
            // inverse of Eq. 9; exp(y) - 1 loses only absolute precision
            // near y = 0, where S itself is ~0
            c4[0] = fmaxf(0.0f, y[0]);
            c4[1] = fmaxf(0.0f, y[1]);
            c4[2] = fmaxf(0.0f, (__expf(y[2]) - 1.0f) * (1.0f / kSpecK));
            c4[3] = fmaxf(0.0f, (__expf(y[3]) - 1.0f) * (1.0f / kSpecK));
          }
          if (out_comps) store_row4(out_comps, p, c4[0], c4[1], c4[2], c4[3]);
          const float4 *al = reinterpret_cast<const float4 *>(alb + (mat < 0 ? 0 : mat) * 12);
          const float4 k0 = al[0], k1 = al[1], k2 = al[2];   // kd_warp, kd_weft, ks_warp, ks_weft (RGB each)
          out_rgb[3 * p + 0] = k0.x * c4[0] + k0.w * c4[1] + k1.z * c4[2] + k2.y * c4[3];
          out_rgb[3 * p + 1] = k0.y * c4[0] + k1.x * c4[1] + k1.w * c4[2] + k2.z * c4[3];
          out_rgb[3 * p + 2] = k0.z * c4[0] + k1.y * c4[1] + k2.x * c4[2] + k2.w * c4[3];
        }
      }
    }
  }

  ok = !wg_sync_or<PT>(wg, !ok);   // one outcome per pipeline
teardown:
  if (!ok) {
    if (tid == 0) atomicOr(a.status, kStatusTimeout);
    // let any copy or product still in flight land before the memory goes away
    tc::mbar_wait(bar_w, 0, kWaitCycles);
    tc::mbar_wait(my_bar, phase ^ 1u, kWaitCycles);   // the phase whose wait expired (passes if none issued)
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(*tmem_slot, kColsPerTile * WG);
  }
}

size_t tc_smem_bytes(int n_mat, int k1, bool f8) {
  const BlobLayout L = blob_layout(n_mat, k1, f8);
  return 1024 /* alignment slack */ + 1024 /* barriers */ + align1k(L.total);
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

// ---- self-test with the A operand in tensor memory: row i of A in lane i,
// two bf16 per 32-bit column (K along the columns), B in shared memory.
__global__ void __launch_bounds__(128, 1) selftest_ts_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                             int n, int k, float *__restrict__ D, int *status) {
  __shared__ __align__(1024) uint8_t sb[64 * 64 * 2];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < n * k; e += 128) {
    const int r = e / k, c = e % k;
    put_bf16(sb, tc::core_offset(r, c, k), B[e]);
  }
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&slot, 256);
  tc::fence_proxy_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = slot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  uint32_t w[32];
#pragma unroll
  for (int j = 0; j < 32; ++j)
    w[j] = (2 * j < k) ? tc::pack_bf16(A[tid * k + 2 * j], A[tid * k + 2 * j + 1]) : 0u;
  for (int c = 0; c < k / 16; ++c) tc::tmem_st8(tmem + lane_base + 64 + 8 * c, w + 8 * c);
  tc::tmem_st_wait();
  tc::tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    tc::tc_fence_after();
    for (int kk = 0; kk < k / 16; ++kk) {
      const uint64_t bd = tc::smem_desc(tc::smem_addr(sb) + kk * 256u, 128u, (uint32_t)k * 16u);
      tc::mma_f16_ts(tmem, tmem + 64 + 8 * kk, bd, tc::idesc_bf16(128, n), kk > 0 ? 1u : 0u);
    }
    tc::mma_commit(&bar);
  }
  const bool ok = tc::mbar_wait(&bar, 0, kWaitCycles);
  if (!ok && tid == 0) atomicOr(status, kStatusTimeout);
  tc::tc_fence_after();
  if (__syncthreads_and(ok)) {
    for (int c = 0; c < n; c += 16) {
      float v[16];
      tc::tmem_ld16(tmem + lane_base + c, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int e = 0; e < 16; ++e) D[tid * n + c + e] = v[e];
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 256);
  }
}

// ---- self-test of the E4M3 path: A in tensor memory (four bytes per
// column), B in shared memory (core_offset8), kind::f8f6f4, K = 32 per step.
__global__ void __launch_bounds__(128, 1) selftest_f8_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                             int n, int k, float *__restrict__ D, int *status) {
  __shared__ __align__(1024) uint8_t sb[64 * 64];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < n * k; e += 128) {
    const int r = e / k, c = e % k;
    sb[tc::core_offset8(r, c, k)] = to_e4m3(B[e]);
  }
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&slot, 128);
  tc::fence_proxy_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = slot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  uint32_t w[16];
#pragma unroll
  for (int j = 0; j < 16; ++j)
    w[j] = (4 * j < k) ? tc::pack4_e4m3(A[tid * k + 4 * j], A[tid * k + 4 * j + 1], A[tid * k + 4 * j + 2],
                                        A[tid * k + 4 * j + 3])
                       : 0u;
  for (int c = 0; c < k / 32; ++c) tc::tmem_st8(tmem + lane_base + 64 + 8 * c, w + 8 * c);
  tc::tmem_st_wait();
  tc::tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    tc::tc_fence_after();
    for (int kk = 0; kk < k / 32; ++kk) {
      const uint64_t bd = tc::smem_desc(tc::smem_addr(sb) + kk * 256u, 128u, (uint32_t)k * 8u);
      tc::mma_f8_ts(tmem, tmem + 64 + 8 * kk, bd, tc::idesc_e4m3(128, n), kk > 0 ? 1u : 0u);
    }
    tc::mma_commit(&bar);
  }
  const bool ok = tc::mbar_wait(&bar, 0, kWaitCycles);
  if (!ok && tid == 0) atomicOr(status, kStatusTimeout);
  tc::tc_fence_after();
  if (__syncthreads_and(ok)) {
    for (int c = 0; c < n; c += 16) {
      float v[16];
      tc::tmem_ld16(tmem + lane_base + c, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int e = 0; e < 16; ++e) D[tid * n + c + e] = v[e];
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 128);
  }
}

template <int PR, int WG, int H, bool MULTI>
const void *kernel_ptr() {
  return reinterpret_cast<const void *>(decoder_tc_kernel<PR, WG, H, MULTI>);
}

// Supported shapes: 1, 2 or 4 tile pipelines per CTA (128 tensor-memory
// columns each) of one warpgroup, or 1 or 2 pipelines of two warpgroups.
int norm_wg(int wg) { return wg == 2 || wg == 4 ? wg : 1; }
int norm_h(int h, int wg) { return (h == 2 && wg <= 2) ? 2 : 1; }

template <int PR, bool MULTI>
const void *pick_kernel_pm(int wg, int h) {
  if (h == 2) return wg == 1 ? kernel_ptr<PR, 1, 2, MULTI>() : kernel_ptr<PR, 2, 2, MULTI>();
  return wg == 1 ? kernel_ptr<PR, 1, 1, MULTI>() : wg == 2 ? kernel_ptr<PR, 2, 1, MULTI>()
                                                           : kernel_ptr<PR, 4, 1, MULTI>();
}
template <bool MULTI>
const void *pick_kernel_m(int pr, int wg, int h) {
  return pr == kPrF16 ? pick_kernel_pm<kPrF16, MULTI>(wg, h)
                      : pr == kPrE4M3 ? pick_kernel_pm<kPrE4M3, MULTI>(wg, h) : pick_kernel_pm<kPrBF16, MULTI>(wg, h);
}
const void *pick_kernel(int pr, int wg, int h, bool multi = false) {
  return multi ? pick_kernel_m<true>(pr, wg, h) : pick_kernel_m<false>(pr, wg, h);
}

// CTAs of the decoder that fit on one SM, counted from the kernel's
// registers (allocated per warp in units of 8), its shared memory (plus the
// 1 KB the driver reserves per CTA) and the 512 tensor-memory columns.
int tc_resident_ctas(const void *fn, size_t smem, int wg, int h) {
  int dev = 0, smem_sm = 0, regs_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaFuncAttributes fa;
  int regs = 128;
  size_t static_smem = 0;
  if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess) {
    regs = fa.numRegs;
    static_smem = fa.sharedSizeBytes;
  }
  cudaGetLastError();
  const int by_smem = (int)(smem_sm / (smem + static_smem + 1024));
  const int by_regs = regs_sm / (((regs + 7) & ~7) * kTile * wg * h);
  const int by_tmem = 512 / (int)(kColsPerTile * wg);
  int occ = by_smem < by_regs ? by_smem : by_regs;
  if (occ > by_tmem) occ = by_tmem;
  return occ < 1 ? 1 : occ;
}

}  // namespace

int tc_k1(int n_mat) { return tc_k1_of(n_mat); }

size_t tc_blob_bytes(int n_mat) { return tc_blob_bytes_of(n_mat); }

cudaError_t launch_tc_pack(const float *dec, const float *latents, const DevMaterial *mats, int n_mat, int precision,
                           void *blob, cudaStream_t s) {
  const int k1 = tc_k1(n_mat);
  if (k1 < 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)n_mat * kHidden * sizeof(float);
  uint8_t *out = static_cast<uint8_t *>(blob);
  switch (prec_code(precision)) {
    case kPrF16: pack_kernel<kPrF16><<<1, 256, smem, s>>>(dec, latents, mats, n_mat, k1, out); break;
    case kPrE4M3: pack_kernel<kPrE4M3><<<1, 256, smem, s>>>(dec, latents, mats, n_mat, k1, out); break;
    default: pack_kernel<kPrBF16><<<1, 256, smem, s>>>(dec, latents, mats, n_mat, k1, out); break;
  }
  return cudaGetLastError();
}

int tc_default_ctas_per_sm(int n_mat, int precision) {
  const int k1 = tc_k1(n_mat);
  if (k1 < 0) return 1;
  const int wg = 1;
  const int pr = prec_code(precision);
  const void *fn = pick_kernel(pr, wg, 1, false);
  ensure_max_dyn_smem(fn, 200 * 1024);
  return tc_resident_ctas(fn, tc_smem_bytes(n_mat, k1, pr == kPrE4M3), wg, 1);
}

static cudaError_t launch_tc(TcArgs &a, bool multi, int precision, int sm_count, int ctas_per_sm, int warpgroups,
                             int tile_wgs, cudaStream_t s) {
  const int pr = prec_code(precision);
  const int wg = norm_wg(warpgroups);
  const int h = norm_h(tile_wgs, wg);
  const size_t smem = tc_smem_bytes(a.n_mat, a.k1, pr == kPrE4M3);
  const void *fn = pick_kernel(pr, wg, h, multi);
  {
    const cudaError_t e = ensure_max_dyn_smem(fn, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  const int resident = tc_resident_ctas(fn, smem, wg, h);
  int per_sm = ctas_per_sm > 0 ? ctas_per_sm : resident;
  if (per_sm > resident) per_sm = resident;
  int64_t grid = (int64_t)sm_count * per_sm;
  const int64_t need = (a.n_tiles + wg - 1) / wg;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  // Pad the dynamic shared memory so that no SM can take more than per_sm
  // CTAs: one more would wait in tcgen05.alloc until a resident CTA (which
  // runs to the end of the grid's work) frees its tensor memory.
  size_t launch_smem = smem;
  {
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const size_t floor_smem = (size_t)smem_sm / (size_t)(per_sm + 1) - 1024 + 1;   // (per_sm + 1) CTAs overflow
    const size_t roomy = (size_t)smem_sm / (size_t)per_sm - 1024;                     // per_sm CTAs still fit
    if (floor_smem > launch_smem && floor_smem <= roomy && floor_smem <= 200 * 1024) launch_smem = floor_smem;
    // batched: the segment table in the spare shared memory, when it fits
    // without lowering the CTAs per SM
    a.seg_in_smem = 0;
    if (multi) {
      const size_t table = ((size_t)a.n_segs + 1) * sizeof(int64_t);
      if (smem + table <= launch_smem) {
        a.seg_in_smem = 1;
      } else if (smem + table <= roomy && smem + table <= 200 * 1024) {
        launch_smem = smem + table;
        a.seg_in_smem = 1;
      }
    }
  }
  void *args[] = {&a};
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kTile * wg * h), args, launch_smem, s);
}

cudaError_t launch_decoder_tc(const fabric_gbuffer &g, const void *blob, int n_mat, int precision, float *rgb,
                              float *comps, int *status, int sm_count, int ctas_per_sm, int warpgroups,
                              int tile_wgs, cudaStream_t s) {
  const int k1 = tc_k1(n_mat);
  if (k1 < 0) return cudaErrorInvalidValue;
  TcArgs a = {};
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
  return launch_tc(a, false, precision, sm_count, ctas_per_sm, warpgroups, tile_wgs, s);
}

int64_t tc_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

cudaError_t launch_decoder_tc_segments(const SegDesc *segs, const int64_t *seg_tile0, int n_segs, int64_t n_tiles,
                                       const void *blob, int n_mat, int precision, int *status, int sm_count,
                                       int ctas_per_sm, int warpgroups, int tile_wgs, cudaStream_t s) {
  const int k1 = tc_k1(n_mat);
  if (k1 < 0) return cudaErrorInvalidValue;
  TcArgs a = {};
  a.n_tiles = n_tiles;
  a.blob = static_cast<const uint8_t *>(blob);
  a.n_mat = n_mat;
  a.k1 = k1;
  a.status = status;
  a.segs = segs;
  a.seg_tile0 = seg_tile0;
  a.n_segs = n_segs;
  return launch_tc(a, true, precision, sm_count, ctas_per_sm, warpgroups, tile_wgs, s);
}

// ---- self-test of the bounded waits: an mbarrier that nothing arrives on.
// Every thread waits on it with the same helpers the kernels use (spinning,
// or try_wait with a suspend hint); each wait gives up after `max_cycles`,
// the block records a timeout in the status word and returns normally.
__global__ void __launch_bounds__(64, 1) selftest_wait_kernel(int sleep, long long max_cycles, int *status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);   // one arrival expected; none ever comes
    tc::fence_mbar_init();
  }
  __syncthreads();
  const bool ok = sleep ? tc::mbar_wait_sleep(&bar, 0, max_cycles) : tc::mbar_wait(&bar, 0, max_cycles);
  const bool expired = __syncthreads_or(!ok);
  if (expired && threadIdx.x == 0) atomicOr(status, kStatusTimeout);
}

cudaError_t launch_selftest_wait(int sleep, int *status, cudaStream_t s) {
  selftest_wait_kernel<<<1, 64, 0, s>>>(sleep, 2000000ll /* about 1 ms */, status);
  return cudaGetLastError();
}

cudaError_t launch_selftest_mma(const float *a, const float *b, int n, int k, int a_in_tmem, float *d, int *status,
                                cudaStream_t s) {
  if (a_in_tmem == 2)
    selftest_f8_kernel<<<1, 128, 0, s>>>(a, b, n, k, d, status);
  else if (a_in_tmem)
    selftest_ts_kernel<<<1, 128, 0, s>>>(a, b, n, k, d, status);
  else
    selftest_kernel<<<1, 128, 0, s>>>(a, b, n, k, d, status);
  return cudaGetLastError();
}

}  // namespace fab
