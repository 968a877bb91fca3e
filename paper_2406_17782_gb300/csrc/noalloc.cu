// noalloc.cu -- fabric_shade_neural_noalloc: the tensor-core neural shading
// call with its per-call scratch (the packed decoder operands) in a
// file-scope device array instead of context-owned memory.  Nothing here
// allocates device memory.
#include <atomic>

#include "decoder_blob.h"
#include "fabric_internal.h"

namespace {

// Largest packed-operand blob this entry point accepts.  The array lives on
// every GPU that loads the library until the process exits.
constexpr size_t kNoAllocBlobBytes = 64 * 1024;

static __device__ __align__(256) uint8_t g_noalloc_blob[kNoAllocBlobBytes];

// The decoder's own material limit (89) is the one that binds in practice:
// its largest packed blob fits the array.
static_assert(fab::tc_blob_bytes_of(fab::kTcMaxMaterials) <= kNoAllocBlobBytes,
              "the packed operands of the largest material table must fit the static scratch");

constexpr int kMaxDevices = 64;
// Device address of g_noalloc_blob per device, resolved once with that
// device current (host code must not use the symbol itself as an address).
// Host threads that make their first call on one device at the same time
// may both resolve it; they store the same address.
std::atomic<void *> g_blob_addr[kMaxDevices] = {};

}  // namespace

extern "C" fabric_status fabric_shade_neural_noalloc(fabric_ctx *ctx, const fabric_gbuffer *g,
                                                     const float *latents_dev, fabric_precision prec,
                                                     float *rgb_dev, float *comps_dev, void *stream) {
  using namespace fab;
  if (!ctx) return FABRIC_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  if (!check_gbuffer(ctx, g)) return FABRIC_ERR_INVALID_ARG;
  if (prec != FABRIC_PREC_FP16 && prec != FABRIC_PREC_BF16 && prec != FABRIC_PREC_FP8)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "the no-allocation call runs the FP16, BF16 or FP8 tensor-core decoder only");
  if (g->n == 0) return FABRIC_OK;
  if (!rgb_dev || !latents_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "rgb output or latents is NULL");
  if (comps_dev && !is_aligned4(comps_dev))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "comps output must be float-aligned");
  if (ctx->n_mat == 0) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no materials set");
  if (tc_k1(ctx->n_mat) < 0)
    return fail(ctx, FABRIC_ERR_UNSUPPORTED, "tensor-core decoder supports at most 89 materials (have %d)",
                ctx->n_mat);
  const size_t need = tc_blob_bytes(ctx->n_mat);
  if (need > kNoAllocBlobBytes)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "packed operands need %zu bytes, the static scratch holds %zu", need,
                kNoAllocBlobBytes);
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return fail(ctx, FABRIC_ERR_UNSUPPORTED, "device index %d beyond %d", ctx->device, kMaxDevices);
  void *blob = g_blob_addr[ctx->device].load(std::memory_order_acquire);
  if (!blob) {
    // one-time set-up on this device (the device is current here)
    const cudaError_t e = cudaGetSymbolAddress(&blob, g_noalloc_blob);
    if (e != cudaSuccess || !blob) return cuda_fail(ctx, e, "cudaGetSymbolAddress(g_noalloc_blob)");
    g_blob_addr[ctx->device].store(blob, std::memory_order_release);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_tc_pack(ctx->d_dec, latents_dev, ctx->d_mat, ctx->n_mat, (int)prec, blob, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pack");
  e = launch_decoder_tc(*g, blob, ctx->n_mat, (int)prec, rgb_dev, comps_dev, ctx->d_status, ctx->sm_count,
                        ctx->tc_ctas_per_sm, ctx->tc_warpgroups, ctx->tc_tile_wgs, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core decoder launch");
  return FABRIC_OK;
}
