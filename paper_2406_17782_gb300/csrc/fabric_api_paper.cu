// fabric_api_paper.cu -- C ABI of the paper's decoder structure (Sec. 4.2,
// "Decoder"; Fig. 3): parameters, operand packing and tensor-core shading.
#include <cstring>

#include "fabric_internal.h"
#include "paper_net.h"

namespace fab {

void paper_release(fabric_ctx *ctx) {
  cudaFree(ctx->d_pn_dec);
  cudaFree(ctx->d_pn_enc);
  cudaFree(ctx->d_pn_adam);
  cudaFree(ctx->d_pn_blob);
  ctx->d_pn_dec = ctx->d_pn_enc = ctx->d_pn_adam = nullptr;
  ctx->d_pn_blob = nullptr;
  ctx->pn_width = 0;
}

namespace {

constexpr int kPnMaxMaterials = 104;   // 24 one-blob channels + 104 one-hot columns = K 128

// Shared memory the decoder needs for n_mat materials at width w (the
// blob plus 2 KB of alignment and barriers); at most 227 KB per CTA.
bool paper_fits(int w, int n_mat) { return paper_blob_bytes(w, n_mat) + 2048 + 1024 <= 227u * 1024u; }

uint64_t pn_state(const fabric_ctx *ctx) { return ctx->version * 0x9E3779B97F4A7C15ull ^ ctx->pn_version; }

}  // namespace
}  // namespace fab

using namespace fab;

#define PN_CHECK_CTX(ctx)                                           \
  do {                                                              \
    if (!(ctx)) return FABRIC_ERR_INVALID_ARG;                      \
    (ctx)->last_error.clear();                                      \
    if (cudaSetDevice((ctx)->device) != cudaSuccess)                \
      return cuda_fail((ctx), cudaGetLastError(), "cudaSetDevice"); \
  } while (0)

#define PN_CUDA(ctx, expr, what)                                   \
  do {                                                             \
    cudaError_t e_ = (expr);                                       \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, (what));    \
  } while (0)

extern "C" {

int64_t fabric_paper_param_count(int width, int encoder) {
  if (encoder) return kPnEncParams;
  return paper_width_ok(width) ? paper_offsets(width).total : -1;
}

fabric_status fabric_paper_set_params(fabric_ctx *ctx, int width, const float *decoder, const float *encoder) {
  PN_CHECK_CTX(ctx);
  if (!paper_width_ok(width)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "width must be 64 or 128 (got %d)", width);
  if (width != ctx->pn_width) {
    if (!decoder || !encoder)
      return fail(ctx, FABRIC_ERR_INVALID_ARG, "a new width needs both decoder and encoder parameters");
    paper_release(ctx);
    const size_t nd = (size_t)paper_offsets(width).total, ne = (size_t)kPnEncParams;
    if (cudaMalloc(&ctx->d_pn_dec, nd * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&ctx->d_pn_enc, ne * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&ctx->d_pn_adam, 2 * (nd + ne) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&ctx->d_pn_blob, paper_blob_bytes(width, kPnMaxMaterials)) != cudaSuccess) {
      paper_release(ctx);
      cudaGetLastError();
      return fail(ctx, FABRIC_ERR_OOM, "paper network buffers");
    }
    ctx->pn_width = width;
  }
  const size_t nd = (size_t)paper_offsets(width).total, ne = (size_t)kPnEncParams;
  if (decoder) PN_CUDA(ctx, cudaMemcpy(ctx->d_pn_dec, decoder, nd * sizeof(float), cudaMemcpyHostToDevice), "params");
  if (encoder) PN_CUDA(ctx, cudaMemcpy(ctx->d_pn_enc, encoder, ne * sizeof(float), cudaMemcpyHostToDevice), "params");
  PN_CUDA(ctx, cudaMemset(ctx->d_pn_adam, 0, 2 * (nd + ne) * sizeof(float)), "adam reset");
  ctx->pn_adam_step = 0;
  ctx->pn_version += 1;
  PN_CUDA(ctx, cudaDeviceSynchronize(), "set params");
  return FABRIC_OK;
}

fabric_status fabric_paper_get_params(fabric_ctx *ctx, float *decoder, float *encoder) {
  PN_CHECK_CTX(ctx);
  if (!ctx->pn_width) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no paper network parameters set");
  PN_CUDA(ctx, cudaDeviceSynchronize(), "get params");
  const size_t nd = (size_t)paper_offsets(ctx->pn_width).total, ne = (size_t)kPnEncParams;
  if (decoder) PN_CUDA(ctx, cudaMemcpy(decoder, ctx->d_pn_dec, nd * sizeof(float), cudaMemcpyDeviceToHost), "params");
  if (encoder) PN_CUDA(ctx, cudaMemcpy(encoder, ctx->d_pn_enc, ne * sizeof(float), cudaMemcpyDeviceToHost), "params");
  return FABRIC_OK;
}

fabric_status fabric_paper_prepare(fabric_ctx *ctx, const float *latents_dev, fabric_precision prec, void *stream) {
  PN_CHECK_CTX(ctx);
  if (prec != FABRIC_PREC_FP16 && prec != FABRIC_PREC_BF16)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "the paper network runs with FP16 or BF16 operands (got %d)", (int)prec);
  if (!ctx->pn_width) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no paper network parameters set");
  if (!latents_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "latents are NULL");
  if (ctx->n_mat == 0) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no materials set");
  if (paper_k1(ctx->n_mat) < 0 || !paper_fits(ctx->pn_width, ctx->n_mat))
    return fail(ctx, FABRIC_ERR_UNSUPPORTED, "the paper network takes at most %d materials (have %d)",
                kPnMaxMaterials, ctx->n_mat);
  ctx->pn_prepared_prec = -1;
  PN_CUDA(ctx,
          launch_paper_pack(ctx->pn_width, (int)prec, ctx->d_pn_dec, latents_dev, ctx->d_mat, ctx->n_mat,
                            ctx->d_pn_blob, static_cast<cudaStream_t>(stream)),
          "paper network pack");
  ctx->pn_prepared_prec = (int)prec;
  ctx->pn_prepared_version = pn_state(ctx);
  return FABRIC_OK;
}

fabric_status fabric_paper_shade_prepared(fabric_ctx *ctx, const fabric_gbuffer *g, fabric_precision prec,
                                          float *rgb_dev, float *comps_dev, void *stream) {
  PN_CHECK_CTX(ctx);
  if (!check_gbuffer(ctx, g)) return FABRIC_ERR_INVALID_ARG;
  if (ctx->pn_prepared_prec != (int)prec || ctx->pn_prepared_version != pn_state(ctx))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "no prepared paper network for this precision, materials and parameters");
  if (g->n == 0) return FABRIC_OK;
  if (!rgb_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "rgb output is NULL");
  if (comps_dev && !is_aligned16(comps_dev))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "comps output must be 16-byte aligned");
  PN_CUDA(ctx,
          launch_paper_decoder(ctx->pn_width, (int)prec, *g, ctx->d_pn_blob, ctx->n_mat, rgb_dev, comps_dev,
                               ctx->d_status, ctx->sm_count, static_cast<cudaStream_t>(stream)),
          "paper network decoder launch");
  return FABRIC_OK;
}

fabric_status fabric_paper_shade_neural(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev,
                                        fabric_precision prec, float *rgb_dev, float *comps_dev, void *stream) {
  PN_CHECK_CTX(ctx);
  if (!check_gbuffer(ctx, g)) return FABRIC_ERR_INVALID_ARG;
  if (g->n == 0) return FABRIC_OK;
  const fabric_status st = fabric_paper_prepare(ctx, latents_dev, prec, stream);
  if (st != FABRIC_OK) return st;
  return fabric_paper_shade_prepared(ctx, g, prec, rgb_dev, comps_dev, stream);
}

}  // extern "C"
