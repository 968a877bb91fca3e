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
  cudaFree(ctx->d_pn_grad);
  ctx->d_pn_dec = ctx->d_pn_enc = ctx->d_pn_adam = ctx->d_pn_grad = nullptr;
  ctx->d_pn_blob = nullptr;
  ctx->pn_width = 0;
  ctx->pn_ablation = 0;
}

namespace {

constexpr int kPnMaxMaterials = 104;   // 24 one-blob channels + 104 one-hot columns = K 128

// Shared memory the decoder needs for n_mat materials at width w (the
// blob plus 2 KB of alignment and barriers); at most 227 KB per CTA.
bool paper_fits(int w, int n_mat) { return paper_blob_bytes(w, n_mat) + 2048 + 1024 <= 227u * 1024u; }

uint64_t pn_state(const fabric_ctx *ctx) { return ctx->version * 0x9E3779B97F4A7C15ull ^ ctx->pn_version; }

bool ablation_ok(int a) { return a == kPnFull || a == kPnNoOneBlob || a == kPnNoFusion; }

size_t n_dec(const fabric_ctx *ctx) { return (size_t)paper_offsets_ablation(ctx->pn_width, ctx->pn_ablation).total; }

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

int64_t fabric_paper_structure_param_count(int width, int ablation) {
  return paper_width_ok(width) && ablation_ok(ablation) ? paper_offsets_ablation(width, ablation).total : -1;
}

fabric_status fabric_paper_set_structure(fabric_ctx *ctx, int width, int ablation, const float *decoder,
                                         const float *encoder) {
  PN_CHECK_CTX(ctx);
  if (!paper_width_ok(width)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "width must be 64 or 128 (got %d)", width);
  if (!ablation_ok(ablation)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "unknown structure %d", ablation);
  const size_t nd = (size_t)paper_offsets_ablation(width, ablation).total, ne = (size_t)kPnEncParams;
  if (width != ctx->pn_width || ablation != ctx->pn_ablation) {
    if (!decoder || !encoder)
      return fail(ctx, FABRIC_ERR_INVALID_ARG, "a new width or structure needs both decoder and encoder parameters");
    paper_release(ctx);
    if (cudaMalloc(&ctx->d_pn_dec, nd * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&ctx->d_pn_enc, ne * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&ctx->d_pn_adam, 2 * (nd + ne) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&ctx->d_pn_grad, (nd + ne) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&ctx->d_pn_blob, paper_blob_bytes(width, kPnMaxMaterials)) != cudaSuccess) {
      paper_release(ctx);
      cudaGetLastError();
      return fail(ctx, FABRIC_ERR_OOM, "paper network buffers");
    }
    ctx->pn_width = width;
    ctx->pn_ablation = ablation;
  }
  if (decoder) PN_CUDA(ctx, cudaMemcpy(ctx->d_pn_dec, decoder, nd * sizeof(float), cudaMemcpyHostToDevice), "params");
  if (encoder) PN_CUDA(ctx, cudaMemcpy(ctx->d_pn_enc, encoder, ne * sizeof(float), cudaMemcpyHostToDevice), "params");
  PN_CUDA(ctx, cudaMemset(ctx->d_pn_adam, 0, 2 * (nd + ne) * sizeof(float)), "adam reset");
  PN_CUDA(ctx, cudaMemset(ctx->d_pn_grad, 0, (nd + ne) * sizeof(float)), "gradient reset");
  ctx->pn_adam_step = 0;
  ctx->pn_version += 1;
  PN_CUDA(ctx, cudaDeviceSynchronize(), "set params");
  return FABRIC_OK;
}

fabric_status fabric_paper_set_params(fabric_ctx *ctx, int width, const float *decoder, const float *encoder) {
  return fabric_paper_set_structure(ctx, width, kPnFull, decoder, encoder);
}

fabric_status fabric_paper_get_params(fabric_ctx *ctx, float *decoder, float *encoder) {
  PN_CHECK_CTX(ctx);
  if (!ctx->pn_width) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no paper network parameters set");
  PN_CUDA(ctx, cudaDeviceSynchronize(), "get params");
  const size_t nd = n_dec(ctx), ne = (size_t)kPnEncParams;
  if (decoder) PN_CUDA(ctx, cudaMemcpy(decoder, ctx->d_pn_dec, nd * sizeof(float), cudaMemcpyDeviceToHost), "params");
  if (encoder) PN_CUDA(ctx, cudaMemcpy(encoder, ctx->d_pn_enc, ne * sizeof(float), cudaMemcpyDeviceToHost), "params");
  return FABRIC_OK;
}

fabric_status fabric_paper_prepare(fabric_ctx *ctx, const float *latents_dev, fabric_precision prec, void *stream) {
  PN_CHECK_CTX(ctx);
  if (prec != FABRIC_PREC_FP16 && prec != FABRIC_PREC_BF16)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "the paper network runs with FP16 or BF16 operands (got %d)", (int)prec);
  if (!ctx->pn_width) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no paper network parameters set");
  if (ctx->pn_ablation != kPnFull)
    return fail(ctx, FABRIC_ERR_UNSUPPORTED, "the tensor-core decoder runs the full structure only; "
                                             "ablations shade with fabric_paper_shade_fp32");
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
  if (comps_dev && !is_aligned4(comps_dev))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "comps output must be float-aligned");
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

fabric_status fabric_paper_encode_params(fabric_ctx *ctx, const fabric_material *m, int n_mat, float *latents_dev,
                                         void *stream) {
  PN_CHECK_CTX(ctx);
  if (!ctx->pn_width) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no paper network parameters set");
  if (n_mat == 0) return FABRIC_OK;
  if (!m || !latents_dev || n_mat < 0 || n_mat > 65535)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "need materials, a latent buffer and 0..65535 records");
  for (int k = 0; k < n_mat; ++k) {
    DevMaterial tmp;
    std::string why;
    if (!build_material(m[k], &tmp, &why)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "material %d: %s", k, why.c_str());
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (ctx->enc_raw_cap < n_mat) {
    PN_CUDA(ctx, cudaStreamSynchronize(s), "encode staging");
    cudaFree(ctx->d_enc_raw);
    ctx->d_enc_raw = nullptr;
    ctx->enc_raw_cap = 0;
    PN_CUDA(ctx, cudaMalloc(&ctx->d_enc_raw, n_mat * sizeof(fabric_material)), "encode staging");
    ctx->enc_raw_cap = n_mat;
  }
  PN_CUDA(ctx, cudaMemcpyAsync(ctx->d_enc_raw, m, n_mat * sizeof(fabric_material), cudaMemcpyHostToDevice, s),
          "encode upload");
  PN_CUDA(ctx, launch_paper_encoder(ctx->d_enc_raw, n_mat, ctx->d_pn_enc, latents_dev, s), "paper encoder");
  return FABRIC_OK;
}

fabric_status fabric_paper_train_step(fabric_ctx *ctx, const fabric_train_batch *batch, float lr, double *loss_dev,
                                      void *stream) {
  PN_CHECK_CTX(ctx);
  if (!ctx->pn_width) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no paper network parameters set");
  if (!batch) return fail(ctx, FABRIC_ERR_INVALID_ARG, "batch is NULL");
  const fabric_gbuffer &q = batch->queries;
  if (!check_gbuffer(ctx, &q)) return FABRIC_ERR_INVALID_ARG;
  if (q.n < 1 || q.n > (1 << 20)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "batch size must be 1..1048576");
  if (!batch->target) return fail(ctx, FABRIC_ERR_INVALID_ARG, "targets are NULL");
  if (!(lr >= 0.0f)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "learning rate must be >= 0");
  if (ctx->n_train_mat < 1) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no training materials set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int M = ctx->n_train_mat;
  if (M > paper_train_max_materials(ctx->pn_width))
    return fail(ctx, FABRIC_ERR_UNSUPPORTED, "paper network training takes at most %d materials at width %d",
                paper_train_max_materials(ctx->pn_width), ctx->pn_width);
  const size_t need = ((paper_train_work_bytes(ctx->pn_width, q.n, M) + 255) & ~size_t(255)) + 256;
  void *work = scratch(ctx, need);
  if (!work) return fail(ctx, FABRIC_ERR_OOM, "training scratch (%zu bytes)", need);
  double *loss = loss_dev ? loss_dev
                          : reinterpret_cast<double *>(static_cast<uint8_t *>(work) + need - 256);
  PN_CUDA(ctx,
          launch_paper_train(ctx->pn_width, ctx->pn_ablation, q, batch->target, ctx->loss_mode, ctx->d_train_raw, M, ctx->d_pn_dec,
                             ctx->d_pn_enc, ctx->d_pn_grad, loss, work, ctx->d_status, s),
          "paper network forward/backward");
  ctx->pn_adam_step += 1;
  ctx->pn_version += 1;
  const size_t nd = n_dec(ctx), ne = (size_t)kPnEncParams;
  float *m = ctx->d_pn_adam, *v = ctx->d_pn_adam + nd + ne;
  PN_CUDA(ctx,
          launch_adam(ctx->d_pn_dec, (int64_t)nd, ctx->d_pn_enc, (int64_t)ne, ctx->d_pn_grad, m, v, lr,
                      ctx->pn_adam_step, s),
          "adam");
  return FABRIC_OK;
}

fabric_status fabric_paper_shade_fp32(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev,
                                      float *rgb_dev, float *comps_dev, void *stream) {
  PN_CHECK_CTX(ctx);
  if (!check_gbuffer(ctx, g)) return FABRIC_ERR_INVALID_ARG;
  if (!ctx->pn_width) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no paper network parameters set");
  if (g->n == 0) return FABRIC_OK;
  if (!latents_dev || !rgb_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "latents or rgb output is NULL");
  if (ctx->n_mat == 0) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no materials set");
  if (comps_dev && !is_aligned4(comps_dev))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "comps output must be float-aligned");
  const size_t need = paper_forward_work_bytes(ctx->pn_width, g->n);
  void *work = scratch(ctx, need);
  if (!work) return fail(ctx, FABRIC_ERR_OOM, "forward scratch (%zu bytes)", need);
  PN_CUDA(ctx,
          launch_paper_forward(ctx->pn_width, ctx->pn_ablation, *g, latents_dev, ctx->d_mat, ctx->n_mat,
                               ctx->d_pn_dec, rgb_dev, comps_dev, work, ctx->d_status,
                               static_cast<cudaStream_t>(stream)),
          "paper network FP32 forward");
  return FABRIC_OK;
}

fabric_status fabric_paper_get_gradient(fabric_ctx *ctx, float *grad) {
  PN_CHECK_CTX(ctx);
  if (!ctx->pn_width || !grad) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no paper network, or grad is NULL");
  PN_CUDA(ctx, cudaDeviceSynchronize(), "get gradient");
  const size_t n = n_dec(ctx) + kPnEncParams;
  PN_CUDA(ctx, cudaMemcpy(grad, ctx->d_pn_grad, n * sizeof(float), cudaMemcpyDeviceToHost), "gradient");
  return FABRIC_OK;
}

}  // extern "C"
