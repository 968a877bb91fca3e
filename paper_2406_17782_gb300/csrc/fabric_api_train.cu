// fabric_api_train.cu -- C ABI entry points of the encoder, the training step
// and the autograd building blocks (include/fabric.h).  Host code only.
#include <cmath>

#include "fabric_internal.h"

using namespace fab;

namespace {

#define FAB_CHECK_CTX(ctx)                                                \
  do {                                                                    \
    if (!(ctx)) return FABRIC_ERR_INVALID_ARG;                            \
    (ctx)->last_error.clear();                                            \
    if (cudaSetDevice((ctx)->device) != cudaSuccess)                      \
      return cuda_fail((ctx), cudaGetLastError(), "cudaSetDevice");       \
  } while (0)

#define FAB_CUDA(ctx, expr, what)                                         \
  do {                                                                    \
    cudaError_t e_ = (expr);                                              \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, (what));           \
  } while (0)

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Bump allocator over the context's scratch arena.
struct Carve {
  uint8_t *base;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    T *p = reinterpret_cast<T *>(base + off);
    off = align_up(off + count * sizeof(T));
    return p;
  }
};

bool check_materials(fabric_ctx *ctx, const fabric_material *m, int n) {
  for (int k = 0; k < n; ++k) {
    DevMaterial tmp;
    std::string why;
    if (!build_material(m[k], &tmp, &why)) {
      fail(ctx, FABRIC_ERR_INVALID_ARG, "material %d: %s", k, why.c_str());
      return false;
    }
  }
  return true;
}

}  // namespace

extern "C" {

fabric_status fabric_encode_params(fabric_ctx *ctx, const fabric_material *m, int n_mat, float *latents_dev,
                                   void *stream) {
  FAB_CHECK_CTX(ctx);
  if (n_mat == 0) return FABRIC_OK;
  if (!m || !latents_dev || n_mat < 0 || n_mat > 65535)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "need materials, a latent buffer and 0..65535 records");
  if (!check_materials(ctx, m, n_mat)) return FABRIC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (ctx->enc_raw_cap < n_mat) {
    FAB_CUDA(ctx, cudaStreamSynchronize(s), "encode staging");
    cudaFree(ctx->d_enc_raw);
    ctx->d_enc_raw = nullptr;
    ctx->enc_raw_cap = 0;
    FAB_CUDA(ctx, cudaMalloc(&ctx->d_enc_raw, n_mat * sizeof(fabric_material)), "encode staging");
    ctx->enc_raw_cap = n_mat;
  }
  FAB_CUDA(ctx, cudaMemcpyAsync(ctx->d_enc_raw, m, n_mat * sizeof(fabric_material), cudaMemcpyHostToDevice, s),
           "encode upload");
  FAB_CUDA(ctx, launch_encoder_raw(ctx->d_enc_raw, n_mat, ctx->d_enc, nullptr, latents_dev, nullptr, s), "encoder");
  return FABRIC_OK;
}

fabric_status fabric_train_step(fabric_ctx *ctx, const fabric_train_batch *batch, float lr, double *loss_dev,
                                void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!batch) return fail(ctx, FABRIC_ERR_INVALID_ARG, "batch is NULL");
  const fabric_gbuffer &q = batch->queries;
  if (!check_gbuffer(ctx, &q)) return FABRIC_ERR_INVALID_ARG;
  if (q.n < 1 || q.n > (1 << 20)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "batch size must be 1..1048576");
  if (!batch->target) return fail(ctx, FABRIC_ERR_INVALID_ARG, "targets are NULL");
  if (!(lr >= 0.0f)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "learning rate must be >= 0");
  if (ctx->n_train_mat < 1) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no training materials set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int M = ctx->n_train_mat;
  // the backward's work area: [grid][width] gradient partials, [grid] loss
  // partials and [n][32] latent-gradient rows
  const bool tc = ctx->train_prec == FABRIC_PREC_BF16;
  const int tc_grid = train_tc_grid(q.n, ctx->sm_count), tc_width = train_tc_partial_width(M);
  const size_t tc_work = align_up((size_t)tc_grid * tc_width * 4) + align_up((size_t)tc_grid * 8) +
                         align_up((size_t)q.n * kLatent * 4);
  const size_t dwork_bytes = tc ? tc_work : decoder_backward_work_bytes(q.n, ctx->sm_count);
  const size_t need = align_up((size_t)M * kEncIn * 4) + align_up((size_t)M * kLatent * 4) +
                      align_up((size_t)M * 2 * kEncHidden * 4) +
                      align_up(((size_t)kDecParams + kEncParams) * 4) + align_up((size_t)M * kLatent * 4) +
                      align_up(encoder_backward_work_floats(M) * 4) +
                      align_up(dwork_bytes) + align_up(8) +
                      align_up(train_tc_blob_bytes());
  void *base = scratch(ctx, need);
  if (!base) return fail(ctx, FABRIC_ERR_OOM, "training scratch (%zu bytes)", need);
  Carve c{static_cast<uint8_t *>(base)};
  float *feats = c.take<float>((size_t)M * kEncIn);
  float *z = c.take<float>((size_t)M * kLatent);
  float *acts = c.take<float>((size_t)M * 2 * kEncHidden);
  float *grad = c.take<float>((size_t)kDecParams + kEncParams);
  float *dz = c.take<float>((size_t)M * kLatent);
  float *ework = c.take<float>(encoder_backward_work_floats(M));
  uint8_t *dwork = c.take<uint8_t>(dwork_bytes);
  double *loss_tmp = c.take<double>(1);
  void *tc_blob = c.take<uint8_t>(train_tc_blob_bytes());
  double *loss = loss_dev ? loss_dev : loss_tmp;
  FAB_CUDA(ctx, launch_encoder_raw(ctx->d_train_raw, M, ctx->d_enc, feats, z, acts, s), "encoder forward");
  const float *dec_partial = nullptr;   // tensor-core path: the decoder's per-CTA gradient partials
  if (tc) {
    Carve w{dwork};
    float *partial = w.take<float>((size_t)tc_grid * tc_width);
    double *loss_part = w.take<double>((size_t)tc_grid);
    float *rows = w.take<float>((size_t)q.n * kLatent);
    FAB_CUDA(ctx,
             launch_train_tc(q, z, M, ctx->d_dec, batch->target, ctx->loss_mode, tc_blob, partial, loss_part, rows,
                             ctx->sm_count, ctx->d_status, s),
             "tensor-core decoder forward/backward");
    // the decoder's gradient sums and Adam update run beside the encoder's
    // gradients (DecAdamArgs below)
    FAB_CUDA(ctx, launch_decoder_grad_finish(q, M, partial, tc_grid, tc_width, loss_part, rows, nullptr, loss, dz, s),
             "latent-gradient and loss sums");
    dec_partial = partial;
  } else {
    FAB_CUDA(ctx,
             launch_decoder_backward(q, z, M, ctx->d_dec, nullptr, batch->target, ctx->loss_mode, grad, dz, loss,
                                     dwork, ctx->sm_count, ctx->d_status, s),
             "decoder forward/backward");
  }
  ctx->adam_step += 1;
  ctx->version += 1;
  const size_t np = (size_t)kDecParams + kEncParams;
  float *m = ctx->d_adam, *v = ctx->d_adam + np;
  DecAdamArgs da{};
  if (dec_partial) {
    da.partial = dec_partial;
    da.n_part = tc_grid;
    da.stride = tc_width;
    da.n = kDecParams;
    da.p = ctx->d_dec;
    da.m = m;
    da.v = v;
    da.lr = lr;
    adam_bias(ctx->adam_step, &da.bc1, &da.bc2);
  }
  FAB_CUDA(ctx,
           launch_encoder_backward(feats, M, ctx->d_enc, acts, dz, grad + kDecParams, ework, s,
                                   dec_partial ? &da : nullptr),
           "encoder backward");
  if (dec_partial)
    FAB_CUDA(ctx,
             launch_adam(ctx->d_enc, kEncParams, nullptr, 0, grad + kDecParams, m + kDecParams, v + kDecParams, lr,
                         ctx->adam_step, s),
             "adam");
  else
    FAB_CUDA(ctx, launch_adam(ctx->d_dec, kDecParams, ctx->d_enc, kEncParams, grad, m, v, lr, ctx->adam_step, s),
             "adam");
  return FABRIC_OK;
}

fabric_status fabric_train_steps(fabric_ctx *ctx, const fabric_train_batch *data, int64_t batch, int n_steps,
                                 int64_t first_step, int64_t total_steps, double lr0, double lr1, double *loss_dev,
                                 void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!data) return fail(ctx, FABRIC_ERR_INVALID_ARG, "dataset is NULL");
  const fabric_gbuffer &g = data->queries;
  if (batch < 1 || batch > g.n || batch > (1 << 20))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "batch must be 1..min(n, 1048576)");
  if (n_steps < 0 || total_steps < 1 || first_step < 0)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "n_steps >= 0, total_steps >= 1 and first_step >= 0 required");
  const int64_t per_epoch = g.n / batch;
  for (int k = 0; k < n_steps; ++k) {
    const int64_t off = (k % per_epoch) * batch;
    fabric_train_batch b;
    b.queries = g;
    b.queries.u = g.u ? g.u + off : nullptr;
    b.queries.v = g.v ? g.v + off : nullptr;
    b.queries.radius = g.radius ? g.radius + off : nullptr;
    b.queries.wi = g.wi ? g.wi + 3 * off : nullptr;
    b.queries.wo = g.wo ? g.wo + 3 * off : nullptr;
    b.queries.material = g.material ? g.material + off : nullptr;
    b.queries.n = batch;
    b.target = data->target ? data->target + 4 * off : nullptr;
    const double t = (double)(first_step + k);
    const float lr = (float)(lr1 + 0.5 * (lr0 - lr1) * (1.0 + std::cos(3.141592653589793 * t / (double)total_steps)));
    const fabric_status st = fabric_train_step(ctx, &b, lr, loss_dev ? loss_dev + k : nullptr, stream);
    if (st != FABRIC_OK) return st;
  }
  return FABRIC_OK;
}

fabric_status fabric_shuffle_dataset(fabric_ctx *ctx, const fabric_train_batch *src, const fabric_dataset_out *dst,
                                     uint64_t seed, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!src || !dst) return fail(ctx, FABRIC_ERR_INVALID_ARG, "dataset is NULL");
  const fabric_gbuffer &g = src->queries;
  if (!check_gbuffer(ctx, &g)) return FABRIC_ERR_INVALID_ARG;
  if (g.n < 1 || g.n > (1ll << 31)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "dataset size must be 1..2^31");
  if (!dst->u || !dst->v || !dst->radius || !dst->wi || !dst->wo || !dst->material)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "output array is NULL");
  if (!src->target != !dst->target)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "targets must be given on both sides or on neither");
  const void *f[] = {dst->u, dst->v, dst->radius, dst->wi, dst->wo, dst->target, src->target};
  for (const void *p : f)
    if (reinterpret_cast<uintptr_t>(p) & 3u) return fail(ctx, FABRIC_ERR_INVALID_ARG, "arrays must be float-aligned");
  if (reinterpret_cast<uintptr_t>(dst->material) & 1u)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "material array must be 2-byte aligned");
  FAB_CUDA(ctx, launch_shuffle_dataset(*src, *dst, seed, ctx->sm_count, static_cast<cudaStream_t>(stream)),
           "dataset shuffle");
  return FABRIC_OK;
}

fabric_status fabric_decoder_forward(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev, int n_lat,
                                     const float *dec_dev, float *y_dev, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!check_gbuffer(ctx, g)) return FABRIC_ERR_INVALID_ARG;
  if (g->n == 0) return FABRIC_OK;
  if (!latents_dev || !dec_dev || !y_dev || n_lat < 1)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "NULL pointer or n_lat < 1");
  if (!is_aligned4(y_dev)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "y must be float-aligned");
  FAB_CUDA(ctx, launch_decoder_raw(*g, latents_dev, n_lat, dec_dev, y_dev, ctx->d_status,
                                   static_cast<cudaStream_t>(stream)),
           "decoder forward");
  return FABRIC_OK;
}

fabric_status fabric_decoder_backward(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev,
                                      int n_lat, const float *dec_dev, const float *dy_dev, float *ddec_dev,
                                      float *dlatents_dev, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!check_gbuffer(ctx, g)) return FABRIC_ERR_INVALID_ARG;
  if (!latents_dev || !dec_dev || !dy_dev || !ddec_dev || n_lat < 1)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "NULL pointer or n_lat < 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (g->n == 0) {
    FAB_CUDA(ctx, cudaMemsetAsync(ddec_dev, 0, kDecParams * sizeof(float), s), "zero");
    if (dlatents_dev) FAB_CUDA(ctx, cudaMemsetAsync(dlatents_dev, 0, (size_t)n_lat * kLatent * 4, s), "zero");
    return FABRIC_OK;
  }
  void *work = scratch(ctx, decoder_backward_work_bytes(g->n, ctx->sm_count));
  if (!work) return fail(ctx, FABRIC_ERR_OOM, "scratch");
  FAB_CUDA(ctx,
           launch_decoder_backward(*g, latents_dev, n_lat, dec_dev, dy_dev, nullptr, 0, ddec_dev, dlatents_dev, nullptr,
                                   work, ctx->sm_count, ctx->d_status, s),
           "decoder backward");
  return FABRIC_OK;
}

fabric_status fabric_encoder_forward(fabric_ctx *ctx, const float *feats_dev, int n, const float *enc_dev,
                                     float *z_dev, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (n == 0) return FABRIC_OK;
  if (!feats_dev || !enc_dev || !z_dev || n < 0) return fail(ctx, FABRIC_ERR_INVALID_ARG, "bad arguments");
  FAB_CUDA(ctx, launch_encoder_feats(feats_dev, n, enc_dev, z_dev, nullptr, static_cast<cudaStream_t>(stream)),
           "encoder forward");
  return FABRIC_OK;
}

fabric_status fabric_encoder_backward(fabric_ctx *ctx, const float *feats_dev, int n, const float *enc_dev,
                                      const float *dz_dev, float *denc_dev, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!feats_dev || !enc_dev || !dz_dev || !denc_dev || n < 1)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "bad arguments");
  float *work = static_cast<float *>(scratch(ctx, encoder_backward_work_floats(n) * 4));
  if (!work) return fail(ctx, FABRIC_ERR_OOM, "scratch");
  FAB_CUDA(ctx,
           launch_encoder_backward(feats_dev, n, enc_dev, nullptr, dz_dev, denc_dev, work,
                                   static_cast<cudaStream_t>(stream)),
           "encoder backward");
  return FABRIC_OK;
}

}  // extern "C"
