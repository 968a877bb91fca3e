// host_pipeline.cu -- fabric_shade_neural_host: neural shading of a G-buffer
// that lives in host memory.  When all buffers are mapped page-locked host
// memory the decoder reads and writes them directly over the host link (one
// launch on the caller's stream).  Otherwise, or when a chunk size is given,
// the frame is cut into chunks that cycle through three context-owned device
// staging slots, each with its own stream, so that the host-to-device copy of
// one chunk, the decoder on the next and the device-to-host copy of a third
// overlap; the caller's stream orders the whole call (the slots start after
// the work already queued on it, and it waits for all of them).
#include "fabric_internal.h"

namespace {

using namespace fab;

constexpr int64_t kDefaultChunk = 262144;   // points per chunk (2048 tiles)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Staging layout of one slot for `chunk` points.
struct SlotLayout {
  size_t u, v, r, wi, wo, mat, rgb, comps, total;
};
SlotLayout slot_layout(int64_t chunk) {
  SlotLayout L;
  const size_t n = (size_t)chunk;
  L.u = 0;
  L.v = L.u + align256(n * 4);
  L.r = L.v + align256(n * 4);
  L.wi = L.r + align256(n * 4);
  L.wo = L.wi + align256(n * 12);
  L.mat = L.wo + align256(n * 12);
  L.rgb = L.mat + align256(n * 2);
  L.comps = L.rgb + align256(n * 12);
  L.total = L.comps + align256(n * 16);
  return L;
}

fabric_status ensure_slots(fabric_ctx *ctx, int64_t chunk) {
  if (!ctx->host_start) {
    for (int k = 0; k < fabric_ctx::kHostSlots; ++k) {
      if (cudaStreamCreateWithFlags(&ctx->host_stream[k], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->host_done[k], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "host pipeline streams");
    }
    if (cudaEventCreateWithFlags(&ctx->host_start, cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(ctx, cudaGetLastError(), "host pipeline event");
  }
  const size_t need = slot_layout(chunk).total;
  if (ctx->host_slot_bytes < need) {
    // earlier calls may still use the old staging: let them finish first
    for (int k = 0; k < fabric_ctx::kHostSlots; ++k) cudaStreamSynchronize(ctx->host_stream[k]);
    cudaFree(ctx->host_stage);
    ctx->host_stage = nullptr;
    ctx->host_slot_bytes = 0;
    if (cudaMalloc(&ctx->host_stage, need * fabric_ctx::kHostSlots) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, FABRIC_ERR_OOM, "host pipeline staging (%zu bytes)", need * fabric_ctx::kHostSlots);
    }
    ctx->host_slot_bytes = need;
  }
  return FABRIC_OK;
}

// Device address of host memory that the GPU may read and write directly
// (page-locked memory mapped into the unified address space), else null.
void *mapped(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace

void fab::host_pipeline_release(fabric_ctx *ctx) {
  for (int k = 0; k < fabric_ctx::kHostSlots; ++k) {
    if (ctx->host_stream[k]) cudaStreamDestroy(ctx->host_stream[k]);
    if (ctx->host_done[k]) cudaEventDestroy(ctx->host_done[k]);
  }
  if (ctx->host_start) cudaEventDestroy(ctx->host_start);
  cudaFree(ctx->host_stage);
}

extern "C" fabric_status fabric_shade_neural_host(fabric_ctx *ctx, const fabric_gbuffer *g_host,
                                                  fabric_precision prec, float *rgb_host, float *comps_host,
                                                  int64_t chunk_points, void *stream) {
  if (!ctx) return FABRIC_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  if (!g_host) return fail(ctx, FABRIC_ERR_INVALID_ARG, "G-buffer is NULL");
  if (g_host->n < 0) return fail(ctx, FABRIC_ERR_INVALID_ARG, "G-buffer n = %lld < 0", (long long)g_host->n);
  if (ctx->prepared_prec != (int)prec || ctx->prepared_version != ctx->version)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "no prepared state for this precision, materials and parameters");
  if (g_host->n == 0) return FABRIC_OK;
  if (!g_host->u || !g_host->v || !g_host->radius || !g_host->wi || !g_host->wo || !g_host->material || !rgb_host)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "a G-buffer field or the rgb output is NULL");
  if (chunk_points < 0) return fail(ctx, FABRIC_ERR_INVALID_ARG, "chunk_points < 0");
  if (comps_host && !is_aligned4(comps_host))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "comps output must be float-aligned");
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (chunk_points == 0) {
    // Direct: when every buffer is mapped page-locked memory the decoder
    // reads the G-buffer and writes its outputs over the host link itself,
    // in one launch and without staging copies.
    fabric_gbuffer d;
    d.u = static_cast<const float *>(mapped(g_host->u));
    d.v = static_cast<const float *>(mapped(g_host->v));
    d.radius = static_cast<const float *>(mapped(g_host->radius));
    d.wi = static_cast<const float *>(mapped(g_host->wi));
    d.wo = static_cast<const float *>(mapped(g_host->wo));
    d.material = static_cast<const uint16_t *>(mapped(g_host->material));
    d.n = g_host->n;
    float *rgb = static_cast<float *>(mapped(rgb_host));
    float *comps = comps_host ? static_cast<float *>(mapped(comps_host)) : nullptr;
    if (d.u && d.v && d.radius && d.wi && d.wo && d.material && rgb && (comps || !comps_host)) {
      if (prec == FABRIC_PREC_FP32)
        e = launch_decoder_fp32(d, ctx->d_mat, ctx->n_mat, ctx->prepared_latents, ctx->d_dec, rgb, comps, nullptr,
                                ctx->d_status, caller);
      else
        e = launch_decoder_tc(d, ctx->d_blob, ctx->n_mat, (int)prec, rgb, comps, ctx->d_status, ctx->sm_count,
                              ctx->tc_ctas_per_sm, ctx->tc_warpgroups, ctx->tc_tile_wgs, caller);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "decoder launch");
      return FABRIC_OK;
    }
  }
  int64_t chunk = chunk_points ? chunk_points : kDefaultChunk;
  chunk = (chunk + 127) / 128 * 128;
  if (chunk > g_host->n) chunk = (g_host->n + 127) / 128 * 128;
  fabric_status st = ensure_slots(ctx, chunk);
  if (st != FABRIC_OK) return st;
  const SlotLayout L = slot_layout(chunk);
  e = cudaEventRecord(ctx->host_start, caller);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host pipeline start");
  for (int k = 0; k < fabric_ctx::kHostSlots; ++k) {
    e = cudaStreamWaitEvent(ctx->host_stream[k], ctx->host_start, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "host pipeline start");
  }
  const int64_t n_chunks = (g_host->n + chunk - 1) / chunk;
  for (int64_t c = 0; c < n_chunks; ++c) {
    const int slot = (int)(c % fabric_ctx::kHostSlots);
    cudaStream_t s = ctx->host_stream[slot];
    uint8_t *base = static_cast<uint8_t *>(ctx->host_stage) + (size_t)slot * ctx->host_slot_bytes;
    const int64_t p0 = c * chunk;
    const int64_t n = (g_host->n - p0) < chunk ? (g_host->n - p0) : chunk;
    fabric_gbuffer d;
    d.u = reinterpret_cast<float *>(base + L.u);
    d.v = reinterpret_cast<float *>(base + L.v);
    d.radius = reinterpret_cast<float *>(base + L.r);
    d.wi = reinterpret_cast<float *>(base + L.wi);
    d.wo = reinterpret_cast<float *>(base + L.wo);
    d.material = reinterpret_cast<uint16_t *>(base + L.mat);
    d.n = n;
    float *rgb = reinterpret_cast<float *>(base + L.rgb);
    float *comps = comps_host ? reinterpret_cast<float *>(base + L.comps) : nullptr;
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice, d2h = cudaMemcpyDeviceToHost;
    if ((e = cudaMemcpyAsync((void *)d.u, g_host->u + p0, n * 4, h2d, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void *)d.v, g_host->v + p0, n * 4, h2d, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void *)d.radius, g_host->radius + p0, n * 4, h2d, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void *)d.wi, g_host->wi + 3 * p0, n * 12, h2d, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void *)d.wo, g_host->wo + 3 * p0, n * 12, h2d, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void *)d.material, g_host->material + p0, n * 2, h2d, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "host-to-device copy");
    if (prec == FABRIC_PREC_FP32)
      e = launch_decoder_fp32(d, ctx->d_mat, ctx->n_mat, ctx->prepared_latents, ctx->d_dec, rgb, comps, nullptr,
                              ctx->d_status, s);
    else
      e = launch_decoder_tc(d, ctx->d_blob, ctx->n_mat, (int)prec, rgb, comps, ctx->d_status, ctx->sm_count,
                            ctx->tc_ctas_per_sm, ctx->tc_warpgroups, ctx->tc_tile_wgs, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "decoder launch");
    if ((e = cudaMemcpyAsync(rgb_host + 3 * p0, rgb, n * 12, d2h, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "device-to-host copy");
    if (comps_host && (e = cudaMemcpyAsync(comps_host + 4 * p0, comps, n * 16, d2h, s)) != cudaSuccess)
      return cuda_fail(ctx, e, "device-to-host copy");
  }
  for (int k = 0; k < fabric_ctx::kHostSlots; ++k) {
    if ((e = cudaEventRecord(ctx->host_done[k], ctx->host_stream[k])) != cudaSuccess ||
        (e = cudaStreamWaitEvent(caller, ctx->host_done[k], 0)) != cudaSuccess)
      return cuda_fail(ctx, e, "host pipeline join");
  }
  return FABRIC_OK;
}
