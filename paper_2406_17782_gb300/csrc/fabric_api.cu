// fabric_api.cu -- the C ABI of include/fabric.h: context lifecycle, argument
// checking, material tables, parameter storage, checkpoints and dispatch to
// the kernels.  Host code only.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <fstream>
#include <new>

#include "fabric_internal.h"

namespace fab {

fabric_status fail(fabric_ctx *ctx, fabric_status s, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return s;
}

fabric_status cuda_fail(fabric_ctx *ctx, cudaError_t e, const char *what) {
  const fabric_status s = (e == cudaErrorMemoryAllocation) ? FABRIC_ERR_OOM : FABRIC_ERR_CUDA;
  return fail(ctx, s, "%s: %s", what, cudaGetErrorString(e));
}

bool is_aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool is_aligned4(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

void *scratch(fabric_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return ctx->scratch;
  if (ctx->scratch) {
    cudaDeviceSynchronize();
    cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
  }
  const size_t want = (bytes + (1u << 20) - 1) & ~size_t((1u << 20) - 1);
  if (cudaMalloc(&ctx->scratch, want) != cudaSuccess) {
    cudaGetLastError();
    ctx->scratch = nullptr;
    return nullptr;
  }
  ctx->scratch_bytes = want;
  return ctx->scratch;
}

// ---------------------------------------------------------------------------
// Weaves, written out row by row from their textile definitions (row i runs
// along v and indexes the weft, column j runs along u and indexes the warp;
// '1' = warp over weft).
// ---------------------------------------------------------------------------
struct Weave {
  int rows, cols;
  const char *cells[kMaxPatternDim];
};

static const Weave kWeaves[kNumWeaves] = {
    {2, 2, {"10", "01"}},                                            // plain
    {3, 3, {"101", "110", "011"}},                                   // 2/1 twill
    {4, 4, {"1011", "1101", "1110", "0111"}},                        // 3/1 twill
    {5, 5, {"01111", "11101", "10111", "11110", "11011"}},           // 4/1 satin, warp-faced
    {5, 5, {"10000", "00100", "00001", "01000", "00010"}},           // 5-harness satin, weft-faced
    {4, 4, {"1100", "1100", "0011", "0011"}},                        // 2x2 basket
    {4, 8, {"10011100", "11001001", "01100011", "00110110"}},        // herringbone
    {4, 2, {"10", "10", "01", "01"}},                                // warp rib
    {5, 5, {"10111", "11011", "11101", "11110", "01111"}},           // 4/1 twill
    {8, 8, {"10111111", "11011111", "11101111", "11110111",          // 7/1 twill
            "11111011", "11111101", "11111110", "01111111"}},
    {8, 8, {"10000000", "00010000", "00000010", "01000000",          // 8-harness satin, weft-faced
            "00001000", "00000001", "00100000", "00000100"}},
    {10, 5, {"10000", "10000", "00100", "00100", "00001",            // 5-harness satin, picks doubled
             "00001", "01000", "01000", "00010", "00010"}},
};

// Offset and length of the float through cell `pos` of a cyclic line whose
// cells are `on[k]` (true where the yarn in question lies on top).
static void float_run(const bool *on, int n, int pos, int *len, int *off) {
  int count_on = 0;
  for (int k = 0; k < n; ++k) count_on += on[k];
  if (count_on == n) {
    *len = n;
    *off = pos;
    return;
  }
  int back = 0;
  while (on[((pos - back - 1) % n + n) % n]) ++back;
  int ahead = 0;
  while (on[(pos + ahead + 1) % n]) ++ahead;
  *len = back + ahead + 1;
  *off = back;
}

bool build_material(const fabric_material &m, DevMaterial *d, std::string *why) {
  char buf[256];
  if (m.pattern_id < 0 || m.pattern_id >= kNumWeaves) {
    snprintf(buf, sizeof(buf), "unknown pattern_id %d (built-in weaves are 0..%d)", m.pattern_id, kNumWeaves - 1);
    *why = buf;
    return false;
  }
  for (int y = 0; y < 2; ++y) {
    if (!(m.alpha[y] > 0.f && m.alpha[y] <= 1.f) || !(m.beta[y] >= 0.f && m.beta[y] <= 4.f)) {
      snprintf(buf, sizeof(buf), "alpha must be in (0,1] and beta in [0,4] (yarn %d: %g, %g)", y, m.alpha[y],
               m.beta[y]);
      *why = buf;
      return false;
    }
  }
  if (!(m.gap >= 0.f && m.gap < 1.f) || !(m.w_blend >= 0.f && m.w_blend <= 1.f) ||
      !(std::fabs(m.twist_deg) <= 89.f) || !(std::fabs(m.incl_deg) <= 89.f)) {
    *why = "gap in [0,1), w_blend in [0,1], |twist|, |incl| <= 89 required";
    return false;
  }
  std::memset(d, 0, sizeof(*d));
  const Weave &w = kWeaves[m.pattern_id];
  d->rows = w.rows;
  d->cols = w.cols;
  d->gap_fixed = (uint32_t)std::floor(0.5 * (double)m.gap * 4294967296.0);
  d->inv_one_minus_gap = (float)(1.0 / (1.0 - (double)m.gap));
  const double psi = (double)m.twist_deg * M_PI / 180.0;
  d->cos_psi = (float)std::cos(psi);
  d->sin_psi = (float)std::sin(psi);
  d->w_blend = m.w_blend;
  for (int y = 0; y < 2; ++y) {
    const double a = m.alpha[y];
    d->alpha[y] = m.alpha[y];
    d->inv_alpha2_minus1[y] = (float)(1.0 / (a * a) - 1.0);
    d->one_minus_alpha2[y] = (float)(1.0 - a * a);
    d->inv_pi_alpha[y] = (float)(1.0 / (M_PI * a));
    d->slope_scale[y] = (float)(-(double)m.beta[y] * M_PI / 2.0);
    for (int c = 0; c < 3; ++c) {
      d->kd[y][c] = m.kd[y][c];
      d->ks[y][c] = m.ks[y][c];
    }
  }
  const double incl = (double)m.incl_deg * M_PI / 180.0;
  double rise_max = 0.0;
  for (int i = 0; i < w.rows; ++i) {
    for (int j = 0; j < w.cols; ++j) {
      const bool warp = w.cells[i][j] == '1';
      if (warp) d->top[i] |= 1u << j;
      bool line[kMaxPatternDim];
      int len, off;
      if (warp) {
        for (int k = 0; k < w.rows; ++k) line[k] = w.cells[k][j] == '1';
        float_run(line, w.rows, i, &len, &off);
      } else {
        for (int k = 0; k < w.cols; ++k) line[k] = w.cells[i][k] == '0';
        float_run(line, w.cols, j, &len, &off);
      }
      // theta(t) = incl (1 - 2 (off + t) / len) = theta0 - theta1 t
      d->theta[i * kMaxPatternDim + j] =
          make_float2((float)(incl * (1.0 - 2.0 * off / len)), (float)(2.0 * incl / len));
      // the float's rise, the integral of tan(theta) along it:
      // (ln cos theta(t) - ln cos incl) / (theta1 N_along)
      const int n_along = warp ? w.rows : w.cols;
      d->rise[i * kMaxPatternDim + j] = incl != 0.0 ? (float)(len / (2.0 * incl * n_along)) : 0.0f;
      if (incl > 0.0) rise_max = std::max(rise_max, len / (double)n_along * -std::log(std::cos(incl)) / (2.0 * incl));
    }
  }
  d->crest[0] = (float)((double)m.beta[0] * (1.0 - (double)m.gap) / (2.0 * w.cols));
  d->crest[1] = (float)((double)m.beta[1] * (1.0 - (double)m.gap) / (2.0 * w.rows));
  d->lncos_incl = (float)std::log(std::cos(incl));
  d->h_max = (float)(std::max((double)d->crest[0], (double)d->crest[1]) + rise_max);
  d->v_delta = (float)(1.0 / (16.0 * std::max(w.rows, w.cols)));
  return true;
}

bool check_gbuffer(fabric_ctx *ctx, const fabric_gbuffer *g) {
  if (!g) {
    fail(ctx, FABRIC_ERR_INVALID_ARG, "G-buffer is NULL");
    return false;
  }
  if (g->n < 0) {
    fail(ctx, FABRIC_ERR_INVALID_ARG, "G-buffer n = %lld < 0", (long long)g->n);
    return false;
  }
  if (g->n == 0) return true;
  if (!g->u || !g->v || !g->radius || !g->wi || !g->wo || !g->material) {
    fail(ctx, FABRIC_ERR_INVALID_ARG, "G-buffer has a NULL array");
    return false;
  }
  const void *f[] = {g->u, g->v, g->radius, g->wi, g->wo};
  for (const void *p : f)
    if (reinterpret_cast<uintptr_t>(p) & 3u) {
      fail(ctx, FABRIC_ERR_INVALID_ARG, "G-buffer float arrays must be 4-byte aligned");
      return false;
    }
  if (reinterpret_cast<uintptr_t>(g->material) & 1u) {
    fail(ctx, FABRIC_ERR_INVALID_ARG, "G-buffer material array must be 2-byte aligned");
    return false;
  }
  return true;
}

// CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320), bytewise.
struct Crc32Table {
  uint32_t v[256];
  Crc32Table() {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      v[i] = c;
    }
  }
};

static uint32_t crc32_update(uint32_t crc, const void *data, size_t n) {
  static const Crc32Table tab;   // initialised once, thread-safe
  const uint32_t *table = tab.v;
  const uint8_t *p = static_cast<const uint8_t *>(data);
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
  return ~crc;
}

}  // namespace fab

using namespace fab;

#define FAB_CHECK_CTX(ctx)                                  \
  do {                                                      \
    if (!(ctx)) return FABRIC_ERR_INVALID_ARG;              \
    (ctx)->last_error.clear();                              \
    if (cudaSetDevice((ctx)->device) != cudaSuccess)        \
      return cuda_fail((ctx), cudaGetLastError(), "cudaSetDevice"); \
  } while (0)

#define FAB_CUDA(ctx, expr, what)                           \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, (what)); \
  } while (0)

extern "C" {

const char *fabric_status_string(fabric_status s) {
  switch (s) {
    case FABRIC_OK: return "FABRIC_OK";
    case FABRIC_ERR_INVALID_ARG: return "FABRIC_ERR_INVALID_ARG";
    case FABRIC_ERR_CUDA: return "FABRIC_ERR_CUDA";
    case FABRIC_ERR_OOM: return "FABRIC_ERR_OOM";
    case FABRIC_ERR_TIMEOUT: return "FABRIC_ERR_TIMEOUT";
    case FABRIC_ERR_IO: return "FABRIC_ERR_IO";
    case FABRIC_ERR_UNSUPPORTED: return "FABRIC_ERR_UNSUPPORTED";
    case FABRIC_ERR_DEVICE: return "FABRIC_ERR_DEVICE";
  }
  return "unknown status";
}

fabric_status fabric_create(fabric_ctx **out, int device) {
  if (!out) return FABRIC_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return FABRIC_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return FABRIC_ERR_CUDA;
  fabric_ctx *ctx = new (std::nothrow) fabric_ctx();
  if (!ctx) return FABRIC_ERR_OOM;
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  const size_t np = (size_t)kDecParams + kEncParams;
  if (cudaMalloc(&ctx->d_dec, kDecParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&ctx->d_enc, kEncParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&ctx->d_adam, 2 * np * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_blob, tc_blob_bytes(89)) != cudaSuccess ||
      cudaMalloc(&ctx->d_err_work, error_stats_work_bytes(0)) != cudaSuccess) {
    fabric_destroy(ctx);
    return FABRIC_ERR_OOM;
  }
  cudaMemset(ctx->d_dec, 0, kDecParams * sizeof(float));
  cudaMemset(ctx->d_enc, 0, kEncParams * sizeof(float));
  cudaMemset(ctx->d_adam, 0, 2 * np * sizeof(float));
  cudaMemset(ctx->d_status, 0, sizeof(int));
  if (cudaDeviceSynchronize() != cudaSuccess) {
    fabric_destroy(ctx);
    return FABRIC_ERR_CUDA;
  }
  *out = ctx;
  return FABRIC_OK;
}

void fabric_destroy(fabric_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->d_mat);
  cudaFree(ctx->d_train_raw);
  cudaFree(ctx->d_dec);
  cudaFree(ctx->d_enc);
  cudaFree(ctx->d_adam);
  cudaFree(ctx->d_status);
  cudaFree(ctx->scratch);
  cudaFree(ctx->d_enc_raw);
  cudaFree(ctx->d_blob);
  cudaFree(ctx->d_err_work);
  host_pipeline_release(ctx);
  paper_release(ctx);
  delete ctx;
}

const char *fabric_last_error(const fabric_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int fabric_sm_count(const fabric_ctx *ctx) { return ctx ? ctx->sm_count : 0; }

fabric_status fabric_set_launch_config(fabric_ctx *ctx, int decoder_ctas_per_sm, int decoder_warpgroups,
                                       int reference_lanes) {
  if (!ctx) return FABRIC_ERR_INVALID_ARG;
  ctx->last_error.clear();
  const bool lanes_ok = reference_lanes == 0 || reference_lanes == 1 || reference_lanes == 2 ||
                        reference_lanes == 4 || reference_lanes == 8 || reference_lanes == 16 ||
                        reference_lanes == 32;
  if (decoder_ctas_per_sm < 0 || decoder_ctas_per_sm > 8 || decoder_warpgroups < 0 || decoder_warpgroups > 4 ||
      !lanes_ok)
    return fail(ctx, FABRIC_ERR_INVALID_ARG,
                "decoder CTAs per SM in 0..8, warpgroups in 0..4, reference lanes in {0,1,2,4,8,16,32}");
  ctx->tc_ctas_per_sm = decoder_ctas_per_sm;
  ctx->tc_warpgroups = decoder_warpgroups;
  ctx->ref_lanes = reference_lanes;
  return FABRIC_OK;
}

fabric_status fabric_set_train_precision(fabric_ctx *ctx, fabric_precision prec) {
  if (!ctx) return FABRIC_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (prec != FABRIC_PREC_FP32 && prec != FABRIC_PREC_BF16)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "training runs in FP32 or BF16 (got %d)", (int)prec);
  ctx->train_prec = (int)prec;
  return FABRIC_OK;
}

fabric_status fabric_set_train_loss(fabric_ctx *ctx, fabric_loss loss) {
  if (!ctx) return FABRIC_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (loss != FABRIC_LOSS_EQ11 && loss != FABRIC_LOSS_RENDERED)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "unknown loss %d", (int)loss);
  ctx->loss_mode = (int)loss;
  return FABRIC_OK;
}

fabric_status fabric_set_visibility(fabric_ctx *ctx, int on) {
  if (!ctx) return FABRIC_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (on != 0 && on != 1) return fail(ctx, FABRIC_ERR_INVALID_ARG, "visibility is 0 or 1 (got %d)", on);
  ctx->visibility = on;
  return FABRIC_OK;
}

fabric_status fabric_set_decoder_tile_warpgroups(fabric_ctx *ctx, int warpgroups_per_tile) {
  if (!ctx) return FABRIC_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (warpgroups_per_tile < 0 || warpgroups_per_tile > 2)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "warpgroups per tile in 0..2");
  ctx->tc_tile_wgs = warpgroups_per_tile;
  return FABRIC_OK;
}

fabric_status fabric_sync_status(fabric_ctx *ctx, void *stream) {
  FAB_CHECK_CTX(ctx);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FAB_CUDA(ctx, cudaStreamSynchronize(s), "stream synchronize");
  int word = 0;
  FAB_CUDA(ctx, cudaMemcpy(&word, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  FAB_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)), "clear status");
  if (word & kStatusTimeout) return fail(ctx, FABRIC_ERR_TIMEOUT, "a kernel wait expired");
  if (word & kStatusBadMaterial)
    return fail(ctx, FABRIC_ERR_DEVICE, "a G-buffer material index was outside the material table");
  return FABRIC_OK;
}

static fabric_status upload_materials(fabric_ctx *ctx, const fabric_material *m, int n_mat) {
  std::vector<DevMaterial> host(n_mat);
  for (int k = 0; k < n_mat; ++k) {
    std::string why;
    if (!build_material(m[k], &host[k], &why))
      return fail(ctx, FABRIC_ERR_INVALID_ARG, "material %d: %s", k, why.c_str());
  }
  DevMaterial *d = nullptr;
  FAB_CUDA(ctx, cudaMalloc(&d, n_mat * sizeof(DevMaterial)), "material table");
  cudaError_t e = cudaMemcpy(d, host.data(), n_mat * sizeof(DevMaterial), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(ctx, e, "material upload");
  }
  cudaDeviceSynchronize();
  cudaFree(ctx->d_mat);
  ctx->d_mat = d;
  ctx->n_mat = n_mat;
  ctx->version += 1;
  ctx->h_mat.assign(m, m + n_mat);
  return FABRIC_OK;
}

fabric_status fabric_set_materials(fabric_ctx *ctx, const fabric_material *m, int n_mat) {
  FAB_CHECK_CTX(ctx);
  if (!m || n_mat < 1 || n_mat > 65535)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "need 1..65535 materials (got %d)", n_mat);
  return upload_materials(ctx, m, n_mat);
}

fabric_status fabric_set_train_materials(fabric_ctx *ctx, const fabric_material *m, int n_mat) {
  FAB_CHECK_CTX(ctx);
  if (!m || n_mat < 1 || n_mat > 65535)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "need 1..65535 training materials (got %d)", n_mat);
  for (int k = 0; k < n_mat; ++k) {
    DevMaterial tmp;
    std::string why;
    if (!build_material(m[k], &tmp, &why))
      return fail(ctx, FABRIC_ERR_INVALID_ARG, "training material %d: %s", k, why.c_str());
  }
  fabric_material *d = nullptr;
  FAB_CUDA(ctx, cudaMalloc(&d, n_mat * sizeof(fabric_material)), "training materials");
  cudaError_t e = cudaMemcpy(d, m, n_mat * sizeof(fabric_material), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(ctx, e, "training material upload");
  }
  cudaDeviceSynchronize();
  cudaFree(ctx->d_train_raw);
  ctx->d_train_raw = d;
  ctx->n_train_mat = n_mat;
  return FABRIC_OK;
}

int64_t fabric_decoder_param_count(void) { return kDecParams; }
int64_t fabric_encoder_param_count(void) { return kEncParams; }

fabric_status fabric_set_params(fabric_ctx *ctx, const float *decoder, const float *encoder) {
  FAB_CHECK_CTX(ctx);
  if (decoder)
    FAB_CUDA(ctx, cudaMemcpy(ctx->d_dec, decoder, kDecParams * sizeof(float), cudaMemcpyHostToDevice), "params");
  if (encoder)
    FAB_CUDA(ctx, cudaMemcpy(ctx->d_enc, encoder, kEncParams * sizeof(float), cudaMemcpyHostToDevice), "params");
  const size_t np = (size_t)kDecParams + kEncParams;
  FAB_CUDA(ctx, cudaMemset(ctx->d_adam, 0, 2 * np * sizeof(float)), "adam reset");
  ctx->adam_step = 0;
  ctx->version += 1;
  FAB_CUDA(ctx, cudaDeviceSynchronize(), "set params");
  return FABRIC_OK;
}

fabric_status fabric_get_params(fabric_ctx *ctx, float *decoder, float *encoder) {
  FAB_CHECK_CTX(ctx);
  FAB_CUDA(ctx, cudaDeviceSynchronize(), "get params");
  if (decoder)
    FAB_CUDA(ctx, cudaMemcpy(decoder, ctx->d_dec, kDecParams * sizeof(float), cudaMemcpyDeviceToHost), "params");
  if (encoder)
    FAB_CUDA(ctx, cudaMemcpy(encoder, ctx->d_enc, kEncParams * sizeof(float), cudaMemcpyDeviceToHost), "params");
  return FABRIC_OK;
}

fabric_status fabric_param_pointers(fabric_ctx *ctx, float **decoder_dev, float **encoder_dev) {
  FAB_CHECK_CTX(ctx);
  if (decoder_dev) *decoder_dev = ctx->d_dec;
  if (encoder_dev) *encoder_dev = ctx->d_enc;
  return FABRIC_OK;
}

static const char kCkptMagic[8] = {'F', 'A', 'B', 'C', 'K', 'P', 'T', '1'};

fabric_status fabric_checkpoint_save(fabric_ctx *ctx, const char *path) {
  FAB_CHECK_CTX(ctx);
  if (!path) return fail(ctx, FABRIC_ERR_INVALID_ARG, "path is NULL");
  const size_t np = (size_t)kDecParams + kEncParams;
  std::vector<float> dec(kDecParams), enc(kEncParams), adam(2 * np);
  FAB_CUDA(ctx, cudaDeviceSynchronize(), "checkpoint");
  FAB_CUDA(ctx, cudaMemcpy(dec.data(), ctx->d_dec, dec.size() * 4, cudaMemcpyDeviceToHost), "checkpoint");
  FAB_CUDA(ctx, cudaMemcpy(enc.data(), ctx->d_enc, enc.size() * 4, cudaMemcpyDeviceToHost), "checkpoint");
  FAB_CUDA(ctx, cudaMemcpy(adam.data(), ctx->d_adam, adam.size() * 4, cudaMemcpyDeviceToHost), "checkpoint");
  std::vector<uint8_t> buf;
  auto put = [&](const void *p, size_t n) {
    const uint8_t *b = static_cast<const uint8_t *>(p);
    buf.insert(buf.end(), b, b + n);
  };
  const uint32_t version = 1, nd = kDecParams, ne = kEncParams;
  put(kCkptMagic, 8);
  put(&version, 4);
  put(&nd, 4);
  put(&ne, 4);
  put(&ctx->adam_step, 8);
  put(dec.data(), dec.size() * 4);
  put(enc.data(), enc.size() * 4);
  put(adam.data(), adam.size() * 4);
  const uint32_t crc = crc32_update(0, buf.data(), buf.size());
  put(&crc, 4);
  std::ofstream f(path, std::ios::binary | std::ios::trunc);
  if (!f) return fail(ctx, FABRIC_ERR_IO, "cannot open %s for writing", path);
  f.write(reinterpret_cast<const char *>(buf.data()), (std::streamsize)buf.size());
  if (!f) return fail(ctx, FABRIC_ERR_IO, "write to %s failed", path);
  return FABRIC_OK;
}

fabric_status fabric_checkpoint_load(fabric_ctx *ctx, const char *path) {
  FAB_CHECK_CTX(ctx);
  if (!path) return fail(ctx, FABRIC_ERR_INVALID_ARG, "path is NULL");
  std::ifstream f(path, std::ios::binary);
  if (!f) return fail(ctx, FABRIC_ERR_IO, "cannot open %s", path);
  std::vector<uint8_t> buf((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
  const size_t np = (size_t)kDecParams + kEncParams;
  const size_t want = 8 + 4 + 4 + 4 + 8 + 4 * (np + 2 * np) + 4;
  if (buf.size() != want) return fail(ctx, FABRIC_ERR_IO, "%s: size %zu, expected %zu", path, buf.size(), want);
  if (std::memcmp(buf.data(), kCkptMagic, 8) != 0) return fail(ctx, FABRIC_ERR_IO, "%s: bad magic", path);
  uint32_t crc_file;
  std::memcpy(&crc_file, buf.data() + want - 4, 4);
  if (crc32_update(0, buf.data(), want - 4) != crc_file) return fail(ctx, FABRIC_ERR_IO, "%s: CRC mismatch", path);
  uint32_t version, nd, ne;
  std::memcpy(&version, buf.data() + 8, 4);
  std::memcpy(&nd, buf.data() + 12, 4);
  std::memcpy(&ne, buf.data() + 16, 4);
  if (version != 1 || nd != (uint32_t)kDecParams || ne != (uint32_t)kEncParams)
    return fail(ctx, FABRIC_ERR_IO, "%s: unsupported version or shapes", path);
  int64_t step;
  std::memcpy(&step, buf.data() + 20, 8);
  const uint8_t *p = buf.data() + 28;
  FAB_CUDA(ctx, cudaDeviceSynchronize(), "checkpoint");
  FAB_CUDA(ctx, cudaMemcpy(ctx->d_dec, p, 4 * (size_t)kDecParams, cudaMemcpyHostToDevice), "checkpoint");
  p += 4 * (size_t)kDecParams;
  FAB_CUDA(ctx, cudaMemcpy(ctx->d_enc, p, 4 * (size_t)kEncParams, cudaMemcpyHostToDevice), "checkpoint");
  p += 4 * (size_t)kEncParams;
  FAB_CUDA(ctx, cudaMemcpy(ctx->d_adam, p, 4 * 2 * np, cudaMemcpyHostToDevice), "checkpoint");
  ctx->adam_step = step;
  ctx->version += 1;
  FAB_CUDA(ctx, cudaDeviceSynchronize(), "checkpoint");
  return FABRIC_OK;
}

fabric_status fabric_shade_reference(fabric_ctx *ctx, const fabric_gbuffer *g, int spp_x, int spp_y,
                                     uint64_t seed, float *rgb_dev, float *comps_dev, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!check_gbuffer(ctx, g)) return FABRIC_ERR_INVALID_ARG;
  if (spp_x < 1 || spp_y < 1 || spp_x > 4096 || spp_y > 4096)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "spp_x, spp_y must be in 1..4096 (got %d, %d)", spp_x, spp_y);
  if (g->n == 0) return FABRIC_OK;
  if (!rgb_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "rgb output is NULL");
  if (comps_dev && !is_aligned4(comps_dev))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "comps output must be float-aligned");
  if (ctx->n_mat == 0) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no materials set");
  const int spp = spp_x * spp_y;
  // lanes per point: a whole warp for large sample counts, fewer otherwise
  const int lanes = ctx->ref_lanes > 0 ? ctx->ref_lanes
                    : spp >= 256 ? 32 : spp >= 64 ? 16 : spp >= 16 ? 8 : spp >= 4 ? 4 : 1;
  FAB_CUDA(ctx,
           launch_reference(*g, ctx->d_mat, ctx->n_mat, spp_x, spp_y, seed, rgb_dev, comps_dev, ctx->d_status,
                            lanes, ctx->sm_count, static_cast<cudaStream_t>(stream), ctx->visibility != 0),
           "reference kernel launch");
  return FABRIC_OK;
}

fabric_status fabric_prepare_neural(fabric_ctx *ctx, const float *latents_dev, fabric_precision prec,
                                    void *stream) {
  FAB_CHECK_CTX(ctx);
  if (prec != FABRIC_PREC_FP32 && prec != FABRIC_PREC_BF16 && prec != FABRIC_PREC_FP8 &&
      prec != FABRIC_PREC_FP16)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
  if (!latents_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "latents are NULL");
  if (ctx->n_mat == 0) return fail(ctx, FABRIC_ERR_INVALID_ARG, "no materials set");
  ctx->prepared_prec = -1;
  if (prec != FABRIC_PREC_FP32) {
    if (tc_k1(ctx->n_mat) < 0)
      return fail(ctx, FABRIC_ERR_UNSUPPORTED, "tensor-core decoder supports at most 89 materials (have %d)",
                  ctx->n_mat);
    FAB_CUDA(ctx,
             launch_tc_pack(ctx->d_dec, latents_dev, ctx->d_mat, ctx->n_mat, (int)prec, ctx->d_blob,
                            static_cast<cudaStream_t>(stream)),
             "pack");
  }
  ctx->prepared_prec = (int)prec;
  ctx->prepared_latents = latents_dev;
  ctx->prepared_version = ctx->version;
  return FABRIC_OK;
}

fabric_status fabric_shade_neural_prepared(fabric_ctx *ctx, const fabric_gbuffer *g, fabric_precision prec,
                                           float *rgb_dev, float *comps_dev, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!check_gbuffer(ctx, g)) return FABRIC_ERR_INVALID_ARG;
  if (ctx->prepared_prec != (int)prec || ctx->prepared_version != ctx->version)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "no prepared state for this precision, materials and parameters");
  if (g->n == 0) return FABRIC_OK;
  if (!rgb_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "rgb output is NULL");
  if (comps_dev && !is_aligned4(comps_dev))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "comps output must be float-aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (prec == FABRIC_PREC_FP32) {
    FAB_CUDA(ctx,
             launch_decoder_fp32(*g, ctx->d_mat, ctx->n_mat, ctx->prepared_latents, ctx->d_dec, rgb_dev, comps_dev,
                                 nullptr, ctx->d_status, s),
             "fp32 decoder launch");
    return FABRIC_OK;
  }
  FAB_CUDA(ctx,
           launch_decoder_tc(*g, ctx->d_blob, ctx->n_mat, (int)prec, rgb_dev, comps_dev, ctx->d_status, ctx->sm_count,
                             ctx->tc_ctas_per_sm, ctx->tc_warpgroups, ctx->tc_tile_wgs, s),
           "tensor-core decoder launch");
  return FABRIC_OK;
}

fabric_status fabric_shade_neural(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev,
                                  fabric_precision prec, float *rgb_dev, float *comps_dev, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!check_gbuffer(ctx, g)) return FABRIC_ERR_INVALID_ARG;
  if (prec != FABRIC_PREC_FP32 && prec != FABRIC_PREC_BF16 && prec != FABRIC_PREC_FP8 &&
      prec != FABRIC_PREC_FP16)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
  if (g->n == 0) return FABRIC_OK;
  if (!rgb_dev || !latents_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "rgb output or latents is NULL");
  if (comps_dev && !is_aligned4(comps_dev))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "comps output must be float-aligned");
  const fabric_status st = fabric_prepare_neural(ctx, latents_dev, prec, stream);
  if (st != FABRIC_OK) return st;
  return fabric_shade_neural_prepared(ctx, g, prec, rgb_dev, comps_dev, stream);
}

fabric_status fabric_selftest_mma(fabric_ctx *ctx, const float *a_dev, const float *b_dev, int n, int k,
                                  int a_in_tmem, float *d_dev, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!a_dev || !b_dev || !d_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "NULL pointer");
  if (!(k == 16 || k == 32 || k == 48 || k == 64) || !(n == 16 || n == 32 || n == 64))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "k must be 16/32/48/64 and n 16/32/64");
  FAB_CUDA(ctx,
           launch_selftest_mma(a_dev, b_dev, n, k, a_in_tmem ? 1 : 0, d_dev, ctx->d_status,
                               static_cast<cudaStream_t>(stream)),
           "selftest launch");
  return FABRIC_OK;
}

fabric_status fabric_selftest_mma_e4m3(fabric_ctx *ctx, const float *a_dev, const float *b_dev, int n, int k,
                                       float *d_dev, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!a_dev || !b_dev || !d_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "NULL pointer");
  if (!(k == 32 || k == 64) || !(n == 16 || n == 32 || n == 64))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "k must be 32/64 and n 16/32/64");
  FAB_CUDA(ctx, launch_selftest_mma(a_dev, b_dev, n, k, 2, d_dev, ctx->d_status, static_cast<cudaStream_t>(stream)),
           "selftest launch");
  return FABRIC_OK;
}

fabric_status fabric_selftest_wait_timeout(fabric_ctx *ctx, int sleep, void *stream) {
  FAB_CHECK_CTX(ctx);
  FAB_CUDA(ctx, launch_selftest_wait(sleep ? 1 : 0, ctx->d_status, static_cast<cudaStream_t>(stream)),
           "selftest launch");
  return FABRIC_OK;
}

fabric_status fabric_selftest_mma_mn(fabric_ctx *ctx, const float *a_dev, const float *b_dev, int n, int k,
                                     float *d_dev, void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!a_dev || !b_dev || !d_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "NULL pointer");
  if (!(k == 16 || k == 32 || k == 48 || k == 64) || !(n == 16 || n == 32 || n == 64))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "k must be 16/32/48/64 and n 16/32/64");
  FAB_CUDA(ctx, launch_selftest_mn(a_dev, b_dev, n, k, d_dev, ctx->d_status, static_cast<cudaStream_t>(stream)),
           "selftest launch");
  return FABRIC_OK;
}

fabric_status fabric_error_stats(fabric_ctx *ctx, const float *a_dev, const float *b_dev, int64_t n,
                                 const float *weights_dev, int group, int weight_stride, double *out_dev,
                                 void *stream) {
  FAB_CHECK_CTX(ctx);
  if (!a_dev || !b_dev || !out_dev || n < 0) return fail(ctx, FABRIC_ERR_INVALID_ARG, "bad arguments");
  if (weights_dev && (group < 1 || weight_stride < 1))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "group and weight_stride must be >= 1 with weights");
  FAB_CUDA(ctx,
           launch_error_stats(a_dev, b_dev, n, weights_dev, group < 1 ? 1 : group,
                              weight_stride < 1 ? 1 : weight_stride, out_dev, ctx->d_err_work,
                              static_cast<cudaStream_t>(stream)),
           "error stats launch");
  return FABRIC_OK;
}

}  // extern "C"
