// fabric_internal.h -- private declarations shared by the library's
// translation units (context, device material record, launch helpers).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "../../include/fabric.h"

namespace fab {

// Programmatic dependent launch: a kernel launched with launch_dependent()
// may be scheduled while the kernel before it in the stream is still
// finishing, which hides the gap between dependent launches.  Every such
// kernel calls grid_dependency_wait() before it reads anything an earlier
// kernel wrote (the wait returns once those kernels have completed and
// their memory is visible; without a pending dependency it returns at
// once), and grid_dependents_launch() once the next kernel may be
// scheduled.
#ifdef __CUDACC__
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Row p of a [n][4] float output: one 16-byte store when the array is
// 16-byte aligned, else four 4-byte stores (the caller's array need only be
// float-aligned; the test is the same for every thread, so it does not
// diverge).
__device__ __forceinline__ void store_row4(float *out, int64_t p, float x0, float x1, float x2, float x3) {
  if ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
    reinterpret_cast<float4 *>(out)[p] = make_float4(x0, x1, x2, x3);
  } else {
    float *q = out + 4 * p;
    q[0] = x0;
    q[1] = x1;
    q[2] = x2;
    q[3] = x3;
  }
}
#endif

// Raise a kernel's dynamic shared-memory limit once per (kernel, device):
// the setting belongs to the device's context, so a process that drives
// several GPUs sets it on each.  Thread-safe.
inline cudaError_t ensure_max_dyn_smem(const void *kernel, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({kernel, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert({kernel, dev});
  return e;
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                   Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

constexpr int kLatent = 32;
constexpr int kHidden = 64;
constexpr int kQueryFeat = 39;          // enc(u) 16 | enc(v) 16 | l | wi 3 | wo 3
constexpr int kDecIn = kLatent + kQueryFeat;
constexpr int kOut = 4;
constexpr int kPatternSlots = 16;   // one-hot width of the weave id in the encoder input
constexpr int kNumWeaves = 12;      // built-in weave tables
constexpr int kEncIn = kPatternSlots + 6;
constexpr int kEncHidden = 128;
constexpr int kMaxPatternDim = 16;

// flat decoder parameter offsets (weights [out][in])
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHidden * kDecIn;
constexpr int kOffW2 = kOffB1 + kHidden;
constexpr int kOffB2 = kOffW2 + kHidden * kHidden;
constexpr int kOffW3 = kOffB2 + kHidden;
constexpr int kOffB3 = kOffW3 + kHidden * kHidden;
constexpr int kOffW4 = kOffB3 + kHidden;
constexpr int kOffB4 = kOffW4 + kOut * kHidden;
constexpr int kDecParams = kOffB4 + kOut;

constexpr int kOffE1 = 0;
constexpr int kOffEb1 = kOffE1 + kEncHidden * kEncIn;
constexpr int kOffE2 = kOffEb1 + kEncHidden;
constexpr int kOffEb2 = kOffE2 + kEncHidden * kEncHidden;
constexpr int kOffE3 = kOffEb2 + kEncHidden;
constexpr int kOffEb3 = kOffE3 + kLatent * kEncHidden;
constexpr int kEncParams = kOffEb3 + kLatent;

// log-footprint feature l = (ln max(r, 2^-20) - c0) / c1 maps [1e-4, 1e-1] to [-1, 1]
constexpr float kLogRC0 = -5.756462732485114f;   // (ln 1e-4 + ln 1e-1) / 2
constexpr float kLogRInvC1 = 0.28952965460216784f; // 2 / (ln 1e-1 - ln 1e-4)
constexpr float kRFloor = 9.5367431640625e-07f;    // 2^-20
constexpr float kSpecK = 100.0f;                    // g(x) = ln(100 x + 1)

// Device status word values (OR-ed).
constexpr int kStatusBadMaterial = 1;
constexpr int kStatusTimeout = 2;

// Per-material record on the device: weave bits, per-cell inclination
// (theta = theta0 - theta1 * t along the float) and shading constants.
struct alignas(16) DevMaterial {
  uint32_t rows, cols, gap_fixed, pad0;
  uint32_t top[kMaxPatternDim];        // bit j of top[i]: warp over weft at (i, j)
  float inv_one_minus_gap;             // 1 / (1 - g)
  float cos_psi, sin_psi, w_blend;
  float alpha[2];
  float inv_alpha2_minus1[2];          // 1/alpha^2 - 1
  float one_minus_alpha2[2];           // 1 - alpha^2
  float inv_pi_alpha[2];               // 1 / (pi alpha)
  float slope_scale[2];                // -beta pi / 2
  float kd[2][3];
  float ks[2][3];
  float2 theta[kMaxPatternDim * kMaxPatternDim];
  // the proposed inter-yarn visibility model (height field and ray march)
  float crest[2];                      // beta w: cross-section height of each yarn, w its half-width
  float lncos_incl;                    // ln cos(inclination)
  float h_max;                         // largest surface height (repeat units)
  float v_delta;                       // horizontal march step: 1 / (16 max(rows, cols)) repeats
  float pad1[3];
  float rise[kMaxPatternDim * kMaxPatternDim];   // per cell 1 / (theta1 N_along), 0 without inclination
};

// One segment of a batched draw, as the kernel reads it.
struct SegDesc {
  const float *u, *v, *radius, *wi, *wo;
  const uint16_t *material;
  float *rgb, *comps;
  int64_t n;
};

}  // namespace fab

struct fabric_plan {
  int device = 0;
  int n_segs = 0;
  int64_t n_tiles = 0;
  int64_t n_points = 0;
  fab::SegDesc *d_segs = nullptr;
  int64_t *d_tile0 = nullptr;   // [n_segs + 1] first tile of each segment
};

struct fabric_ctx {
  int device = 0;
  int sm_count = 0;
  std::string last_error;
  // materials for shading
  int n_mat = 0;
  fab::DevMaterial *d_mat = nullptr;
  std::vector<fabric_material> h_mat;
  // materials for training
  int n_train_mat = 0;
  fabric_material *d_train_raw = nullptr;
  // parameters (FP32 master) and Adam state
  float *d_dec = nullptr;
  float *d_enc = nullptr;
  float *d_adam = nullptr;          // [m | v] over [dec | enc]
  int64_t adam_step = 0;
  // device status word
  int *d_status = nullptr;
  // growable scratch arena
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  // staging for host material records (encoder)
  fabric_material *d_enc_raw = nullptr;
  int enc_raw_cap = 0;
  // packed tensor-core weights (fixed size, largest material table) and
  // partial sums of the error reduction
  void *d_blob = nullptr;
  double *d_err_work = nullptr;
  // state of the last fabric_prepare_neural: precision (-1 = none), latents
  // and the material / parameter versions it was built from
  int prepared_prec = -1;
  const float *prepared_latents = nullptr;
  uint64_t prepared_version = 0;
  uint64_t version = 1;            // bumped when materials or parameters change
  // launch configuration (0 = automatic)
  int tc_ctas_per_sm = 0;
  int tc_warpgroups = 0;
  int tc_tile_wgs = 0;         // warpgroups per decoder tile pipeline (0 or 1: one, 2: two)
  int loss_mode = 0;           // FABRIC_LOSS_EQ11 or FABRIC_LOSS_RENDERED
  int visibility = 0;          // the reference's proposed inter-yarn visibility model on
  int train_prec = 0;          // FABRIC_PREC_FP32 (SIMT) or FABRIC_PREC_BF16 (tensor cores)
  int ref_lanes = 0;
  // host-buffer pipeline (fabric_shade_neural_host): per-slot stream, event
  // and device staging for one chunk's G-buffer and outputs
  static constexpr int kHostSlots = 3;
  cudaStream_t host_stream[kHostSlots] = {};
  cudaEvent_t host_done[kHostSlots] = {};
  cudaEvent_t host_start = nullptr;
  void *host_stage = nullptr;   // kHostSlots x host_slot_bytes
  size_t host_slot_bytes = 0;
  // the paper's decoder structure (fabric_paper_*): width, FP32 master
  // parameters, Adam moments over [decoder | encoder], packed operands and
  // the state of the last fabric_paper_prepare
  int pn_width = 0;
  int pn_ablation = 0;              // 0 the full structure, 1 without one-blob, 2 without spatial fusion
  float *d_pn_dec = nullptr;
  float *d_pn_enc = nullptr;
  float *d_pn_adam = nullptr;
  float *d_pn_grad = nullptr;       // the last training step's gradient [decoder | encoder]
  int64_t pn_adam_step = 0;
  void *d_pn_blob = nullptr;
  uint64_t pn_version = 1;          // bumped when the paper network's parameters change
  int pn_prepared_prec = -1;
  uint64_t pn_prepared_version = 0;  // (ctx->version, pn_version) folded at prepare time
};

namespace fab {

fabric_status fail(fabric_ctx *ctx, fabric_status s, const char *fmt, ...);
fabric_status cuda_fail(fabric_ctx *ctx, cudaError_t e, const char *what);
// Make sure the scratch arena holds `bytes`; returns nullptr on failure.
void *scratch(fabric_ctx *ctx, size_t bytes);
bool build_material(const fabric_material &m, DevMaterial *out, std::string *why);
bool check_gbuffer(fabric_ctx *ctx, const fabric_gbuffer *g);
bool is_aligned16(const void *p);
bool is_aligned4(const void *p);
// Free the host-pipeline streams, events and staging of a context.
void host_pipeline_release(fabric_ctx *ctx);
// Free the paper network's parameters and buffers of a context.
void paper_release(fabric_ctx *ctx);

// Launchers implemented in the kernel translation units.
cudaError_t launch_reference(const fabric_gbuffer &g, const DevMaterial *mats, int n_mat, int spp_x, int spp_y,
                             uint64_t seed, float *rgb, float *comps, int *status, int lanes_per_point,
                             int sm_count, cudaStream_t s, bool visibility = false);
cudaError_t launch_decoder_fp32(const fabric_gbuffer &g, const DevMaterial *mats, int n_mat, const float *latents,
                                const float *dec, float *rgb, float *comps, float *y_raw, int *status,
                                cudaStream_t s);
size_t tc_blob_bytes(int n_mat);
int tc_k1(int n_mat);
cudaError_t launch_tc_pack(const float *dec, const float *latents, const DevMaterial *mats, int n_mat,
                           int precision, void *blob, cudaStream_t s);
int tc_default_ctas_per_sm(int n_mat, int precision);
cudaError_t launch_decoder_tc(const fabric_gbuffer &g, const void *blob, int n_mat, int precision, float *rgb,
                              float *comps, int *status, int sm_count, int ctas_per_sm, int warpgroups, int tile_wgs,
                              cudaStream_t s);
int64_t tc_tiles(int64_t n);
cudaError_t launch_decoder_tc_segments(const SegDesc *segs, const int64_t *seg_tile0, int n_segs, int64_t n_tiles,
                                       const void *blob, int n_mat, int precision, int *status, int sm_count,
                                       int ctas_per_sm, int warpgroups, int tile_wgs, cudaStream_t s);
cudaError_t launch_selftest_mma(const float *a, const float *b, int n, int k, int a_in_tmem, float *d, int *status,
                                cudaStream_t s);
cudaError_t launch_encoder_raw(const fabric_material *raw, int n, const float *enc, float *z, cudaStream_t s);
cudaError_t launch_encoder_feats(const float *feats, int n, const float *enc, float *z, float *acts,
                                 cudaStream_t s);
// The decoder's gradient summed from per-CTA partials and its Adam update,
// run by extra blocks of the encoder-gradient launch, beside that work
// instead of before it.  The sums are the ones launch_decoder_grad_finish
// forms, in the same order.
struct DecAdamArgs {
  const float *partial;   // [n_part][stride]; the decoder's n columns first
  int n_part, stride, n;
  float *p, *m, *v;       // the decoder's parameters and their Adam moments
  float lr, bc1, bc2;
};
cudaError_t launch_encoder_backward(const float *feats, int n, const float *enc, const float *acts,
                                    const float *dz, float *denc, float *work, cudaStream_t s,
                                    const DecAdamArgs *dec_adam = nullptr);
// Adam's bias corrections 1 - beta^t for step t.
void adam_bias(int64_t step, float *bc1, float *bc2);
size_t encoder_backward_work_floats(int n);
// Encoder forward with the input features computed from the material
// records (and written to feats_out, when not null, for the backward pass).
cudaError_t launch_encoder_raw(const fabric_material *raw, int n, const float *enc, float *feats_out, float *z,
                               float *acts, cudaStream_t s);
cudaError_t launch_decoder_raw(const fabric_gbuffer &g, const float *latents, int n_lat, const float *dec,
                               float *y_raw, int *status, cudaStream_t s);
cudaError_t launch_decoder_backward(const fabric_gbuffer &g, const float *latents, int n_lat, const float *dec,
                                    const float *dy, const float *target, int loss_mode, float *ddec, float *dlat,
                                    double *loss, void *work, int sm_count, int *status, cudaStream_t s);
size_t decoder_backward_work_bytes(int64_t n, int sm_count);
// The fixed-order sums after a backward pass that wrote per-CTA partials
// ([grid][width] floats): parameter gradients (left to a DecAdamArgs launch
// when ddec is null), the loss, and the per-material latent gradients (from
// the partials' columns past kDecParams when width > kDecParams, else from
// the per-row latent gradients `rows`).
cudaError_t launch_decoder_grad_finish(const fabric_gbuffer &g, int n_lat, const float *partial, int grid, int width,
                                      const double *loss_part, const float *rows, float *ddec, double *loss,
                                      float *dlat, cudaStream_t s);
// Tensor-core (BF16) decoder training forward + backward: per-CTA gradient
// partials [grid][kDecParams], loss partials [grid], latent-gradient rows [n][32].
size_t train_tc_blob_bytes();
int train_tc_grid(int64_t n, int sm_count);
int train_tc_partial_width(int n_lat);
cudaError_t launch_selftest_wait(int sleep, int *status, cudaStream_t s);
cudaError_t launch_selftest_mn(const float *a, const float *b, int n, int k, float *d, int *status, cudaStream_t s);
cudaError_t launch_train_tc(const fabric_gbuffer &g, const float *latents, int n_lat, const float *dec,
                            const float *target, int loss_mode, void *blob, float *partial, double *loss_partial,
                            float *dlat_rows, int sm_count, int *status, cudaStream_t s);
// dst[p] = src[pi(p)] for the dataset's fields (fabric_shuffle_dataset).
cudaError_t launch_shuffle_dataset(const fabric_train_batch &src, const fabric_dataset_out &dst, uint64_t seed,
                                   int sm_count, cudaStream_t s);
cudaError_t launch_adam(float *p0, int64_t n0, float *p1, int64_t n1, const float *grad, float *m, float *v, float lr,
                        int64_t step, cudaStream_t s);
// The paper's decoder structure (paper_decoder.cu): K of its first layer for
// n_mat materials (-1 beyond 104), packed-operand bytes, packing and the
// tensor-core decoder (FP16 or BF16 operands), width 64 or 128.
int paper_k1(int n_mat);
size_t paper_blob_bytes(int width, int n_mat);
cudaError_t launch_paper_pack(int width, int precision, const float *params, const float *latents,
                              const DevMaterial *mats, int n_mat, void *blob, cudaStream_t s);
cudaError_t launch_paper_decoder(int width, int precision, const fabric_gbuffer &g, const void *blob, int n_mat,
                                 float *rgb, float *comps, int *status, int sm_count, cudaStream_t s);
// Its FP32 training forward, loss and backward (paper_train.cu): the
// gradient [decoder | encoder] and the batch loss; and its encoder alone.
size_t paper_train_work_bytes(int width, int64_t batch, int n_mat);
int paper_train_max_materials(int width);
cudaError_t launch_paper_train(int width, int ablation, const fabric_gbuffer &q, const float *target, int loss_mode,
                               const fabric_material *raw, int n_mat, const float *dec, const float *enc, float *grad,
                               double *loss, void *work, int *status, cudaStream_t s);
// Its FP32 forward over a G-buffer (any ablation): components and RGB.
size_t paper_forward_work_bytes(int width, int64_t n);
cudaError_t launch_paper_forward(int width, int ablation, const fabric_gbuffer &g, const float *z,
                                 const DevMaterial *mats, int n_mat, const float *dec, float *rgb, float *comps,
                                 void *work, int *status, cudaStream_t s);
cudaError_t launch_paper_encoder(const fabric_material *raw, int n_mat, const float *enc, float *z, cudaStream_t s);
cudaError_t launch_error_stats(const float *a, const float *b, int64_t n, const float *w, int group, int w_stride,
                               double *out, void *work, cudaStream_t s);
size_t error_stats_work_bytes(int64_t n);

}  // namespace fab
