/*
 * fabric.h -- C ABI of the GB300 (sm_103a) footprint-filtered woven-fabric
 * reflectance library: the per-shading-point path of Chen, Wang and Wang,
 * "Real-time Neural Woven Fabric Rendering" (SIGGRAPH 2024).
 *
 * Conventions shared by every call
 * ---------------------------------
 *  - Plain C types only.  `stream` is a cudaStream_t passed as void* (NULL =
 *    the legacy default stream).  Pointers named *_dev are device pointers
 *    owned by the caller; pointers without the suffix are host pointers.
 *  - The context owns what it allocates: pattern and material tables,
 *    network parameters (FP32 master copy), Adam moments, packed tensor-core
 *    weights and per-call scratch.  It never frees caller memory.
 *  - Every call that takes a stream is asynchronous on it and returns before
 *    the GPU work finishes, except where a call says otherwise.  Arguments
 *    are checked on the host before any launch; a rejected call launches
 *    nothing and returns FABRIC_ERR_INVALID_ARG with a message available from
 *    fabric_last_error().  No C++ exception and no process exit crosses the
 *    ABI; device code never traps.
 *  - Errors found on the device (a material index outside the material
 *    table, an expired wait inside a kernel) are recorded in a device status
 *    word; the faulty point's outputs are NaN.  fabric_sync_status() reports
 *    and clears it.
 *  - n = 0 is a no-op that returns FABRIC_OK.  NaN inputs propagate to the
 *    affected point only.
 *  - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef FABRIC_H
#define FABRIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FABRIC_OK = 0,
  FABRIC_ERR_INVALID_ARG = 1,
  FABRIC_ERR_CUDA = 2,
  FABRIC_ERR_OOM = 3,
  FABRIC_ERR_TIMEOUT = 4,
  FABRIC_ERR_IO = 5,
  FABRIC_ERR_UNSUPPORTED = 6,
  FABRIC_ERR_DEVICE = 7
} fabric_status;

typedef enum {
  FABRIC_PREC_FP32 = 0,   /* SIMT FP32 decoder (accuracy anchor)                */
  FABRIC_PREC_BF16 = 1,   /* tcgen05 tensor cores, BF16 operands, FP32 accum.   */
  FABRIC_PREC_FP8 = 2,    /* tcgen05 tensor cores, E4M3 operands, FP32 accum.   */
  FABRIC_PREC_FP16 = 3    /* tcgen05 tensor cores, FP16 operands, FP32 accum.   */
} fabric_precision;

/*
 * Material record (host memory, 84 bytes, no padding): the shading-model
 * parameters of Table 1 plus the procedural weave of Sec. 5.1.
 *   pattern_id  built-in weave 0..11: plain, 2/1 twill, 3/1 twill, 4/1 satin
 *               (warp-faced), 5-harness satin (weft-faced), 2x2 basket,
 *               herringbone, warp rib, 4/1 twill, 7/1 twill, 8-harness
 *               satin (weft-faced), 5-harness satin with doubled picks
 *               (10 x 5); the encoder's one-hot has 16 slots
 *   twist_deg   ply twist psi, degrees (Table 2)
 *   incl_deg    yarn inclination u, degrees (Table 2)
 *   alpha, beta roughness and height-field scale, [0] warp, [1] weft (Table 1)
 *   kd, ks      diffuse / specular RGB albedos, [yarn][rgb]; they enter only
 *               through Eq. 8, never the network (Sec. 4.1)
 *   gap         gap ratio of a yarn's width (0.2 in Sec. 5.1)
 *   w_blend     blended-Lambertian weight w of Eq. 1
 * Accepted ranges: 0 < alpha <= 1, 0 <= beta <= 4, 0 <= gap < 1,
 * 0 <= w_blend <= 1, |twist|, |incl| <= 89.
 */
typedef struct {
  int32_t pattern_id;
  float twist_deg;
  float incl_deg;
  float alpha[2];
  float beta[2];
  float kd[2][3];
  float ks[2][3];
  float gap;
  float w_blend;
} fabric_material;

/*
 * G-buffer of n shading points, structure of arrays, device memory, all
 * arrays 4-byte aligned (16-byte alignment enables the vectorised paths).
 * The same holds for every output array: a [n][4] output (comps_dev and
 * the like) that is 16-byte aligned takes one 16-byte store per point, any
 * other float-aligned one four 4-byte stores; FABRIC_ERR_INVALID_ARG only
 * for an output that is not float-aligned.
 * The query of Eq. 6: footprint centre (u, v) in pattern repeats (1 uv unit =
 * one weave repeat), footprint half side `radius` in the same units (box
 * kernel k_P over [u-r, u+r] x [v-r, v+r], Eq. 3), wi and wo as [n][3] unit
 * vectors in the local shading frame (z = macro normal n_s, x along u, y
 * along v), and a material index into the context's material table.
 */
typedef struct {
  const float *u;
  const float *v;
  const float *radius;
  const float *wi;
  const float *wo;
  const uint16_t *material;
  int64_t n;
} fabric_gbuffer;

typedef struct fabric_ctx fabric_ctx;

/* ------------------------------------------------------------------ */
/* Lifecycle and status                                               */
/* ------------------------------------------------------------------ */

/* Create a context on CUDA device `device` (becomes current for the calling
 * thread).  Synchronous.  *out is NULL on failure. */
fabric_status fabric_create(fabric_ctx **out, int device);

/* Release everything the context owns (waits for its streams' work). */
void fabric_destroy(fabric_ctx *ctx);

/* Message describing the last failed call on this context ("" if none). */
const char *fabric_last_error(const fabric_ctx *ctx);

/* Name of a status code. */
const char *fabric_status_string(fabric_status s);

/* Synchronise `stream`, then read and clear the device status word:
 * FABRIC_OK, FABRIC_ERR_DEVICE (bad material index) or FABRIC_ERR_TIMEOUT. */
fabric_status fabric_sync_status(fabric_ctx *ctx, void *stream);

/* Number of streaming multiprocessors of the context's device. */
int fabric_sm_count(const fabric_ctx *ctx);

/*
 * Launch configuration (no counterpart in the paper; set by the autotuner):
 *   decoder_ctas_per_sm  resident CTAs per SM of the persistent tensor-core
 *                        decoder (0 = as many as fit; capped at what fits)
 *   decoder_warpgroups   independent 128-point tile pipelines per decoder
 *                        CTA sharing one copy of the weights, 1, 2 or 4
 *                        (0 or 3 = 1); each uses 128 of the SM's 512
 *                        tensor-memory columns
 *   reference_lanes      lanes per shading point of the reference kernel,
 *                        1, 2, 4, 8, 16 or 32 (0 = by sample count)
 * Takes effect for the following calls.  FABRIC_ERR_INVALID_ARG on values
 * outside those sets.
 */
fabric_status fabric_set_launch_config(fabric_ctx *ctx, int decoder_ctas_per_sm, int decoder_warpgroups,
                                       int reference_lanes);

/* Warpgroups per decoder tile pipeline: 1 (0 = 1) or 2.  With 2, the two
 * threads of each tile row split the encoding and the epilogues' columns;
 * this applies with 1 or 2 pipelines per CTA (with 4 the setting is ignored).
 * FABRIC_ERR_INVALID_ARG outside 0..2. */
fabric_status fabric_set_decoder_tile_warpgroups(fabric_ctx *ctx, int warpgroups_per_tile);

/* ------------------------------------------------------------------ */
/* Materials                                                          */
/* ------------------------------------------------------------------ */

/* Copy n_mat (1..65535) host material records into the context's material
 * table (used by the shading calls: G-buffer material indices refer to it).
 * Builds the weave and float-run tables.  Synchronous. */
fabric_status fabric_set_materials(fabric_ctx *ctx, const fabric_material *m, int n_mat);

/* ------------------------------------------------------------------ */
/* Network parameters                                                 */
/* ------------------------------------------------------------------ */

/* Flat FP32 parameter counts.  Decoder layout (weights [out][in]):
 *   W1[64][71] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[4][64] b4[4]
 * with input [latent(32) | enc(u)(16) | enc(v)(16) | l | wi(3) | wo(3)],
 * output the four components of Eq. 7 (C_warp, C_weft, S'_warp, S'_weft).
 * Encoder layout: E1[128][14] e1[128] E2[128][128] e2[128] E3[32][128] e3[32]
 * (parameters -> latent, residual block of Sec. 4.2). */
int64_t fabric_decoder_param_count(void);
int64_t fabric_encoder_param_count(void);

/* Copy host FP32 parameters into the context (either pointer may be NULL to
 * leave that network unchanged).  Resets the Adam state.  Synchronous. */
fabric_status fabric_set_params(fabric_ctx *ctx, const float *decoder, const float *encoder);

/* Copy the context's parameters to host memory (NULL skips).  Synchronous. */
fabric_status fabric_get_params(fabric_ctx *ctx, float *decoder, float *encoder);

/* Device pointers to the context's FP32 master parameters (valid until the
 * context is destroyed); for callers that drive training themselves. */
fabric_status fabric_param_pointers(fabric_ctx *ctx, float **decoder_dev, float **encoder_dev);

/* Checkpoint: parameters, Adam moments and step counter in a versioned
 * binary file with a CRC-32.  Synchronous.  Load fails with FABRIC_ERR_IO on
 * a missing, truncated or corrupted file and leaves the context unchanged. */
fabric_status fabric_checkpoint_save(fabric_ctx *ctx, const char *path);
fabric_status fabric_checkpoint_load(fabric_ctx *ctx, const char *path);

/* ------------------------------------------------------------------ */
/* The four calls of the shading path                                 */
/* ------------------------------------------------------------------ */

/*
 * Encoder (Sec. 4.2, "Encoder"; run only when materials change, Sec. 4.4):
 * material parameters -> latent z in R^32 for n_mat host records, written
 * to latents_dev [n_mat][32] FP32.  Input features: one-hot weave (8),
 * psi/30, u/45, alpha_warp, beta_warp, alpha_weft, beta_weft.
 */
fabric_status fabric_encode_params(fabric_ctx *ctx, const fabric_material *m, int n_mat,
                                   float *latents_dev, void *stream);

/*
 * Supersampled reference (the plain method, Eq. 3-5 with the components of
 * Eq. 7 and Eq. 8): for every point, spp_x * spp_y stratified samples over
 * the footprint square, jittered by SplitMix64(seed, point index, sample),
 * shaded with the model of Eq. 1-2, summed with warp-level reductions.
 * Outputs rgb_dev [n][3] (Eq. 8 with the material's albedos) and, if not
 * NULL, comps_dev [n][4] = (C_warp, C_weft, S_warp, S_weft).
 * 1 <= spp_x, spp_y <= 4096.
 */
fabric_status fabric_shade_reference(fabric_ctx *ctx, const fabric_gbuffer *g, int spp_x, int spp_y,
                                     uint64_t seed, float *rgb_dev, float *comps_dev, void *stream);

/*
 * Inter-yarn visibility V(x_p, w) of Eq. 3-5 in fabric_shade_reference (and
 * so in data generated with it): 0 (default) V = 1; 1 this library's
 * proposed model (the paper defers its own to a supplementary that is not
 * available).  The surface is the height field whose slopes the shading
 * frame uses, in repeat units: on a top yarn's body beta w cos(pi x / 2) plus
 * the float's rise (the integral of tan(theta) along the float), w the yarn's
 * half-width (1 - g) / (2 N), N the pattern size across the yarn; under a gap
 * the under-yarn, level, at beta' w' (cos(pi x' / 2) - 1).  V = 1 when a
 * march from the surface point along w with horizontal steps of
 * 1 / (16 max(rows, cols)) repeats stays above the surface until the ray
 * rises above the material's largest height (at most 4096 steps), else 0;
 * the numerators carry V(x_p, wi) V(x_p, wo) and A carries V(x_p, wo).
 * Costs one or two marches per sample.  FABRIC_ERR_INVALID_ARG for values
 * other than 0 and 1.
 */
fabric_status fabric_set_visibility(fabric_ctx *ctx, int on);

/*
 * Neural shading (Sec. 4.4, "Rendering"): decoder over the G-buffer with the
 * per-material latents latents_dev [n_mat][32] (n_mat = size of the material
 * table), then C = max(0, y), S = max(0, expm1(y')/100) (inverse of Eq. 9)
 * and Eq. 8.  Outputs as for fabric_shade_reference.  FP32 runs the SIMT
 * decoder; FP16 / BF16 / FP8 run the tensor-core decoder (material table of at most
 * 89 entries).  FP8: layer 1 keeps FP16 operands (its weights carry the folded
 * latent); layers 2-4 take E4M3 activations (unscaled, saturating at 448)
 * and E4M3 weights scaled per layer by 2^(8 - E), where max |W| = m 2^E with
 * m in [0.5, 1); the scale is undone and the bias added in FP32.
 */
fabric_status fabric_shade_neural(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev,
                                  fabric_precision prec, float *rgb_dev, float *comps_dev, void *stream);

/*
 * fabric_shade_neural split in its two stages, for renderers that edit
 * materials rarely and draw frames often (Sec. 4.4: only the decoder runs per
 * frame, the encoder and the latent fold run on edits):
 *  - fabric_prepare_neural folds latents_dev [n_mat][32] into the first layer
 *    and packs the operands of `prec` into the context (one small kernel);
 *    latents_dev must stay valid for FP32 frames.
 *  - fabric_shade_neural_prepared draws one G-buffer with the last prepared
 *    state of the same precision (FABRIC_ERR_INVALID_ARG if none, or if the
 *    material table or parameters changed since).
 */
fabric_status fabric_prepare_neural(fabric_ctx *ctx, const float *latents_dev, fabric_precision prec,
                                    void *stream);
fabric_status fabric_shade_neural_prepared(fabric_ctx *ctx, const fabric_gbuffer *g, fabric_precision prec,
                                           float *rgb_dev, float *comps_dev, void *stream);

/*
 * Training batch: queries (material indices refer to the training material
 * table set by fabric_set_train_materials) and ground-truth components
 * target_dev [n][4] (C_warp, C_weft, S_warp, S_weft), e.g. from
 * fabric_shade_reference.
 */
typedef struct {
  fabric_gbuffer queries;
  const float *target;
} fabric_train_batch;

/* Copy the training material table (1..65535 records).  Synchronous. */
fabric_status fabric_set_train_materials(fabric_ctx *ctx, const fabric_material *m, int n_mat);

/*
 * One training step (Sec. 4.3, Sec. 5.2): encoder over the training
 * materials, decoder over the batch, the loss of Eq. 11 (specular mapped by
 * g(x) = ln(100 x + 1), Eq. 9; lambda_S = 0.4, lambda_C = 0.1), backward
 * through both networks with deterministic reductions, one Adam update
 * (beta1 0.9, beta2 0.999, eps 1e-8) of the context's parameters.
 * *loss_dev (device double) receives the batch loss before the update.
 * Batch size 1..1048576.
 */
fabric_status fabric_train_step(fabric_ctx *ctx, const fabric_train_batch *batch, float lr,
                                double *loss_dev, void *stream);

/*
 * n_steps training steps of fabric_train_step over one dataset, without a
 * host round trip between them: step k (k = 0 .. n_steps - 1) takes the
 * `batch` queries and targets starting at point (k mod (n / batch)) * batch
 * of data (n = data->queries.n, so an epoch is n / batch steps over
 * consecutive slices; shuffle the dataset between calls), with learning rate
 *   lr(t) = lr1 + (lr0 - lr1) (1 + cos(pi t / total_steps)) / 2,
 * t = first_step + k, evaluated in double and rounded to float (a cosine
 * decay over total_steps steps).  loss_dev (device doubles, optional) gets
 * step k's loss at loss_dev[k].  The results are bitwise those of the same
 * single steps.  batch 1..min(n, 1048576); n_steps >= 0; total_steps >= 1;
 * first_step >= 0; else FABRIC_ERR_INVALID_ARG.  Errors of a step end the
 * call with that step's status (the steps before it are applied).
 */
fabric_status fabric_train_steps(fabric_ctx *ctx, const fabric_train_batch *data, int64_t batch, int n_steps,
                                 int64_t first_step, int64_t total_steps, double lr0, double lr1,
                                 double *loss_dev, void *stream);

/* Output arrays of fabric_shuffle_dataset: device memory of the caller, the
 * layout of fabric_train_batch (wi, wo [n][3], target [n][4]), not
 * overlapping the input. */
typedef struct {
  float *u;
  float *v;
  float *radius;
  float *wi;
  float *wo;
  uint16_t *material;
  float *target;   /* NULL when the input has no targets */
} fabric_dataset_out;

/*
 * A shuffled copy of a training dataset in one pass on the device (the data
 * loader between epochs): dst[p] = src[pi(p)] for every field, p < n, where
 * pi is the pseudo-random permutation of [0, n) that `seed` selects: a
 * four-round Feistel network on [0, 4^k), 4^k >= n, whose round function is
 * the SplitMix64 finaliser of (seed, round, half), walked along its cycles
 * until it lands in [0, n).  pi depends only on n and seed.  n 1..2^31;
 * FABRIC_ERR_INVALID_ARG for NULL or misaligned arrays.  Asynchronous.
 */
fabric_status fabric_shuffle_dataset(fabric_ctx *ctx, const fabric_train_batch *src, const fabric_dataset_out *dst,
                                     uint64_t seed, void *stream);

/* Training loss of fabric_train_step (default FABRIC_LOSS_EQ11):
 *   FABRIC_LOSS_EQ11      the paper's Eq. 11, as above;
 *   FABRIC_LOSS_RENDERED  this library's option: (1/B) sum over queries and
 *       the four components of ((c_hat - c) max(<wi . n_s>, 0))^2, where
 *       c_hat is the decoded component (C = y; S = (exp(min(y, 12)) - 1)/100,
 *       the inverse of Eq. 9 without the clamp at 0): the error of the
 *       components as they light the frame under a directional light.
 * FABRIC_ERR_INVALID_ARG for other values. */
typedef enum { FABRIC_LOSS_EQ11 = 0, FABRIC_LOSS_RENDERED = 1 } fabric_loss;
fabric_status fabric_set_train_loss(fabric_ctx *ctx, fabric_loss loss);

/* Arithmetic of the decoder's forward and backward in fabric_train_step
 * (default FABRIC_PREC_FP32): FABRIC_PREC_FP32 runs them as FP32 SIMT
 * kernels; FABRIC_PREC_BF16 runs every product on the tensor cores with BF16
 * operands and FP32 accumulation (the weight gradients accumulate over each
 * CTA's queries in tensor memory).  Both keep FP32 master parameters, the
 * encoder in FP32, FP64 loss sums and fixed-order reductions, so both are
 * bitwise repeatable.  FABRIC_ERR_INVALID_ARG for other precisions. */
fabric_status fabric_set_train_precision(fabric_ctx *ctx, fabric_precision prec);

/* ------------------------------------------------------------------ */
/* Building blocks for a torch.autograd.Function                      */
/* ------------------------------------------------------------------ */

/* Raw decoder head y_dev [n][4] (no output activation) for the G-buffer,
 * with latents_dev [n_lat][32] indexed by g->material and explicit FP32
 * decoder parameters dec_dev (layout above).  FP32 SIMT. */
fabric_status fabric_decoder_forward(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev,
                                     int n_lat, const float *dec_dev, float *y_dev, void *stream);

/* Gradients of sum(dy * y): ddec_dev [decoder params] and dlatents_dev
 * [n_lat][32] are overwritten (not accumulated).  Deterministic. */
fabric_status fabric_decoder_backward(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev,
                                      int n_lat, const float *dec_dev, const float *dy_dev,
                                      float *ddec_dev, float *dlatents_dev, void *stream);

/* Encoder on explicit features feats_dev [n][14] -> z_dev [n][32]. */
fabric_status fabric_encoder_forward(fabric_ctx *ctx, const float *feats_dev, int n, const float *enc_dev,
                                     float *z_dev, void *stream);

/* Gradients of sum(dz * z): denc_dev [encoder params] overwritten. */
fabric_status fabric_encoder_backward(fabric_ctx *ctx, const float *feats_dev, int n, const float *enc_dev,
                                      const float *dz_dev, float *denc_dev, void *stream);

/* ------------------------------------------------------------------ */
/* Image-wide error (FP64 on the device)                              */
/* ------------------------------------------------------------------ */

/* out_dev[0] = sum (w(a-b))^2, out_dev[1] = sum (w b)^2, out_dev[2] =
 * max |w(a-b)| over n floats (device double[3]); RMSE = sqrt(out0/n),
 * rel-L2 = sqrt(out0/out1).  w = 1 when weights_dev is NULL, else
 * weights_dev[i / group] (one weight per group of `group` consecutive
 * floats, e.g. per RGB pixel), read with stride weight_stride floats, so
 * that for instance the z of a [n][3] direction array can weight RGB
 * (renderers multiply f_P by <wi . n_s> under direct light).  Deterministic. */
fabric_status fabric_error_stats(fabric_ctx *ctx, const float *a_dev, const float *b_dev, int64_t n,
                                 const float *weights_dev, int group, int weight_stride, double *out_dev,
                                 void *stream);

/* ------------------------------------------------------------------ */
/* Batched draws                                                      */
/* ------------------------------------------------------------------ */

/* One segment of a batched draw: a G-buffer and its own outputs (device
 * memory, caller-owned; comps_dev may be NULL). */
typedef struct {
  fabric_gbuffer g;
  float *rgb_dev;     /* [g.n][3] */
  float *comps_dev;   /* [g.n][4] or NULL */
} fabric_segment;

typedef struct fabric_plan fabric_plan;

/*
 * Batching (the paper renders one view per frame; a renderer with several
 * views, cameras or ragged tiles per frame wants them in one launch):
 * fabric_plan_create checks and uploads a table of 1..1048576 segments once
 * (synchronous; the plan keeps the device pointers, not the data).
 * fabric_plan_shade then shades every segment with the prepared neural
 * state (fabric_prepare_neural, FP16, BF16 or FP8) in one persistent
 * tensor-core launch over all segments' 128-point tiles: asynchronous, no
 * host-side work besides the launch, so it can be captured in a CUDA graph
 * and replayed.  Results equal per-segment fabric_shade_neural_prepared
 * calls bit for bit.
 */
fabric_status fabric_plan_create(fabric_ctx *ctx, const fabric_segment *segs, int n_segs, fabric_plan **out);
fabric_status fabric_plan_shade(fabric_ctx *ctx, const fabric_plan *plan, fabric_precision prec, void *stream);
int64_t fabric_plan_points(const fabric_plan *plan);
void fabric_plan_destroy(fabric_plan *plan);

/*
 * Neural shading of a G-buffer in HOST memory, with the prepared state of
 * fabric_prepare_neural for `prec`.  g_host's pointers and rgb_host [n][3]
 * (and comps_host [n][4], or NULL) are host pointers that
 * must stay valid until `stream` has passed this call.  Asynchronous on
 * `stream`.
 *  - chunk_points = 0 and every buffer page-locked and mapped (as
 *    cudaHostAlloc gives it): the decoder reads the G-buffer and writes the
 *    outputs directly over the host link, one launch on `stream`.
 *  - otherwise: the frame is cut into chunks of chunk_points (0 = 262144;
 *    rounded up to a multiple of 128) that cycle through three
 *    context-owned device staging slots on their own streams, so that one
 *    chunk's upload, the next one's decoder and a third one's download
 *    overlap (pageable memory works but serialises the copies).  The chunks
 *    start after the work queued on `stream`, and it waits for all of them.
 *    The staging (about 90 bytes per chunk point per slot) is allocated on
 *    first use and grown when a larger chunk is asked for; calls on several
 *    streams of one context share the slots and are serialised by them.
 * Errors as for fabric_shade_neural_prepared.
 */
fabric_status fabric_shade_neural_host(fabric_ctx *ctx, const fabric_gbuffer *g_host, fabric_precision prec,
                                       float *rgb_host, float *comps_host, int64_t chunk_points, void *stream);

/* ------------------------------------------------------------------ */
/* The paper's decoder structure                                      */
/* ------------------------------------------------------------------ */

/*
 * The decoder of Sec. 4.2 ("Decoder", Fig. 3) beside the workload's: the
 * footprint centre (frac u, frac v) and size one-blob encoded (3 inputs ->
 * 24 channels, 8 Gaussian bins each of standard deviation 1/8; the centre's
 * Gaussians wrap around the weave repeat; size t = ln(max(r, 2^-20) / 1e-4) /
 * ln(2.5e4)), fused with a 64-wide material latent z by two fully connected
 * layers of width W (the spatial feature h), then with wi (x, y, z) and
 * wo (x, y) decoded by five fully connected layers with one skip:
 *   k1 = lrelu(A1 [h | wi | wo.xy] + a1),
 *   k3 = lrelu(A3 lrelu(A2 k1 + a2) + a3 + k1),
 *   y  = A5 lrelu(A4 k3 + a4) + a5,
 * leaky ReLU of slope 0.01, W = 64 or 128; y becomes the four components and
 * RGB exactly as for fabric_shade_neural.  Flat FP32 parameters, weights
 * [out][in]:
 *   S1[W][88] s1[W] S2[W][W] s2[W] A1[W][W+5] a1[W] A2[W][W] a2[W]
 *   A3[W][W] a3[W] A4[W][W] a4[W] A5[4][W] a5[4]
 * (S1's inputs are [z (64) | one-blob (24)]); the encoder is the workload's
 * with a 64-wide output: E1[128][22] e1 E2[128][128] e2 E3[64][128] e3.
 * One paper network per context, separate from the workload's network.
 */

/* Parameter count of the paper decoder of width 64 or 128 (encoder != 0: of
 * its encoder); -1 for another width. */
int64_t fabric_paper_param_count(int width, int encoder);

/* Copy host FP32 parameters in (either pointer NULL leaves that network
 * unchanged; a width different from the current one needs both).  Resets
 * the paper network's Adam state.  Synchronous. */
fabric_status fabric_paper_set_params(fabric_ctx *ctx, int width, const float *decoder, const float *encoder);

/* Copy the paper network's parameters out (NULL skips).  Synchronous. */
fabric_status fabric_paper_get_params(fabric_ctx *ctx, float *decoder, float *encoder);

/*
 * The two ablations of Sec. 6.3 ("Ablation study") beside the full
 * structure (FABRIC_PAPER_FULL, what fabric_paper_set_params sets):
 *   FABRIC_PAPER_NO_ONEBLOB: the footprint's three inputs enter S1 as they
 *     are, [z (64) | frac u | frac v | t] -> S1[W][67];
 *   FABRIC_PAPER_NO_FUSION: space and angle are queried together; as the
 *     section adds hidden layers to the angular decoder for a fair
 *     comparison, the S1 and S2 slots hold its two added first layers,
 *     [z (64) | one-blob (24) | wi | wo.xy] -> S1[W][93] -> S2[W][W], and
 *     A1 becomes [W][W] over their output (same size as the full
 *     structure).
 * Parameter layout otherwise as above.  Ablations
 * train (fabric_paper_train_step) and shade in FP32
 * (fabric_paper_shade_fp32); the tensor-core decoder (fabric_paper_prepare,
 * fabric_paper_shade_*) refuses them with FABRIC_ERR_UNSUPPORTED.
 */
enum { FABRIC_PAPER_FULL = 0, FABRIC_PAPER_NO_ONEBLOB = 1, FABRIC_PAPER_NO_FUSION = 2 };

/* Decoder parameter count of `ablation` at width 64 or 128; -1 otherwise. */
int64_t fabric_paper_structure_param_count(int width, int ablation);

/* fabric_paper_set_params for a structure: a change of width or structure
 * needs both parameter arrays (fabric_paper_structure_param_count(width,
 * ablation) and fabric_paper_param_count(width, 1) floats).  Resets the
 * paper network's Adam state.  Synchronous. */
fabric_status fabric_paper_set_structure(fabric_ctx *ctx, int width, int ablation, const float *decoder,
                                         const float *encoder);

/* The paper network (any structure) in FP32 on CUDA cores, one thread per
 * point and layer GEMMs over the G-buffer: latents_dev [n_mat][64] for the
 * material table; rgb_dev [n][3], comps_dev [n][4] or
 * NULL.  Uses the context's scratch (at most (5 W + 230) * 4 bytes a point).
 * A material index beyond the table gives NaN outputs and
 * FABRIC_ERR_DEVICE at the next fabric_sync_status. */
fabric_status fabric_paper_shade_fp32(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev,
                                      float *rgb_dev, float *comps_dev, void *stream);

/* Fold latents_dev [n_mat][64] (n_mat = the material table's size, at most
 * 104) into the first layer and pack the operands for FABRIC_PREC_FP16 or
 * FABRIC_PREC_BF16 (one small kernel on `stream`). */
fabric_status fabric_paper_prepare(fabric_ctx *ctx, const float *latents_dev, fabric_precision prec, void *stream);

/* Shade a G-buffer with the last prepared paper network of `prec` (one
 * persistent tensor-core launch); outputs, alignment and errors as for
 * fabric_shade_neural_prepared. */
fabric_status fabric_paper_shade_prepared(fabric_ctx *ctx, const fabric_gbuffer *g, fabric_precision prec,
                                          float *rgb_dev, float *comps_dev, void *stream);

/* fabric_paper_prepare followed by fabric_paper_shade_prepared. */
fabric_status fabric_paper_shade_neural(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev,
                                        fabric_precision prec, float *rgb_dev, float *comps_dev, void *stream);

/* The paper network's encoder (Sec. 4.2, "Encoder"; residual block):
 * n_mat host records -> latents_dev [n_mat][64] FP32, features as for
 * fabric_encode_params. */
fabric_status fabric_paper_encode_params(fabric_ctx *ctx, const fabric_material *m, int n_mat, float *latents_dev,
                                         void *stream);

/* One training step of the paper network (Sec. 4.3, Sec. 5.2), as
 * fabric_train_step does for the workload's network: its encoder over the
 * training material table, the decoder over the batch in FP32, the loss set
 * by fabric_set_train_loss, the backward pass (fixed-order reductions:
 * bitwise repeatable), one Adam update of the paper network's parameters.
 * *loss_dev (device double, or NULL) receives the batch loss before the
 * update.  Batch size 1..1048576; at most 1600 training materials
 * (FABRIC_ERR_UNSUPPORTED beyond). */
fabric_status fabric_paper_train_step(fabric_ctx *ctx, const fabric_train_batch *batch, float lr, double *loss_dev,
                                      void *stream);

/* Copy the gradient [decoder | encoder] of the last fabric_paper_train_step
 * to host memory (fabric_paper_structure_param_count(width, ablation) +
 * fabric_paper_param_count(width, 1) floats).
 * Synchronous.  Used by the tests. */
fabric_status fabric_paper_get_gradient(fabric_ctx *ctx, float *grad);

/* ------------------------------------------------------------------ */
/* Neural shading without any device allocation                       */
/* ------------------------------------------------------------------ */

/*
 * The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory while they draw, such as a host application
 * that owns all device memory and forbids plug-ins to allocate at draw time.
 *
 * Same arguments, outputs and errors as fabric_shade_neural with
 * prec = FABRIC_PREC_FP16, FABRIC_PREC_BF16 or FABRIC_PREC_FP8 (anything else
 * is FABRIC_ERR_INVALID_ARG).  It uses the context's material table and
 * parameters, set up beforehand, and keeps its per-call scratch (the packed
 * decoder operands, at most 64 KiB) in one static device array that every
 * GPU loading the library holds until the process exits.  It never calls
 * cudaMalloc, cudaFree or any allocating routine.
 *  - The limit that applies in practice is the tensor-core decoder's own:
 *    beyond 89 materials the call returns FABRIC_ERR_UNSUPPORTED as
 *    fabric_shade_neural does.  The packed operands of 89 materials
 *    (about 43 KiB) fit the array, which the library checks when it is
 *    compiled; a table that did not fit would be rejected with
 *    FABRIC_ERR_INVALID_ARG.
 *  - The first call on each device looks up the array's device address (a
 *    host-side query that allocates nothing); later calls reuse it.
 *  - All calls share the one array and overwrite all of it that they read,
 *    so nothing needs clearing between calls, but calls that overlap on the
 *    GPU (other streams, other host threads, other contexts on the same
 *    device) race on it: order them on one stream.
 */
fabric_status fabric_shade_neural_noalloc(fabric_ctx *ctx, const fabric_gbuffer *g, const float *latents_dev,
                                          fabric_precision prec, float *rgb_dev, float *comps_dev,
                                          void *stream);

/* ------------------------------------------------------------------ */
/* Diagnostics                                                        */
/* ------------------------------------------------------------------ */

/* One 128 x N x K BF16 tensor-core product through the same shared-memory
 * layouts, descriptors and tensor-memory path as the decoder:
 * d_dev[128][n] = a_dev[128][k] * b_dev[n][k]^T with a, b given as FP32 and
 * rounded to BF16.  k in {16, 32, 48, 64}, n in {16, 32, 64}.  a_in_tmem = 1
 * places A in tensor memory (written with tcgen05.st), 0 in shared memory.
 * Used by the tests to check the tensor-core data layouts in isolation. */
fabric_status fabric_selftest_mma(fabric_ctx *ctx, const float *a_dev, const float *b_dev, int n, int k,
                                  int a_in_tmem, float *d_dev, void *stream);

/* The same product with E4M3 operands (kind::f8f6f4), A in tensor memory
 * (four E4M3 values per 32-bit column), B in shared memory: a, b given as
 * FP32 and rounded to E4M3 (nearest even, saturating).  k in {32, 64},
 * n in {16, 32, 64}. */
fabric_status fabric_selftest_mma_e4m3(fabric_ctx *ctx, const float *a_dev, const float *b_dev, int n, int k,
                                       float *d_dev, void *stream);

/* The bounded-wait path of the kernels, exercised on purpose: one CTA waits
 * on an mbarrier that nothing ever completes (spinning when sleep = 0, with
 * try_wait and a suspend hint otherwise), gives up after about a
 * millisecond, records a timeout in the status word and returns; the next
 * fabric_sync_status returns FABRIC_ERR_TIMEOUT and clears it, and the
 * context stays usable.  Nothing faults or hangs.  Used by the tests. */
fabric_status fabric_selftest_wait_timeout(fabric_ctx *ctx, int sleep, void *stream);

/* The same BF16 product with both operands in shared memory in the MN-major
 * (transposed) layout the tensor-core training kernel uses for its weight
 * gradients: element (i, q) of a (and of b) stored with the 8 consecutive i
 * of one q in 16 contiguous bytes.  k in {16, 32, 48, 64}, n in {16, 32, 64}. */
fabric_status fabric_selftest_mma_mn(fabric_ctx *ctx, const float *a_dev, const float *b_dev, int n, int k,
                                     float *d_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FABRIC_H */
