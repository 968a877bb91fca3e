// fabric_plan.cu -- batched draws: many G-buffer segments (views, ragged
// tiles) shaded by one persistent tensor-core launch.  Host code only.
#include <vector>

#include "fabric_internal.h"

using namespace fab;

extern "C" {

fabric_status fabric_plan_create(fabric_ctx *ctx, const fabric_segment *segs, int n_segs, fabric_plan **out) {
  if (!ctx || !out) return FABRIC_ERR_INVALID_ARG;
  *out = nullptr;
  ctx->last_error.clear();
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  if (!segs || n_segs < 1 || n_segs > (1 << 20))
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "need 1..1048576 segments (got %d)", n_segs);
  std::vector<SegDesc> host(n_segs);
  std::vector<int64_t> tile0(n_segs + 1);
  int64_t tiles = 0, points = 0;
  for (int s = 0; s < n_segs; ++s) {
    const fabric_segment &g = segs[s];
    if (!check_gbuffer(ctx, &g.g)) return fail(ctx, FABRIC_ERR_INVALID_ARG, "segment %d: %s", s,
                                               ctx->last_error.c_str());
    if (g.g.n > 0 && !g.rgb_dev) return fail(ctx, FABRIC_ERR_INVALID_ARG, "segment %d: rgb output is NULL", s);
    if (g.comps_dev && !is_aligned4(g.comps_dev))
      return fail(ctx, FABRIC_ERR_INVALID_ARG, "segment %d: comps output must be float-aligned", s);
    host[s] = SegDesc{g.g.u, g.g.v, g.g.radius, g.g.wi, g.g.wo, g.g.material, g.rgb_dev, g.comps_dev, g.g.n};
    tile0[s] = tiles;
    tiles += tc_tiles(g.g.n);
    points += g.g.n;
  }
  tile0[n_segs] = tiles;
  fabric_plan *p = new (std::nothrow) fabric_plan();
  if (!p) return FABRIC_ERR_OOM;
  p->device = ctx->device;
  p->n_segs = n_segs;
  p->n_tiles = tiles;
  p->n_points = points;
  if (cudaMalloc(&p->d_segs, n_segs * sizeof(SegDesc)) != cudaSuccess ||
      cudaMalloc(&p->d_tile0, (n_segs + 1) * sizeof(int64_t)) != cudaSuccess ||
      cudaMemcpy(p->d_segs, host.data(), n_segs * sizeof(SegDesc), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_tile0, tile0.data(), (n_segs + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    fabric_plan_destroy(p);
    return cuda_fail(ctx, e, "plan upload");
  }
  *out = p;
  return FABRIC_OK;
}

void fabric_plan_destroy(fabric_plan *plan) {
  if (!plan) return;
  cudaSetDevice(plan->device);
  cudaDeviceSynchronize();
  cudaFree(plan->d_segs);
  cudaFree(plan->d_tile0);
  delete plan;
}

int64_t fabric_plan_points(const fabric_plan *plan) { return plan ? plan->n_points : 0; }

fabric_status fabric_plan_shade(fabric_ctx *ctx, const fabric_plan *plan, fabric_precision prec, void *stream) {
  if (!ctx) return FABRIC_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (!plan || plan->device != ctx->device) return fail(ctx, FABRIC_ERR_INVALID_ARG, "plan is NULL or on another device");
  if (prec != FABRIC_PREC_FP16 && prec != FABRIC_PREC_BF16 && prec != FABRIC_PREC_FP8)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "batched draws run the FP16, BF16 or FP8 tensor-core decoder");
  if (ctx->prepared_prec != (int)prec || ctx->prepared_version != ctx->version)
    return fail(ctx, FABRIC_ERR_INVALID_ARG, "no prepared state for this precision, materials and parameters");
  if (plan->n_tiles == 0) return FABRIC_OK;
  const cudaError_t e = launch_decoder_tc_segments(plan->d_segs, plan->d_tile0, plan->n_segs, plan->n_tiles,
                                                   ctx->d_blob, ctx->n_mat, (int)prec, ctx->d_status, ctx->sm_count,
                                                   ctx->tc_ctas_per_sm, ctx->tc_warpgroups, ctx->tc_tile_wgs,
                                                   static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batched decoder launch");
  return FABRIC_OK;
}

}  // extern "C"
