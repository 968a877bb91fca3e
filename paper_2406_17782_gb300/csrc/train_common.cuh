// train_common.cuh -- device helpers shared by the FP32 (SIMT) and the
// tensor-core training kernels: the accurate query features and the
// per-output loss gradient of Eq. 9-11 or the rendered-space option.
#pragma once

#include <cmath>

#include "fabric_internal.h"

namespace fab {

constexpr float kLambdaS = 0.4f;      // Eq. 11
constexpr float kLambdaC = 0.1f;
constexpr float kYClamp = 12.0f;      // head pre-activation limit of the rendered-space loss

// sin / cos of 2 pi 2^k frac(x), k = 0..7 (sinpi/cospi of the exact reduced
// argument per octave); f16[2k] = sin, f16[2k + 1] = cos.
__device__ __forceinline__ void octaves_accurate(float x, float *f16) {
  const float f0 = x - floorf(x);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float sc = f0 * (float)(1 << k);
    const float fk = sc - floorf(sc);
    float s, c;
    sincospif(2.0f * fk, &s, &c);
    f16[2 * k] = s;
    f16[2 * k + 1] = c;
  }
}

// The 39 query features enc(u) | enc(v) | log footprint | wi | wo from the
// point's record r = (u, v, radius, wi[3], wo[3]).
__device__ __forceinline__ void query_features_of(const float *r, float *q) {
  octaves_accurate(r[0], q);
  octaves_accurate(r[1], q + 16);
  q[32] = (logf(fmaxf(r[2], kRFloor)) - kLogRC0) * kLogRInvC1;
  for (int i = 0; i < 6; ++i) q[33 + i] = r[3 + i];
}

// The G-buffer record of point p, as query_features_of reads it.
__device__ __forceinline__ void load_record(const fabric_gbuffer &g, int64_t p, float *r) {
  r[0] = g.u[p];
  r[1] = g.v[p];
  r[2] = g.radius[p];
  for (int i = 0; i < 3; ++i) {
    r[3 + i] = g.wi[3 * p + i];
    r[6 + i] = g.wo[3 * p + i];
  }
}

// The 39 query features of point p.
__device__ __forceinline__ void query_features(const fabric_gbuffer &g, int64_t p, float *q) {
  float r[9];
  load_record(g, p, r);
  query_features_of(r, q);
}

// d loss / d y_k for output k of one query (scaled by inv_batch); adds the
// query's loss term to *loss in the accumulator's type T.  y: raw head; tg:
// target component; wz: the query's <wi . n_s> (rendered-space loss only).
// T = double adds every term in FP64; T = float lets a caller sum a query's
// four terms in FP32 and only the per-query totals in FP64 (FP64 arithmetic
// issues at a small fraction of the FP32 rate).
template <typename T>
__device__ __forceinline__ float loss_grad(int k, float y, float tg, float wz, int mode, float inv_batch, T *loss) {
  if (mode == FABRIC_LOSS_RENDERED) {
    // ((c_hat - c) max(<wi.n_s>, 0))^2, c_hat = y (C) or (exp(min(y, 12)) - 1) / k (S)
    const float w = fmaxf(wz, 0.0f);
    float c = y, dc = 1.0f;
    if (k >= 2) {
      // expm1: near y = 0, exp(y) - 1 in FP32 would lose the relative
      // precision of the small S values the loss compares
      const float ys = fminf(y, kYClamp);
      c = expm1f(ys) * (1.0f / kSpecK);
      dc = y < kYClamp ? expf(ys) * (1.0f / kSpecK) : 0.0f;
    }
    const float diff = (c - tg) * w;
    *loss += (T)diff * (T)diff * (T)inv_batch;
    return 2.0f * diff * w * dc * inv_batch;
  }
  const float tt = k < 2 ? tg : logf(kSpecK * tg + 1.0f);   // g(x) = ln(k x + 1), Eq. 9
  const float lam = k < 2 ? kLambdaC : kLambdaS;
  const float diff = y - tt;
  *loss += (T)lam * (T)diff * (T)diff * (T)inv_batch;
  return 2.0f * lam * diff * inv_batch;
}

}  // namespace fab
