// reference.cu -- supersampled footprint integral of the woven-fabric shading
// model (the plain method): Eq. 3-5 estimated with spp_x * spp_y stratified
// samples per shading point, shaded with Eq. 1-2, split into the components
// of Eq. 7 and recombined by Eq. 8.
//
// Work mapping: L lanes (L = 1..32, a power of two) share one shading point;
// each lane takes samples lane, lane + L, ... and the five running sums are
// combined with warp shuffles.  Every discrete decision (cell, gap, visible
// yarn) is taken in 0.32 fixed-point integers from a SplitMix64 jitter
// (Steele, Lea and Flood 2014) so that it is exactly reproducible; the
// shading itself runs in FP32.
#include "fabric_internal.h"

namespace fab {
namespace {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoNeg32 = 2.3283064365386963e-10f;   // 2^-32

__device__ __forceinline__ uint64_t splitmix_finalise(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Footprint centre in 0.32 fixed-point pattern coordinates (mod one repeat).
__device__ __forceinline__ uint32_t centre_fixed(float u) {
  const float f = __fsub_rn(u, floorf(u));
  return (uint32_t)(unsigned long long)__float2ll_rn(__fmul_rn(f, 4294967296.0f));
}

// Offset of stratum k jittered by xi: ((k + xi) * (2/n) - 1) * r, every step
// rounded to nearest in FP32 without contraction, then to 0.32 fixed point.
__device__ __forceinline__ uint32_t offset_fixed(int k, float xi, float two_over_n, float r) {
  float t = __fadd_rn((float)k, xi);
  t = __fmul_rn(t, two_over_n);
  t = __fsub_rn(t, 1.0f);
  t = __fmul_rn(t, r);
  return (uint32_t)(unsigned long long)__float2ll_rn(__fmul_rn(t, 4294967296.0f));
}

// sin and cos for |x| <= pi/2 from their Maclaurin series up to x^11 and
// x^12 (truncation below 6e-8 and 7e-9 there), Horner form with FMA.  The
// frame's angles (pi x / 2 across a yarn, theta along a float) stay in that
// range; the series keep the normal's error near one FP32 rounding, where the
// fast intrinsics' absolute error (about 4e-7) reached 2e-4 relative in the
// components of rays grazing the yarns.
__device__ __forceinline__ float sin_half_pi(float x) {
  const float x2 = x * x;
  float p = -2.505210838544172e-08f;     // -1/11!
  p = fmaf(p, x2, 2.7557319223985893e-06f);
  p = fmaf(p, x2, -1.984126984126984e-04f);
  p = fmaf(p, x2, 8.333333333333333e-03f);
  p = fmaf(p, x2, -1.6666666666666666e-01f);
  return fmaf(p * x2, x, x);
}
__device__ __forceinline__ float cos_half_pi(float x) {
  const float x2 = x * x;
  float p = 2.08767569878681e-09f;       // 1/12!
  p = fmaf(p, x2, -2.755731922398589e-07f);
  p = fmaf(p, x2, 2.48015873015873e-05f);
  p = fmaf(p, x2, -1.388888888888889e-03f);
  p = fmaf(p, x2, 4.1666666666666664e-02f);
  p = fmaf(p, x2, -0.5f);
  return fmaf(p, x2, 1.0f);
}

struct PointMaterial {
  uint32_t rows, cols, gap;
  float inv_1mg, cos_psi, sin_psi;
  float slope[2], ia2m1[2], oma2[2], ipa[2];
};

struct Sums {
  float c0, c1, s0, s1, a;
};

// ---- the proposed inter-yarn visibility model (V of Eq. 3-5).  The surface
// is the height field whose slopes the frame below uses, in repeat units:
// on a top yarn's body beta w cos(pi x / 2) plus the float's rise (the
// integral of tan(theta) along it); under a gap the under-yarn, level, one
// cross-section height below the top yarns' edges, beta' w' (cos(pi x'/2) - 1).
// V(x_p, w) = 1 when a march from (p, H(p)) along w, with horizontal steps
// of 1 / (16 max(rows, cols)) repeats, stays above H until the ray rises
// above the material's largest height (at most 4096 steps); 0 otherwise and
// below the horizon.  Steps are integer multiples of one 0.32 fixed-point
// increment per ray.
constexpr int kVisMaxSteps = 4096;

__device__ __forceinline__ float surface_height(const DevMaterial *__restrict__ m, const PointMaterial &pm,
                                                uint32_t pu, uint32_t pv) {
  const uint32_t j = __umulhi(pu, pm.cols), su = pu * pm.cols;
  const uint32_t i = __umulhi(pv, pm.rows), sv = pv * pm.rows;
  const bool warp_top = (__ldg(&m->top[i]) >> j) & 1u;
  const uint32_t s_top = warp_top ? su : sv;
  if ((s_top >= pm.gap) && (s_top <= 0xFFFFFFFFu - pm.gap)) {
    const float s = (float)s_top * kTwoNeg32;
    const float x = (2.0f * s - 1.0f) * pm.inv_1mg;
    float h = __ldg(&m->crest[warp_top ? 0 : 1]) * cosf(x * (0.5f * kPi));
    const float rs = __ldg(&m->rise[i * kMaxPatternDim + j]);
    if (rs != 0.0f) {
      const float t = (float)(warp_top ? sv : su) * kTwoNeg32;
      const float2 th = __ldg(&m->theta[i * kMaxPatternDim + j]);
      h += rs * (logf(cosf(th.x - th.y * t)) - __ldg(&m->lncos_incl));
    }
    return h;
  }
  const float s2 = (float)(warp_top ? sv : su) * kTwoNeg32;
  const float x = fminf(1.0f, fmaxf(-1.0f, (2.0f * s2 - 1.0f) * pm.inv_1mg));
  return __ldg(&m->crest[warp_top ? 1 : 0]) * (cosf(x * (0.5f * kPi)) - 1.0f);
}

__device__ bool visible(const DevMaterial *__restrict__ m, const PointMaterial &pm, uint32_t pu, uint32_t pv,
                        float3 w) {
  if (!(w.z > 0.0f)) return false;
  const float rho2 = w.x * w.x + w.y * w.y;
  if (rho2 == 0.0f) return true;
  const float rho = sqrtf(rho2);
  const float delta = __ldg(&m->v_delta);
  const uint32_t inc_u = (uint32_t)(unsigned long long)__float2ll_rn(w.x / rho * delta * 4294967296.0f);
  const uint32_t inc_v = (uint32_t)(unsigned long long)__float2ll_rn(w.y / rho * delta * 4294967296.0f);
  const float dz = delta * (w.z / rho);
  const float h0 = surface_height(m, pm, pu, pv);
  const float span = (__ldg(&m->h_max) - h0) / dz;
  int K = span < (float)kVisMaxSteps ? (int)floorf(span) + 1 : kVisMaxSteps;
  if (K < 1) K = 1;
  uint32_t qu = pu, qv = pv;
  for (int k = 1; k <= K; ++k) {
    qu += inc_u;
    qv += inc_v;
    if (surface_height(m, pm, qu, qv) > h0 + (float)k * dz) return false;
  }
  return true;
}

template <bool VIS>
__device__ __forceinline__ void shade_sample(const DevMaterial *__restrict__ m, const PointMaterial &pm,
                                             uint32_t pu, uint32_t pv, float3 wi, float3 wo, float3 h,
                                             bool h_ok, float diff_k, float diff_c, Sums &acc) {
  const uint32_t j = __umulhi(pu, pm.cols), su = pu * pm.cols;
  const uint32_t i = __umulhi(pv, pm.rows), sv = pv * pm.rows;
  const bool warp_top = (__ldg(&m->top[i]) >> j) & 1u;
  const uint32_t s_top = warp_top ? su : sv;
  const bool body = (s_top >= pm.gap) && (s_top <= 0xFFFFFFFFu - pm.gap);
  int yarn;
  float x, st, ct;
  if (body) {
    yarn = warp_top ? 0 : 1;
    const float s = (float)s_top * kTwoNeg32;
    const float t = (float)(warp_top ? sv : su) * kTwoNeg32;
    x = (2.0f * s - 1.0f) * pm.inv_1mg;
    const float2 th = __ldg(&m->theta[i * kMaxPatternDim + j]);
    const float theta = th.x - th.y * t;
    st = sin_half_pi(theta);
    ct = cos_half_pi(theta);
  } else {
    // gap of the top yarn: the yarn underneath shows, level, at its edge
    yarn = warp_top ? 1 : 0;
    const float s2 = (float)(warp_top ? sv : su) * kTwoNeg32;
    x = fminf(1.0f, fmaxf(-1.0f, (2.0f * s2 - 1.0f) * pm.inv_1mg));
    st = 0.0f;
    ct = 1.0f;
  }
  // cross-section slope of the height profile beta cos(pi x / 2)
  const float hc = (yarn ? pm.slope[1] : pm.slope[0]) * sin_half_pi(x * (0.5f * kPi));
  // n_p ~ cos(theta) (z - hc c) - sin(theta) a ; t0 = cos(theta) a + sin(theta) z
  float3 nv, t0;
  if (yarn == 0) {   // warp: a = +y, c = +x
    nv = make_float3(-hc * ct, -st, ct);
    t0 = make_float3(0.0f, ct, st);
  } else {           // weft: a = +x, c = +y
    nv = make_float3(-st, -hc * ct, ct);
    t0 = make_float3(ct, 0.0f, st);
  }
  const float inv = rsqrtf(nv.x * nv.x + nv.y * nv.y + nv.z * nv.z);
  const float3 n = make_float3(nv.x * inv, nv.y * inv, nv.z * inv);
  const float3 b = make_float3(n.y * t0.z - n.z * t0.y, n.z * t0.x - n.x * t0.z, n.x * t0.y - n.y * t0.x);
  const float3 tp = make_float3(pm.cos_psi * t0.x + pm.sin_psi * b.x, pm.cos_psi * t0.y + pm.sin_psi * b.y,
                                pm.cos_psi * t0.z + pm.sin_psi * b.z);
  const float ci = fmaxf(0.0f, wi.x * n.x + wi.y * n.y + wi.z * n.z);
  const float co = fmaxf(0.0f, wo.x * n.x + wo.y * n.y + wo.z * n.z);
  const float J = 1.0f / n.z;                      // 1 / <n_s . n_p>
  float coJ = co * J;
  bool lit = true;                                 // V(x_p, wi) V(x_p, wo)
  if (VIS && co > 0.0f) {
    // V(x_p, wo) weighs A and the numerators; V(x_p, wi) only matters with <wi.n_p> > 0
    if (!visible(m, pm, pu, pv, wo)) {
      coJ = 0.0f;
      lit = false;
    } else if (ci > 0.0f) {
      lit = visible(m, pm, pu, pv, wi);
    }
  }
  acc.a += coJ;                                    // A of Eq. 4
  if (VIS && !lit) return;
  const float diff = (diff_k * ci + diff_c) * ci * coJ;
  float spec = 0.0f;
  if (ci > 0.0f && co > 0.0f && h_ok) {
    const float tau = h.x * tp.x + h.y * tp.y + h.z * tp.z;
    const float q = 1.0f + tau * tau * (yarn ? pm.ia2m1[1] : pm.ia2m1[0]);
    const float D = (yarn ? pm.ipa[1] : pm.ipa[0]) / (q * q);   // 1 / (pi alpha q^2)
    const float ti = wi.x * tp.x + wi.y * tp.y + wi.z * tp.z;
    const float to = wo.x * tp.x + wo.y * tp.y + wo.z * tp.z;
    const float oma2 = yarn ? pm.oma2[1] : pm.oma2[0];
    const float si = sqrtf(fmaxf(0.0f, 1.0f - oma2 * ti * ti));
    const float so = sqrtf(fmaxf(0.0f, 1.0f - oma2 * to * to));
    const float X = si * co + so * ci;
    const float cc = ci * co;
    const float G = cc * (-expm1f(-2.0f * X / cc)) / X;   // Eq. 2, T rho = 2
    spec = D * G * 0.25f * J;
  }
  if (yarn == 0) {
    acc.c0 += diff;
    acc.s0 += spec;
  } else {
    acc.c1 += diff;
    acc.s1 += spec;
  }
}

struct RefArgs {
  const float *u, *v, *radius, *wi, *wo;
  const uint16_t *material;
  int64_t n;
  const DevMaterial *mats;
  int n_mat;
  int nx, ny, nx_log2;
  float two_over_nx, two_over_ny;
  uint64_t seed;
  float *rgb, *comps;
  int *status;
};

// Four CTAs per SM (64 registers): the V = 1 kernel needs no more, and with
// the visibility model the extra warps on the divergent marches outweigh a
// few spilled registers (73 -> 60 ms per 1080p frame at 256 spp, against 94
// registers unbounded).
template <int L, bool VIS>
__global__ void __launch_bounds__(256, 4) reference_kernel(const RefArgs a) {
  const int lane_g = threadIdx.x & (L - 1);
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L;
  const bool in_range = p < a.n;
  Sums acc = {0.f, 0.f, 0.f, 0.f, 0.f};
  int mat = 0;
  bool ok = false;
  if (in_range) {
    mat = a.material[p];
    ok = mat < a.n_mat;
    if (!ok && lane_g == 0) atomicOr(a.status, kStatusBadMaterial);
  }
  const DevMaterial *m = a.mats + (ok ? mat : 0);
  if (ok) {
    PointMaterial pm;
    pm.rows = m->rows;
    pm.cols = m->cols;
    pm.gap = m->gap_fixed;
    pm.inv_1mg = m->inv_one_minus_gap;
    pm.cos_psi = m->cos_psi;
    pm.sin_psi = m->sin_psi;
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      pm.slope[y] = m->slope_scale[y];
      pm.ia2m1[y] = m->inv_alpha2_minus1[y];
      pm.oma2[y] = m->one_minus_alpha2[y];
      pm.ipa[y] = m->inv_pi_alpha[y];
    }
    const float u = a.u[p], v = a.v[p], r = a.radius[p];
    const float3 wi = make_float3(a.wi[3 * p], a.wi[3 * p + 1], a.wi[3 * p + 2]);
    const float3 wo = make_float3(a.wo[3 * p], a.wo[3 * p + 1], a.wo[3 * p + 2]);
    float3 h = make_float3(wi.x + wo.x, wi.y + wo.y, wi.z + wo.z);
    const float hn2 = h.x * h.x + h.y * h.y + h.z * h.z;
    const bool h_ok = hn2 > 0.0f;
    if (h_ok) {
      const float hi = rsqrtf(hn2);
      h = make_float3(h.x * hi, h.y * hi, h.z * hi);
    }
    const float w = m->w_blend;
    const float diff_k = w / (kPi * fmaxf(wi.z, 1e-3f));
    const float diff_c = (1.0f - w) / kPi;
    const uint32_t cu = centre_fixed(u), cv = centre_fixed(v);
    const uint64_t hp = splitmix_finalise(a.seed + 0x9E3779B97F4A7C15ull * (uint64_t)(p + 1));
    const int spp = a.nx * a.ny;
    for (int k = lane_g; k < spp; k += L) {
      const uint64_t hk = splitmix_finalise(hp + (uint64_t)k);
      const float xi_x = (float)(uint32_t)(hk >> 40) * 5.9604644775390625e-08f;           // 2^-24
      const float xi_y = (float)(uint32_t)((hk >> 16) & 0xFFFFFFu) * 5.9604644775390625e-08f;
      int iy, ix;
      if (a.nx_log2 >= 0) {
        iy = k >> a.nx_log2;
        ix = k & (a.nx - 1);
      } else {
        iy = k / a.nx;
        ix = k - iy * a.nx;
      }
      const uint32_t pu = cu + offset_fixed(ix, xi_x, a.two_over_nx, r);
      const uint32_t pv = cv + offset_fixed(iy, xi_y, a.two_over_ny, r);
      shade_sample<VIS>(m, pm, pu, pv, wi, wo, h, h_ok, diff_k, diff_c, acc);
    }
  }
  // warp-level reduction inside each group of L lanes
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) {
    acc.c0 += __shfl_xor_sync(0xFFFFFFFFu, acc.c0, off);
    acc.c1 += __shfl_xor_sync(0xFFFFFFFFu, acc.c1, off);
    acc.s0 += __shfl_xor_sync(0xFFFFFFFFu, acc.s0, off);
    acc.s1 += __shfl_xor_sync(0xFFFFFFFFu, acc.s1, off);
    acc.a += __shfl_xor_sync(0xFFFFFFFFu, acc.a, off);
  }
  if (!in_range || lane_g != 0) return;
  float c[4];
  if (!ok) {
    c[0] = c[1] = c[2] = c[3] = __int_as_float(0x7FC00000);
  } else if (acc.a > 0.0f) {
    const float ia = 1.0f / acc.a;
    c[0] = acc.c0 * ia;
    c[1] = acc.c1 * ia;
    c[2] = acc.s0 * ia;
    c[3] = acc.s1 * ia;
  } else {
    c[0] = c[1] = c[2] = c[3] = 0.0f;
  }
  if (a.comps) store_row4(a.comps, p, c[0], c[1], c[2], c[3]);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float val = c[0];
    if (ok)
      val = m->kd[0][ch] * c[0] + m->kd[1][ch] * c[1] + m->ks[0][ch] * c[2] + m->ks[1][ch] * c[3];
    a.rgb[3 * p + ch] = val;
  }
}

}  // namespace

cudaError_t launch_reference(const fabric_gbuffer &g, const DevMaterial *mats, int n_mat, int spp_x, int spp_y,
                             uint64_t seed, float *rgb, float *comps, int *status, int lanes_per_point,
                             int sm_count, cudaStream_t s, bool visibility) {
  (void)sm_count;
  RefArgs a;
  a.u = g.u;
  a.v = g.v;
  a.radius = g.radius;
  a.wi = g.wi;
  a.wo = g.wo;
  a.material = g.material;
  a.n = g.n;
  a.mats = mats;
  a.n_mat = n_mat;
  a.nx = spp_x;
  a.ny = spp_y;
  a.nx_log2 = -1;
  for (int b = 0; b < 13; ++b)
    if ((1 << b) == spp_x) a.nx_log2 = b;
  a.two_over_nx = 2.0f / (float)spp_x;
  a.two_over_ny = 2.0f / (float)spp_y;
  a.seed = seed;
  a.rgb = rgb;
  a.comps = comps;
  a.status = status;
  const int threads = 256;
  const int64_t total = g.n * (int64_t)lanes_per_point;
  const unsigned blocks = (unsigned)((total + threads - 1) / threads);
  if (visibility) {
    switch (lanes_per_point) {
      case 1: reference_kernel<1, true><<<blocks, threads, 0, s>>>(a); break;
      case 2: reference_kernel<2, true><<<blocks, threads, 0, s>>>(a); break;
      case 4: reference_kernel<4, true><<<blocks, threads, 0, s>>>(a); break;
      case 8: reference_kernel<8, true><<<blocks, threads, 0, s>>>(a); break;
      case 16: reference_kernel<16, true><<<blocks, threads, 0, s>>>(a); break;
      default: reference_kernel<32, true><<<blocks, threads, 0, s>>>(a); break;
    }
    return cudaGetLastError();
  }
  switch (lanes_per_point) {
    case 1: reference_kernel<1, false><<<blocks, threads, 0, s>>>(a); break;
    case 2: reference_kernel<2, false><<<blocks, threads, 0, s>>>(a); break;
    case 4: reference_kernel<4, false><<<blocks, threads, 0, s>>>(a); break;
    case 8: reference_kernel<8, false><<<blocks, threads, 0, s>>>(a); break;
    case 16: reference_kernel<16, false><<<blocks, threads, 0, s>>>(a); break;
    default: reference_kernel<32, false><<<blocks, threads, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace fab
