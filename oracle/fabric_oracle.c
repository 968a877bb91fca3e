/*
 * fabric_oracle.c -- plain, slow FP64 CPU oracle for the footprint-filtered
 * woven-fabric reflectance of Chen, Wang and Wang, "Real-time Neural Woven
 * Fabric Rendering" (SIGGRAPH 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant generator
 * with the CUDA library; both follow the paper (and the readings listed in the
 * design notes) independently.
 *
 * What it computes, per query (u, v, r, wi, wo, material):
 *   f_P = (1/A_P) * integral over the footprint P of
 *           f_p(wi, wo) <wi . n_p> V A(p, wo) k_P(p) dp          (Eq. 3)
 *   A(p, wo) = <wo . n_p> / <n_s . n_p> * V                       (Eq. 4)
 *   A_P = integral of A k_P dp                                    (Eq. 5)
 * split into the four albedo-free components {C_warp, C_weft, S_warp,
 * S_weft} of Eq. 7 and recombined with the albedos by Eq. 8.  The shading
 * model f_p is the specular fibre-microflake term plus the blended Lambertian
 * term of Eq. 1, with D and G of Eq. 2 (S = diag(1,1,alpha^2) along the ply
 * direction t_p, T*rho = 2).  The footprint kernel k_P is a box over the
 * square [u-r, u+r] x [v-r, v+r] (Sec. 3.1 only requires it to integrate to 1);
 * the integral is estimated with n_x * n_y stratified samples, one per
 * stratum, jittered by a counter-based hash (SplitMix64, Steele, Lea and
 * Flood, OOPSLA 2014) so that the GPU path can draw the very same positions.
 * Every discrete decision (cell, gap, yarn type, float run) is taken in
 * integers on 32-bit fixed-point pattern coordinates; shading is FP64.
 *
 * The yarn geometry is not in the paper (it defers to its supplementary
 * material, Sec. 3.1); the reading implemented here is:
 *   - 1 uv unit = one pattern repeat; cell (i, j) = (floor(v R), floor(u C));
 *     P[i][j] = 1 means the warp yarn (running along v) is on top.
 *   - on top yarn: axis a, across direction c, across coordinate s, along
 *     coordinate t (warp: a = +y, c = +x, s = local u, t = local v; weft the
 *     other way round).  Body iff s in [g/2, 1 - g/2]; x = (2s-1)/(1-g).
 *     Otherwise the under-yarn shows, with its own across coordinate clamped
 *     to [-1, 1] and no inclination.
 *   - float position y = (o + t)/L on the maximal cyclic run of cells in
 *     which the yarn stays on top; inclination theta = u_incl (1 - 2y).
 *   - slopes dh/dc = -beta (pi/2) sin(pi x / 2) (height profile
 *     beta cos(pi x / 2)), dh/da = tan(theta).
 *   - n_p = normalize(z - dh/dc c - dh/da a); t0 = normalize(a + tan(theta) z);
 *     t_p = cos(psi) t0 + sin(psi) (n_p x t0).
 *   - V = 1 by default (inter-yarn shadowing is in the missing
 *     supplementary).  With visibility on, V is this build's proposed model
 *     (see "inter-yarn visibility" below): a ray march through the height
 *     field whose slopes the frame above uses.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Material record: 21 doubles per material, converted exactly from the       */
/* float32 inputs the caller generated.                                       */
/*   [0] pattern id  [1] twist psi (deg)  [2] inclination u (deg)             */
/*   [3] alpha_warp  [4] alpha_weft  [5] beta_warp  [6] beta_weft             */
/*   [7..9] kd_warp  [10..12] kd_weft  [13..15] ks_warp  [16..18] ks_weft     */
/*   [19] gap ratio g  [20] Lambertian blend weight w                          */
/* ------------------------------------------------------------------------- */
enum { M_PAT = 0, M_PSI, M_INCL, M_ALPHA_W, M_ALPHA_F, M_BETA_W, M_BETA_F,
       M_KD_W, M_KD_F = 10, M_KS_W = 13, M_KS_F = 16, M_GAP = 19, M_WBLEND = 20,
       M_STRIDE = 21 };

#define ORA_NPAT 12
#define ORA_MAXDIM 16

/* ---------------------------- weave patterns ----------------------------- */
/* Textile definitions of the twelve weaves; row i runs along v (weft index),*/
/* column j along u (warp index); 1 = warp over weft.                         */
static int pat_rows(int pid) {
  static const int R[ORA_NPAT] = {2, 3, 4, 5, 5, 4, 4, 4, 5, 8, 8, 10};
  return R[pid];
}
static int pat_cols(int pid) {
  static const int C[ORA_NPAT] = {2, 3, 4, 5, 5, 4, 8, 2, 5, 8, 8, 5};
  return C[pid];
}
static int imod(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }

static int pat_bit(int pid, int i, int j) {
  switch (pid) {
    case 0: return (i + j) % 2 == 0;                     /* plain */
    case 1: return imod(i - j, 3) < 2;                   /* 2/1 twill */
    case 2: return imod(i - j, 4) < 3;                   /* 3/1 twill */
    case 3: return imod(i - 2 * j, 5) != 0;              /* 4/1 satin, warp-faced */
    case 4: return imod(i - 3 * j, 5) == 0;              /* 5-harness satin, weft-faced */
    case 5: return ((i / 2) + (j / 2)) % 2 == 0;         /* 2x2 basket */
    case 6: return j < 4 ? imod(i - j, 4) < 2            /* herringbone: 2/2 twill */
                         : imod(i + j, 4) < 2;           /*   reversed at j = 4 */
    case 7: return ((i / 2) + j) % 2 == 0;               /* warp rib */
    case 8: return imod(i - j, 5) < 4;                   /* 4/1 twill (5 x 5) */
    case 9: return imod(i - j, 8) < 7;                   /* 7/1 twill (8 x 8) */
    case 10: return imod(i - 3 * j, 8) == 0;             /* 8-harness satin, weft-faced */
    case 11: return imod(i / 2 - 3 * j, 5) == 0;         /* 5-harness satin, picks doubled (10 x 5) */
  }
  return 0;
}

/* Float run of the yarn on top at (i, j): length L and offset o of the cell
 * inside the maximal cyclic run along that yarn's axis.                      */
static void pat_run(int pid, int i, int j, int *L, int *o) {
  const int R = pat_rows(pid), C = pat_cols(pid);
  const int top = pat_bit(pid, i, j);
  if (top) {                       /* warp on top: walk the column j along i */
    int all = 1;
    for (int k = 0; k < R; ++k) all &= pat_bit(pid, k, j);
    if (all) { *L = R; *o = i; return; }
    int start = i, len = 0;
    while (pat_bit(pid, imod(start - 1, R), j)) start = imod(start - 1, R);
    for (int k = 0; k < R && pat_bit(pid, imod(start + k, R), j); ++k) ++len;
    *L = len; *o = imod(i - start, R);
  } else {                         /* weft on top: walk the row i along j */
    int all = 1;
    for (int k = 0; k < C; ++k) all &= !pat_bit(pid, i, k);
    if (all) { *L = C; *o = j; return; }
    int start = j, len = 0;
    while (!pat_bit(pid, i, imod(start - 1, C))) start = imod(start - 1, C);
    for (int k = 0; k < C && !pat_bit(pid, i, imod(start + k, C)); ++k) ++len;
    *L = len; *o = imod(j - start, C);
  }
}

/* Exposed for the pattern pins: R, C, bits, run lengths and offsets. */
int ora_pattern_info(int pid, int *R, int *C, uint8_t *bits, uint8_t *runlen,
                     uint8_t *runoff) {
  if (pid < 0 || pid >= ORA_NPAT) return -1;
  *R = pat_rows(pid); *C = pat_cols(pid);
  for (int i = 0; i < *R; ++i)
    for (int j = 0; j < *C; ++j) {
      int L, o;
      pat_run(pid, i, j, &L, &o);
      bits[i * ORA_MAXDIM + j] = (uint8_t)pat_bit(pid, i, j);
      runlen[i * ORA_MAXDIM + j] = (uint8_t)L;
      runoff[i * ORA_MAXDIM + j] = (uint8_t)o;
    }
  return 0;
}

/* ------------------------------ small vectors ---------------------------- */
static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void normalize3(double *a) {
  double n = sqrt(dot3(a, a));
  a[0] /= n; a[1] /= n; a[2] /= n;
}
static void cross3(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------ SplitMix64 ------------------------------- */
#define ORA_GOLDEN 0x9E3779B97F4A7C15ULL
uint64_t ora_mix64(uint64_t z) {          /* SplitMix64 output finaliser */
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Gap threshold in 0.32 fixed point: floor((g/2) 2^32). */
static uint32_t gap_fixed(double g) { return (uint32_t)floor(0.5 * g * 4294967296.0); }

/* --------------------------- geometry (frame) ---------------------------- */
/* Frame at the pattern-space fixed-point position (pu, pv): visible yarn
 * (0 warp, 1 weft), ply normal n_p and ply orientation t_p.                   */
int ora_frame(const double *m, uint32_t pu, uint32_t pv, double *n_p, double *t_p) {
  const int pid = (int)m[M_PAT];
  const int R = pat_rows(pid), C = pat_cols(pid);
  const uint64_t wu = (uint64_t)pu * (uint64_t)C, wv = (uint64_t)pv * (uint64_t)R;
  const int j = (int)(wu >> 32), i = (int)(wv >> 32);
  const uint32_t su = (uint32_t)wu, sv = (uint32_t)wv;   /* local 0.32 coords */
  const double au = (double)su * 0x1p-32, av = (double)sv * 0x1p-32;
  const uint32_t G = gap_fixed(m[M_GAP]);
  const double g = m[M_GAP];
  const int warp_top = pat_bit(pid, i, j);

  /* across coordinate of the top yarn and its body test */
  const uint32_t s_top = warp_top ? su : sv;
  const int body = (s_top >= G) && (s_top <= 0xFFFFFFFFu - G);

  int yarn;               /* visible yarn: 0 warp, 1 weft */
  double x, theta;
  if (body) {
    yarn = warp_top ? 0 : 1;
    const double s = warp_top ? au : av, t = warp_top ? av : au;
    int L, o;
    pat_run(pid, i, j, &L, &o);
    x = (2.0 * s - 1.0) / (1.0 - g);
    const double y = ((double)o + t) / (double)L;
    theta = m[M_INCL] * (ORA_PI / 180.0) * (1.0 - 2.0 * y);
  } else {                /* gap of the top yarn: the under-yarn shows */
    yarn = warp_top ? 1 : 0;
    const double s2 = warp_top ? av : au;     /* under-yarn across coordinate */
    x = (2.0 * s2 - 1.0) / (1.0 - g);
    if (x < -1.0) x = -1.0;
    if (x > 1.0) x = 1.0;
    theta = 0.0;
  }
  const double beta = yarn == 0 ? m[M_BETA_W] : m[M_BETA_F];
  /* axis a and across c of the visible yarn */
  double a[3] = {0, 0, 0}, c[3] = {0, 0, 0};
  if (yarn == 0) { a[1] = 1.0; c[0] = 1.0; } else { a[0] = 1.0; c[1] = 1.0; }
  const double hc = -beta * (ORA_PI / 2.0) * sin(ORA_PI * x / 2.0);
  const double ha = tan(theta);
  double n[3], t0[3], nxt[3];
  for (int k = 0; k < 3; ++k) n[k] = -hc * c[k] - ha * a[k];
  n[2] += 1.0;
  normalize3(n);
  t0[0] = a[0]; t0[1] = a[1]; t0[2] = ha;
  normalize3(t0);
  cross3(n, t0, nxt);
  const double psi = m[M_PSI] * (ORA_PI / 180.0);
  for (int k = 0; k < 3; ++k) {
    n_p[k] = n[k];
    t_p[k] = cos(psi) * t0[k] + sin(psi) * nxt[k];
  }
  return yarn;
}

/* SGGX fibre distribution of Eq. 2 with S = I - (1 - alpha^2) t t^T:
 * q = h^T S^{-1} h = 1 - tau^2 + tau^2 / alpha^2, D = 1 / (pi alpha q^2).    */
double ora_sggx_D(double alpha, const double *t, const double *h) {
  const double tau = dot3(h, t);
  const double q = 1.0 - tau * tau + tau * tau / (alpha * alpha);
  return 1.0 / (ORA_PI * alpha * q * q);
}
/* projected area sigma(w) = sqrt(w^T S w) of Eq. 2 */
double ora_sggx_sigma(double alpha, const double *t, const double *w) {
  const double c = dot3(w, t);
  return sqrt(1.0 - (1.0 - alpha * alpha) * c * c);
}

/* ------------------------ inter-yarn visibility V ------------------------- */
/* A proposed model of the binary visibility V(x_p, w) of Eq. 3-5 (the paper
 * defers its own to the missing supplementary).  The surface is the height
 * field whose slopes the frame uses, in repeat units:
 *   top yarn body:  beta w cos(pi x / 2) + (L / N_a) (ln cos(u (1 - 2y)) - ln cos u) / (2 u)
 *                   (the cross-section, plus the float's rise: the integral of
 *                   tan(theta) along the float), w = (1 - g) / (2 N_c) the
 *                   half-width of the yarn, N_c / N_a the pattern size across /
 *                   along the yarn, u the inclination in radians;
 *   under a gap:    beta' w' (cos(pi x' / 2) - 1), the under-yarn, level, one
 *                   cross-section height below the top yarns' edges.
 * V(x_p, w) = 1 when the ray from (p, H(p)) along w stays above H at every
 * step of a march with horizontal step 1 / (16 max(R, C)) repeats, until it
 * rises above the largest height of the material (at most 4096 steps); 0
 * otherwise, and 0 for w below the horizon.  Step positions are integer
 * multiples of one rounded 0.32 fixed-point increment per ray.             */
#define ORA_V_STEPS_PER_CELL 16
#define ORA_V_MAX_STEPS 4096

static double hump(double incl, int L, int n_along, double y) {
  if (incl == 0.0) return 0.0;
  return (double)L / (double)n_along * (log(cos(incl * (1.0 - 2.0 * y))) - log(cos(incl))) / (2.0 * incl);
}

double ora_height(const double *m, uint32_t pu, uint32_t pv) {
  const int pid = (int)m[M_PAT];
  const int R = pat_rows(pid), C = pat_cols(pid);
  const uint64_t wu = (uint64_t)pu * (uint64_t)C, wv = (uint64_t)pv * (uint64_t)R;
  const int j = (int)(wu >> 32), i = (int)(wv >> 32);
  const uint32_t su = (uint32_t)wu, sv = (uint32_t)wv;
  const double au = (double)su * 0x1p-32, av = (double)sv * 0x1p-32;
  const uint32_t G = gap_fixed(m[M_GAP]);
  const double g = m[M_GAP];
  const int warp_top = pat_bit(pid, i, j);
  const uint32_t s_top = warp_top ? su : sv;
  const int body = (s_top >= G) && (s_top <= 0xFFFFFFFFu - G);
  if (body) {
    const int yarn = warp_top ? 0 : 1;
    const double s = warp_top ? au : av, t = warp_top ? av : au;
    const int n_across = yarn == 0 ? C : R, n_along = yarn == 0 ? R : C;
    const double w = (1.0 - g) / (2.0 * n_across);
    const double beta = yarn == 0 ? m[M_BETA_W] : m[M_BETA_F];
    int L, o;
    pat_run(pid, i, j, &L, &o);
    const double x = (2.0 * s - 1.0) / (1.0 - g);
    return beta * w * cos(ORA_PI * x / 2.0) + hump(m[M_INCL] * (ORA_PI / 180.0), L, n_along, ((double)o + t) / L);
  }
  const int under = warp_top ? 1 : 0;
  const double s2 = warp_top ? av : au;
  double x = (2.0 * s2 - 1.0) / (1.0 - g);
  if (x < -1.0) x = -1.0;
  if (x > 1.0) x = 1.0;
  const int n_across = under == 0 ? C : R;
  const double w = (1.0 - g) / (2.0 * n_across);
  const double beta = under == 0 ? m[M_BETA_W] : m[M_BETA_F];
  return beta * w * (cos(ORA_PI * x / 2.0) - 1.0);
}

/* Largest height of the material: the thicker yarn's crest plus the
 * highest float rise of the pattern (none for a negative inclination). */
double ora_height_max(const double *m) {
  const int pid = (int)m[M_PAT];
  const int R = pat_rows(pid), C = pat_cols(pid);
  const double g = m[M_GAP], incl = m[M_INCL] * (ORA_PI / 180.0);
  const double cw = m[M_BETA_W] * (1.0 - g) / (2.0 * C), cf = m[M_BETA_F] * (1.0 - g) / (2.0 * R);
  double rise = 0.0;
  for (int i = 0; i < R; ++i)
    for (int j = 0; j < C; ++j) {
      int L, o;
      pat_run(pid, i, j, &L, &o);
      const double r = hump(incl, L, pat_bit(pid, i, j) ? R : C, 0.5);
      if (r > rise) rise = r;
    }
  return (cw > cf ? cw : cf) + rise;
}

/* V(x_p, w) of the model above at the fixed-point position (pu, pv).  When
 * amb is given it is set to 1 if no step lies below the surface by more than
 * eps while some step lies within eps of it (a decision that rounding could
 * turn), else 0.                                                            */
int ora_visible(const double *m, uint32_t pu, uint32_t pv, const double *w, double eps, int *amb) {
  if (amb) *amb = 0;
  if (w[2] <= 0.0) return 0;
  const double rho = sqrt(w[0] * w[0] + w[1] * w[1]);
  if (rho == 0.0) return 1;
  const int pid = (int)m[M_PAT];
  const int R = pat_rows(pid), C = pat_cols(pid);
  const double delta = 1.0 / (ORA_V_STEPS_PER_CELL * (R > C ? R : C));
  const uint32_t inc_u = (uint32_t)(uint64_t)(int64_t)llrint(w[0] / rho * delta * 4294967296.0);
  const uint32_t inc_v = (uint32_t)(uint64_t)(int64_t)llrint(w[1] / rho * delta * 4294967296.0);
  const double dz = delta * (w[2] / rho);
  const double h0 = ora_height(m, pu, pv);
  const double span = (ora_height_max(m) - h0) / dz;
  int K = span < (double)ORA_V_MAX_STEPS ? (int)floor(span) + 1 : ORA_V_MAX_STEPS;
  if (K < 1) K = 1;
  int vis = 1, clear = 0, near = 0;
  uint32_t qu = pu, qv = pv;
  for (int k = 1; k <= K; ++k) {
    qu += inc_u;
    qv += inc_v;
    const double d = ora_height(m, qu, qv) - (h0 + k * dz);
    if (d > 0.0) vis = 0;
    if (d > eps) clear = 1;
    if (fabs(d) <= eps) near = 1;
  }
  if (amb) *amb = !clear && near;
  return vis;
}

/* Integrand of Eq. 3-5 at one point, with k_d = k_s = 1 (Eq. 7):
 * out[0..3] += numerators of (C_warp, C_weft, S_warp, S_weft); out[4] += A.
 * The Eq. 1 specular denominator 4 cos_i cos_o cancels against <wi.n_p> of
 * Eq. 3 and <wo.n_p> of Eq. 4; cosines are taken with respect to n_p.  With
 * `vis`, the numerators carry V(x_p, wi) V(x_p, wo) and A carries
 * V(x_p, wo); a visibility that cannot change the sums (wo with <wo.n_p> = 0,
 * wi with <wi.n_p> = 0) is not marched.  *amb |= an ambiguous march.       */
static void point_contrib(const double *m, uint32_t pu, uint32_t pv, const double *wi,
                          const double *wo, int vis, double eps, double *out, int *amb) {
  double n_p[3], t_p[3];
  const int yarn = ora_frame(m, pu, pv, n_p, t_p);
  const double ci = fmax(0.0, dot3(wi, n_p));
  const double co = fmax(0.0, dot3(wo, n_p));
  const double J = 1.0 / n_p[2];                     /* 1 / <n_s . n_p> */
  const double w = m[M_WBLEND];
  const double alpha = yarn == 0 ? m[M_ALPHA_W] : m[M_ALPHA_F];
  /* blended Lambertian of Eq. 1 (k_d = 1), <wi . n_s> clamped at 1e-3 */
  const double fd = w * ci / (ORA_PI * fmax(wi[2], 1e-3)) + (1.0 - w) / ORA_PI;
  const double s_diff = fd * ci * co * J;
  double s_spec = 0.0;
  if (ci > 0.0 && co > 0.0) {
    double h[3] = {wi[0] + wo[0], wi[1] + wo[1], wi[2] + wo[2]};
    const double hn = sqrt(dot3(h, h));
    if (hn > 0.0) {
      h[0] /= hn; h[1] /= hn; h[2] /= hn;
      const double D = ora_sggx_D(alpha, t_p, h);
      const double si = ora_sggx_sigma(alpha, t_p, wi);
      const double so = ora_sggx_sigma(alpha, t_p, wo);
      /* Eq. 2 with T rho = 2: G = (1 - exp(-2 (Li + Lo))) / (Li + Lo),
       * L = sigma / cos; written over the common denominator ci co.          */
      const double X = si * co + so * ci;
      const double G = ci * co * (-expm1(-2.0 * X / (ci * co))) / X;
      s_spec = D * G / 4.0 * J;
    }
  }
  double vi = 1.0, vo = 1.0;
  if (vis && co > 0.0) {
    int a1 = 0, a2 = 0;
    vo = ora_visible(m, pu, pv, wo, eps, &a1);
    if (vo > 0.0 && ci > 0.0) vi = ora_visible(m, pu, pv, wi, eps, &a2);
    if (amb) *amb |= a1 | a2;
  }
  out[yarn] += s_diff * vi * vo;
  out[2 + yarn] += s_spec * vi * vo;
  out[4] += co * J * vo;
}

void ora_point_contrib(const double *m, uint32_t pu, uint32_t pv, const double *wi,
                       const double *wo, double *out) {
  point_contrib(m, pu, pv, wi, wo, 0, 0.0, out, NULL);
}

/* --------------------------- sample positions ---------------------------- */
/* Fixed-point pattern coordinate of the footprint centre: frac(u) * 2^32. */
static uint32_t centre_fixed(float u) {
  const float f = u - floorf(u);
  return (uint32_t)(uint64_t)llrintf(f * 4294967296.0f);
}
/* Offset of stratum index k in [0, n) jittered by xi in [0,1), in FP32
 * round-to-nearest without contraction: ((k + xi) (2/n) - 1) r, then 0.32
 * fixed point rounded to nearest even.                                       */
static int64_t offset_fixed(int k, float xi, int n, float r) {
  volatile float t1 = (float)k + xi;
  volatile float t2 = t1 * (2.0f / (float)n);
  volatile float t3 = t2 - 1.0f;
  volatile float d = t3 * r;
  volatile float d32 = d * 4294967296.0f;
  return (int64_t)llrintf(d32);
}

/* Sample k of point `pixel`: stratum (k mod nx, k div nx), SplitMix64 jitter. */
void ora_sample_position(float u, float v, float r, int64_t pixel, int k, int nx,
                         int ny, uint64_t seed, uint32_t *pu, uint32_t *pv) {
  const uint64_t hp = ora_mix64(seed + ORA_GOLDEN * (uint64_t)(pixel + 1));
  const uint64_t h = ora_mix64(hp + (uint64_t)k);
  const float xi_x = (float)(uint32_t)(h >> 40) * 0x1p-24f;
  const float xi_y = (float)(uint32_t)((h >> 16) & 0xFFFFFFu) * 0x1p-24f;
  const int ix = k % nx, iy = k / nx;
  (void)ny;
  *pu = centre_fixed(u) + (uint32_t)(uint64_t)offset_fixed(ix, xi_x, nx, r);
  *pv = centre_fixed(v) + (uint32_t)(uint64_t)offset_fixed(iy, xi_y, ny, r);
}

/* --------------------------- footprint estimator ------------------------- */
static void shade_one(const double *mats, int n_mat, float u, float v, float r,
                      const float *wi_f, const float *wo_f, int mat, int64_t pixel,
                      int nx, int ny, uint64_t seed, int vis, double eps, double *comps,
                      double *rgb, uint8_t *amb) {
  double acc[5] = {0, 0, 0, 0, 0};
  if (mat < 0 || mat >= n_mat) {
    for (int k = 0; k < 4; ++k) comps[k] = NAN;
    for (int k = 0; k < 3; ++k) rgb[k] = NAN;
    return;
  }
  const double *m = mats + (size_t)mat * M_STRIDE;
  const double wi[3] = {wi_f[0], wi_f[1], wi_f[2]};
  const double wo[3] = {wo_f[0], wo_f[1], wo_f[2]};
  int a = 0;
  for (int k = 0; k < nx * ny; ++k) {
    uint32_t pu, pv;
    ora_sample_position(u, v, r, pixel, k, nx, ny, seed, &pu, &pv);
    point_contrib(m, pu, pv, wi, wo, vis, eps, acc, &a);
  }
  if (amb) *amb = (uint8_t)a;
  for (int k = 0; k < 4; ++k) comps[k] = acc[4] > 0.0 ? acc[k] / acc[4] : 0.0;
  for (int ch = 0; ch < 3; ++ch)   /* Eq. 8 */
    rgb[ch] = m[M_KD_W + ch] * comps[0] + m[M_KD_F + ch] * comps[1] +
              m[M_KS_W + ch] * comps[2] + m[M_KS_F + ch] * comps[3];
}

/* Supersampled footprint integral for n points (structure of arrays).  The
 * sample jitter of point p is keyed by its index in the full G-buffer:
 * pixel_index[p] when given (a subset of a larger buffer), else p.          */
void ora_shade_reference_vis(const double *mats, int n_mat, const float *u, const float *v,
                             const float *r, const float *wi, const float *wo,
                             const uint16_t *mat, int64_t n, int nx, int ny, uint64_t seed,
                             double *comps, double *rgb, int nthreads, const int64_t *pixel_index,
                             int vis, double eps, uint8_t *ambiguous) {
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
  for (int64_t p = 0; p < n; ++p)
    shade_one(mats, n_mat, u[p], v[p], r[p], wi + 3 * p, wo + 3 * p, (int)mat[p],
              pixel_index ? pixel_index[p] : p, nx, ny, seed, vis, eps, comps + 4 * p, rgb + 3 * p,
              ambiguous ? ambiguous + p : NULL);
  (void)nthreads;
}

/* The same with V = 1. */
void ora_shade_reference(const double *mats, int n_mat, const float *u, const float *v,
                         const float *r, const float *wi, const float *wo,
                         const uint16_t *mat, int64_t n, int nx, int ny, uint64_t seed,
                         double *comps, double *rgb, int nthreads, const int64_t *pixel_index) {
  ora_shade_reference_vis(mats, n_mat, u, v, r, wi, wo, mat, n, nx, ny, seed, comps, rgb, nthreads,
                          pixel_index, 0, 0.0, NULL);
}

/* Components at one fixed-point position (the point evaluation f_p <wi.n_p>
 * A / A of Eq. 3-5 at a single p, i.e. the r -> 0 limit).                    */
void ora_point_eval(const double *m, uint32_t pu, uint32_t pv, const double *wi,
                    const double *wo, double *comps) {
  double acc[5] = {0, 0, 0, 0, 0};
  ora_point_contrib(m, pu, pv, wi, wo, acc);
  for (int k = 0; k < 4; ++k) comps[k] = acc[4] > 0.0 ? acc[k] / acc[4] : 0.0;
}

/* Whole-period midpoint quadrature on a grid x grid lattice of fixed-point
 * positions: out[0..3] = period-average numerators, out[4] = average A.      */
void ora_period_quadrature(const double *m, const double *wi, const double *wo,
                           int grid, double *out, int nthreads) {
  for (int k = 0; k < 5; ++k) out[k] = 0.0;
  double tot[5] = {0, 0, 0, 0, 0};
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
  {
    double loc[5] = {0, 0, 0, 0, 0};
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
    for (int a = 0; a < grid; ++a) {
      double row[5] = {0, 0, 0, 0, 0};
      const uint32_t pv = (uint32_t)llrint(((double)a + 0.5) / (double)grid * 4294967296.0);
      for (int b = 0; b < grid; ++b) {
        const uint32_t pu = (uint32_t)llrint(((double)b + 0.5) / (double)grid * 4294967296.0);
        ora_point_contrib(m, pu, pv, wi, wo, row);
      }
      for (int k = 0; k < 5; ++k) loc[k] += row[k];
    }
#ifdef _OPENMP
#pragma omp critical
#endif
    for (int k = 0; k < 5; ++k) tot[k] += loc[k];
  }
  const double cells = (double)grid * (double)grid;
  for (int k = 0; k < 5; ++k) out[k] = tot[k] / cells;
  (void)nthreads;
}
