// paper_net.h -- parameter layout of the paper's decoder structure (Sec. 4.2,
// "Decoder"; Fig. 3): a spatial fusion of the material latent with the
// one-blob-encoded footprint (two layers), then an angular decoder of five
// layers with one skip, leaky ReLU; width W = 64 or 128.
//
// Flat FP32 parameters, weights [out][in]:
//   S1[W][88] s1[W] S2[W][W] s2[W] A1[W][W+5] a1[W] A2[W][W] a2[W]
//   A3[W][W] a3[W] A4[W][W] a4[W] A5[4][W] a5[4]
// S1's inputs are [z (64) | one-blob (24)], A1's are [h (W) | wi (3) | wo.xy (2)].
// Encoder: the workload's parameter encoder with a 64-wide latent,
//   E1[128][22] e1[128] E2[128][128] e2[128] E3[64][128] e3[64].
#pragma once

#include <cstdint>

namespace fab {

constexpr int kPnLatent = 64;
constexpr int kPnBins = 8;
constexpr int kPnBlob = 3 * kPnBins;   // one-blob channels of (frac u, frac v, size)
constexpr int kPnAng = 5;              // wi (x, y, z), wo (x, y)
constexpr float kPnSlope = 0.01f;      // leaky ReLU
// size coordinate t = ln(max(r, 2^-20) / 1e-4) / ln(2.5 / 1e-4)
constexpr float kPnLnRLo = -9.210340371976182f;     // ln 1e-4
constexpr float kPnInvLnSpan = 0.09874952387865506f; // 1 / ln(2.5e4)

struct PaperOffsets {
  int S1, s1, S2, s2, A1, a1, A2, a2, A3, a3, A4, a4, A5, a5, total;
};

__host__ __device__ constexpr PaperOffsets paper_offsets(int w) {
  PaperOffsets o{};
  o.S1 = 0;
  o.s1 = o.S1 + w * (kPnLatent + kPnBlob);
  o.S2 = o.s1 + w;
  o.s2 = o.S2 + w * w;
  o.A1 = o.s2 + w;
  o.a1 = o.A1 + w * (w + kPnAng);
  o.A2 = o.a1 + w;
  o.a2 = o.A2 + w * w;
  o.A3 = o.a2 + w;
  o.a3 = o.A3 + w * w;
  o.A4 = o.a3 + w;
  o.a4 = o.A4 + w * w;
  o.A5 = o.a4 + w;
  o.a5 = o.A5 + 4 * w;
  o.total = o.a5 + 4;
  return o;
}

// Ablations of the structure (Sec. 6.3): the spatial inputs unencoded
// (frac u, frac v, t: S1 becomes [W][67]), or no spatial fusion: the
// angular decoder gains two hidden layers in the fusion's place (the
// section adds hidden layers for a fair comparison), held in the S1, S2
// slots -- [W][93] over [z | one-blob | wi | wo.xy], then [W][W] -- and A1
// becomes [W][W] over their output (same size as the full structure).
constexpr int kPnFull = 0, kPnNoOneBlob = 1, kPnNoFusion = 2;

__host__ __device__ constexpr int paper_spatial_channels(int ablation) { return ablation == kPnNoOneBlob ? 3 : kPnBlob; }
// Inputs of the first layer, and of A1.
__host__ __device__ constexpr int paper_x0_inputs(int ablation) {
  return kPnLatent + paper_spatial_channels(ablation) + (ablation == kPnNoFusion ? kPnAng : 0);
}
__host__ __device__ constexpr int paper_a1_inputs(int w, int ablation) { return ablation == kPnNoFusion ? w : w + kPnAng; }

__host__ __device__ constexpr PaperOffsets paper_offsets_ablation(int w, int ablation) {
  PaperOffsets o{};
  o.S1 = 0;
  o.s1 = o.S1 + w * paper_x0_inputs(ablation);
  o.S2 = o.s1 + w;
  o.s2 = o.S2 + w * w;
  o.A1 = o.s2 + w;
  o.a1 = o.A1 + w * paper_a1_inputs(w, ablation);
  o.A2 = o.a1 + w;
  o.a2 = o.A2 + w * w;
  o.A3 = o.a2 + w;
  o.a3 = o.A3 + w * w;
  o.A4 = o.a3 + w;
  o.a4 = o.A4 + w * w;
  o.A5 = o.a4 + w;
  o.a5 = o.A5 + 4 * w;
  o.total = o.a5 + 4;
  return o;
}

static_assert(paper_offsets_ablation(64, kPnFull).A5 == paper_offsets(64).A5 &&
                  paper_offsets_ablation(128, kPnFull).total == paper_offsets(128).total,
              "the full structure's layout");

// Encoder with a 64-wide latent (same layout as the workload's encoder).
constexpr int kPnEncParams = 128 * 22 + 128 + 128 * 128 + 128 + kPnLatent * 128 + kPnLatent;

constexpr bool paper_width_ok(int w) { return w == 64 || w == 128; }

}  // namespace fab
