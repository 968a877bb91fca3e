// decoder_blob.h -- byte layout of the tensor-core decoder's packed operands
// (folded first layer, layers 2-4, FP8 epilogue block, per-material
// albedos), identical in global and shared memory.  Compile-time so that
// every user of the layout can size its storage statically.
#pragma once

#include <cstddef>
#include <cstdint>

namespace fab {

constexpr int kKH = 80;   // K of 16-bit layers 2-4: 64 inputs + bias column + pad

// E4M3 epilogue block (FP32): per layer l = 0..3 a 64-entry bias row (row 0
// zero: layer 1's bias rides in its folded column; row 3 holds b4 and zeros)
// followed by the four unscaling factors (1 for layer 1).
constexpr int kF8Bias = 0;
constexpr int kF8Inv = 4 * 64;
constexpr uint32_t kF8EpiBytes = (4 * 64 + 4) * 4;

// Layer 1 of the tensor-core decoder has K = 39 query features + one
// one-hot bias column per material, padded to a multiple of 16; at most
// K = 128, i.e. 89 materials.
constexpr int kTcMaxMaterials = 128 - 39;

struct BlobLayout {
  int k1;
  uint32_t w1, w2, w3, w4, epi, alb, total;
};

__host__ __device__ constexpr BlobLayout blob_layout(int n_mat, int k1, bool f8) {
  BlobLayout L{};
  L.k1 = k1;
  L.w1 = 0;
  L.w2 = L.w1 + 64u * (uint32_t)k1 * 2u;
  if (f8) {
    L.w3 = L.w2 + 64u * 64u;
    L.w4 = L.w3 + 64u * 64u;
    L.epi = L.w4 + 16u * 64u;
    L.alb = L.epi + kF8EpiBytes;
  } else {
    L.w3 = L.w2 + 64u * kKH * 2u;
    L.w4 = L.w3 + 64u * kKH * 2u;
    L.epi = L.w4 + 16u * kKH * 2u;
    L.alb = L.epi;
  }
  L.total = L.alb + ((uint32_t)(n_mat * 12 * 4) + 15u) / 16u * 16u;
  return L;
}

// K of layer 1 for n_mat materials, or -1 beyond the decoder's limit.
constexpr int tc_k1_of(int n_mat) {
  return (n_mat >= 1 && n_mat <= kTcMaxMaterials) ? (39 + n_mat + 15) / 16 * 16 : -1;
}

// Largest packed blob over the precisions for n_mat materials.
constexpr size_t tc_blob_bytes_of(int n_mat) {
  const int k1 = tc_k1_of(n_mat) > 0 ? tc_k1_of(n_mat) : 128;
  const uint32_t a = blob_layout(n_mat, k1, false).total, b = blob_layout(n_mat, k1, true).total;
  return a > b ? a : b;
}

}  // namespace fab
