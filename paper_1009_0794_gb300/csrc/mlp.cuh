// The per-tile capacity network: 12 features -> 64 -> 64 -> 64 -> 1, ReLU on
// the hidden layers, BF16 weights, FP32 biases and FP32 accumulation.
//
// Parameter layout (shared by the C ABI, the training kernels and the CPU
// oracle): weights row-major [out][in], layers concatenated,
//   W0 [64][12] at 0, W1 [64][64] at 768, W2 [64][64] at 4864, W3 [1][64] at 8960
//   (9024 weights); biases b0[64] at 0, b1[64] at 64, b2[64] at 128, b3[1] at 192
//   (193 biases).
#pragma once

#include <cuda_bf16.h>

namespace ldni {

constexpr int kMlpIn = 12;
constexpr int kMlpHidden = 64;
constexpr int kMlpWeights = kMlpHidden * kMlpIn + 2 * kMlpHidden * kMlpHidden + kMlpHidden;  // 9024
constexpr int kMlpBiases = 3 * kMlpHidden + 1;                                              // 193
constexpr int kW0 = 0, kW1 = kMlpHidden * kMlpIn, kW2 = kW1 + kMlpHidden * kMlpHidden,
              kW3 = kW2 + kMlpHidden * kMlpHidden;
constexpr int kB0 = 0, kB1 = kMlpHidden, kB2 = 2 * kMlpHidden, kB3 = 3 * kMlpHidden;

// Raw tile feature accumulators (features kernel) and their normalised form.
// Every accumulator adds with an order-independent result, so the features,
// the capacities and a network trained on them are the same run to run:
// the count and the histogram bins add whole numbers (exact in FP32 below
// 2^24), and the area and the |n_a| sum are kept as unsigned fixed-point
// words (1/16 pixel, 1/256) in their float slots.
constexpr int kRawFeat = 11;  // count, area, sum |n_a|, 8-bin depth histogram
constexpr float kAreaFix = 16.0f, kNormalFix = 256.0f;

__device__ __forceinline__ unsigned to_fixed(float x, float scale) { return __float2uint_rn(x * scale); }

// x[0] log1p(count), x[1] log1p(area in pixels), x[2] mean |n_a|,
// x[3..10] depth histogram / count, x[11] fraction of the tile inside the image
__device__ __forceinline__ void normalise_features(const float *raw, float npix_frac, float *x) {
    const float c = raw[0];
    const float inv = c > 0.0f ? 1.0f / c : 0.0f;
    x[0] = log1pf(c);
    x[1] = log1pf((float)__float_as_uint(raw[1]) * (1.0f / kAreaFix));
    x[2] = (float)__float_as_uint(raw[2]) * (1.0f / kNormalFix) * inv;
#pragma unroll
    for (int k = 0; k < 8; ++k) x[3 + k] = raw[3 + k] * inv;
    x[11] = npix_frac;
}

// One forward pass for one feature row, by one thread (inference is one
// thread per tile; a few thousand tiles).
__device__ __forceinline__ float mlp_forward_row(const __nv_bfloat16 *__restrict__ W, const float *__restrict__ b,
                                                 const float *x) {
    float h0[kMlpHidden], h1[kMlpHidden];
    for (int o = 0; o < kMlpHidden; ++o) {
        float s = b[kB0 + o];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) s = fmaf(__bfloat162float(W[kW0 + o * kMlpIn + i]), x[i], s);
        h0[o] = fmaxf(s, 0.0f);
    }
    for (int o = 0; o < kMlpHidden; ++o) {
        float s = b[kB1 + o];
        for (int i = 0; i < kMlpHidden; ++i) s = fmaf(__bfloat162float(W[kW1 + o * kMlpHidden + i]), h0[i], s);
        h1[o] = fmaxf(s, 0.0f);
    }
    for (int o = 0; o < kMlpHidden; ++o) {
        float s = b[kB2 + o];
        for (int i = 0; i < kMlpHidden; ++i) s = fmaf(__bfloat162float(W[kW2 + o * kMlpHidden + i]), h1[i], s);
        h0[o] = fmaxf(s, 0.0f);
    }
    float y = b[kB3];
    for (int i = 0; i < kMlpHidden; ++i) y = fmaf(__bfloat162float(W[kW3 + i]), h0[i], y);
    return y;
}

}  // namespace ldni
