// Double-float sums for volumes: each FP32 difference is split exactly into
// a rounded value and its rounding error (TwoSum, Knuth, TAOCP vol. 2,
// 4.2.2), and sums are kept as unevaluated FP32 pairs (Dekker 1971), which
// keeps the per-ray work in FP32 (GB300 runs FP64 at a small fraction of its
// FP32 rate) while the sum stays within about 1e-13 relative of the exact one.
#pragma once

#include <cuda_runtime.h>

namespace ldni {

// s + e == a + b exactly (round-to-nearest FP32 arithmetic, no FMA)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF x, DF y) {
    float s, e;
    two_sum(x.hi, y.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    DF r;
    two_sum(s, e, r.hi, r.lo);
    return r;
}

// x + y keeping the rounding error of the high parts in the low part, without
// renormalising: 8 operations instead of df_add's 14.  For sums of many
// non-negative terms (inside lengths) the low part stays below 2^-24 of the
// high part per term, so the pair's value (hi + lo, taken in FP64 at the
// end) is within about 2^-47 of the exact sum.
__device__ __forceinline__ DF df_add_lazy(DF x, DF y) {
    float s, e;
    two_sum(x.hi, y.hi, s, e);
    return DF{s, __fadd_rn(__fadd_rn(x.lo, y.lo), e)};
}

// hi - lo as an exact pair
__device__ __forceinline__ DF df_diff(float hi, float lo) {
    DF d;
    two_sum(hi, -lo, d.hi, d.lo);
    return d;
}

// Block sum of one DF per thread in a fixed order (warp trees, then the
// warps in order); the result is valid in thread 0.  sh: NT / 32 entries.
template <int NT>
__device__ __forceinline__ DF df_block_sum(DF acc, DF *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF y{__shfl_down_sync(0xffffffffu, acc.hi, o), __shfl_down_sync(0xffffffffu, acc.lo, o)};
        acc = df_add(acc, y);
    }
    if (lane == 0) sh[warp] = acc;
    __syncthreads();
    DF t{0.0f, 0.0f};
    if (threadIdx.x == 0) {
        t = sh[0];
        for (int w = 1; w < NT / 32; ++w) t = df_add(t, sh[w]);
    }
    return t;
}

// FP64 sum of n partials in a fixed order by one block (strided per thread,
// then a fixed tree); valid in thread 0.  shd: NT entries.
template <int NT>
__device__ __forceinline__ double fixed_order_sum(const double *p, int n, double *shd) {
    constexpr int kU = 8;  // loads in flight per thread (L2 reads: written by other blocks)
    double sum = 0.0;
    for (int k0 = threadIdx.x; k0 < n; k0 += NT * kU) {
        double v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) v[u] = k0 + u * NT < n ? __ldcg(p + k0 + u * NT) : 0.0;
#pragma unroll
        for (int u = 0; u < kU; ++u) sum += v[u];
    }
    shd[threadIdx.x] = sum;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) shd[threadIdx.x] += shd[threadIdx.x + w];
        __syncthreads();
    }
    return shd[0];
}

}  // namespace ldni
