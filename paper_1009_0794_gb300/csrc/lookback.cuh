// Single-pass prefix sums across thread blocks by decoupled look-back: each
// block publishes its aggregate, then walks back over its predecessors'
// published words until it meets an inclusive prefix, and publishes its own
// inclusive prefix.  Blocks take their chunk index from a ticket counter, so
// a block only ever waits for blocks that are already running.  Every wait is
// bounded: after kSpinLimit polls the block records LDNI_ST_TIMEOUT in the
// call's info block and treats the missing word as zero, so the kernel always
// terminates (the result is then flagged as invalid, never silently wrong).
// The same bounded poll serves the self-test of ldni_wait_selftest.
#pragma once

#include <cstdint>

#include "ldni.h"

namespace ldni {

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;
// Polls of a look-back wait before it gives up: a kernel argument, from the
// process-wide setting of ldni_set_wait_limit (default kDefaultWaitPolls).

__device__ __forceinline__ unsigned long long ld_status(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ void st_status(unsigned long long *p, unsigned long long v) {
    atomicExch(p, v);  // value and flag travel in one 64-bit word
}

// Called by ALL 32 lanes of one warp (the same warp in every block).
// Returns, in every lane, the exclusive prefix of chunk `c` given its
// aggregate (>= 0).  One probe inspects 32 * P predecessors (each lane reads
// P consecutive words with independent loads): it waits until all of them
// have published something, adds the aggregates down to the nearest inclusive
// prefix, and moves on by a whole window if none was found.  Blocks of one wave finish their local work at about the same time,
// so a chunk usually walks back through its wave's chunks before any of them
// holds a prefix; a wide window keeps that walk to a few probes.
// A smaller P (words per lane) costs more probes and fewer registers.
constexpr int kLookbackPerLane = 8;

template <int P = kLookbackPerLane>
__device__ __forceinline__ long long lookback_warp(unsigned long long *status, int c, long long aggregate,
                                                   ldni_info_t *info, int spin_limit) {
    const int lane = threadIdx.x & 31;
    const unsigned long long agg = (unsigned long long)aggregate & kValueMask;
    if (c == 0) {
        if (lane == 0) st_status(status, kFlagPrefix | agg);
        return 0;
    }
    if (lane == 0) st_status(status + c, kFlagAgg | agg);
    long long excl = 0;
    int hi = c - 1;  // nearest predecessor not yet accounted for
    bool timed_out = false;
    while (hi >= 0) {
        // lane l holds chunks hi - l*P - j, j = 0 (nearest) .. P-1; before chunk 0: prefix 0
        unsigned long long w[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int k = hi - lane * P - j;
            w[j] = k >= 0 ? ld_status(status + k) : kFlagPrefix;
        }
        int spins = 0;
        while (true) {
            bool missing = false;
#pragma unroll
            for (int j = 0; j < P; ++j) missing |= (w[j] & ~kValueMask) == 0;
            if (!__any_sync(0xffffffffu, missing)) break;
            if (++spins > spin_limit) {
                timed_out = true;
                break;
            }
            __nanosleep(32);
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const int k = hi - lane * P - j;
                if ((w[j] & ~kValueMask) == 0) w[j] = ld_status(status + k);
            }
        }
        if (timed_out) break;
        // nearest inclusive prefix: the first j in the first lane that has one
        int jp = P;
#pragma unroll
        for (int j = P - 1; j >= 0; --j)
            if ((w[j] & ~kValueMask) == kFlagPrefix) jp = j;
        const unsigned prefix_lanes = __ballot_sync(0xffffffffu, jp < P);
        const int stop_lane = prefix_lanes ? __ffs(prefix_lanes) - 1 : 32;
        long long v = 0;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const bool take = lane < stop_lane || (lane == stop_lane && j <= jp);
            if (take) v += (long long)(w[j] & kValueMask);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (prefix_lanes) break;
        hi -= 32 * P;
    }
    if (timed_out && lane == 0 && info) atomicOr(&info->status, LDNI_ST_TIMEOUT);
    if (lane == 0) st_status(status + c, kFlagPrefix | (((unsigned long long)(excl + aggregate)) & kValueMask));
    return excl;
}

// Block-wide exclusive scan of one long long per thread (blockDim.x == NT,
// a multiple of 32, at most 1024).  Returns the exclusive prefix; *total gets
// the block sum.  `sh` holds at least NT/32 + 1 entries.
template <int NT>
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *sh, long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < NT / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) sh[lane] = w;
    }
    __syncthreads();
    const long long excl = x - v + (warp > 0 ? sh[warp - 1] : 0);
    *total = sh[NT / 32 - 1];
    __syncthreads();
    return excl;
}

// The same scan with a carry-in: every thread's prefix also holds the sum of
// carry[0 .. NT/32 - 1], one partial per warp, stored by the warps before the
// call (read after its first barrier).  Warp 0 scans the carry partials and
// then the warp totals as one list of 2 NT/32 values, so the carry costs no
// step of its own.  *total is the block's own sum, without the carry.
template <int NT>
__device__ __forceinline__ long long block_exclusive_scan_carry(long long v, const long long *carry, long long *sh,
                                                                long long *total) {
    constexpr int W = NT / 32;
    static_assert(2 * W <= 32, "carry partials and warp totals share one warp");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < W ? carry[lane] : (lane < 2 * W ? sh[lane - W] : 0);
#pragma unroll
        for (int o = 1; o < 2 * W; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane >= W && lane < 2 * W) sh[lane - W] = w;  // carry + warps 0 .. lane - W
        if (lane == W - 1) sh[W] = w;                     // the carry
    }
    __syncthreads();
    const long long excl = x - v + (warp > 0 ? sh[warp - 1] : sh[W]);
    *total = sh[W - 1] - sh[W];
    __syncthreads();
    return excl;
}

}  // namespace ldni
