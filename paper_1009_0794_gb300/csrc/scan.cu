// Exclusive prefix sum of per-ray counts into CSR row offsets: the step that
// replaces the paper's per-pixel depth-complexity readback (Section 3:
// n_p from the stencil buffer, then n_max = max n_p) with one device pass.
//
// One kernel per call: every block scans a chunk of kChunk counts (coalesced
// 16-byte loads), finds the chunk's starting offset by decoupled look-back
// over its predecessors, and writes its offsets.  All images of a call are
// scanned by the same launch (blockIdx.y = image).
#include <climits>

#include "ldni_host.h"
#include "lookback.cuh"

namespace ldni {
namespace {

constexpr int kThreads = 256;
constexpr int kVec = 4;                      // counts per 16-byte load
constexpr int kSlices = 4;                   // 16-byte loads per thread
constexpr int kSlice = kThreads * kVec;      // 1024 counts per slice
constexpr int kChunk = kSlice * kSlices;     // 4096 counts per block
static_assert(kChunk == kScanChunk, "chunk size is part of the scan's interface");

struct AxisPtrs {
    const int *counts[3];
    int *offsets[3];
    int2 *tinfo[3];
};

// 16-byte load when the address allows it (c + e aligned), scalar otherwise
__device__ __forceinline__ int4 load4(const int *c, long long e, long long N, bool vec) {
    if (vec && e + 3 < N) return *reinterpret_cast<const int4 *>(c + e);
    int4 v = make_int4(0, 0, 0, 0);
    if (e < N) v.x = c[e];
    if (e + 1 < N) v.y = c[e + 1];
    if (e + 2 < N) v.z = c[e + 2];
    if (e + 3 < N) v.w = c[e + 3];
    return v;
}

__device__ __forceinline__ int clamp_int(long long x) { return (int)(x < INT_MAX ? x : INT_MAX); }

__global__ void __launch_bounds__(kThreads) scan_lookback(AxisPtrs ap, long long N, int nchunk,
                                                          unsigned long long *words, ldni_info_t *info,
                                                          int info_base) {
    __shared__ long long sh[kThreads / 32 + 1];
    __shared__ int s_chunk;
    __shared__ long long s_base;
    const int a = blockIdx.y;
    unsigned long long *status = words + (long long)a * (nchunk + 1);
    unsigned long long *ticket = status + nchunk;
    if (threadIdx.x == 0) s_chunk = (int)atomicAdd(ticket, 1ull);
    __syncthreads();
    const int c = s_chunk;
    const int *cnt = ap.counts[a];
    int *out = ap.offsets[a];
    const long long base = (long long)c * kChunk;

    // e is a multiple of 4, so 16-byte access is legal iff the base is aligned
    const bool vec_in = ((reinterpret_cast<uintptr_t>(cnt) & 15) == 0);
    int4 v[kSlices];
    long long tsum[kSlices];
#pragma unroll
    for (int m = 0; m < kSlices; ++m) {
        v[m] = load4(cnt, base + (long long)m * kSlice + threadIdx.x * kVec, N, vec_in);
        tsum[m] = (long long)v[m].x + v[m].y + v[m].z + v[m].w;
    }
    long long excl[kSlices];
    long long carry = 0;
#pragma unroll
    for (int m = 0; m < kSlices; ++m) {
        long long tot;
        excl[m] = carry + block_exclusive_scan<kThreads>(tsum[m], sh, &tot);
        carry += tot;
    }
    if (threadIdx.x < 32) {
        const long long b = lookback_warp(status, c, carry, info);
        if (threadIdx.x == 0) s_base = b;
    }
    __syncthreads();
    const long long b0 = s_base;
    if (ap.tinfo[a] && threadIdx.x == 0) ap.tinfo[a][c] = make_int2(clamp_int(b0), clamp_int(carry));
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
#pragma unroll
    for (int m = 0; m < kSlices; ++m) {
        const long long e = base + (long long)m * kSlice + threadIdx.x * kVec;
        const long long o0 = b0 + excl[m];
        const int4 w = make_int4(clamp_int(o0), clamp_int(o0 + v[m].x), clamp_int(o0 + v[m].x + v[m].y),
                                 clamp_int(o0 + v[m].x + v[m].y + v[m].z));
        if (vec_ok && e + 3 < N) {
            *reinterpret_cast<int4 *>(out + e) = w;
        } else {
            if (e < N) out[e] = w.x;
            if (e + 1 < N) out[e + 1] = w.y;
            if (e + 2 < N) out[e + 2] = w.z;
            if (e + 3 < N) out[e + 3] = w.w;
        }
    }
    if (c == nchunk - 1 && threadIdx.x == 0) {
        const long long total = b0 + carry;
        if (info) info->n[info_base + a] = total;
        if (total > INT_MAX && info) atomicOr(&info->status, LDNI_ST_TOOLARGE);
        out[N] = clamp_int(total);
    }
}

__global__ void scan_empty(AxisPtrs ap, ldni_info_t *info, int info_base) {
    const int a = blockIdx.x;
    ap.offsets[a][0] = 0;
    if (info) info->n[info_base + a] = 0;
}

}  // namespace

size_t csr_scan_partials(long long N) {
    const long long n = (N + kChunk - 1) / kChunk;
    return (size_t)(n + 1);  // one status word per chunk + the ticket
}

int csr_scan(const int *const *counts, int *const *offsets, int naxes, long long N, long long *partials,
             ldni_info_t *info, int info_base, cudaStream_t s, int2 *const *tinfo) {
    AxisPtrs ap{};
    for (int a = 0; a < naxes; ++a) {
        ap.counts[a] = counts[a];
        ap.offsets[a] = offsets[a];
        ap.tinfo[a] = tinfo ? tinfo[a] : nullptr;
    }
    const int nchunk = (int)((N + kChunk - 1) / kChunk);
    if (nchunk == 0) {
        LDNI_LAUNCH(K_SCAN_TOP, s, scan_empty<<<naxes, 1, 0, s>>>(ap, info, info_base));
        return cuda_status();
    }
    unsigned long long *words = reinterpret_cast<unsigned long long *>(partials);
    if (cudaMemsetAsync(words, 0, sizeof(unsigned long long) * (size_t)(nchunk + 1) * naxes, s) != cudaSuccess)
        return LDNI_ECUDA;
    LDNI_LAUNCH(K_SCAN_DOWN, s,
                scan_lookback<<<dim3(nchunk, naxes), kThreads, 0, s>>>(ap, N, nchunk, words, info, info_base));
    return cuda_status();
}

}  // namespace ldni
