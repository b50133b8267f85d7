// Exclusive prefix sum of per-ray counts into CSR row offsets: the step that
// replaces the paper's per-pixel depth-complexity readback (Section 3:
// n_p from the stencil buffer) with one device scan.
//
// Three phases over chunks of kChunk counts: per-chunk totals, a scan of the
// totals per axis, then a per-chunk scan that adds the chunk's prefix.
#include <climits>

#include "ldni_host.h"

namespace ldni {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr int kChunk = kThreads * kPerThread;

struct AxisPtrs {
    const int *counts[3];
    int *offsets[3];
};

__device__ __forceinline__ long long block_sum(long long v, long long *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (kThreads / 32) ? sh[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kThreads) chunk_totals(AxisPtrs ap, long long N, int nchunk, long long *partials) {
    __shared__ long long sh[kThreads / 32];
    const int a = blockIdx.y;
    const int *c = ap.counts[a];
    const long long base = (long long)blockIdx.x * kChunk;
    long long s = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const long long i = base + (long long)k * kThreads + threadIdx.x;
        if (i < N) s += c[i];
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[(long long)a * nchunk + blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) scan_totals(AxisPtrs ap, long long N, int nchunk, long long *partials,
                                                     ldni_info_t *info, int info_base) {
    __shared__ long long sh[32];
    __shared__ long long carry;
    const int a = blockIdx.x;
    long long *P = partials + (long long)a * nchunk;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nchunk; base += 1024) {
        const int i = base + threadIdx.x;
        const long long v = i < nchunk ? P[i] : 0;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sh[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long w = sh[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            sh[lane] = w;
        }
        __syncthreads();
        const long long incl = x + (warp > 0 ? sh[warp - 1] : 0) + carry;
        if (i < nchunk) P[i] = incl - v;  // exclusive
        __syncthreads();
        if (threadIdx.x == 1023) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long total = carry;
        if (info) info->n[info_base + a] = total;
        if (total > INT_MAX) {
            if (info) atomicOr(&info->status, LDNI_ST_TOOLARGE);
        }
        ap.offsets[a][N] = (int)min(total, (long long)INT_MAX);
    }
}

__global__ void __launch_bounds__(kThreads) chunk_scan(AxisPtrs ap, long long N, int nchunk,
                                                       const long long *partials) {
    __shared__ long long sh[kThreads / 32];
    const int a = blockIdx.y;
    const int *c = ap.counts[a];
    int *out = ap.offsets[a];
    const long long base = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * kPerThread;
    int v[kPerThread];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const long long i = base + k;
        v[k] = i < N ? c[i] : 0;
        s += v[k];
    }
    // exclusive scan of per-thread sums across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < (kThreads / 32) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (kThreads / 32)) sh[lane] = w;
    }
    __syncthreads();
    long long run = partials[(long long)a * nchunk + blockIdx.x] + (x - s) + (warp > 0 ? sh[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const long long i = base + k;
        if (i < N) out[i] = (int)min(run, (long long)INT_MAX);
        run += v[k];
    }
}

}  // namespace

size_t csr_scan_partials(long long N) {
    const long long n = (N + kChunk - 1) / kChunk;
    return (size_t)(n > 0 ? n : 1);
}

int csr_scan(const int *const *counts, int *const *offsets, int naxes, long long N, long long *partials,
             ldni_info_t *info, int info_base, cudaStream_t s) {
    AxisPtrs ap{};
    for (int a = 0; a < naxes; ++a) {
        ap.counts[a] = counts[a];
        ap.offsets[a] = offsets[a];
    }
    const int nchunk = (int)((N + kChunk - 1) / kChunk);
    if (nchunk > 0)
        LDNI_LAUNCH(K_SCAN_CHUNK, s, chunk_totals<<<dim3(nchunk, naxes), kThreads, 0, s>>>(ap, N, nchunk, partials));
    LDNI_LAUNCH(K_SCAN_TOP, s, scan_totals<<<naxes, 1024, 0, s>>>(ap, N, nchunk, partials, info, info_base));
    if (nchunk > 0)
        LDNI_LAUNCH(K_SCAN_DOWN, s, chunk_scan<<<dim3(nchunk, naxes), kThreads, 0, s>>>(ap, N, nchunk, partials));
    return cuda_status();
}

}  // namespace ldni
