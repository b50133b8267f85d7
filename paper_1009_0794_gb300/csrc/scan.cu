// Exclusive prefix sum of per-ray counts into CSR row offsets: the step that
// replaces the paper's per-pixel depth-complexity readback (Section 3:
// n_p from the stencil buffer, then n_max = max n_p) with one device pass.
//
// Every block scans a chunk of kChunk counts (coalesced 16-byte loads) and
// writes its offsets; all images of a call share each launch (blockIdx.y =
// image).  A chunk's starting offset comes either from a first launch that
// sums every chunk (the second launch then adds the sums before its chunk,
// read directly: no block waits for another; used up to kMaxSumChunks chunks
// per image) or, for larger images, from decoupled look-back over its
// predecessors in one launch.
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
    ScanVerify ver;
    bool verify;
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

// ---- two-launch form (at most kMaxSumChunks chunks per image) -----------------
//
// Pass 1 sums every chunk; pass 2 gives every chunk the sum of the sums before
// it by reading them directly, so no block ever waits for another.
constexpr int kMaxSumChunks = 1024;
#ifndef LDNI_SCAN_ONE_LAUNCH
#define LDNI_SCAN_ONE_LAUNCH 0
#endif

__device__ __forceinline__ void load_chunk(const int *cnt, long long base, long long N, int4 (&v)[kSlices],
                                           long long (&tsum)[kSlices]) {
    const bool vec_in = ((reinterpret_cast<uintptr_t>(cnt) & 15) == 0);
#pragma unroll
    for (int m = 0; m < kSlices; ++m) {
        v[m] = load4(cnt, base + (long long)m * kSlice + threadIdx.x * kVec, N, vec_in);
        tsum[m] = (long long)v[m].x + v[m].y + v[m].z + v[m].w;
    }
}

// Two-layer check of one-pass sampling (ScanVerify) for chunk c of image a.
__device__ __forceinline__ void verify_chunk(const AxisPtrs &ap, int a, int c, long long base, long long N,
                                             const int4 (&v)[kSlices]) {
    if (!ap.verify || ap.ver.kcap[a][c] != 2) return;  // block-uniform
    const int *ex = ap.ver.exitc[a];
    const bool vec_ex = ((reinterpret_cast<uintptr_t>(ex) & 15) == 0);
    bool bad = false;
#pragma unroll
    for (int m = 0; m < kSlices; ++m) {
        const int4 x = load4(ex, base + (long long)m * kSlice + threadIdx.x * kVec, N, vec_ex);
        bad |= !(v[m].x == 0 || (v[m].x == 2 && x.x == 1));
        bad |= !(v[m].y == 0 || (v[m].y == 2 && x.y == 1));
        bad |= !(v[m].z == 0 || (v[m].z == 2 && x.z == 1));
        bad |= !(v[m].w == 0 || (v[m].w == 2 && x.w == 1));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) {
        ap.ver.over[a][c] = 1;
        *ap.ver.any_over = 1;
    }
}

constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ long long warp_sum(long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ long long warp_inclusive(long long x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// ---- one-launch form: decoupled look-back ---------------------------------------

__global__ void __launch_bounds__(kThreads, 6) scan_lookback(AxisPtrs ap, long long N, int nchunk,
                                                             unsigned long long *words, ldni_info_t *info,
                                                             int info_base, int spin_limit) {
    __shared__ long long sh[kSlices][kThreads / 32];  // per slice: warp totals
    __shared__ int4 sv[kSlices][kThreads];            // the chunk's counts, until the offsets are written
    __shared__ int s_chunk;
    __shared__ long long s_base;
    const int a = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long *status = words + (long long)a * (nchunk + 1);
    unsigned long long *ticket = status + nchunk;
    if (threadIdx.x == 0) s_chunk = (int)atomicAdd(ticket, 1ull);
    __syncthreads();
    const int c = s_chunk;
    int *out = ap.offsets[a];
    const long long base = (long long)c * kChunk;
    // as in scan_prefix: counts in shared memory, one 64-bit value per slice in registers, one
    // barrier for the chunk's scan
    long long xin[kSlices];
    {
        int4 v[kSlices];
        long long tsum[kSlices];
        load_chunk(ap.counts[a], base, N, v, tsum);
        verify_chunk(ap, a, c, base, N, v);
#pragma unroll
        for (int m = 0; m < kSlices; ++m) {
            sv[m][threadIdx.x] = v[m];
            const long long incl = warp_inclusive(tsum[m], lane);
            if (lane == 31) sh[m][warp] = incl;
            xin[m] = incl - tsum[m];
        }
    }
    __syncthreads();
    long long excl[kSlices];
    long long carry = 0;  // rays of the slices before m; at the end, the chunk's total
#pragma unroll
    for (int m = 0; m < kSlices; ++m) {
        long long lead = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            const long long t = sh[m][w];
            tot += t;
            if (w < warp) lead += t;
        }
        excl[m] = carry + lead + xin[m];
        carry += tot;
    }
    if (threadIdx.x < 32) {
        const long long b = lookback_warp<4>(status, c, carry, info, spin_limit);
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
        const int4 v = sv[m][threadIdx.x];  // this thread's own counts
        const int4 w = make_int4(clamp_int(o0), clamp_int(o0 + v.x), clamp_int(o0 + v.x + v.y),
                                 clamp_int(o0 + v.x + v.y + v.z));
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

// ---- two-launch form: the kernels ------------------------------------------------
//
// Each kernel meets at one barrier: warps reduce or scan with shuffles and
// leave one value per warp (and per slice) in shared memory, which every
// thread then adds up itself.

__global__ void __launch_bounds__(kThreads) scan_sums(AxisPtrs ap, long long N, int nchunk, long long *sums) {
    __shared__ long long sh[kWarps];
    const int a = blockIdx.y, c = blockIdx.x;
    const long long base = (long long)c * kChunk;
    int4 v[kSlices];
    long long tsum[kSlices];
    load_chunk(ap.counts[a], base, N, v, tsum);
    verify_chunk(ap, a, c, base, N, v);
    const long long ws = warp_sum(tsum[0] + tsum[1] + tsum[2] + tsum[3]);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = ws;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long total = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) total += sh[w];
        sums[(size_t)a * nchunk + c] = total;
    }
}

__global__ void __launch_bounds__(kThreads, 6) scan_prefix(AxisPtrs ap, long long N, int nchunk, const long long *sums,
                                                        ldni_info_t *info, int info_base) {
    __shared__ long long sh[kSlices + 1][kWarps];  // per slice: warp totals; last row: warp sums of `before`
    __shared__ int4 sv[kSlices][kThreads];          // the chunk's counts, until the offsets are written
    const int a = blockIdx.y, c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)c * kChunk;
    // Registers: the counts wait in shared memory and each slice keeps one 64-bit value (the
    // thread's exclusive prefix within its warp), so six blocks fit per SM and the chunks of
    // three 1024^2 images run in one wave.
    long long xin[kSlices];
    {
        int4 v[kSlices];
        long long tsum[kSlices];
        load_chunk(ap.counts[a], base, N, v, tsum);
#pragma unroll
        for (int m = 0; m < kSlices; ++m) {
            sv[m][threadIdx.x] = v[m];
            const long long incl = warp_inclusive(tsum[m], lane);
            if (lane == 31) sh[m][warp] = incl;
            xin[m] = incl - tsum[m];
        }
    }
    long long before = 0;  // this thread's share of the chunk sums before c
    for (int k = threadIdx.x; k < c; k += kThreads) before += sums[(size_t)a * nchunk + k];
    before = warp_sum(before);
    if (lane == 0) sh[kSlices][warp] = before;
    __syncthreads();
    long long b0 = 0;  // offset of the chunk's first ray
#pragma unroll
    for (int w = 0; w < kWarps; ++w) b0 += sh[kSlices][w];
    long long excl[kSlices];
    long long carry = 0;  // rays of the slices before m
#pragma unroll
    for (int m = 0; m < kSlices; ++m) {
        long long lead = 0, tot = 0;  // warps before this one in slice m; the whole slice
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const long long t = sh[m][w];
            tot += t;
            if (w < warp) lead += t;
        }
        excl[m] = carry + lead + xin[m];
        carry += tot;
    }
    int *out = ap.offsets[a];
    if (ap.tinfo[a] && threadIdx.x == 0) ap.tinfo[a][c] = make_int2(clamp_int(b0), clamp_int(carry));
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
#pragma unroll
    for (int m = 0; m < kSlices; ++m) {
        const long long e = base + (long long)m * kSlice + threadIdx.x * kVec;
        const long long o0 = b0 + excl[m];
        const int4 v = sv[m][threadIdx.x];  // this thread's own counts: no barrier needed
        const int4 w = make_int4(clamp_int(o0), clamp_int(o0 + v.x), clamp_int(o0 + v.x + v.y),
                                 clamp_int(o0 + v.x + v.y + v.z));
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
             ldni_info_t *info, int info_base, cudaStream_t s, int2 *const *tinfo, const ScanVerify *verify) {
    AxisPtrs ap{};
    if (verify) {
        ap.ver = *verify;
        ap.verify = true;
    }
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
    if (!LDNI_SCAN_ONE_LAUNCH && nchunk <= kMaxSumChunks) {
        LDNI_LAUNCH(K_SCAN_TOP, s, scan_sums<<<dim3(nchunk, naxes), kThreads, 0, s>>>(ap, N, nchunk, partials));
        LDNI_LAUNCH(K_SCAN_DOWN, s,
                    scan_prefix<<<dim3(nchunk, naxes), kThreads, 0, s>>>(ap, N, nchunk, partials, info, info_base));
        return cuda_status();
    }
    unsigned long long *words = reinterpret_cast<unsigned long long *>(partials);
    if (int rc_ = cuda_check(cudaMemsetAsync(words, 0, sizeof(unsigned long long) * (size_t)(nchunk + 1) * naxes, s))) return rc_;
    LDNI_LAUNCH(K_SCAN_DOWN, s,
                scan_lookback<<<dim3(nchunk, naxes), kThreads, 0, s>>>(ap, N, nchunk, words, info, info_base,
                                                                        wait_limit()));
    return cuda_status();
}

}  // namespace ldni
