// Per-ray Boolean of two LDNIs on one grid (Section 4.1) with small-interval
// removal (Section 4.1.1).
//
// The paper slices A's segments by B's samples and keeps, merges or removes
// segments per operation.  Restated as a merge of two sorted sample lists
// with inside-counters: walking the distinct depths in order, every sample
// toggles its solid's state (odd-to-even ranges are inside, Section 2);
// equal depths of A and B are one event; the output state op(inA, inB)
// changes exactly at the result's boundary samples.  An emitted sample is
// A's when A's state flipped at that depth, else B's (normal inverted for a
// difference, Section 4.1).  Entering samples wait in registers until their
// exit is known, so an interval thinner than eps is dropped without a second
// pass over the output.
//
// Three forms share that merge:
//   - one launch per image (bool_tiled): a block stages its tile's sample
//     arrays in shared memory with bulk copies, counts its rays, scans,
//     finds its first output slot by decoupled look-back and writes;
//   - two launches per image (bool_count, bool_write): no block ever waits
//     for another; a write tile's first output slot is the sum of the tile
//     and super-tile totals before it, read directly; the result's volume,
//     when asked for, is summed by the count pass and finished by the last
//     write block of the image;
//   - the two-pass form behind ldni_boolean_static (bool_pass + csr_scan).
// Launch shapes are chosen by the tuning knobs (ldni_set_tuning).
#include <climits>
#include <mutex>

#include <cuda.h>

#include "bulk.cuh"
#include "dfloat.cuh"
#include "ldni_host.h"
#include "lookback.cuh"
#include "merge.cuh"

namespace ldni {
namespace {

constexpr int kThreads = 256;
constexpr int kBoolThreads = 256;

// Normals are FP32 in nx, ny, nz, or packed 8-bit words in nx with ny = nz =
// nullptr (Section 3 item 1); the operands and the output of a call share the
// format.  An inverted packed normal has every code q replaced by 255 - q.
struct Side {
    long long cap;  // samples beyond capacity are never read
    const int *off;
    const float *d;
    const float *nx;
    const float *ny;
    const float *nz;
    const int *tri;
};

struct Out {
    const int *off;
    float *d;
    float *nx;
    float *ny;
    float *nz;
    int *tri;
    long long cap;
};

// Elements i, i + 1 of a 4-byte array as one 8-byte access (i even, the
// array 8-byte aligned).
template <class T>
__device__ __forceinline__ uint2 ld_pair(const T *a, long long i) {
    return *reinterpret_cast<const uint2 *>(a + i);
}
template <class T>
__device__ __forceinline__ void st_pair(T *a, long long i, uint2 v) {
    *reinterpret_cast<uint2 *>(a + i) = v;
}

// The images of one call: job j is out[j] = A[j] op B[j], all on one grid.
// Kernels take it as a __grid_constant__ parameter and index it by job.
constexpr int kMaxJobs = LDNI_MAX_IMAGES;
struct BoolJobs {
    Side A[kMaxJobs];
    Side B[kMaxJobs];
    Out o[kMaxJobs];
    ldni_info_t *info[kMaxJobs];
    double *vol[kMaxJobs];  // optional: volume of each result
    bool packed;            // 8-bit normals (one word) instead of FP32 nx, ny, nz, for every image of the call
    bool pairs8;            // every sample array of the call 8-byte aligned: a pair at an even index is one 8-byte access
};

// One output sample at slot `at` from sample idx of A or B.
__device__ __forceinline__ void emit_global(bool from_b, long long idx, const Side &A, const Side &B, int op,
                                            const Out &o, long long at, ldni_info_t *info) {
    if (at >= o.cap) {
        set_status(info, LDNI_ST_CAPACITY);
        return;
    }
    if (!from_b) {
        o.d[at] = A.d[idx];
        o.nx[at] = A.nx[idx];
        if (o.ny) {
            o.ny[at] = A.ny[idx];
            o.nz[at] = A.nz[idx];
        }
        o.tri[at] = A.tri[idx];
    } else {
        const bool inv = op == LDNI_OP_DIFF;
        const float sg = inv ? -1.0f : 1.0f;
        o.d[at] = B.d[idx];
        if (o.ny) {
            o.nx[at] = sg * B.nx[idx];
            o.ny[at] = sg * B.ny[idx];
            o.nz[at] = sg * B.nz[idx];
        } else {
            o.nx[at] = __uint_as_float(__float_as_uint(B.nx[idx]) ^ (inv ? kInvert8 : 0u));
        }
        o.tri[at] = (int)((unsigned)B.tri[idx] | 0x80000000u);
    }
}

__device__ __forceinline__ void finish_output(const Out &o, long long N, long long n_out, ldni_info_t *info) {
    const_cast<int *>(o.off)[N] = (int)min(n_out, (long long)INT_MAX);
    info->n[0] = n_out;
    if (n_out > INT_MAX) set_status(info, LDNI_ST_TOOLARGE);
    if (n_out > o.cap) set_status(info, LDNI_ST_CAPACITY);
}

// Ray kinds answered without the general merge: 1 = A alone, entering and
// leaving once; 2 = B alone, likewise.  Their interval is kept unless it is
// empty (both samples at one depth cancel) or thinner than eps; it belongs to
// a union, to a difference only from A, and to no intersection.  4 = one
// interval in each operand (two_two).  0 = no samples, 3 = anything else.
__device__ __forceinline__ int ray_kind(long long na, long long nb) {
    if ((na | nb) == 0) return 0;
    if (nb == 0 && na == 2) return 1;
    if (na == 0 && nb == 2) return 2;
    if (na == 2 && nb == 2) return 4;
    return 3;
}

// merge_core in closed form for one interval [a0, a1] of A and [b0, b1] of B
// (same events, same tie rules: at a shared depth A's sample is the one
// emitted, touching intervals of a union merge, a zero-length interval
// cancels).  Returns the output count; bits 2k, 2k + 1 of *src name output
// k's source (src_of): 0, 1 = A's first, second sample; 2, 3 = B's.  The
// sources travel packed in one register, not in an indexed array, which
// would live in local memory.
__device__ __forceinline__ int src_of(unsigned src, int k) { return (int)(src >> (2 * k)) & 3; }

// A ray that takes the general merge: more than one interval in an operand,
// or rows beyond an operand's capacity (then clamped to it).
__device__ __forceinline__ bool general_ray(int a, int ae, int b, int be, int capA, int capB) {
    const int na = ae - a, nb = be - b;
    return ae > capA || be > capB || !((na == 0 || na == 2) && (nb == 0 || nb == 2));
}

// Bit s set when one of the first c outputs copies sample s.
__device__ __forceinline__ unsigned src_needs(unsigned src, int c) {
    unsigned need = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (m < c) need |= 1u << src_of(src, m);
    return need;
}

// The count pass's word of a ray in closed form (not general_ray): the count
// (at most 4) in the low bits, the outputs' sources from bit kSrcShift on.
// A general ray's word is its count.
constexpr int kSrcShift = 3;

// v[i] of four values a0, a1, b0, b1, without an indexed array
__device__ __forceinline__ float pick4(int i, float a0, float a1, float b0, float b1) {
    return i < 2 ? (i ? a1 : a0) : (i == 2 ? b0 : b1);
}
__device__ __forceinline__ uint32_t pick4u(int i, uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1) {
    return i < 2 ? (i ? a1 : a0) : (i == 2 ? b0 : b1);
}

// The ends of the kept intervals, in order (x0, y0), (x1, y1), come back in *ends.
struct Ends {
    float x0, y0, x1, y1;
};

__device__ __forceinline__ int two_two(int op, float eps, float a0, float a1, float b0, float b1, unsigned &src,
                                       Ends *ends = nullptr) {
    int n = 0;
    src = 0;
    auto put = [&](int s0, int s1, float d0, float d1) {
        if (!(__fsub_rn(d1, d0) < eps)) {
            src |= (unsigned)(s0 | (s1 << 2)) << (2 * n);
            if (ends) {
                if (n == 0) {
                    ends->x0 = d0;
                    ends->y0 = d1;
                } else {
                    ends->x1 = d0;
                    ends->y1 = d1;
                }
            }
            n += 2;
        }
    };
    const bool za = a0 == a1, zb = b0 == b1;
    if (za || zb) {
        if (!zb && op == LDNI_OP_UNION) put(2, 3, b0, b1);  // A cancels: B alone
        if (!za && zb && op != LDNI_OP_INTER) put(0, 1, a0, a1);  // B cancels: A alone
        return n;
    }
    if (op == LDNI_OP_UNION) {
        if (a1 < b0) {
            put(0, 1, a0, a1);
            put(2, 3, b0, b1);
        } else if (b1 < a0) {
            put(2, 3, b0, b1);
            put(0, 1, a0, a1);
        } else {
            const bool in_a = !(b0 < a0), out_a = !(a1 < b1);
            put(in_a ? 0 : 2, out_a ? 1 : 3, in_a ? a0 : b0, out_a ? a1 : b1);
        }
    } else if (op == LDNI_OP_INTER) {
        const bool in_a = !(a0 < b0), out_a = !(b1 < a1);
        const float lo = in_a ? a0 : b0, hi = out_a ? a1 : b1;
        if (lo < hi) put(in_a ? 0 : 2, out_a ? 1 : 3, lo, hi);
    } else {  // A \ B: the parts of A before B and after B
        if (a0 < b0) {
            const bool out_a = !(b0 < a1);
            put(0, out_a ? 1 : 2, a0, out_a ? a1 : b0);
        }
        if (b1 < a1) {
            const bool in_a = !(a0 < b1);
            put(in_a ? 0 : 3, 1, in_a ? a0 : b1, a1);
        }
    }
    return n;
}

__device__ __forceinline__ int two_count(int kind, int op, float d0, float d1, float eps) {
    if (op == LDNI_OP_INTER || (kind == 2 && op == LDNI_OP_DIFF)) return 0;
    return (d0 == d1 || __fsub_rn(d1, d0) < eps) ? 0 : 2;
}

// merge_core with kinds 1 and 2 answered directly.
template <class Idx, class EmitF>
__device__ __forceinline__ int merge_ray_fast(const float *dA, Idx a, Idx ae, const float *dB, Idx b, Idx be, int op,
                                              float eps, EmitF emit) {
    const int kind = ray_kind(ae - a, be - b);
    if (kind == 1 || kind == 2) {
        const float *d = kind == 1 ? dA : dB;
        const Idx i = kind == 1 ? a : b;
        const int c = two_count(kind, op, d[i], d[i + 1], eps);
        if (c) emit(kind == 2, i, kind == 2, i + 1, 0);
        return c;
    }
    if (kind == 4) {
        unsigned src;
        const int c = two_two(op, eps, dA[a], dA[a + 1], dB[b], dB[b + 1], src);
        for (int k = 0; k < c; k += 2) {
            const int s0 = src_of(src, k), s1 = src_of(src, k + 1);
            emit(s0 >= 2, (s0 >= 2 ? b : a) + (s0 & 1), s1 >= 2, (s1 >= 2 ? b : a) + (s1 & 1), k);
        }
        return c;
    }
    return merge_core<Idx>(dA, a, ae, dB, b, be, op, eps, emit);
}

// ---- two-pass form (ldni_boolean_static) ------------------------------------

template <bool kWrite>
__global__ void __launch_bounds__(kThreads) bool_pass(long long nrays, Side A, Side B, int op, float eps,
                                                      int *out_count, Out o, ldni_info_t *info) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nrays;
         p += (long long)gridDim.x * blockDim.x) {
        long long a = A.off[p];
        long long ae = A.off[p + 1];
        long long b = B.off[p];
        long long be = B.off[p + 1];
        if (!kWrite && (((ae - a) | (be - b)) & 1)) {
            atomicAdd(&info->odd_rays, 1u);
            set_status(info, LDNI_ST_ODD);
        }
        if (ae > A.cap || be > B.cap) {
            // an operand whose samples were cut off by its own capacity
            set_status(info, LDNI_ST_CAPACITY);
            ae = min(ae, A.cap);
            be = min(be, B.cap);
            a = min(a, ae);
            b = min(b, be);
        }
        if (!kWrite) {
            out_count[p] = merge_ray_fast<long long>(A.d, a, ae, B.d, b, be, op, eps, NoEmit{});
        } else {
            const long long base = o.off[p];
            merge_ray_fast<long long>(A.d, a, ae, B.d, b, be, op, eps,
                                      [&](bool pb, long long pi, bool cb, long long ci, int m) {
                                          emit_global(pb, pi, A, B, op, o, base + m, info);
                                          emit_global(cb, ci, A, B, op, o, base + m + 1, info);
                                      });
        }
    }
}

// ---- one launch per image, tile staged in shared memory ------------------------
//
// One block owns a tile of kR * 256 consecutive rays; thread t owns the kR
// consecutive rays t*kR .. t*kR + kR - 1, so one block scan orders the tile
// and offsets move as vectors.  The samples of the tile are contiguous in
// both operands (CSR rows in ray order): one thread copies the two ranges of
// every sample array (depths, normals, triangle ids) into shared memory with
// asynchronous bulk copies, the depths on one barrier and the rest on
// another, so the normals are still landing while the block merges.  The
// block then
//   1. counts every ray's output samples from the staged depths,
//   2. scans the counts, obtains the tile's first output slot by decoupled
//      look-back and writes the tile's CSR offsets,
//   3. merges again, recording for each output sample its source (operand
//      and index) in shared memory, and sums the result's inside lengths
//      when the volume is asked for,
//   4. writes the tile's output samples in order from shared memory;
//      consecutive threads write consecutive samples.
// A tile whose two ranges exceed the shared-memory budget (or a budget of 0)
// merges every ray from global memory instead; results are the same.  When
// an array does not start on a 16-byte boundary, the staging uses plain
// loads instead of bulk copies.
constexpr int kStageUnroll = 8;  // staged loads in flight per thread (plain staging)
constexpr int kGather = 4;       // output samples written per thread and step

__device__ __forceinline__ int clamp_local(long long x, long long cap_rel) {  // x >= 0
    return cap_rel < 0 ? 0 : (int)min(x, cap_rel);
}

// Copy elements [g0, g1) of a 4-byte array to dst[i - floor4(g0)] with plain
// loads, kStageUnroll in flight per thread.
__device__ __forceinline__ void stage_plain(const uint32_t *__restrict__ src, long long g0, long long g1,
                                            uint32_t *dst) {
    const long long s = g0 & ~3ll;
    const int n = (int)(g1 - g0), off = (int)(g0 - s);
    for (int k0 = threadIdx.x; k0 < n; k0 += kBoolThreads * kStageUnroll) {
        uint32_t v[kStageUnroll];
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
            const int k = k0 + u * kBoolThreads;
            v[u] = k < n ? src[g0 + k] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
            const int k = k0 + u * kBoolThreads;
            if (k < n) dst[off + k] = v[u];
        }
    }
}

// Rows of rays q .. q + kR (rows past the tile's end repeat its end).
template <int kR>
__device__ __forceinline__ void load_rows(const int *off, long long p0, int q, int nr, int (&r)[kR + 1]) {
    if (kR >= 4 && (reinterpret_cast<uintptr_t>(off) & 15) == 0 && q + kR <= nr) {
#pragma unroll
        for (int v = 0; v < kR; v += 4) {
            const int4 x = *reinterpret_cast<const int4 *>(off + p0 + q + v);
            r[v] = x.x; r[v + 1] = x.y; r[v + 2] = x.z; r[v + 3] = x.w;
        }
        r[kR] = off[p0 + q + kR];
    } else {
#pragma unroll
        for (int k = 0; k <= kR; ++k) r[k] = off[p0 + min(q + k, nr)];
    }
}

// kR ints of this thread to a[p0 + q ..], as 16-byte stores when possible.
template <int kR>
__device__ __forceinline__ void store_rows(int *dst, long long p0, int q, int nr, const int (&w)[kR]) {
    if (kR >= 4 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0 && q + kR <= nr) {
#pragma unroll
        for (int v = 0; v < kR; v += 4)
            *reinterpret_cast<int4 *>(dst + p0 + q + v) = make_int4(w[v], w[v + 1], w[v + 2], w[v + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < kR; ++k)
            if (q + k < nr) dst[p0 + q + k] = w[k];
    }
}

// The staged copy of one operand's tile range: array k (0 depth, then the
// normal arrays, last the triangle ids) at arr(k), element i of the range
// (tile-local) at arr(k)[off + i].
struct StagedSide {
    uint32_t *base;  // array k at base + k * stride
    int stride;
    int narr;  // 5 (FP32 normals) or 3 (packed normals)
    int off;
    __device__ __forceinline__ uint32_t *arr(int k) const { return base + k * stride; }
    __device__ __forceinline__ const float *d() const { return reinterpret_cast<const float *>(base) + off; }
};

template <int kR>
struct TileIn {
    int la[kR + 1], lb[kR + 1];  // rows q0 .. q0 + kR, tile-local and clamped to capacity
    unsigned odd;                // bit k: ray q0 + k has an odd count in A or B
    long long ga0, gb0;          // first kept sample of the tile
    int LA, LB;                  // kept samples of the tile
    bool staged;
    StagedSide sa, sb;
};

__device__ __forceinline__ const uint32_t *side_array(const Side &S, int k, int narr) {
    if (k == 0) return reinterpret_cast<const uint32_t *>(S.d);
    if (k == narr - 1) return reinterpret_cast<const uint32_t *>(S.tri);
    return reinterpret_cast<const uint32_t *>(k == 1 ? S.nx : (k == 2 ? S.ny : S.nz));
}

// Rows of this thread's rays and the tile's sample ranges; if they fit the
// budget, the staging of every sample array is started: depths complete on
// bars[0], the other arrays on bars[1] (bulk copies when `bulk`, else plain
// loads, complete on return).  Ends with a barrier after which the depths
// are in shared memory (or the tile is not staged).  False when a bounded
// wait gave up (LDNI_ST_TIMEOUT recorded).
template <int kR>
__device__ __forceinline__ bool tile_prologue(const Side &A, const Side &B, long long p_begin, int nr, int budget,
                                              int narr, bool bulk, uint32_t *stage, uint64_t *bars, long long *sh4,
                                              TileIn<kR> &T, ldni_info_t *info) {
    const int q0 = threadIdx.x * kR;
    int ra[kR + 1], rb[kR + 1];
    load_rows<kR>(A.off, p_begin, q0, nr, ra);
    load_rows<kR>(B.off, p_begin, q0, nr, rb);
    if (threadIdx.x == 0) {
        sh4[0] = ra[0];
        sh4[1] = rb[0];
        if (bulk) {
            mbar_init(bars, 1);
            mbar_init(bars + 1, 1);
        }
    }
    if (q0 < nr && q0 + kR >= nr) {  // this thread holds the tile's end row
#pragma unroll
        for (int k = 1; k <= kR; ++k)
            if (q0 + k == nr) {
                sh4[2] = ra[k];
                sh4[3] = rb[k];
            }
    }
    __syncthreads();
    const int rawA0 = (int)sh4[0], rawB0 = (int)sh4[1];
    const int endA = (int)sh4[2], endB = (int)sh4[3];
    T.ga0 = min((long long)rawA0, A.cap);
    T.gb0 = min((long long)rawB0, B.cap);
    const long long capA = A.cap - rawA0, capB = B.cap - rawB0;  // capacities relative to the tile
    T.LA = clamp_local((long long)(endA - rawA0), capA);
    T.LB = clamp_local((long long)(endB - rawB0), capB);
    T.odd = 0;
#pragma unroll
    for (int k = 0; k <= kR; ++k) {
        T.la[k] = clamp_local((long long)(ra[k] - rawA0), capA);
        T.lb[k] = clamp_local((long long)(rb[k] - rawB0), capB);
        if (k < kR && q0 + k < nr && (((ra[k + 1] - ra[k]) | (rb[k + 1] - rb[k])) & 1)) T.odd |= 1u << k;
    }
    if (threadIdx.x == 0 && (endA > A.cap || endB > B.cap)) set_status(info, LDNI_ST_CAPACITY);
    T.sa.narr = T.sb.narr = narr;
    T.sa.off = (int)(T.ga0 & 3);
    T.sb.off = (int)(T.gb0 & 3);
    const int SA = (T.sa.off + T.LA + 3) & ~3, SB = (T.sb.off + T.LB + 3) & ~3;  // words per staged array
    T.staged = budget > 0 && SA + SB <= budget;
    if (!T.staged) return true;  // block-uniform
    T.sa.base = stage;
    T.sa.stride = SA;
    T.sb.base = stage + narr * SA;
    T.sb.stride = SB;
    const long long ga1 = T.ga0 + T.LA, gb1 = T.gb0 + T.LB;
    if (bulk) {
        if (threadIdx.x == 0) {
            const uint32_t bA = (uint32_t)max(0ll, ((ga1 & ~3ll) - (T.ga0 & ~3ll)) * 4);
            const uint32_t bB = (uint32_t)max(0ll, ((gb1 & ~3ll) - (T.gb0 & ~3ll)) * 4);
            mbar_arrive_expect(bars, bA + bB);
            bulk_range4(T.sa.arr(0), A.d, T.ga0, ga1, bars);
            bulk_range4(T.sb.arr(0), B.d, T.gb0, gb1, bars);
            mbar_arrive_expect(bars + 1, (uint32_t)(narr - 1) * (bA + bB));
            for (int k = 1; k < narr; ++k) {
                bulk_range4(T.sa.arr(k), side_array(A, k, narr), T.ga0, ga1, bars + 1);
                bulk_range4(T.sb.arr(k), side_array(B, k, narr), T.gb0, gb1, bars + 1);
            }
        }
        // the at most three elements past each body, by plain loads (threads 4 (2k + s) .. + 3)
        const int grp = threadIdx.x >> 2;
        if (grp < 2 * narr) {
            const int k = grp >> 1;
            const bool sb = grp & 1;
            const long long g0 = sb ? T.gb0 : T.ga0, g1 = sb ? gb1 : ga1;
            const long long e = g1 & ~3ll, i = e + (threadIdx.x & 3);
            if (i < g1 && i >= g0) (sb ? T.sb : T.sa).arr(k)[i - (g0 & ~3ll)] = side_array(sb ? B : A, k, narr)[i];
        }
    } else {
        for (int k = 0; k < narr; ++k) {
            stage_plain(side_array(A, k, narr), T.ga0, ga1, T.sa.arr(k));
            stage_plain(side_array(B, k, narr), T.gb0, gb1, T.sb.arr(k));
        }
    }
    __syncthreads();  // plain loads visible
    if (!bulk) return true;
    const bool landed = mbar_wait(bars, 0);
    if (__syncthreads_and(landed)) return true;  // the same answer in every thread
    if (threadIdx.x == 0) set_status(info, LDNI_ST_TIMEOUT);
    return false;
}

// Output counts of this thread's rays (and the odd-count check).
template <int kR>
__device__ __forceinline__ int tile_counts(const TileIn<kR> &T, const Side &A, const Side &B, int op, float eps,
                                           int nr, int (&cnt)[kR], ldni_info_t *info) {
    const int q0 = threadIdx.x * kR;
    const float *sA = T.sa.d(), *sB = T.sb.d();
    int mine = 0;
#pragma unroll
    for (int k = 0; k < kR; ++k) {
        cnt[k] = 0;
        if (q0 + k >= nr) continue;
        if (T.odd & (1u << k)) {
            atomicAdd(&info->odd_rays, 1u);
            set_status(info, LDNI_ST_ODD);
        }
        const int a = T.la[k], ae = T.la[k + 1], b = T.lb[k], be = T.lb[k + 1];
        if (a == ae && b == be) continue;
        if (T.staged)
            cnt[k] = merge_ray_fast<int>(sA, a, ae, sB, b, be, op, eps, NoEmit{});
        else
            cnt[k] = merge_ray_fast<long long>(A.d, T.ga0 + a, T.ga0 + ae, B.d, T.gb0 + b, T.gb0 + be, op, eps,
                                               NoEmit{});
        mine += cnt[k];
    }
    return mine;
}

// CSR offsets of this thread's rays, then the tile's output samples from
// output slot `base` on (this thread's first sample is at base + excl).
// vacc gains the inside lengths of this thread's rays when want_vol.
template <int kR>
__device__ __forceinline__ bool tile_emit(const TileIn<kR> &T, const Side &A, const Side &B, int op, float eps,
                                          const Out &o, long long p_begin, int nr, const int (&cnt)[kR], int excl,
                                          long long base, long long total, int *pick, bool bulk, uint64_t *bars,
                                          bool want_vol, DF &vacc, ldni_info_t *info) {
    const int q0 = threadIdx.x * kR;
    {
        int w[kR];
        int run = excl;
#pragma unroll
        for (int k = 0; k < kR; ++k) {
            w[k] = (int)min(base + run, (long long)INT_MAX);
            run += cnt[k];
        }
        store_rows<kR>(const_cast<int *>(o.off), p_begin, q0, nr, w);
    }
    if (!T.staged) {
        int run = excl;
#pragma unroll
        for (int k = 0; k < kR; ++k) {
            if (cnt[k] > 0) {
                const long long at = base + run;
                merge_ray_fast<long long>(A.d, T.ga0 + T.la[k], T.ga0 + T.la[k + 1], B.d, T.gb0 + T.lb[k],
                                          T.gb0 + T.lb[k + 1], op, eps,
                                          [&](bool pb, long long pi, bool cb, long long ci, int m) {
                                              emit_global(pb, pi, A, B, op, o, at + m, info);
                                              emit_global(cb, ci, A, B, op, o, at + m + 1, info);
                                              if (want_vol)
                                                  vacc = df_add(vacc, df_diff((cb ? B.d : A.d)[ci],
                                                                              (pb ? B.d : A.d)[pi]));
                                          });
            }
            run += cnt[k];
        }
        return true;  // block-uniform: no barrier follows on this path
    }
    const float *sA = T.sa.d(), *sB = T.sb.d();
    {
        int run = excl;
#pragma unroll
        for (int k = 0; k < kR; ++k) {
            if (cnt[k] > 0) {
                const int at = run;
                merge_ray_fast<int>(sA, T.la[k], T.la[k + 1], sB, T.lb[k], T.lb[k + 1], op, eps,
                                    [&](bool pb, int pi, bool cb, int ci, int m) {
                                        pick[at + m] = pb ? (int)(0x80000000u | (unsigned)pi) : pi;
                                        pick[at + m + 1] = cb ? (int)(0x80000000u | (unsigned)ci) : ci;
                                        if (want_vol) vacc = df_add(vacc, df_diff((cb ? sB : sA)[ci], (pb ? sB : sA)[pi]));
                                    });
            }
            run += cnt[k];
        }
    }
    bool ok = true;
    if (bulk && !mbar_wait(bars + 1, 0)) {
        set_status(info, LDNI_ST_TIMEOUT);
        ok = false;
    }
    __syncthreads();
    const int tot = (int)total;
    const bool inv = op == LDNI_OP_DIFF;
    const bool three = T.sa.narr == 5;
    const int kt = T.sa.narr - 1;
    for (int k0 = threadIdx.x; k0 < tot; k0 += kBoolThreads * kGather) {
        uint32_t d[kGather], x[kGather], y[kGather], z[kGather], t[kGather];
#pragma unroll
        for (int u = 0; u < kGather; ++u) {
            const int k = k0 + u * kBoolThreads;
            if (k < tot) {
                const int code = pick[k];
                const bool fb = code < 0;
                const int stride = fb ? T.sb.stride : T.sa.stride;
                const uint32_t *src = (fb ? T.sb.base : T.sa.base) + (code & 0x7fffffff) + (fb ? T.sb.off : T.sa.off);
                d[u] = src[0];
                x[u] = src[stride];
                y[u] = three ? src[2 * stride] : 0u;
                z[u] = three ? src[3 * stride] : 0u;
                t[u] = src[kt * stride];
                if (fb) {
                    if (inv) {  // FP32: negate; packed: every code q -> 255 - q
                        const uint32_t m = three ? 0x80000000u : kInvert8;
                        x[u] ^= m;
                        y[u] ^= three ? m : 0u;
                        z[u] ^= three ? m : 0u;
                    }
                    t[u] |= 0x80000000u;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kGather; ++u) {
            const int k = k0 + u * kBoolThreads;
            if (k >= tot) continue;
            const long long at = base + k;
            if (at >= o.cap) {
                set_status(info, LDNI_ST_CAPACITY);
                continue;
            }
            o.d[at] = __uint_as_float(d[u]);
            o.nx[at] = __uint_as_float(x[u]);
            if (three) {
                o.ny[at] = __uint_as_float(y[u]);
                o.nz[at] = __uint_as_float(z[u]);
            }
            o.tri[at] = (int)t[u];
        }
    }
    return ok;
}

// Tickets run over all jobs' tiles in order: ticket t is tile t % tpj of job
// t / tpj; each job has its own look-back words (words + job * tpj); word
// tpj * njobs is the ticket counter, the next one counts finished tiles.
// With volumes asked for, each tile leaves its summed inside lengths in
// tile_vol[ticket], and the block that finishes last adds every job's
// partials in a fixed order.
template <int kR>
__global__ void __launch_bounds__(kBoolThreads) bool_tiled(long long N, const __grid_constant__ BoolJobs J, int op,
                                                           float eps, unsigned long long *words, int tpj, int njobs,
                                                           int budget, bool bulk, double *tile_vol, double h2,
                                                           int spin_limit) {
    constexpr int kRays = kR * kBoolThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int narr = J.packed ? 3 : 5;
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem_raw);      // [narr][budget] words
    int *pick = reinterpret_cast<int *>(stage + narr * budget);    // [budget] source of every output sample
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ long long sh[kBoolThreads / 32 + 1];
    __shared__ long long sh4[4];
    __shared__ int s_tile;
    __shared__ long long s_base;
    __shared__ DF s_df[kBoolThreads / 32];
    __shared__ bool s_last;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(words + (size_t)tpj * njobs, 1ull);
    __syncthreads();
    const int ticket = s_tile;
    const int job = ticket / tpj, tile = ticket - job * tpj;
    const Side &A = J.A[job];
    const Side &B = J.B[job];
    const Out &o = J.o[job];
    ldni_info_t *info = J.info[job];
    const long long p_begin = (long long)tile * kRays;
    const int nr = (int)min((long long)kRays, N - p_begin);
    TileIn<kR> T;
    const bool ok = tile_prologue<kR>(A, B, p_begin, nr, budget, narr, bulk, stage, bars, sh4, T, info);
    int cnt[kR];
    const int mine = ok ? tile_counts<kR>(T, A, B, op, eps, nr, cnt, info) : 0;
    if (!ok)
#pragma unroll
        for (int k = 0; k < kR; ++k) cnt[k] = 0;
    long long total;
    const int excl = (int)block_exclusive_scan<kBoolThreads>(mine, sh, &total);
    if (threadIdx.x < 32) {
        const long long b = lookback_warp(words + (size_t)job * tpj, tile, total, info, spin_limit);
        if (threadIdx.x == 0) s_base = b;
    }
    __syncthreads();
    const long long base = s_base;
    if (tile == tpj - 1 && threadIdx.x == 0) finish_output(o, N, base + total, info);
    const bool want_vol = tile_vol != nullptr;
    DF vacc{0.0f, 0.0f};
    if (ok) tile_emit<kR>(T, A, B, op, eps, o, p_begin, nr, cnt, excl, base, total, pick, bulk, bars, want_vol, vacc,
                          info);
    else if (T.staged && bulk)  // a copy may still be landing: give it a bounded while before the block ends
        mbar_wait(bars + 1, 0);
    if (!want_vol) return;  // block-uniform
    const DF tsum = df_block_sum<kBoolThreads>(vacc, s_df);
    if (threadIdx.x == 0) {
        tile_vol[ticket] = (double)tsum.hi + (double)tsum.lo;
        __threadfence();
        s_last = atomicAdd(words + (size_t)tpj * njobs + 1, 1ull) == (unsigned long long)(tpj * njobs - 1);
    }
    __syncthreads();
    if (!s_last) return;  // block-uniform
    __threadfence();
    double *shd = reinterpret_cast<double *>(smem_raw);  // the stage is no longer needed
    for (int j = 0; j < njobs; ++j) {
        const double v = fixed_order_sum<kBoolThreads>(tile_vol + (size_t)j * tpj, tpj, shd);
        if (threadIdx.x == 0) *J.vol[j] = v * h2;
        __syncthreads();
    }
}

// ---- two launches per image -------------------------------------------------
//
// Super-tiles of 2^gshift write tiles, at most kMaxSupers per image: a write
// block reads at most kMaxSupers super-tile totals and 2^gshift - 1 tile
// totals to find its first output slot.
constexpr int kMaxSupers = 256;
//
// No block waits for another.  Each thread owns kR consecutive rays and reads
// their rows and depths straight from global memory.  A ray with at most one
// interval per operand (kinds 0, 1, 2 and 4) is answered in closed form from
// its depths, issued for all the thread's rays before any is used; every
// other ray runs the general merge.  Both passes are compiled per operation.

// Pass 1: output count of every ray (kept in the output's offset array,
// which pass 3 overwrites in place; a closed-form ray keeps its outputs'
// sources beside the count, from bit kSrcShift on), of every tile of the
// write pass (tile_total, cleared before the launch; 2^wshift rays per tile,
// tpjw tiles per job) and of every super-tile of 2^gshift write tiles
// (super_total, kMaxSupers per job, cleared).  The count pass has its own
// rays per thread (kR): a warp's 32 * kR rays lie in one write tile, so each
// warp adds its sum to that tile's and that super-tile's totals.  tpj: count
// blocks per job.
#ifndef LDNI_BOOL_COUNT_BLOCKS
#define LDNI_BOOL_COUNT_BLOCKS 8
#endif
template <int kR, int kOp>
__global__ void __launch_bounds__(kBoolThreads, LDNI_BOOL_COUNT_BLOCKS)
    bool_count(int N, const __grid_constant__ BoolJobs J, float eps, unsigned long long *tile_total,
               unsigned long long *super_total, int tpj, int wshift, int gshift, int tpjw, float2 *vol_part) {
    // Index arithmetic is 32-bit: rays (at most 8192^2) and rows (int) fit.
    constexpr int kRays = kR * kBoolThreads;
    const int job = blockIdx.y, tile = blockIdx.x;  // the grid is tpj x jobs
    const Side &A = J.A[job];
    const Side &B = J.B[job];
    const Out &o = J.o[job];
    ldni_info_t *info = J.info[job];
    const int p0 = tile * kRays;
    const int nr = min(kRays, N - p0);
    const int q0 = threadIdx.x * kR;
    const int capA = (int)min(A.cap, (long long)INT_MAX), capB = (int)min(B.cap, (long long)INT_MAX);
    int ra[kR + 1], rb[kR + 1];
    load_rows<kR>(A.off + p0, 0, q0, nr, ra);
    load_rows<kR>(B.off + p0, 0, q0, nr, rb);
    // a ray whose rows run beyond an operand's capacity takes the general (clamping) path
    if (ra[kR] > capA || rb[kR] > capB) set_status(info, LDNI_ST_CAPACITY);
    // Every ray with at most one interval per operand (kinds 0, 1, 2 and 4) takes
    // the closed form, an absent operand as the empty interval (0, 0): the
    // lanes of a warp run the same instructions whatever their rays' kinds.
    bool gen[kR];
    float a0[kR], a1[kR], b0[kR], b1[kR];
#pragma unroll
    for (int k = 0; k < kR; ++k) {
        const int na = ra[k + 1] - ra[k], nb = rb[k + 1] - rb[k];
        if ((na | nb) & 1) {
            atomicAdd(&info->odd_rays, 1u);
            set_status(info, LDNI_ST_ODD);
        }
        gen[k] = general_ray(ra[k], ra[k + 1], rb[k], rb[k + 1], capA, capB);
        const bool pa = !gen[k] && na == 2 && range_ok(ra[k], ra[k] + 2, capA, info);
        const bool pb = !gen[k] && nb == 2 && range_ok(rb[k], rb[k] + 2, capB, info);
        a0[k] = a1[k] = b0[k] = b1[k] = 0.0f;
        if (J.pairs8 && ((ra[k] | rb[k]) & 1) == 0) {  // even rows: each depth pair is one 8-byte load
            if (pa) {
                const uint2 v = ld_pair(A.d, ra[k]);
                a0[k] = __uint_as_float(v.x);
                a1[k] = __uint_as_float(v.y);
            }
            if (pb) {
                const uint2 v = ld_pair(B.d, rb[k]);
                b0[k] = __uint_as_float(v.x);
                b1[k] = __uint_as_float(v.y);
            }
        } else {
            a0[k] = pa ? A.d[ra[k]] : 0.0f;
            a1[k] = pa ? A.d[ra[k] + 1] : 0.0f;
            b0[k] = pb ? B.d[rb[k]] : 0.0f;
            b1[k] = pb ? B.d[rb[k] + 1] : 0.0f;
        }
    }
    int cnt[kR], word[kR];
    int mine = 0;
    // inside lengths of the result (its volume, when asked for): each kept interval [x, y] adds
    // y - x as an exact pair of floats, summed in double-float (FP32 arithmetic: this GPU's FP64
    // rate would double the pass)
    const bool want_vol = vol_part != nullptr;
    DF len{0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < kR; ++k) {
        if (gen[k]) {
            const long long a = min((long long)ra[k], A.cap), b = min((long long)rb[k], B.cap);
            const int na = (int)(min((long long)ra[k + 1], A.cap) - a), nb = (int)(min((long long)rb[k + 1], B.cap) - b);
            const float *dA = A.d + a, *dB = B.d + b;
            if (want_vol)
                cnt[k] = merge_core<int>(dA, 0, na, dB, 0, nb, kOp, eps, [&](bool pb, int pi, bool cb, int ci, int) {
                    len = df_add_lazy(len, df_diff((cb ? dB : dA)[ci], (pb ? dB : dA)[pi]));
                });
            else
                cnt[k] = merge_core<int>(dA, 0, na, dB, 0, nb, kOp, eps, NoEmit{});
            word[k] = cnt[k];
        } else {
            unsigned src;
            Ends e{0.0f, 0.0f, 0.0f, 0.0f};
            cnt[k] = two_two(kOp, eps, a0[k], a1[k], b0[k], b1[k], src, &e);
            if (want_vol) {
                if (cnt[k] >= 2) len = df_add_lazy(len, df_diff(e.y0, e.x0));
                if (cnt[k] == 4) len = df_add_lazy(len, df_diff(e.y1, e.x1));
            }
            word[k] = cnt[k] | (int)(src << kSrcShift);
        }
        mine += cnt[k];
    }
    store_rows<kR>(const_cast<int *>(o.off) + p0, 0, q0, nr, word);
    mine = (int)__reduce_add_sync(0xffffffffu, (unsigned)mine);  // at most 2^31 - 1: counts are int rows
    if ((threadIdx.x & 31) == 0 && mine) {
        const int pw = p0 + (threadIdx.x >> 5) * 32 * kR;  // the warp's first ray
        atomicAdd(tile_total + (size_t)job * tpjw + (pw >> wshift), (unsigned long long)mine);
        atomicAdd(super_total + (size_t)job * kMaxSupers + (pw >> (wshift + gshift)), (unsigned long long)mine);
    }
    if (!want_vol) return;  // block-uniform
#pragma unroll
    for (int w = 16; w > 0; w >>= 1)  // a fixed tree; one partial per warp (no barrier)
        len = df_add_lazy(len, DF{__shfl_down_sync(0xffffffffu, len.hi, w), __shfl_down_sync(0xffffffffu, len.lo, w)});
    if ((threadIdx.x & 31) == 0)
        vol_part[((size_t)job * tpj + tile) * (kBoolThreads / 32) + (threadIdx.x >> 5)] = make_float2(len.hi, len.lo);
}

// One sample's fields as loaded (normals as raw words: FP32 or one packed word).
struct Smp {
    float d;
    uint32_t x, y, z, t;
};

// Sample i of side S into v when `on` (zeros otherwise); y, z only for FP32 normals.
__device__ __forceinline__ void load_smp(const Side &S, bool on, bool three, long long i, Smp &v) {
    v.d = on ? S.d[i] : 0.0f;
    v.x = on ? reinterpret_cast<const uint32_t *>(S.nx)[i] : 0u;
    v.y = on && three ? reinterpret_cast<const uint32_t *>(S.ny)[i] : 0u;
    v.z = on && three ? reinterpret_cast<const uint32_t *>(S.nz)[i] : 0u;
    v.t = on ? reinterpret_cast<const uint32_t *>(S.tri)[i] : 0u;
}

#ifndef LDNI_BOOL_WRITE_BLOCKS
#define LDNI_BOOL_WRITE_BLOCKS 6
#endif

// Pass 2: the block first writes its tile's offsets (kR rays per thread),
// listing every ray with output samples in shared memory, and then its
// threads take the listed rays in turn: first the closed-form rays, which
// copy samples of their one or two pairs (their sources come from pass 1, so
// samples a ray drops are not read; every sample a ray copies is loaded
// before any of its stores), then the rays of the general merge.  Rays without samples (often half of an image) thus leave no
// thread idle while the others wait on memory, and a block covers kR times
// as many rays with the same registers per thread.
struct CopyItem {
    long long at;  // first output slot; copies: the outputs' sources and count from bit kItemSrcShift on
    int ra;        // copies: A's row; merges: the ray
    int rb;        // copies: B's row
};
constexpr int kItemSrcShift = 48;  // output slots stay below 2^48

// The tile's first output slot is the sum of the totals of every earlier tile
// of its image, which pass 1 left complete: the super-tile totals before the
// tile's super-tile, then the tile totals of its own super-tile before it,
// read directly.  With volumes asked for (vol_part), the volume of image j
// is summed by the block of tile j mod tpj of the first image, one of the
// first blocks to start: after its own rays it adds all of the count warps'
// partials of image j in a fixed order (pass 1 left them complete: nothing
// waits).  The block of an image's last tile writes the image's total.
template <int kR, int kOp>
__global__ void __launch_bounds__(kBoolThreads, LDNI_BOOL_WRITE_BLOCKS)
    bool_write(int N, const __grid_constant__ BoolJobs J, float eps, const unsigned long long *tile_total,
               const unsigned long long *super_total, int tpj, int gshift, const float2 *vol_part, int nvol,
               double h2) {
    constexpr int op = kOp;
    constexpr int kRays = kR * kBoolThreads;
    constexpr int kItemBits = 20;  // items per tile < 2^20 in the low bits of the scanned word
    __shared__ long long sh[kBoolThreads / 32 + 1];
    __shared__ long long s_pre[kBoolThreads / 32];
    __shared__ CopyItem items[kRays];  // copies from the front, merges from the back
    __shared__ int s_merges;
    const int job = blockIdx.y, tile = blockIdx.x;  // the grid is tpj x jobs
    const Side &A = J.A[job];
    const Side &B = J.B[job];
    const Out &o = J.o[job];
    ldni_info_t *info = J.info[job];
    const int p0 = tile * kRays;  // 32-bit index arithmetic, as in pass 1
    const int nr = min(kRays, N - p0);
    const int q0 = threadIdx.x * kR;
    const int lane = threadIdx.x & 31;
    // the totals of the earlier tiles: one load each from the first threads, issued before the rows and
    // used after them (tiles beyond the first kBoolThreads of a super-tile: only for images of more than
    // 2^24 rays)
    const int sup = tile >> gshift, first = sup << gshift;  // sup < kMaxSupers
    const unsigned long long sv = (int)threadIdx.x < sup ? super_total[(size_t)job * kMaxSupers + threadIdx.x] : 0ull;
    const unsigned long long tv = first + (int)threadIdx.x < tile ? tile_total[(size_t)job * tpj + first + threadIdx.x]
                                                                  : 0ull;
    const int capA = (int)min(A.cap, (long long)INT_MAX), capB = (int)min(B.cap, (long long)INT_MAX);
    const bool three = !J.packed;
    if (threadIdx.x == 0) s_merges = 0;  // ordered before its first use by the block scan's barriers
    int ra[kR + 1], rb[kR + 1], cnt[kR + 1];
    load_rows<kR>(A.off + p0, 0, q0, nr, ra);
    load_rows<kR>(B.off + p0, 0, q0, nr, rb);
    load_rows<kR>(o.off + p0, 0, q0, nr, cnt);  // pass 1's words (cnt[kR] unused)
    long long pre = (long long)(sv + tv);
    for (int k = first + (int)threadIdx.x + kBoolThreads; k < tile; k += kBoolThreads)
        pre += (long long)tile_total[(size_t)job * tpj + k];
    // each warp's share of the carry (warps that loaded nothing skip the sum)
    const int first_idle = max(sup, tile - first);  // threads from here on loaded nothing
    if ((int)(threadIdx.x & ~31u) < first_idle) {  // warp-uniform
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) pre += __shfl_xor_sync(0xffffffffu, pre, w);
    }
    // read by the block scan after its first barrier, shifted past the item bits of the scanned word
    if (lane == 0) s_pre[threadIdx.x >> 5] = pre << kItemBits;
    bool gen[kR];
    unsigned src[kR];
    long long mine = 0;
    int listed = 0;
#pragma unroll
    for (int k = 0; k < kR; ++k) {
        if (q0 + k >= nr) cnt[k] = 0;
        gen[k] = general_ray(ra[k], ra[k + 1], rb[k], rb[k + 1], capA, capB);
        src[k] = gen[k] ? 0u : (unsigned)cnt[k] >> kSrcShift;
        cnt[k] = gen[k] ? cnt[k] : cnt[k] & 7;
        mine += cnt[k];
        listed += !gen[k] && cnt[k] > 0;
    }
    long long total;
    // the earlier tiles' total enters the scan as its carry
    const long long ex = block_exclusive_scan_carry<kBoolThreads>((mine << kItemBits) | listed, s_pre, sh, &total);
    if (tile == tpj - 1 && threadIdx.x == 0) finish_output(o, N, (ex >> kItemBits) + (total >> kItemBits), info);
    const long long base = ex >> kItemBits;
    const int nitems = (int)(total & ((1 << kItemBits) - 1));
    {
        int w[kR];
        int slot = (int)(ex & ((1 << kItemBits) - 1));
        long long run = base;
#pragma unroll
        for (int k = 0; k < kR; ++k) {
            w[k] = (int)min(run, (long long)INT_MAX);
            if (cnt[k] > 0 && !gen[k])
                items[slot++] = CopyItem{run | (long long)(src[k] | ((unsigned)cnt[k] << 8)) << kItemSrcShift, ra[k],
                                         rb[k]};
            else if (cnt[k] > 0)
                items[kRays - 1 - atomicAdd(&s_merges, 1)] = CopyItem{run, q0 + k, 0};
            run += cnt[k];
        }
        store_rows<kR>(const_cast<int *>(o.off) + p0, 0, q0, nr, w);
    }
    __syncthreads();
    const int nmerges = s_merges;
    const uint32_t flip = op != LDNI_OP_DIFF ? 0u : (three ? 0x80000000u : kInvert8);  // an inverted normal
    for (int i = threadIdx.x; i < nitems; i += kBoolThreads) {
        const CopyItem it = items[i];
        const unsigned src = (unsigned)(it.at >> kItemSrcShift) & 0xffu;
        const int c = (int)(it.at >> (kItemSrcShift + 8));
        const long long at0 = it.at & ((1ll << kItemSrcShift) - 1);
        if (!range_ok(it.ra, it.ra + ((src_needs(src, c) & 3u) ? 2 : 0), capA, info) ||
            !range_ok(it.rb, it.rb + ((src_needs(src, c) & 12u) ? 2 : 0), capB, info))
            continue;
        if (c == 2 && (src == 0x4u || src == 0xEu) && at0 + 1 < o.cap) {
            // one operand's pair, in order (most rays): a plain copy
            const bool fb = src == 0xEu;
            const Side &S = fb ? B : A;
            const int i0 = fb ? it.rb : it.ra;
            const uint32_t f = fb ? flip : 0u;
            const uint32_t tb = fb ? 0x80000000u : 0u;
            if (J.pairs8 && ((i0 | (int)at0) & 1) == 0) {
                // rows and output slots of closed solids are even: each field's pair is one 8-byte access
                const uint2 d = ld_pair(S.d, i0), x = ld_pair(S.nx, i0), t = ld_pair(S.tri, i0);
                st_pair(o.d, at0, d);
                st_pair(o.nx, at0, make_uint2(x.x ^ f, x.y ^ f));
                if (three) {
                    const uint2 y = ld_pair(S.ny, i0), z = ld_pair(S.nz, i0);
                    st_pair(o.ny, at0, make_uint2(y.x ^ f, y.y ^ f));
                    st_pair(o.nz, at0, make_uint2(z.x ^ f, z.y ^ f));
                }
                st_pair(o.tri, at0, make_uint2(t.x | tb, t.y | tb));
                continue;
            }
            Smp v0, v1;
            load_smp(S, true, three, i0, v0);
            load_smp(S, true, three, i0 + 1, v1);
            o.d[at0] = v0.d;
            o.d[at0 + 1] = v1.d;
            o.nx[at0] = __uint_as_float(v0.x ^ f);
            o.nx[at0 + 1] = __uint_as_float(v1.x ^ f);
            if (three) {
                o.ny[at0] = __uint_as_float(v0.y ^ f);
                o.ny[at0 + 1] = __uint_as_float(v1.y ^ f);
                o.nz[at0] = __uint_as_float(v0.z ^ f);
                o.nz[at0 + 1] = __uint_as_float(v1.z ^ f);
            }
            o.tri[at0] = (int)(v0.t | tb);
            o.tri[at0 + 1] = (int)(v1.t | tb);
            continue;
        }
        const unsigned need = src_needs(src, c);
        Smp a0, a1, b0, b1;  // every sample the ray copies, loaded before any store
        load_smp(A, need & 1u, three, it.ra, a0);
        load_smp(A, need & 2u, three, it.ra + 1, a1);
        load_smp(B, need & 4u, three, it.rb, b0);
        load_smp(B, need & 8u, three, it.rb + 1, b1);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (m >= c) break;
            const long long at = at0 + m;
            if (at >= o.cap) {
                set_status(info, LDNI_ST_CAPACITY);
                continue;
            }
            const int sm = src_of(src, m);
            const uint32_t f = sm >= 2 ? flip : 0u;
            o.d[at] = pick4(sm, a0.d, a1.d, b0.d, b1.d);
            o.nx[at] = __uint_as_float(pick4u(sm, a0.x, a1.x, b0.x, b1.x) ^ f);
            if (three) {
                o.ny[at] = __uint_as_float(pick4u(sm, a0.y, a1.y, b0.y, b1.y) ^ f);
                o.nz[at] = __uint_as_float(pick4u(sm, a0.z, a1.z, b0.z, b1.z) ^ f);
            }
            o.tri[at] = (int)pick4u(sm, a0.t, a1.t, b0.t | 0x80000000u, b1.t | 0x80000000u);
        }
    }
    for (int i = threadIdx.x; i < nmerges; i += kBoolThreads) {
        const CopyItem it = items[kRays - 1 - i];
        const int p = p0 + it.ra;  // the ray (its rows again: cached)
        const long long a0 = min((long long)A.off[p], A.cap), b0 = min((long long)B.off[p], B.cap);
        const int na = (int)(min((long long)A.off[p + 1], A.cap) - a0);
        const int nb = (int)(min((long long)B.off[p + 1], B.cap) - b0);
        const long long at0 = it.at;
        merge_core<int>(A.d + a0, 0, na, B.d + b0, 0, nb, op, eps, [&](bool pb, int pi, bool cb, int ci, int m) {
            emit_global(pb, (pb ? b0 : a0) + pi, A, B, op, o, at0 + m, info);
            emit_global(cb, (cb ? b0 : a0) + ci, A, B, op, o, at0 + m + 1, info);
        });
    }
    if (!vol_part || job != 0) return;  // block-uniform
    __shared__ DF shdf[kBoolThreads / 32];
    for (int vjob = tile; vjob < (int)gridDim.y; vjob += tpj) {  // the images whose volumes this block sums
        // the image's nvol partials, strided per thread in a fixed order, then a fixed tree
        constexpr int kU = 8;
        const float2 *vp = vol_part + (size_t)vjob * nvol;
        DF acc{0.0f, 0.0f};
        for (int k0 = threadIdx.x; k0 < nvol; k0 += kBoolThreads * kU) {
            float2 v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u)
                v[u] = k0 + u * kBoolThreads < nvol ? vp[k0 + u * kBoolThreads] : make_float2(0.0f, 0.0f);
#pragma unroll
            for (int u = 0; u < kU; ++u) acc = df_add_lazy(acc, DF{v[u].x, v[u].y});
        }
        const DF t = df_block_sum<kBoolThreads>(acc, shdf);
        if (threadIdx.x == 0) *J.vol[vjob] = ((double)t.hi + (double)t.lo) * h2;
        __syncthreads();  // shdf is reused by the next image
    }
}

// ---- host side ------------------------------------------------------------------

int grid_blocks(long long work) {
    long long b = (work + kThreads - 1) / kThreads;
    const long long lim = (long long)num_sms() * 16;
    if (b > lim) b = lim;
    return (int)(b > 0 ? b : 1);
}

struct BoolWs {
    int *count;
    long long *partials;
};

BoolWs carve_bool_ws(Carver &c, int res) {
    BoolWs w;
    const long long N = (long long)res * res;
    w.count = c.take<int>((size_t)N);
    w.partials = c.take<long long>(csr_scan_partials(N));
    return w;
}

Side side_of(const ldni_layers_t &L) {
    float *x, *y, *z;
    normal_arrays(L, x, y, z);
    return Side{L.capacity, L.offsets, L.depth, x, y, z, L.tri_id};
}

Out out_of(const ldni_layers_t &L) {
    float *x, *y, *z;
    normal_arrays(L, x, y, z);
    return Out{L.offsets, L.depth, x, y, z, L.tri_id, L.capacity};
}

bool layers_ok(const ldni_layers_t *L, bool need) {
    if (!L || !L->offsets || L->capacity < 0) return false;
    if (need && !samples_ok(*L)) return false;
    return true;
}

constexpr int kMinTileRays = 256;  // the workspace is sized for the smallest tile
#ifndef LDNI_BOOL_COUNT_RAYS
#define LDNI_BOOL_COUNT_RAYS 2
#endif
// rays per thread of the count pass (1, 2, 4 or 8), whatever the write pass's tile
constexpr int kBoolCountRays = LDNI_BOOL_COUNT_RAYS;
constexpr int kMaxDynSmem = 220 * 1024;  // dynamic shared memory of one Boolean block, at most

size_t bool_ws_words(long long N) { return (size_t)((N + kMinTileRays - 1) / kMinTileRays); }

// bulk copies need every staged array to start on a 16-byte boundary
bool bulk_aligned(const BoolJobs &J, int njobs, bool rows) {
    bool ok = true;
    for (int j = 0; j < njobs; ++j) {
        for (const Side *S : {&J.A[j], &J.B[j]}) {
            for (const void *p : {(const void *)S->d, (const void *)S->nx, (const void *)S->ny, (const void *)S->nz,
                                  (const void *)S->tri})
                ok &= (reinterpret_cast<uintptr_t>(p) & 15) == 0;
            if (rows) ok &= (reinterpret_cast<uintptr_t>(S->off) & 15) == 0;
        }
        if (rows) ok &= (reinterpret_cast<uintptr_t>(J.o[j].off) & 15) == 0;
    }
    return ok;
}

template <int kR>
int launch_bool(long long N, const BoolJobs &J, int njobs, int op, float eps, void *ws, int budget, int form,
                double h2, cudaStream_t s) {
    constexpr int kRays = kR * kBoolThreads;
    const int tpj = (int)((N + kRays - 1) / kRays);
    const int nblocks = tpj * njobs;
    // staged arrays per sample (depth, normals, id) plus the output sources, within the
    // shared memory a block can have
    const int narr = J.packed ? 3 : 5;
    unsigned long long *words = static_cast<unsigned long long *>(ws);
    if (form == 0) {
        const int per = 4 * (narr + 1);
        budget = min(budget, (kMaxDynSmem / per) & ~3);
        const bool bulk = bulk_aligned(J, njobs, false);
        // (the block that sums the volumes last reuses the stage for kBoolThreads doubles)
        const size_t smem = max((size_t)per * (size_t)budget, J.vol[0] ? sizeof(double) * kBoolThreads : (size_t)0);
        if (smem > 32 * 1024)  // beyond the default 48 KB with the static shared memory
            if (int rc_ = cuda_check(
                    cudaFuncSetAttribute(bool_tiled<kR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
                return rc_;
        // workspace: look-back words (one per tile) | ticket | finished tiles | tile volumes
        double *tile_vol = J.vol[0] ? reinterpret_cast<double *>(words + nblocks + 2) : nullptr;
        if (int rc_ = cuda_check(cudaMemsetAsync(words, 0, sizeof(unsigned long long) * ((size_t)nblocks + 2), s)))
            return rc_;
        LDNI_LAUNCH(K_BOOL_FUSED, s,
                    bool_tiled<kR><<<nblocks, kBoolThreads, smem, s>>>(N, J, op, eps, words, tpj, njobs, budget, bulk,
                                                                       tile_vol, h2, wait_limit()));
        return cuda_status();
    }
    // super-tiles of 2^gshift write tiles, at most kMaxSupers per job
    int gshift = 5;
    while (((long long)tpj + (1ll << gshift) - 1) >> gshift > kMaxSupers) ++gshift;
    // workspace: tile totals | super-tile totals (cleared together) | volume partials (one per count warp)
    unsigned long long *tile_total = words;
    unsigned long long *super_total = tile_total + nblocks;
    const size_t cleared = (size_t)nblocks + (size_t)kMaxSupers * njobs;
    float2 *vol_part = J.vol[0] ? reinterpret_cast<float2 *>(words + cleared) : nullptr;
    if (int rc_ = cuda_check(cudaMemsetAsync(tile_total, 0, sizeof(unsigned long long) * cleared, s)))
        return rc_;
    constexpr int kRc = kBoolCountRays;
    const int tpjc = (int)((N + kRc * kBoolThreads - 1) / (kRc * kBoolThreads));  // count blocks per job
    const int nvol = tpjc * (kBoolThreads / 32);
    auto count = op == LDNI_OP_UNION   ? bool_count<kRc, LDNI_OP_UNION>
                 : op == LDNI_OP_INTER ? bool_count<kRc, LDNI_OP_INTER>
                                       : bool_count<kRc, LDNI_OP_DIFF>;
    auto write = op == LDNI_OP_UNION   ? bool_write<kR, LDNI_OP_UNION>
                 : op == LDNI_OP_INTER ? bool_write<kR, LDNI_OP_INTER>
                                       : bool_write<kR, LDNI_OP_DIFF>;
    LDNI_LAUNCH(K_BOOL_COUNT, s,
                count<<<dim3(tpjc, njobs), kBoolThreads, 0, s>>>((int)N, J, eps, tile_total, super_total, tpjc,
                                                                 __builtin_ctz(kRays), gshift, tpj, vol_part));
    LDNI_LAUNCH(K_BOOL_WRITE, s,
                write<<<dim3(tpj, njobs), kBoolThreads, 0, s>>>((int)N, J, eps, tile_total, super_total, tpj, gshift,
                                                               vol_part, nvol, h2));
    return cuda_status();
}

bool same_grid(const ldni_grid_t *a, const ldni_grid_t *b) {
    return a->res == b->res && a->width == b->width && a->origin[0] == b->origin[0] &&
           a->origin[1] == b->origin[1] && a->origin[2] == b->origin[2];
}

int boolean_jobs(int32_t count, const ldni_layers_t *A, const ldni_layers_t *B, const ldni_grid_t *grid, int32_t op,
                 float eps, ldni_layers_t *out, ldni_info_t *infos, double *vols, void *ws, size_t ws_bytes,
                 void *stream) {
    if (count < 1 || count > kMaxJobs || !A || !B || !out || !infos || !ws || !grid_valid(grid) ||
        op < LDNI_OP_UNION || op > LDNI_OP_DIFF || !(eps >= 0.0f))
        return LDNI_EINVAL;
    BoolJobs J{};
    {
        const ldni_layers_t *all[3 * kMaxJobs];
        for (int j = 0; j < count; ++j) {
            all[3 * j] = A + j;
            all[3 * j + 1] = B + j;
            all[3 * j + 2] = out + j;
        }
        if (!same_format(all, 3 * count, &J.packed)) return LDNI_EINVAL;
        J.pairs8 = true;
        for (int k = 0; k < 3 * count; ++k) {
            float *x, *y, *z;
            normal_arrays(*all[k], x, y, z);
            for (const void *q : {(const void *)all[k]->depth, (const void *)x, (const void *)y, (const void *)z,
                                  (const void *)all[k]->tri_id})
                J.pairs8 &= (reinterpret_cast<uintptr_t>(q) & 7) == 0;
        }
    }
    for (int j = 0; j < count; ++j) {
        if (!layers_ok(A + j, true) || !layers_ok(B + j, true) || !layers_ok(out + j, true)) return LDNI_EINVAL;
        J.A[j] = side_of(A[j]);
        J.B[j] = side_of(B[j]);
        J.o[j] = out_of(out[j]);
        J.info[j] = infos + j;
        J.vol[j] = vols ? vols + j : nullptr;
    }
    const long long N = (long long)grid->res * grid->res;
    size_t need = 0;
    ldni_boolean_many_workspace_size(grid->res, count, &need);
    if (ws_bytes < need) return LDNI_EWORKSPACE;
    const ldni_tuning_t tune = current_tuning();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int budget = tune.bool_stage_samples;
    const int rays = tune.bool_tile_rays;
    // small images: one staged launch; large ones: count, then write
    const int form = tune.bool_split >= 0 ? tune.bool_split : (N * count / rays > 2 * (long long)num_sms() ? 1 : 0);
    const double h = (double)grid->width / (double)grid->res;
    switch (rays) {
        case 256: return launch_bool<1>(N, J, count, op, eps, ws, budget, form, h * h, s);
        case 512: return launch_bool<2>(N, J, count, op, eps, ws, budget, form, h * h, s);
        case 2048: return launch_bool<8>(N, J, count, op, eps, ws, budget, form, h * h, s);
        default: return launch_bool<4>(N, J, count, op, eps, ws, budget, form, h * h, s);
    }
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_boolean_workspace_size(int32_t res, size_t *bytes) {
    return ldni_boolean_many_workspace_size(res, 1, bytes);
}

extern "C" int ldni_boolean_many_workspace_size(int32_t res, int32_t count, size_t *bytes) {
    if (!bytes || res < 1 || res > 8192 || count < 1 || count > kMaxJobs) return LDNI_EINVAL;
    // look-back words and ticket of the one-launch form, or tile totals,
    // super-tile totals and warp volumes of the two-launch form, for the
    // smallest tile
    *bytes = align_up(sizeof(long long) * ((2 + kBoolThreads / 32) * bool_ws_words((long long)res * res) * count +
                                           (size_t)kMaxSupers * count + 8));
    return LDNI_OK;
}

extern "C" int ldni_boolean(const ldni_layers_t *A, const ldni_grid_t *grid_a, const ldni_layers_t *B,
                            const ldni_grid_t *grid_b, int32_t op, float eps, ldni_layers_t *out, ldni_info_t *info,
                            void *ws, size_t ws_bytes, void *stream) {
    if (!grid_valid(grid_a) || !grid_valid(grid_b)) return LDNI_EINVAL;
    if (!same_grid(grid_a, grid_b)) return LDNI_EGRID_MISMATCH;
    return boolean_jobs(1, A, B, grid_a, op, eps, out, info, nullptr, ws, ws_bytes, stream);
}

extern "C" int ldni_boolean_many(int32_t count, const ldni_layers_t *A, const ldni_layers_t *B,
                                 const ldni_grid_t *grid, int32_t op, float eps, ldni_layers_t *out,
                                 ldni_info_t *infos, double *vols, void *ws, size_t ws_bytes, void *stream) {
    return boolean_jobs(count, A, B, grid, op, eps, out, infos, vols, ws, ws_bytes, stream);
}

// ---- Boolean without a caller workspace -------------------------------------
//
// Some callers cannot allocate device memory at the point where they need a
// Boolean: code running while another framework owns the device allocator
// (a plugin that is only handed input and output buffers), or a latency-
// critical loop where an allocation would synchronise the device.  For them
// ldni_boolean_static keeps its scratch (per-ray output counts and the scan's
// chunk totals) in one static device array instead of a workspace argument.
// Every GPU that loads the library holds this array until the process exits.
namespace ldni {
namespace {

constexpr int kStaticMaxRes = 1024;  // scratch sized for res <= 1024
constexpr size_t kStaticScratchBytes =
    4u * (size_t)kStaticMaxRes * kStaticMaxRes + 8u * 1024u + 2u * kAlign;  // counts + scan chunk totals

static __device__ __align__(256) unsigned char g_bool_static_scratch[kStaticScratchBytes];

// The array's device address belongs to a CUDA context, not to a device
// ordinal: a non-primary context of the same device, or the primary context
// made again after cudaDeviceReset, has its own copy of the array.  Addresses
// are therefore cached per context, keyed by the driver's context id, which
// no later context of the process reuses.  The two driver calls are reached
// through the runtime, so the library links no driver library.
using CtxGetCurrentFn = CUresult(CUDAAPI *)(CUcontext *);
using CtxGetIdFn = CUresult(CUDAAPI *)(CUcontext, unsigned long long *);

constexpr int kMaxContexts = 64;
std::mutex g_static_mu;
struct StaticEntry {
    unsigned long long ctx_id;
    void *ptr;
};
StaticEntry g_static[kMaxContexts] = {};
int g_static_n = 0;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// Id of the calling thread's current context; false when there is none or
// the driver cannot say.  Holds g_static_mu.
bool current_context_id(unsigned long long *id) {
    if (!g_ctx_current || !g_ctx_id) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1) {
            cudaGetLastError();
            return false;
        }
        g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f0);
        g_ctx_id = reinterpret_cast<CtxGetIdFn>(f1);
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_ctx_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the static scratch in the current context.  The
// host-side symbol is only a stand-in, so the address is looked up once per
// context (cudaGetSymbolAddress also makes the device's primary context
// current when the thread has none yet).
int static_scratch(void **out) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    unsigned long long id = 0;
    const bool known = current_context_id(&id);
    if (known)
        for (int k = 0; k < g_static_n; ++k)
            if (g_static[k].ctx_id == id) {
                *out = g_static[k].ptr;
                return LDNI_OK;
            }
    void *p = nullptr;
    if (const cudaError_t e = cudaGetSymbolAddress(&p, g_bool_static_scratch); e != cudaSuccess || !p) {
        cudaGetLastError();
        return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    }
    if (known || current_context_id(&id)) {  // the lookup may have made the context
        int slot = -1;
        for (int k = 0; k < g_static_n && slot < 0; ++k)
            if (g_static[k].ctx_id == id) slot = k;
        if (slot < 0) slot = g_static_n < kMaxContexts ? g_static_n++ : (int)(id % kMaxContexts);
        g_static[slot] = StaticEntry{id, p};
    }
    *out = p;
    return LDNI_OK;
}

}  // namespace
}  // namespace ldni

extern "C" int ldni_boolean_static(const ldni_layers_t *A, const ldni_grid_t *grid_a, const ldni_layers_t *B,
                                   const ldni_grid_t *grid_b, int32_t op, float eps, ldni_layers_t *out,
                                   ldni_info_t *info, void *stream) {
    const ldni_layers_t *all[3] = {A, B, out};
    bool packed = false;
    if (!layers_ok(A, true) || !layers_ok(B, true) || !layers_ok(out, true) || !same_format(all, 3, &packed) ||
        !info || !grid_valid(grid_a) ||
        !grid_valid(grid_b) || op < LDNI_OP_UNION || op > LDNI_OP_DIFF || !(eps >= 0.0f))
        return LDNI_EINVAL;
    if (!same_grid(grid_a, grid_b)) return LDNI_EGRID_MISMATCH;
    const int res = grid_a->res;
    if (res > kStaticMaxRes) return LDNI_ETOOLARGE;
    void *scratch = nullptr;
    int rc = static_scratch(&scratch);
    if (rc != LDNI_OK) return rc;
    // every scratch word is written before it is read (counts by the count
    // pass, chunk totals by the scan), so nothing needs clearing
    Carver c(scratch, kStaticScratchBytes);
    BoolWs w = carve_bool_ws(c, res);
    if (!c.fits()) return LDNI_ETOOLARGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long N = (long long)res * res;
    Side sa = side_of(*A);
    Side sb = side_of(*B);
    Out o = out_of(*out);
    LDNI_LAUNCH(K_BOOL_COUNT, s, bool_pass<false><<<grid_blocks(N), kThreads, 0, s>>>(N, sa, sb, op, eps, w.count, o, info));
    rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    const int *cnt[1] = {w.count};
    int *off[1] = {out->offsets};
    rc = csr_scan(cnt, off, 1, N, w.partials, info, 0, s);
    if (rc != LDNI_OK) return rc;
    LDNI_LAUNCH(K_BOOL_WRITE, s, bool_pass<true><<<grid_blocks(N), kThreads, 0, s>>>(N, sa, sb, op, eps, w.count, o, info));
    return cuda_status();
}
