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
// Two passes: count (one output count per ray), scan to CSR offsets, write.
#include <climits>
#include <mutex>

#include "ldni_host.h"
#include "lookback.cuh"

namespace ldni {
namespace {

constexpr int kThreads = 256;

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

__device__ __forceinline__ bool op_apply(int op, bool a, bool b) {
    return op == LDNI_OP_UNION ? (a || b) : (op == LDNI_OP_INTER ? (a && b) : (a && !b));
}

struct Pick {
    bool from_b;
    long long idx;
    float d;
};

__device__ __forceinline__ void emit(const Pick &s, const Side &A, const Side &B, int op, const Out &o,
                                     long long at, ldni_info_t *info) {
    if (at >= o.cap) {
        set_status(info, LDNI_ST_CAPACITY);
        return;
    }
    o.d[at] = s.d;
    if (!s.from_b) {
        o.nx[at] = A.nx[s.idx];
        o.ny[at] = A.ny[s.idx];
        o.nz[at] = A.nz[s.idx];
        o.tri[at] = A.tri[s.idx];
    } else {
        const float sg = op == LDNI_OP_DIFF ? -1.0f : 1.0f;
        o.nx[at] = sg * B.nx[s.idx];
        o.ny[at] = sg * B.ny[s.idx];
        o.nz[at] = sg * B.nz[s.idx];
        o.tri[at] = (int)((unsigned)B.tri[s.idx] | 0x80000000u);
    }
}

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
        bool inA = false, inB = false, out = false;
        Pick pend{false, 0, 0.0f};
        long long m = 0;
        const long long base = kWrite ? (long long)o.off[p] : 0;
        while (a < ae || b < be) {
            float d;
            if (a < ae && b < be) {
                const float da = A.d[a], db = B.d[b];
                d = da < db ? da : db;
            } else {
                d = a < ae ? A.d[a] : B.d[b];
            }
            const long long fa = a, fb = b;
            while (a < ae && A.d[a] == d) ++a;
            while (b < be && B.d[b] == d) ++b;
            const bool flipA = ((a - fa) & 1) != 0;
            const bool flipB = ((b - fb) & 1) != 0;
            inA ^= flipA;
            inB ^= flipB;
            const bool now = op_apply(op, inA, inB);
            if (now == out) continue;
            out = now;
            const Pick cur = flipA ? Pick{false, fa, d} : Pick{true, fb, d};
            if (now) {
                pend = cur;
            } else if (!(__fsub_rn(d, pend.d) < eps)) {
                if (kWrite) {
                    emit(pend, A, B, op, o, base + m, info);
                    emit(cur, A, B, op, o, base + m + 1, info);
                }
                m += 2;
            }
        }
        if (!kWrite) out_count[p] = (int)m;
    }
}

// ---- fused single-launch Boolean --------------------------------------
//
// One block owns a tile of kTileRays consecutive rays, taken in kRounds
// rounds of kFusedThreads consecutive rays (lane k of a warp holds ray p + k,
// so a warp's loads and stores touch neighbouring CSR rows).  It merges every
// ray once to count its output samples, scans the counts inside the block,
// obtains the tile's starting offset by decoupled look-back, writes the tile's
// CSR offsets, then merges again (inputs now hot in L1/L2) and writes the
// samples.  One launch per image; the workspace is one status word per tile.
constexpr int kFusedThreads = 256;
constexpr int kRounds = 4;
constexpr int kTileRays = kFusedThreads * kRounds;

// Merge one ray.  kWrite = false: returns the output count.  kWrite = true:
// writes the samples from `at` on.
template <bool kWrite>
__device__ __forceinline__ int merge_ray(long long p, const Side &A, const Side &B, int op, float eps,
                                         const Out &o, long long at, ldni_info_t *info) {
    long long a = A.off[p], ae = A.off[p + 1];
    long long b = B.off[p], be = B.off[p + 1];
    if (!kWrite && (((ae - a) | (be - b)) & 1)) {
        atomicAdd(&info->odd_rays, 1u);
        set_status(info, LDNI_ST_ODD);
    }
    if (ae > A.cap || be > B.cap) {
        if (!kWrite) set_status(info, LDNI_ST_CAPACITY);
        ae = min(ae, A.cap);
        be = min(be, B.cap);
        a = min(a, ae);
        b = min(b, be);
    }
    bool inA = false, inB = false, out = false;
    Pick pend{false, 0, 0.0f};
    int m = 0;
    while (a < ae || b < be) {
        const float da = a < ae ? A.d[a] : 0.0f;
        const float db = b < be ? B.d[b] : 0.0f;
        const float d = (a < ae && (b >= be || da <= db)) ? da : db;
        const long long fa = a, fb = b;
        while (a < ae && A.d[a] == d) ++a;
        while (b < be && B.d[b] == d) ++b;
        const bool flipA = ((a - fa) & 1) != 0;
        const bool flipB = ((b - fb) & 1) != 0;
        inA ^= flipA;
        inB ^= flipB;
        const bool now = op_apply(op, inA, inB);
        if (now == out) continue;
        out = now;
        const Pick cur = flipA ? Pick{false, fa, d} : Pick{true, fb, d};
        if (now) {
            pend = cur;
        } else if (!(__fsub_rn(d, pend.d) < eps)) {
            if (kWrite) {
                emit(pend, A, B, op, o, at + m, info);
                emit(cur, A, B, op, o, at + m + 1, info);
            }
            m += 2;
        }
    }
    return m;
}

__global__ void __launch_bounds__(kFusedThreads, 4) bool_fused(long long N, Side A, Side B, int op, float eps,
                                                               Out o, unsigned long long *words, int ntiles,
                                                               ldni_info_t *info) {
    __shared__ long long sh[kFusedThreads / 32 + 1];
    __shared__ int s_tile;
    __shared__ long long s_base;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(words + ntiles, 1ull);
    __syncthreads();
    const int tile = s_tile;
    const long long p0 = (long long)tile * kTileRays + threadIdx.x;  // round r: ray p0 + r * kFusedThreads
    int cnt[kRounds];
    long long excl[kRounds];
    long long total = 0;
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const long long p = p0 + (long long)r * kFusedThreads;
        cnt[r] = p < N ? merge_ray<false>(p, A, B, op, eps, o, 0, info) : 0;
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {  // rays in order: round by round, lane by lane
        long long tot;
        excl[r] = total + block_exclusive_scan<kFusedThreads>(cnt[r], sh, &tot);
        total += tot;
    }
    if (threadIdx.x < 32) {
        const long long b = lookback_warp(words, tile, total, info);
        if (threadIdx.x == 0) s_base = b;
    }
    __syncthreads();
    const long long base = s_base;
    int *off = const_cast<int *>(o.off);
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const long long p = p0 + (long long)r * kFusedThreads;
        if (p < N) off[p] = (int)min(base + excl[r], (long long)INT_MAX);
    }
    if (tile == ntiles - 1 && threadIdx.x == 0) {
        const long long n_out = base + total;
        off[N] = (int)min(n_out, (long long)INT_MAX);
        info->n[0] = n_out;
        if (n_out > INT_MAX) set_status(info, LDNI_ST_TOOLARGE);
        if (n_out > o.cap) set_status(info, LDNI_ST_CAPACITY);
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const long long p = p0 + (long long)r * kFusedThreads;
        if (p < N && cnt[r] > 0) merge_ray<true>(p, A, B, op, eps, o, base + excl[r], info);
    }
}

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

bool layers_ok(const ldni_layers_t *L, bool need) {
    if (!L || !L->offsets || L->capacity < 0) return false;
    if (need && L->capacity > 0 && (!L->depth || !L->nx || !L->ny || !L->nz || !L->tri_id)) return false;
    return true;
}

}  // namespace
}  // namespace ldni

using namespace ldni;

namespace ldni {
namespace {
int fused_tiles(long long N) { return (int)((N + kTileRays - 1) / kTileRays); }
}  // namespace
}  // namespace ldni

extern "C" int ldni_boolean_workspace_size(int32_t res, size_t *bytes) {
    if (!bytes || res < 1 || res > 8192) return LDNI_EINVAL;
    *bytes = align_up(sizeof(unsigned long long) * (size_t)(fused_tiles((long long)res * res) + 1));
    return LDNI_OK;
}

extern "C" int ldni_boolean(const ldni_layers_t *A, const ldni_grid_t *grid_a, const ldni_layers_t *B,
                            const ldni_grid_t *grid_b, int32_t op, float eps, ldni_layers_t *out, ldni_info_t *info,
                            void *ws, size_t ws_bytes, void *stream) {
    if (!layers_ok(A, true) || !layers_ok(B, true) || !layers_ok(out, true) || !info || !ws ||
        !grid_valid(grid_a) || !grid_valid(grid_b) || op < LDNI_OP_UNION || op > LDNI_OP_DIFF || !(eps >= 0.0f))
        return LDNI_EINVAL;
    if (grid_a->res != grid_b->res || grid_a->width != grid_b->width || grid_a->origin[0] != grid_b->origin[0] ||
        grid_a->origin[1] != grid_b->origin[1] || grid_a->origin[2] != grid_b->origin[2])
        return LDNI_EGRID_MISMATCH;
    const int res = grid_a->res;
    const long long N = (long long)res * res;
    const int ntiles = fused_tiles(N);
    if (ws_bytes < sizeof(unsigned long long) * (size_t)(ntiles + 1)) return LDNI_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long *words = static_cast<unsigned long long *>(ws);
    if (cudaMemsetAsync(words, 0, sizeof(unsigned long long) * (size_t)(ntiles + 1), s) != cudaSuccess)
        return LDNI_ECUDA;
    Side sa{A->capacity, A->offsets, A->depth, A->nx, A->ny, A->nz, A->tri_id};
    Side sb{B->capacity, B->offsets, B->depth, B->nx, B->ny, B->nz, B->tri_id};
    Out o{out->offsets, out->depth, out->nx, out->ny, out->nz, out->tri_id, out->capacity};
    LDNI_LAUNCH(K_BOOL_FUSED, s,
                bool_fused<<<ntiles, kFusedThreads, 0, s>>>(N, sa, sb, op, eps, o, words, ntiles, info));
    return cuda_status();
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

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {nullptr};

// Device address of the static scratch on the current device.  The host-side
// symbol is only a stand-in, so the address is looked up once per device.
int static_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LDNI_ECUDA;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bool_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LDNI_ECUDA;
        }
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return LDNI_OK;
}

}  // namespace
}  // namespace ldni

extern "C" int ldni_boolean_static(const ldni_layers_t *A, const ldni_grid_t *grid_a, const ldni_layers_t *B,
                                   const ldni_grid_t *grid_b, int32_t op, float eps, ldni_layers_t *out,
                                   ldni_info_t *info, void *stream) {
    if (!layers_ok(A, true) || !layers_ok(B, true) || !layers_ok(out, true) || !info || !grid_valid(grid_a) ||
        !grid_valid(grid_b) || op < LDNI_OP_UNION || op > LDNI_OP_DIFF || !(eps >= 0.0f))
        return LDNI_EINVAL;
    if (grid_a->res != grid_b->res || grid_a->width != grid_b->width || grid_a->origin[0] != grid_b->origin[0] ||
        grid_a->origin[1] != grid_b->origin[1] || grid_a->origin[2] != grid_b->origin[2])
        return LDNI_EGRID_MISMATCH;
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
    Side sa{A->capacity, A->offsets, A->depth, A->nx, A->ny, A->nz, A->tri_id};
    Side sb{B->capacity, B->offsets, B->depth, B->nx, B->ny, B->nz, B->tri_id};
    Out o{out->offsets, out->depth, out->nx, out->ny, out->nz, out->tri_id, out->capacity};
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
