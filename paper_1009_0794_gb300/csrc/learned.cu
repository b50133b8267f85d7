// LDNI sampling in one traversal with a learned per-tile layer capacity.
//
// The exact form counts every ray's crossings before it can place them
// (Section 3: the stencil pass that finds each pixel's depth complexity n_p,
// then one rendering pass per layer).  Here a small network predicts, for
// every tile of kTilePix rays, how many layers k_t its rays can have, so the
// mesh is traversed once:
//
//   features : per tile, from a 1-in-`stride` subsample of the triangles:
//              triangle count, projected area in pixels, mean |n_a|, and an
//              8-bin histogram of triangle depth (a proxy for layering);
//   mlp      : features -> log1p(k_t) -> an even capacity k_t (mlp.cuh);
//   layout   : every ray of tile t owns k_t slab slots (reserved by the
//              mlp launch with one atomic per tile);
//   one pass : every crossing takes the next slot of its ray (the atomic
//              cursor is also the ray's exact count) and stores (depth, tri)
//              if it fits, else marks its tile as overflowed; two-layer
//              tiles place crossings by orientation instead (see onepass_hit);
//   scan     : exact CSR offsets from the counts; two-layer tiles are
//              checked in the same pass;
//   redo     : tiles that overflowed are filled again by the exact method
//              (a second traversal restricted to them; no-op when none did);
//   gather   : every ray is ordered by (depth, tri_id) and written to its CSR
//              rows, normals from the per-triangle table the pass wrote.
//
// Depths, normals and ordering come from the same device functions as the
// exact two-pass form, so both forms produce identical LDNIs.
#include <cuda_bf16.h>

#include "mlp.cuh"
#include "sample_common.cuh"

namespace ldni {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxLayerCap = 64;   // largest k_t the layout hands out
#ifndef LDNI_ONEPASS_BATCH
#define LDNI_ONEPASS_BATCH 2
#endif
#ifndef LDNI_ONEPASS_BLOCKS
#define LDNI_ONEPASS_BLOCKS 5
#endif
// resident blocks per SM of the one-pass traversal (5 measured fastest of 4, 5, 6 and 8)
constexpr int kOnepassBlocksPerSm = LDNI_ONEPASS_BLOCKS;

struct LImg {
    int *count[3];
    int *exitc[3];               // crossings whose face leaves the solid (two-layer tiles)
    const int *offsets[3];
    float *depth[3];
    float *nx[3];
    float *ny[3];
    float *nz[3];
    int *tri[3];
    long long cap[3];
    // per tile
    float *feat[3];              // [ntiles][kRawFeat]
    int *kcap[3];                // layers per ray
    long long *slab_base[3];     // first slab slot of the tile
    int *over[3];                // 1 = overflowed, redone exactly
    unsigned *deep[3];           // per image, bit c of word w: chunk 32 w + c (rays 32 (32 w + c) ...) has a
                                 // ray of more than kLanePer samples, ordered by order_deep
    int2 *slab;                  // (depth bits, tri) per slot
    float4 *nrm;                 // per-triangle unit normal (x, y, z, 0): one 16-byte load per sample
    long long slab_cap;
    int *any_over;
    ldni_info_t *info;           // the call's status (checked builds report out-of-range indices there)
    bool pairs8;                 // every output array 8-byte aligned (a pair at an even slot: one 8-byte store)
};

template <class T>
__device__ __forceinline__ T pick3(T const (&arr)[3], int a) {
    return a == 0 ? arr[0] : (a == 1 ? arr[1] : arr[2]);
}

// ---- features --------------------------------------------------------------

// Tile of one triangle on image A and its feature contributions; tile -1
// when it covers no pixel centre.
template <int A>
__device__ __forceinline__ int feature_of(const TriView &T, const GridDev &g, float &area_px, int &bin) {
    constexpr int U = (A + 1) % 3, V = (A + 2) % 3;
    const int u0 = T.q[0][U], u1 = T.q[1][U], u2 = T.q[2][U];
    const int v0 = T.q[0][V], v1 = T.q[1][V], v2 = T.q[2][V];
    const int umin = min(u0, min(u1, u2)), umax = max(u0, max(u1, u2));
    const int vmin = min(v0, min(v1, v2)), vmax = max(v0, max(v1, v2));
    const int i0 = max((umin + 127) >> 8, 0), i1 = min((umax - 128) >> 8, g.res - 1);
    const int j0 = max((vmin + 127) >> 8, 0), j1 = min((vmax - 128) >> 8, g.res - 1);
    if (i0 > i1 || j0 > j1) return -1;
    const long long p = (long long)((j0 + j1) >> 1) * g.res + ((i0 + i1) >> 1);
    const float du1 = (float)(u1 - u0), dv1 = (float)(v1 - v0), du2 = (float)(u2 - u0), dv2 = (float)(v2 - v0);
    area_px = fabsf(du1 * dv2 - dv1 * du2) * (0.5f / (kSubpix * kSubpix));
    const float ca = (comp(T.p[0], A) + comp(T.p[1], A) + comp(T.p[2], A)) * (1.0f / 3.0f);
    const float rel = (ca - g.o[A]) * g.s / (float)(kSubpix * g.res);  // 0..1 across the cube
    bin = min(7, max(0, (int)(rel * 8.0f)));
    return (int)(p >> kTileBits);
}

// Every lane of the warp calls this.  The warp walks the distinct tiles its
// lanes hit (usually one or two: neighbouring triangles) and adds each
// tile's sums with one set of atomics.
template <int A>
__device__ __forceinline__ void feature_axis(const TriView &T, bool valid, float w, const GridDev &g, const LImg &o,
                                             float absn) {
    float area = 0.0f;
    int bin = 0;
    const int tile = valid ? feature_of<A>(T, g, area, bin) : -1;
    unsigned todo = __ballot_sync(0xffffffffu, tile >= 0);
    while (todo) {
        const int t = __shfl_sync(0xffffffffu, tile, __ffs(todo) - 1);
        const bool mine = tile == t;
        const unsigned grp = __ballot_sync(0xffffffffu, mine);
        todo &= ~grp;
        float ar = mine ? area * w : 0.0f, an = mine ? absn * w : 0.0f;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            ar += __shfl_xor_sync(0xffffffffu, ar, d);
            an += __shfl_xor_sync(0xffffffffu, an, d);
        }
        unsigned bins[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) bins[k] = __popc(__ballot_sync(0xffffffffu, mine && bin == k));
        if ((threadIdx.x & 31) == 0) {
            float *f = pick3(o.feat, A) + (long long)t * kRawFeat;
            atomicAdd(f + 0, (float)__popc(grp) * w);
            atomicAdd(reinterpret_cast<unsigned *>(f + 1), to_fixed(ar, kAreaFix));
            atomicAdd(reinterpret_cast<unsigned *>(f + 2), to_fixed(an, kNormalFix));
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (bins[k]) atomicAdd(f + 3 + k, (float)bins[k] * w);
        }
    }
}

// Thread = (sampled triangle, image): blockIdx.y is the image, so each
// thread's chain of dependent work is one triangle on one image.  The sample
// is 1 in `stride` triangles taken as runs of kFeatRun consecutive ones
// (sample s is triangle (s / kFeatRun) * kFeatRun * stride + s % kFeatRun): a
// warp's lanes then hold a few groups of neighbouring triangles, which mostly
// share a tile, while the runs still spread over the whole mesh.
constexpr int kFeatRun = 8;
__device__ __host__ __forceinline__ long long feature_samples(long long nt, int stride) {
    const long long run = (long long)kFeatRun * stride;
    return (nt + run - 1) / run * kFeatRun;
}

__global__ void __launch_bounds__(kThreads) features_kernel(const float *__restrict__ verts,
                                                            const int *__restrict__ tris, int nt, int nv, GridDev g,
                                                            int ax_lo, int stride, LImg o) {
    const int a = ax_lo + blockIdx.y;
    const long long nsamp = feature_samples(nt, stride);
    const float w = (float)stride;
    // uniform loop bound per block: whole warps take part in the collectives
    for (long long base = (long long)blockIdx.x * blockDim.x; base < nsamp; base += (long long)gridDim.x * blockDim.x) {
        const long long sidx = base + threadIdx.x;
        TriView T;
        bool valid = false;
        float nx = 0.f, ny = 0.f, nz = 0.f;
        const long long t = (sidx / kFeatRun) * kFeatRun * stride + sidx % kFeatRun;
        if (sidx < nsamp && t < nt) {
            valid = load_tri(verts, tris, (int)t, nv, g, T) == 0;
            if (valid) face_normal(T.p[0], T.p[1], T.p[2], nx, ny, nz);
        }
        if (a == 0)  // block-uniform
            feature_axis<0>(T, valid, w, g, o, fabsf(nx));
        else if (a == 1)
            feature_axis<1>(T, valid, w, g, o, fabsf(ny));
        else
            feature_axis<2>(T, valid, w, g, o, fabsf(nz));
    }
}

// ---- capacity: network or fixed ---------------------------------------------

__device__ __forceinline__ int capacity_from(float y, float margin) {
    const float layers = expm1f(fmaxf(y, 0.0f)) * (1.0f + margin);
    int k = (int)ceilf(layers - 1e-3f);
    k = (k + 1) & ~1;  // rays of closed meshes have even counts
    return min(max(k, 2), kMaxLayerCap);
}

// Two warps per tile, one hidden unit per lane (warp h of the pair owns units
// 32 h .. 32 h + 31); the weights sit in shared memory and the activations of
// the pair's tile in a shared buffer, four inputs per load.  Each unit sums
// its inputs in order with FP32 FMAs on the BF16 weights, so predictions
// agree with ldni_mlp_forward's to FP32 rounding (the capacity is a hint
// either way).  Each tile then reserves its npix * k_t slab slots with one
// atomic on the slab cursor (any order is a valid layout: the gather reads a
// tile's base, and a tile that no longer fits gets k_t = 0, i.e. its
// crossings all go to the exact redo).
constexpr int kCapWarps = 8;
constexpr int kCapTiles = kCapWarps / 2;

__device__ __forceinline__ void reserve_slab(const LImg &o, int a, int tile, long long nrays, int kt,
                                             unsigned long long *cursor) {
    const long long npix = min((long long)kTilePix, nrays - ((long long)tile << kTileBits));
    const unsigned long long need = (unsigned long long)(npix * kt);
    const unsigned long long start = atomicAdd(cursor, need);
    const bool fits = start + need <= (unsigned long long)o.slab_cap;
    pick3(o.kcap, a)[tile] = fits ? kt : 0;
    pick3(o.slab_base, a)[tile] = fits ? (long long)start : 0;
}

__global__ void __launch_bounds__(kCapWarps * 32) capacity_kernel(int ntiles, long long nrays, int ax_lo, int naxes,
                                                                  LImg o, const __nv_bfloat16 *__restrict__ W,
                                                                  const float *__restrict__ b, float margin,
                                                                  int fixed_k, unsigned long long *cursor) {
    // weights row-major [unit][in] as given, rows padded to an odd number of 32-bit words so that the
    // 32 lanes (32 units) reading the same input pair hit 32 different banks
    constexpr int kRow0 = kMlpIn / 2 + 1, kRowH = kMlpHidden / 2 + 1;  // words per padded row
    constexpr int kS1 = kMlpHidden * kRow0, kS2 = kS1 + kMlpHidden * kRowH, kS3 = kS2 + kMlpHidden * kRowH;
    __shared__ unsigned sw[kS3 + kMlpHidden / 2];
    __shared__ float sb[kMlpBiases];
    __shared__ __align__(16) float act[kCapTiles][2][kMlpHidden];
    __shared__ float part[kCapTiles];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pr = warp >> 1, half = warp & 1;
    const int k = blockIdx.x * kCapTiles + pr;
    const bool valid = k < ntiles * naxes;
    const int a = ax_lo + (valid ? k / ntiles : 0), tile = valid ? k % ntiles : 0;
    if (W) {
        // copy in 32-bit words (pairs of inputs of one unit; rows have an even length), every load of
        // the thread issued before the first store
        constexpr int kWords = kMlpWeights / 2, kPer = (kWords + kCapWarps * 32 - 1) / (kCapWarps * 32);
        const bool w_aligned = (reinterpret_cast<uintptr_t>(W) & 3) == 0;
        const unsigned *W2 = reinterpret_cast<const unsigned *>(W);
        const unsigned short *W1 = reinterpret_cast<const unsigned short *>(W);
        unsigned v[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int q = (int)threadIdx.x + r * kCapWarps * 32;
            v[r] = q >= kWords ? 0u
                               : (w_aligned ? W2[q] : ((unsigned)W1[2 * q] | ((unsigned)W1[2 * q + 1] << 16)));
        }
        const float bias = threadIdx.x < kMlpBiases ? b[threadIdx.x] : 0.0f;
        float *x = act[pr][0];
        if (valid && half == 0 && lane == 0) {
            const long long p0 = (long long)tile << kTileBits;
            const float frac = (float)min((long long)kTilePix, nrays - p0) / (float)kTilePix;
            normalise_features(pick3(o.feat, a) + (long long)tile * kRawFeat, frac, x);
        }
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int q = (int)threadIdx.x + r * kCapWarps * 32;
            if (q >= kWords) continue;
            const int i = 2 * q;
            int dst;
            if (i < kW1) {
                dst = (i / kMlpIn) * kRow0 + (i % kMlpIn) / 2;
            } else if (i < kW3) {
                const int base = i < kW2 ? kW1 : kW2, rr = i - base;
                dst = (i < kW2 ? kS1 : kS2) + (rr / kMlpHidden) * kRowH + (rr % kMlpHidden) / 2;
            } else {
                dst = kS3 + (i - kW3) / 2;
            }
            sw[dst] = v[r];
        }
        if (threadIdx.x < kMlpBiases) sb[threadIdx.x] = bias;
    }
    __syncthreads();
    if (!W) {
        if (valid && half == 0 && lane == 0) reserve_slab(o, a, tile, nrays, fixed_k, cursor);
    } else {
        const int u = 32 * half + lane;
        // unit u of a layer: inputs in order, two weights per shared load, four inputs per activation load
        auto unit = [&](const float *in, int n_in, const unsigned *row, int boff) {
            float acc = sb[boff + u];
            const float4 *in4 = reinterpret_cast<const float4 *>(in);
            for (int q = 0; q < n_in / 4; ++q) {
                const float4 v = in4[q];
                const unsigned w01 = row[2 * q], w23 = row[2 * q + 1];
                acc = fmaf(__uint_as_float(w01 << 16), v.x, acc);
                acc = fmaf(__uint_as_float(w01 & 0xffff0000u), v.y, acc);
                acc = fmaf(__uint_as_float(w23 << 16), v.z, acc);
                acc = fmaf(__uint_as_float(w23 & 0xffff0000u), v.w, acc);
            }
            return fmaxf(acc, 0.0f);
        };
        float *b0 = act[pr][0], *b1 = act[pr][1];
        b1[u] = unit(b0, kMlpIn, sw + u * kRow0, kB0);
        __syncthreads();
        b0[u] = unit(b1, kMlpHidden, sw + kS1 + u * kRowH, kB1);  // every read of b0 (layer 0) is before the barrier
        __syncthreads();
        b1[u] = unit(b0, kMlpHidden, sw + kS2 + u * kRowH, kB2);
        __syncthreads();
        const unsigned w3 = sw[kS3 + u / 2];
        float y = __uint_as_float((u & 1) ? (w3 & 0xffff0000u) : (w3 << 16)) * b1[u];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) y += __shfl_xor_sync(0xffffffffu, y, d);
        if (half == 1 && lane == 0) part[pr] = y;
        __syncthreads();
        if (valid && half == 0 && lane == 0)
            reserve_slab(o, a, tile, nrays, capacity_from(y + part[pr] + sb[kB3], margin), cursor);
    }
}

// ---- one pass ----------------------------------------------------------------

// A tile given two layers per ray takes the shortcut of closed meshes: a ray
// crossed twice is entered once and left once, so the entering crossing
// takes slot 0 and the leaving one slot 1 - no returned atomic, only counts.
// The scan (csr_scan with ScanVerify) later sends every tile where some ray
// broke that pattern to the exact redo.
__device__ __forceinline__ void onepass_hit(int a, long long p, float d, int t, const float3 &n, int exiting,
                                            const LImg &o) {
    const int tile = (int)(p >> kTileBits);
    const int kt = pick3(o.kcap, a)[tile];
    if (kt == 2) {
        atomicAdd(pick3(o.count, a) + p, 1);
        if (exiting) atomicAdd(pick3(o.exitc, a) + p, 1);
        const long long slot = pick3(o.slab_base, a)[tile] + (p & (kTilePix - 1)) * 2 + exiting;
        if (range_ok(slot, slot + 1, o.slab_cap, o.info)) o.slab[slot] = make_int2(__float_as_int(d), t);
        return;
    }
    const int k = atomicAdd(pick3(o.count, a) + p, 1);
    if (k < kt) {
        const long long slot = pick3(o.slab_base, a)[tile] + (p & (kTilePix - 1)) * kt + k;
        if (range_ok(slot, slot + 1, o.slab_cap, o.info)) o.slab[slot] = make_int2(__float_as_int(d), t);
    } else {
        pick3(o.over, a)[tile] = 1;
        *o.any_over = 1;
    }
}

// The crossings of one (triangle, image) pair, kHitBatch at a time: their
// tiles' layer counts are read, then every slot of a tile with more than two
// layers is claimed (a returned atomic on the ray's count) before any sample
// is stored, so the claims' round trips overlap instead of following one
// another.  Two-layer tiles take the shortcut of onepass_hit.  m: the box's
// crossings, bit x + w y for pixel (i0 + x, j0 + y).
constexpr int kHitBatch = LDNI_ONEPASS_BATCH;
template <int A>
__device__ __forceinline__ void onepass_hits(const Setup32 &S, unsigned m, int t, const float3 &n, int res,
                                             const LImg &o) {
    const int wdiv = (256 + S.w - 1) / S.w;  // y = (b * wdiv) >> 8 = b / w for b < 16, w <= 16
    int *cnt = pick3(o.count, A);
    const int *kc = pick3(o.kcap, A);
    const long long *sb = pick3(o.slab_base, A);
    while (m) {
        int pr[kHitBatch], kt[kHitBatch], k[kHitBatch];
        float d[kHitBatch];
        long long base[kHitBatch];
        bool v[kHitBatch];
#pragma unroll
        for (int u = 0; u < kHitBatch; ++u) {
            v[u] = m != 0u;
            const int b = v[u] ? __ffs(m) - 1 : 0;
            m &= m - 1u;
            const int y = (b * wdiv) >> 8, x = b - y * S.w;
            int e0, e1, e2;
            S.edges(S.i0 + x, S.j0 + y, e0, e1, e2);
            pr[u] = (S.j0 + y) * res + S.i0 + x;
            d[u] = S.depth_from(e0, e1, e2);
            const int tile = pr[u] >> kTileBits;
            kt[u] = v[u] ? kc[tile] : 2;
            base[u] = v[u] ? sb[tile] : 0;
        }
#pragma unroll
        for (int u = 0; u < kHitBatch; ++u) k[u] = v[u] && kt[u] != 2 ? atomicAdd(cnt + pr[u], 1) : 0;
#pragma unroll
        for (int u = 0; u < kHitBatch; ++u) {
            if (!v[u]) continue;
            const int q = pr[u] & (kTilePix - 1);
            long long slot;
            if (kt[u] == 2) {
                atomicAdd(cnt + pr[u], 1);
                if (S.exiting) atomicAdd(pick3(o.exitc, A) + pr[u], 1);
                slot = base[u] + q * 2 + S.exiting;
            } else if (k[u] < kt[u]) {
                slot = base[u] + (long long)q * kt[u] + k[u];
            } else {
                pick3(o.over, A)[pr[u] >> kTileBits] = 1;
                *o.any_over = 1;
                continue;
            }
            if (range_ok(slot, slot + 1, o.slab_cap, o.info)) o.slab[slot] = make_int2(__float_as_int(d[u]), t);
        }
    }
}

template <int A>
__device__ __forceinline__ void onepass_axis(const TriView &T, int t, const float3 &n, int res, const LImg &o,
                                             int *big_q, long long qcap, int *big_n) {
    Setup32 S;
    const int kind = setup_axis<A>(T, res, S);
    if (kind == kNone) return;
    if (kind == kBig) {
        enqueue_big(big_q, qcap, big_n, t * 4 + A, (long long)S.w * S.h);
        return;
    }
    if (kHitBatch > 1 && (S.w > 2 || S.h > 2)) {  // (boxes of up to 2 x 2 centres: the loop-free visit)
        onepass_hits<A>(S, S.hit_bits(), t, n, res, o);
        return;
    }
    S.for_each_hit([&](int i, int j, int e0, int e1, int e2) {
        onepass_hit(A, (long long)j * res + i, S.depth_from(e0, e1, e2), t, n, S.exiting, o);
    });
}

__global__ void __launch_bounds__(kThreads, kOnepassBlocksPerSm) onepass_kernel(const float *__restrict__ verts,
                                                           const int *__restrict__ tris, int nt, int nv, GridDev g,
                                                           int ax_lo, int ax_hi, LImg o, int *big_q, long long qcap,
                                                           int *big_n,
                                                           ldni_info_t *info) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        TriView T;
        const unsigned bad = load_tri(verts, tris, t, nv, g, T);
        if (bad) {
            set_status(info, bad);
            continue;
        }
        float3 n;
        face_normal(T.p[0], T.p[1], T.p[2], n.x, n.y, n.z);
        // coalesced: the gather looks normals up by triangle (w: the packed
        // 8-bit normal, when the images take packed normals)
        const float w8 = pick3(o.ny, ax_lo) ? 0.0f : __uint_as_float(encode_normal8(n.x, n.y, n.z));
        o.nrm[t] = make_float4(n.x, n.y, n.z, w8);
        if (ax_lo <= 0 && 0 <= ax_hi) onepass_axis<0>(T, t, n, g.res, o, big_q, qcap, big_n);
        if (ax_lo <= 1 && 1 <= ax_hi) onepass_axis<1>(T, t, n, g.res, o, big_q, qcap, big_n);
        if (ax_lo <= 2 && 2 <= ax_hi) onepass_axis<2>(T, t, n, g.res, o, big_q, qcap, big_n);
    }
}

__global__ void __launch_bounds__(kThreads) onepass_big(const float *__restrict__ verts, const int *__restrict__ tris,
                                                        int nv, GridDev g, LImg o, const int *big_q, long long qcap,
                                                        const int *big_n, int huge_blocks) {
    for_each_big(big_q, qcap, big_n, (int)blockIdx.x, (int)gridDim.x, huge_blocks, [&](int code, int first, int step) {
        const int t = code >> 2, a = code & 3;
        TriView T;
        if (load_tri(verts, tris, t, nv, g, T)) return;
        Setup64 S;
        int i0, i1, j0, j1;
        if (!setup_big(T, a, g.res, S, i0, i1, j0, j1)) return;
        float3 n;
        face_normal(T.p[0], T.p[1], T.p[2], n.x, n.y, n.z);
        const int w = i1 - i0 + 1;
        const long long npx = (long long)w * (j1 - j0 + 1);
        for (long long k = first; k < npx; k += step) {
            const int j = j0 + (int)(k / w), i = i0 + (int)(k % w);
            if (S.inside(i, j)) onepass_hit(a, (long long)j * g.res + i, S.depth(i, j), t, n, S.exiting, o);
        }
    });
}

// ---- exact redo of overflowed tiles ------------------------------------------

__device__ __forceinline__ void redo_hit(int a, long long p, float d, int t, const LImg &o, const float3 &n,
                                         ldni_info_t *info) {
    if (!pick3(o.over, a)[p >> kTileBits]) return;
    const int k = atomicSub(pick3(o.count, a) + p, 1) - 1;
    const long long slot = (long long)pick3(o.offsets, a)[p] + k;
    if (k < 0 || slot >= pick3(o.cap, a)) {
        set_status(info, LDNI_ST_CAPACITY);
        return;
    }
    if (!range_ok(slot, slot + 1, pick3(o.cap, a), info)) return;
    pick3(o.depth, a)[slot] = d;
    pick3(o.tri, a)[slot] = t;
    if (float *Y = pick3(o.ny, a)) {
        pick3(o.nx, a)[slot] = n.x;
        Y[slot] = n.y;
        pick3(o.nz, a)[slot] = n.z;
    } else {  // approximate normals (Section 3 item 1)
        pick3(o.nx, a)[slot] = __uint_as_float(encode_normal8(n.x, n.y, n.z));
    }
}

template <int A>
__device__ __forceinline__ void redo_axis(const TriView &T, int t, const float3 &n, int res, const LImg &o,
                                          ldni_info_t *info) {
    {  // skip the edge setup unless the triangle's pixel box reaches a redone tile
        constexpr int U = (A + 1) % 3, V = (A + 2) % 3;
        const int umin = min(T.q[0][U], min(T.q[1][U], T.q[2][U])), umax = max(T.q[0][U], max(T.q[1][U], T.q[2][U]));
        const int vmin = min(T.q[0][V], min(T.q[1][V], T.q[2][V])), vmax = max(T.q[0][V], max(T.q[1][V], T.q[2][V]));
        const int i0 = max((umin + 127) >> 8, 0), i1 = min((umax - 128) >> 8, res - 1);
        const int j0 = max((vmin + 127) >> 8, 0), j1 = min((vmax - 128) >> 8, res - 1);
        if (i0 > i1 || j0 > j1) return;
        const int t0 = (int)(((long long)j0 * res + i0) >> kTileBits);
        const int t1 = (int)(((long long)j1 * res + i1) >> kTileBits);
        if (t1 - t0 < 4) {
            const int *over = pick3(o.over, A);
            bool any = false;
            for (int t = t0; t <= t1; ++t) any |= over[t] != 0;
            if (!any) return;
        }
    }
    Setup32 S;
    if (setup_axis<A>(T, res, S) != kSmall) return;  // big triangles: redo_big
    S.for_each_hit([&](int i, int j, int e0, int e1, int e2) {
        redo_hit(A, (long long)j * res + i, S.depth_from(e0, e1, e2), t, o, n, info);
    });
}

__device__ __forceinline__ void redo_big_block(const float *__restrict__ verts, const int *__restrict__ tris, int nv,
                                               const GridDev &g, const LImg &o, const int *big_q, long long qcap,
                                               const int *big_n, int blk, int nblk, ldni_info_t *info) {
    for_each_big(big_q, qcap, big_n, blk, nblk, max(1, nblk / 3), [&](int code, int first, int step) {
        const int t = code >> 2, a = code & 3;
        TriView T;
        if (load_tri(verts, tris, t, nv, g, T)) return;
        Setup64 S;
        int i0, i1, j0, j1;
        if (!setup_big(T, a, g.res, S, i0, i1, j0, j1)) return;
        float3 n;
        face_normal(T.p[0], T.p[1], T.p[2], n.x, n.y, n.z);
        const int w = i1 - i0 + 1;
        const long long npx = (long long)w * (j1 - j0 + 1);
        for (long long k = first; k < npx; k += step) {
            const int j = j0 + (int)(k / w), i = i0 + (int)(k % w);
            if (S.inside(i, j)) redo_hit(a, (long long)j * g.res + i, S.depth(i, j), t, o, n, info);
        }
    });
}

// One launch for both redo traversals: blocks below tri_blocks walk the
// triangles, the others the big-triangle queue.  Nothing to do (the usual
// case) costs one load per block.
__global__ void __launch_bounds__(kThreads) redo_kernel(const float *__restrict__ verts, const int *__restrict__ tris,
                                                        int nt, int nv, GridDev g, int ax_lo, int ax_hi, LImg o,
                                                        const int *big_q, long long qcap, const int *big_n,
                                                        int tri_blocks,
                                                        ldni_info_t *info) {
    if (*(volatile int *)o.any_over == 0) return;
    if (blockIdx.x >= tri_blocks) {
        redo_big_block(verts, tris, nv, g, o, big_q, qcap, big_n, blockIdx.x - tri_blocks, gridDim.x - tri_blocks,
                       info);
        return;
    }
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += tri_blocks * blockDim.x) {
        TriView T;
        if (load_tri(verts, tris, t, nv, g, T)) continue;
        float3 n;
        face_normal(T.p[0], T.p[1], T.p[2], n.x, n.y, n.z);
        if (ax_lo <= 0 && 0 <= ax_hi) redo_axis<0>(T, t, n, g.res, o, info);
        if (ax_lo <= 1 && 1 <= ax_hi) redo_axis<1>(T, t, n, g.res, o, info);
        if (ax_lo <= 2 && 2 <= ax_hi) redo_axis<2>(T, t, n, g.res, o, info);
    }
}


// ---- gather ----------------------------------------------------------------------

// (n_over, if given: the number of redone tiles, counted by the thread of each
// tile's first ray; cleared before the launch.)
struct SlabSrc {  // a ray's samples in its tile's slab, normals from the table
    const int2 *slab;
    const float4 *nrm;
    long long s0;
    bool packed;  // the packed 8-bit normal (table entry w) in x
    __device__ __forceinline__ void operator()(int i, float &d, int &t, float &x, float &y, float &z) const {
        const int2 v = slab[s0 + i];
        d = __int_as_float(v.x);
        t = v.y;
        const float4 q = nrm[v.y];
        x = packed ? q.w : q.x;
        y = q.y;
        z = q.z;
    }
};

__device__ __forceinline__ void put_sample(const RayOut &o, long long at, float d, int t, float x, float y, float z) {
    o.D[at] = d;
    o.Tr[at] = t;
    o.X[at] = x;
    if (o.Y) {
        o.Y[at] = y;
        o.Z[at] = z;
    }
}

#ifndef LDNI_GATHER_BLOCKS
#define LDNI_GATHER_BLOCKS 8
#endif
__global__ void __launch_bounds__(kThreads, LDNI_GATHER_BLOCKS) gather_kernel(long long nrays, int ax_lo, LImg o,
                                                                             ldni_info_t *info,
                                                          int *n_over) {
    const int a = ax_lo + blockIdx.y;
    const int *off = pick3(o.offsets, a);
    const RayOut r{pick3(o.depth, a), pick3(o.tri, a), pick3(o.nx, a), pick3(o.ny, a), pick3(o.nz, a)};
    const long long cap = pick3(o.cap, a);
    const int *over = pick3(o.over, a);
    const int *kc = pick3(o.kcap, a);
    const long long *sb = pick3(o.slab_base, a);
    unsigned *deep = pick3(o.deep, a);
    const float4 *NRM = o.nrm;
    const int lane = threadIdx.x & 31;
    // a warp takes 32 consecutive rays, which lie in one tile (tiles are
    // multiples of 32 rays): the tile's values are loaded once per warp
    for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); base < nrays;
         base += (long long)gridDim.x * blockDim.x) {
        const long long p = base + lane;
        const bool act = p < nrays;
        const int tile = (int)(base >> kTileBits);
        int t_over = 0, kt = 0;
        long long tbase = 0;
        if (lane == 0) {
            t_over = over[tile];
            kt = kc[tile];
            tbase = sb[tile];
            if (n_over && (base & (kTilePix - 1)) == 0 && t_over) atomicAdd(n_over, 1);
        }
        t_over = __shfl_sync(0xffffffffu, t_over, 0);
        kt = __shfl_sync(0xffffffffu, kt, 0);
        tbase = __shfl_sync(0xffffffffu, tbase, 0);
        const long long b = act ? off[p] : 0;
        long long e = __shfl_down_sync(0xffffffffu, b, 1);
        if (lane == 31 && act) e = off[p + 1];
        if (!act) continue;
        if (lane < 31 && p + 1 == nrays) e = off[p + 1];  // the last ray of the image
        const int c = (int)(e - b);
        if (c & 1) {
            atomicAdd(&info->odd_rays, 1u);
            set_status(info, LDNI_ST_ODD);
        }
        if (c == 0) continue;
        if (e > cap) {
            set_status(info, LDNI_ST_CAPACITY);
            continue;
        }
        if (!t_over && c > kt) {  // cannot happen for a tile that did not overflow
            set_status(info, LDNI_ST_CAPACITY);
            continue;
        }
        if (c > kLanePer) {  // ordered by order_deep, from where the samples are now
            atomicOr(deep + (p >> 10), 1u << ((p >> 5) & 31));
            continue;
        }
        const long long s0 = tbase + (p & (kTilePix - 1)) * kt;
        if (!range_ok(b, e, cap, info) || (!t_over && !range_ok(s0, s0 + c, o.slab_cap, info))) continue;
        if (t_over) {  // filled exactly by the redo pass: order in place
            sort_ray_global(b, e, r.D, r.Tr, r.X, r.Y, r.Z);
            continue;
        }
        if (c == 2) {  // the common case: everything in registers
            int2 v0, v1;
            if ((s0 & 1) == 0) {  // the slot pair is one 16-byte record
                const int4 v = *reinterpret_cast<const int4 *>(o.slab + s0);
                v0 = make_int2(v.x, v.y);
                v1 = make_int2(v.z, v.w);
            } else {
                v0 = o.slab[s0];
                v1 = o.slab[s0 + 1];
            }
            if (key_less(__int_as_float(v1.x), v1.y, __int_as_float(v0.x), v0.y)) {
                const int2 w = v0;
                v0 = v1;
                v1 = w;
            }
            const float4 q0 = NRM[v0.y], q1 = NRM[v1.y];
            if (o.pairs8 && (b & 1) == 0) {  // even slots (closed meshes): one 8-byte store per field
                *reinterpret_cast<int2 *>(r.D + b) = make_int2(v0.x, v1.x);
                *reinterpret_cast<int2 *>(r.Tr + b) = make_int2(v0.y, v1.y);
                if (r.Y) {
                    *reinterpret_cast<float2 *>(r.X + b) = make_float2(q0.x, q1.x);
                    *reinterpret_cast<float2 *>(r.Y + b) = make_float2(q0.y, q1.y);
                    *reinterpret_cast<float2 *>(r.Z + b) = make_float2(q0.z, q1.z);
                } else {
                    *reinterpret_cast<float2 *>(r.X + b) = make_float2(q0.w, q1.w);
                }
                continue;
            }
            r.D[b] = __int_as_float(v0.x);
            r.D[b + 1] = __int_as_float(v1.x);
            r.Tr[b] = v0.y;
            r.Tr[b + 1] = v1.y;
            if (r.Y) {
                r.X[b] = q0.x;
                r.X[b + 1] = q1.x;
                r.Y[b] = q0.y;
                r.Y[b + 1] = q1.y;
                r.Z[b] = q0.z;
                r.Z[b + 1] = q1.z;
            } else {
                r.X[b] = q0.w;
                r.X[b + 1] = q1.w;
            }
            continue;
        }
        const SlabSrc src{o.slab, NRM, s0, r.Y == nullptr};  // 1, 3 or 4 samples: copy, then order in place
        for (int x = 0; x < c; ++x) {
            float d, nx, ny, nz;
            int t;
            src(x, d, t, nx, ny, nz);
            put_sample(r, b + x, d, t, nx, ny, nz);
        }
        sort_ray_global(b, e, r.D, r.Tr, r.X, r.Y, r.Z);
    }
}

// The rays of more than kLanePer samples in the chunks of 32 rays that
// gather marked, ordered by whole warps: from the slab, or in place in a
// redone tile.  A warp reads 32 words of marks, then orders the chunks of
// the set bits one after another.
__global__ void __launch_bounds__(kThreads) order_deep(long long nrays, int ax_lo, LImg o) {
    __shared__ SortStage stage[kThreads / 32];
    const int a = ax_lo + blockIdx.y;
    const unsigned *deep = pick3(o.deep, a);
    const int *off = pick3(o.offsets, a);
    const RayOut r{pick3(o.depth, a), pick3(o.tri, a), pick3(o.nx, a), pick3(o.ny, a), pick3(o.nz, a)};
    const long long cap = pick3(o.cap, a);
    const int *over = pick3(o.over, a);
    const int *kc = pick3(o.kcap, a);
    const long long *sb = pick3(o.slab_base, a);
    const int lane = threadIdx.x & 31;
    SortStage &st = stage[threadIdx.x >> 5];
    const auto in_place = [](long long, long long b, const RayOut &ro) { return InPlace{ro, b}; };
    const bool packed = r.Y == nullptr;
    const auto from_slab = [&](long long s0, long long, const RayOut &) { return SlabSrc{o.slab, o.nrm, s0, packed}; };
    const long long nwords = (nrays + 1023) >> 10;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long w0 = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; w0 < nwords;
         w0 += warps * 32) {
        const unsigned word = w0 + lane < nwords ? deep[w0 + lane] : 0u;
        unsigned any = __ballot_sync(0xffffffffu, word != 0u);
        while (any) {
            const int src = __ffs(any) - 1;
            any &= any - 1;
            unsigned bits = __shfl_sync(0xffffffffu, word, src);
            while (bits) {
                const int bit = __ffs(bits) - 1;
                bits &= bits - 1;
                const long long base = ((w0 + src) * 32 + bit) * 32;  // first ray of the chunk
                const int tile = (int)(base >> kTileBits);
                const int t_over = over[tile], kt = kc[tile];
                const long long p = base + lane;
                long long b = 0;
                int n = 0;
                if (p < nrays) {
                    b = off[p];
                    const long long e = off[p + 1];
                    const int c = (int)(e - b);
                    if (c > kLanePer && e <= cap && (t_over || c <= kt)) n = c;
                    const long long s0 = sb[tile] + (p & (kTilePix - 1)) * kt;
                    if (n && (!range_ok(b, e, cap, o.info) || (!t_over && !range_ok(s0, s0 + c, o.slab_cap, o.info))))
                        n = 0;
                }
                if (t_over)  // the same in every lane: a chunk lies in one tile
                    order_warp_rays<true>(b, n, b, in_place, r, st, lane);
                else
                    order_warp_rays<true>(b, n, sb[tile] + (p & (kTilePix - 1)) * kt, from_slab, r, st, lane);
            }
        }
    }
}

// per-tile training targets: log1p of the largest ray count in the tile
__global__ void tile_label_kernel(long long nrays, const int *off, float *label) {
    __shared__ int mx;
    if (threadIdx.x == 0) mx = 0;
    __syncthreads();
    const long long p0 = (long long)blockIdx.x << kTileBits;
    int m = 0;
    for (int q = threadIdx.x; q < kTilePix && p0 + q < nrays; q += blockDim.x) m = max(m, off[p0 + q + 1] - off[p0 + q]);
    atomicMax(&mx, m);
    __syncthreads();
    if (threadIdx.x == 0) label[blockIdx.x] = log1pf((float)mx);
}

__global__ void normalise_kernel(int ntiles, long long nrays, int naxes, const float *raw, float *X) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ntiles * naxes) return;
    const int tile = k % ntiles;
    const long long p0 = (long long)tile << kTileBits;
    const float frac = (float)min((long long)kTilePix, nrays - p0) / (float)kTilePix;
    normalise_features(raw + (long long)k * kRawFeat, frac, X + (long long)k * kMlpIn);
}

// ---- host side -----------------------------------------------------------------

struct LearnedWs {
    int *count[3];
    int *exitc[3];
    int *big_n;
    int *any_over;
    float *feat[3];
    int *over[3];
    unsigned *deep[3];
    size_t clear_bytes;  // counts, flags, features, overflow and deep-ray marks: one memset
    long long *scan_words;
    int *kcap[3];
    long long *slab_base[3];
    int *big_q;
    long long qcap;
    float4 *nrm;
    int2 *slab;
    long long slab_cap;
};

LearnedWs carve_learned_ws(Carver &c, long long nt, int res, int naxes, long long slab_samples) {
    LearnedWs w{};
    const long long N = (long long)res * res;
    const long long stride = (N + 63) / 64 * 64;
    const long long ntiles = (N + kTilePix - 1) / kTilePix;
    const long long tstride = (ntiles + 63) / 64 * 64;
    // one cleared block: counts | 64 ints (queue counts at 0 and 1, any_over at 8, slab cursor at
    // 10..11) | features | overflow marks | exiting counts | deep-ray marks
    const size_t deep_at = (size_t)(stride * naxes + 64 + tstride * naxes * kRawFeat + tstride * naxes + stride * naxes);
    const long long dstride = ((N + 1023) / 1024 + 63) / 64 * 64;  // words of chunk marks per image
    const size_t ints = deep_at + (size_t)dstride * naxes;
    int *block = c.take<int>(ints);
    for (int a = 0; a < naxes; ++a) {
        w.count[a] = block ? block + (size_t)a * stride : nullptr;
        w.exitc[a] = block ? block + (size_t)stride * naxes + 64 + (size_t)tstride * naxes * kRawFeat +
                                 (size_t)tstride * naxes + (size_t)a * stride
                           : nullptr;
        w.feat[a] = block ? reinterpret_cast<float *>(block + (size_t)stride * naxes + 64) + (size_t)a * tstride * kRawFeat
                          : nullptr;
        w.over[a] = block ? block + (size_t)stride * naxes + 64 + (size_t)tstride * naxes * kRawFeat + (size_t)a * tstride
                          : nullptr;
        w.deep[a] = block ? reinterpret_cast<unsigned *>(block + deep_at) + (size_t)a * dstride : nullptr;
    }
    w.big_n = block ? block + (size_t)stride * naxes : nullptr;
    w.any_over = block ? block + (size_t)stride * naxes + 8 : nullptr;
    w.clear_bytes = sizeof(int) * ints;
    w.scan_words = c.take<long long>(csr_scan_partials(N) * naxes);
    int *kc = c.take<int>((size_t)(tstride * naxes));
    long long *sb = c.take<long long>((size_t)(tstride * naxes));
    for (int a = 0; a < naxes; ++a) {
        w.kcap[a] = kc ? kc + (size_t)a * tstride : nullptr;
        w.slab_base[a] = sb ? sb + (size_t)a * tstride : nullptr;
    }
    w.qcap = nt * naxes > 0 ? nt * naxes : 1;
    w.big_q = c.take<int>((size_t)w.qcap);
    w.nrm = c.take<float4>((size_t)(nt > 0 ? nt : 1));
    w.slab = c.take<int2>((size_t)(slab_samples > 0 ? slab_samples : 1));
    w.slab_cap = slab_samples;
    return w;
}

int feature_blocks(long long nt, int stride) {
    const long long nsamp = feature_samples(nt, stride);
    long long b = (nsamp + kThreads - 1) / kThreads;
    const long long lim = (long long)num_sms() * 8;  // one sampled triangle per thread where possible
    return (int)(b < 1 ? 1 : (b > lim ? lim : b));
}

int grid_blocks(long long work) {
    long long b = (work + kThreads - 1) / kThreads;
    const long long lim = (long long)num_sms() * 16;
    if (b > lim) b = lim;
    return (int)(b > 0 ? b : 1);
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_sample_learned_workspace_size(int64_t nv, int64_t nt, int32_t res, int32_t axis,
                                                  int64_t slab_samples, size_t *bytes) {
    if (!bytes || res < 1 || res > 8192 || nt < 0 || nv < 0 || axis < 0 || axis > LDNI_AXIS_ALL || slab_samples < 0)
        return LDNI_EINVAL;
    Carver c(nullptr, 0);
    carve_learned_ws(c, nt, res, axis == LDNI_AXIS_ALL ? 3 : 1, slab_samples);
    *bytes = align_up(c.off);
    return LDNI_OK;
}

extern "C" int ldni_sample_learned(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                                   const ldni_grid_t *grid, int32_t axis, const ldni_mlp_t *mlp, int32_t fixed_layers,
                                   int32_t feature_stride, int64_t slab_samples, ldni_layers_t *out, ldni_info_t *info,
                                   int32_t *overflow_tiles, void *ws, size_t ws_bytes, void *stream) {
    if (!grid_valid(grid) || !out || !info || !ws || axis < 0 || axis > LDNI_AXIS_ALL || nv <= 0 || nt < 0 ||
        (nt > 0 && (!verts || !tris)) || slab_samples < 0 || feature_stride < 1 ||
        (!mlp && (fixed_layers < 0 || fixed_layers > kMaxLayerCap)) || (mlp && (!mlp->w || !mlp->b)))
        return LDNI_EINVAL;
    if (nt > (INT_MAX / 4) || nv > INT_MAX) return LDNI_ETOOLARGE;
    const int ax_lo = axis == LDNI_AXIS_ALL ? 0 : axis, ax_hi = axis == LDNI_AXIS_ALL ? 2 : axis;
    const int naxes = ax_hi - ax_lo + 1;
    Carver c(ws, ws_bytes);
    LearnedWs w = carve_learned_ws(c, nt, grid->res, naxes, slab_samples);
    if (!c.fits()) return LDNI_EWORKSPACE;
    const GridDev g = make_grid(grid);
    const long long N = (long long)grid->res * grid->res;
    const int ntiles = (int)((N + kTilePix - 1) / kTilePix);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LImg o{};
    for (int k = 0; k < naxes; ++k) {
        const int a = ax_lo + k;
        const ldni_layers_t &L = out[k];
        if (!L.offsets || L.capacity < 0 || !samples_ok(L))
            return LDNI_EINVAL;
        o.count[a] = w.count[k];
        o.exitc[a] = w.exitc[k];
        o.offsets[a] = L.offsets;
        o.depth[a] = L.depth;
        normal_arrays(L, o.nx[a], o.ny[a], o.nz[a]);
        o.tri[a] = L.tri_id;
        o.cap[a] = L.capacity;
        o.feat[a] = w.feat[k];
        o.kcap[a] = w.kcap[k];
        o.slab_base[a] = w.slab_base[k];
        o.over[a] = w.over[k];
        o.deep[a] = w.deep[k];
    }
    o.slab = w.slab;
    o.nrm = w.nrm;
    o.slab_cap = w.slab_cap;
    o.any_over = w.any_over;
    o.info = info;
    o.pairs8 = true;
    for (int a = ax_lo; a <= ax_lo + naxes - 1; ++a)
        for (const void *q : {(const void *)o.depth[a], (const void *)o.nx[a], (const void *)o.ny[a],
                              (const void *)o.nz[a], (const void *)o.tri[a]})
            o.pairs8 &= (reinterpret_cast<uintptr_t>(q) & 7) == 0;

    if (int rc_ = cuda_check(cudaMemsetAsync(w.count[0], 0, w.clear_bytes, s))) return rc_;
    if (overflow_tiles) if (int rc_ = cuda_check(cudaMemsetAsync(overflow_tiles, 0, sizeof(int32_t), s))) return rc_;
    if (mlp && nt > 0)
        LDNI_LAUNCH(K_FEATURES, s,
                    features_kernel<<<dim3(feature_blocks(nt, feature_stride), naxes), kThreads, 0, s>>>(
                        verts, tris, (int)nt, (int)nv, g, ax_lo, feature_stride, o));
    const __nv_bfloat16 *W = mlp ? reinterpret_cast<const __nv_bfloat16 *>(mlp->w) : nullptr;
    const float *B = mlp ? mlp->b : nullptr;
    const float margin = mlp ? mlp->margin : 0.0f;
    LDNI_LAUNCH(K_CAPACITY, s,
                capacity_kernel<<<(ntiles * naxes + kCapTiles - 1) / kCapTiles, kCapWarps * 32, 0, s>>>(
                    ntiles, N, ax_lo, naxes, o, W, B, margin, fixed_layers,
                    reinterpret_cast<unsigned long long *>(w.any_over + 2)));  // 8-byte aligned, cleared
    if (nt > 0) {
        // as many blocks as stay resident (five per SM at the kernel's register bound)
        const int op_blocks = (int)min((long long)grid_blocks(nt), (long long)num_sms() * kOnepassBlocksPerSm);
        LDNI_LAUNCH(K_ONEPASS, s,
                    onepass_kernel<<<op_blocks, kThreads, 0, s>>>(verts, tris, (int)nt, (int)nv, g, ax_lo, ax_hi,
                                                                        o, w.big_q, w.qcap, w.big_n, info));
        LDNI_LAUNCH(K_ONEPASS_BIG, s,
                    onepass_big<<<5 * num_sms(), kThreads, 0, s>>>(verts, tris, (int)nv, g, o, w.big_q, w.qcap,
                                                                   w.big_n, num_sms()));
    }
    const int *cnt[3];
    int *off[3];
    for (int k = 0; k < naxes; ++k) {
        cnt[k] = w.count[k];
        off[k] = const_cast<int *>(o.offsets[ax_lo + k]);
    }
    int rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    ScanVerify ver{};
    for (int k = 0; k < naxes; ++k) {
        ver.exitc[k] = w.exitc[k];
        ver.kcap[k] = w.kcap[k];
        ver.over[k] = w.over[k];
    }
    ver.any_over = w.any_over;
    rc = csr_scan(cnt, off, naxes, N, w.scan_words, info, ax_lo, s, nullptr, &ver);
    if (rc != LDNI_OK) return rc;
    if (nt > 0) {
            // the triangle sweep on as many blocks as stay resident (every block
        // exits at once when no tile overflowed), the big-triangle queue on a
        // few more
        const int tri_blocks = (int)min((long long)grid_blocks(nt), (long long)num_sms() * 4);
        LDNI_LAUNCH(K_REDO, s,
                    redo_kernel<<<tri_blocks + num_sms() / 2, kThreads, 0, s>>>(
                        verts, tris, (int)nt, (int)nv, g, ax_lo, ax_hi, o, w.big_q, w.qcap, w.big_n, tri_blocks, info));
    }
    LDNI_LAUNCH(K_GATHER, s,
                gather_kernel<<<dim3(grid_blocks(N), naxes), kThreads, 0, s>>>(N, ax_lo, o, info, overflow_tiles));
    LDNI_LAUNCH(K_ORDER, s,
                order_deep<<<dim3((unsigned)((N + 1023) / 1024 + 255) / 256, naxes), kThreads, 0, s>>>(N, ax_lo, o));
    return cuda_status();
}

extern "C" int ldni_tile_features(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                                  const ldni_grid_t *grid, int32_t axis, int32_t feature_stride, float *raw, float *X,
                                  void *stream) {
    if (!grid_valid(grid) || axis < 0 || axis > LDNI_AXIS_ALL || nv <= 0 || nt < 0 || (nt > 0 && (!verts || !tris)) ||
        feature_stride < 1 || !raw || !X)
        return LDNI_EINVAL;
    if (nt > (INT_MAX / 4) || nv > INT_MAX) return LDNI_ETOOLARGE;
    const int ax_lo = axis == LDNI_AXIS_ALL ? 0 : axis, ax_hi = axis == LDNI_AXIS_ALL ? 2 : axis;
    const int naxes = ax_hi - ax_lo + 1;
    const long long N = (long long)grid->res * grid->res;
    const int ntiles = (int)((N + kTilePix - 1) / kTilePix);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LImg o{};
    for (int k = 0; k < naxes; ++k) o.feat[ax_lo + k] = raw + (size_t)k * ntiles * kRawFeat;
    if (int rc_ = cuda_check(cudaMemsetAsync(raw, 0, sizeof(float) * (size_t)naxes * ntiles * kRawFeat, s))) return rc_;
    if (nt > 0)
        LDNI_LAUNCH(K_FEATURES, s,
                    features_kernel<<<dim3(feature_blocks(nt, feature_stride), naxes), kThreads, 0, s>>>(
                        verts, tris, (int)nt, (int)nv, make_grid(grid), ax_lo, feature_stride, o));
    LDNI_LAUNCH(K_FEATURES, s,
                normalise_kernel<<<(ntiles * naxes + 127) / 128, 128, 0, s>>>(ntiles, N, naxes, raw, X));
    return cuda_status();
}

extern "C" int ldni_tile_labels(const int32_t *offsets, int32_t res, float *label, void *stream) {
    if (!offsets || !label || res < 1 || res > 8192) return LDNI_EINVAL;
    const long long N = (long long)res * res;
    const int ntiles = (int)((N + kTilePix - 1) / kTilePix);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LDNI_LAUNCH(K_FEATURES, s, tile_label_kernel<<<ntiles, 256, 0, s>>>(N, offsets, label));
    return cuda_status();
}
