// Triangle traversal shared by the exact two-pass and the learned one-pass
// samplers: per-thread triangle setup, the exact crossing test and hit masks.
//
// A tile is kTilePix consecutive rays of one image in CSR order (rows
// p = j * res + i), so a tile's samples occupy one contiguous CSR range.
#pragma once

#include <climits>

#include "ldni_host.h"

namespace ldni {

constexpr int kTileBits = 12;
constexpr int kTilePix = 1 << kTileBits;  // rays per tile (= one scan chunk)
static_assert(kTilePix == kScanChunk, "a tile is one scan chunk");
constexpr int kBigPixels = 16;            // pixel-centre box of a thread-handled triangle (fits one mask)
constexpr int kHugePixels = 2048;         // boxes above this take a whole block, smaller big ones a warp
// Largest snapped extent (fixed-point units) of a triangle handled with
// 32-bit edge functions.  With every vertex and every visited pixel centre
// (plus one step beyond the box) within 32768 units of each other, each edge
// function |d_u (c_v - v) - d_v (c_u - u)| < 2 * 32767^2 < 2^31.
constexpr int kSmallExtent = 32000;

// Depth of a crossing, d = sum_k lambda_k a_k with lambda_k = E_k / A2 from
// the exact edge functions E_k (FP32 values of integers) and inv = 1 / A2:
// every operation is an explicit rounding, so every traversal (direct,
// binned, one-pass, batched) computes the same bits wherever it is inlined.
__device__ __forceinline__ float depth_of(float E0, float E1, float E2, float inv, float a0, float a1, float a2) {
    const float l0 = __fmul_rn(E0, inv), l1 = __fmul_rn(E1, inv), l2 = __fmul_rn(E2, inv);
    return __fmaf_rn(l2, a2, __fmaf_rn(l1, a1, __fmul_rn(l0, a0)));
}

// Per-thread view of one triangle: snapped lattice coordinates of its three
// vertices (all three world axes) and the world positions.
struct TriView {
    int q[3][3];  // [vertex][axis]
    float3 p[3];
};

// 0 = ok, else an LDNI_ST_* bit (bad index, unsnappable vertex)
__device__ __forceinline__ unsigned load_tri(const float *__restrict__ verts, const int *__restrict__ tris, int t,
                                             int nv, const GridDev &g, TriView &T) {
    const int id[3] = {__ldg(tris + 3 * (long long)t), __ldg(tris + 3 * (long long)t + 1),
                       __ldg(tris + 3 * (long long)t + 2)};
    if ((unsigned)id[0] >= (unsigned)nv || (unsigned)id[1] >= (unsigned)nv || (unsigned)id[2] >= (unsigned)nv)
        return LDNI_ST_INDEX;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float *v = verts + 3 * (long long)id[k];
        T.p[k] = make_float3(__ldg(v), __ldg(v + 1), __ldg(v + 2));
        ok &= snap(T.p[k].x, g.o[0], g.s, T.q[k][0]);
        ok &= snap(T.p[k].y, g.o[1], g.s, T.q[k][1]);
        ok &= snap(T.p[k].z, g.o[2], g.s, T.q[k][2]);
    }
    return ok ? 0u : LDNI_ST_RANGE;
}

__device__ __forceinline__ int owns_i(int du, int dv) { return (dv > 0 || (dv == 0 && du < 0)) ? 1 : 0; }

// Counter-clockwise projection of one triangle on one image, 32-bit form.
struct Setup32 {
    int u0, v0, u1, v1, u2, v2;
    float a0, a1, a2;
    int b0, b1, b2;
    float inv;  // 1 / area2
    int i0, j0, w, h;  // pixel-centre box: i0 .. i0+w-1, j0 .. j0+h-1
    int exiting;       // 1 if the face's projection was counter-clockwise (n_a > 0: the ray leaves the solid)

    // biased edge functions at pixel (i, j): inside iff all three are > 0
    __device__ __forceinline__ void edges(int i, int j, int &e0, int &e1, int &e2) const {
        const int cu = i * kSubpix + kHalfSubpix, cv = j * kSubpix + kHalfSubpix;
        e0 = (u1 - u0) * (cv - v0) - (v1 - v0) * (cu - u0) + b0;
        e1 = (u2 - u1) * (cv - v1) - (v2 - v1) * (cu - u1) + b1;
        e2 = (u0 - u2) * (cv - v2) - (v0 - v2) * (cu - u2) + b2;
    }
    // depth from the biased edge functions at a crossing: lambda_k from the
    // exact edge functions (bias removed); the edge opposite vertex k is k+1
    __device__ __forceinline__ float depth_from(int e0, int e1, int e2) const {
        return depth_of(__int2float_rn(e1 - b1), __int2float_rn(e2 - b2), __int2float_rn(e0 - b0), inv, a0, a1, a2);
    }
    __device__ __forceinline__ float depth(int i, int j) const {
        int e0, e1, e2;
        edges(i, j, e0, e1, e2);
        return depth_from(e0, e1, e2);
    }
    // visit every crossed pixel centre of the box: f(i, j, e0, e1, e2), with
    // the biased edge functions at that centre.  A box of at most 2 x 2
    // pixel centres (nearly every triangle of a mesh finer than the pixel
    // grid) is tested without a loop, so that the lanes of a warp, whose
    // boxes differ, run the same instructions; a larger box builds its hit
    // mask first and then visits the mask's bits.  Either way the crossings
    // come in row-major order.
    template <class F>
    __device__ __forceinline__ void for_each_hit(F &&f) const;
    // the box's crossings as bits x + w y (w * h <= kBigPixels)
    __device__ __forceinline__ unsigned hit_bits() const;
};

// 64-bit form for triangles too large for Setup32.
struct Setup64 {
    long long u0, v0, u1, v1, u2, v2;
    float a0, a1, a2;
    long long b0, b1, b2;
    float inv;
    int exiting;
    __device__ __forceinline__ void edges(int i, int j, long long &e0, long long &e1, long long &e2) const {
        const long long cu = (long long)i * kSubpix + kHalfSubpix, cv = (long long)j * kSubpix + kHalfSubpix;
        e0 = (u1 - u0) * (cv - v0) - (v1 - v0) * (cu - u0) + b0;
        e1 = (u2 - u1) * (cv - v1) - (v2 - v1) * (cu - u1) + b1;
        e2 = (u0 - u2) * (cv - v2) - (v0 - v2) * (cu - u2) + b2;
    }
    __device__ __forceinline__ bool inside(int i, int j) const {
        long long e0, e1, e2;
        edges(i, j, e0, e1, e2);
        return e0 > 0 && e1 > 0 && e2 > 0;
    }
    __device__ __forceinline__ float depth(int i, int j) const {
        long long e0, e1, e2;
        edges(i, j, e0, e1, e2);
        return depth_of(__ll2float_rn(e1 - b1), __ll2float_rn(e2 - b2), __ll2float_rn(e0 - b0), inv, a0, a1, a2);
    }
};

enum AxisKind { kNone = 0, kSmall = 1, kBig = 2 };

// Box test and (for small triangles) the 32-bit setup of image A; the
// reciprocal area for depths only when kDepth.
template <int A, bool kDepth = true>
__device__ __forceinline__ int setup_axis(const TriView &T, int res, Setup32 &S) {
    constexpr int U = (A + 1) % 3, V = (A + 2) % 3;
    int u0 = T.q[0][U], u1 = T.q[1][U], u2 = T.q[2][U];
    int v0 = T.q[0][V], v1 = T.q[1][V], v2 = T.q[2][V];
    const int umin = min(u0, min(u1, u2)), umax = max(u0, max(u1, u2));
    const int vmin = min(v0, min(v1, v2)), vmax = max(v0, max(v1, v2));
    // pixel centres 256 i + 128 inside [umin, umax] x [vmin, vmax]
    const int i0 = max((umin + 127) >> 8, 0), i1 = min((umax - 128) >> 8, res - 1);
    const int j0 = max((vmin + 127) >> 8, 0), j1 = min((vmax - 128) >> 8, res - 1);
    if (i0 > i1 || j0 > j1) return kNone;
    S.w = i1 - i0 + 1;
    S.h = j1 - j0 + 1;
    if (umax - umin >= kSmallExtent || vmax - vmin >= kSmallExtent || S.w * S.h > kBigPixels) return kBig;
    int A2 = (u1 - u0) * (v2 - v0) - (v1 - v0) * (u2 - u0);
    if (A2 == 0) return kNone;  // face parallel to the ray (Definition 1 note)
    float a0 = comp(T.p[0], A), a1 = comp(T.p[1], A), a2 = comp(T.p[2], A);
    S.exiting = A2 > 0 ? 1 : 0;
    if (A2 < 0) {  // turn counter-clockwise
        int x = u1; u1 = u2; u2 = x;
        x = v1; v1 = v2; v2 = x;
        const float y = a1; a1 = a2; a2 = y;
        A2 = -A2;
    }
    S.u0 = u0; S.v0 = v0; S.u1 = u1; S.v1 = v1; S.u2 = u2; S.v2 = v2;
    S.a0 = a0; S.a1 = a1; S.a2 = a2;
    S.b0 = owns_i(u1 - u0, v1 - v0);
    S.b1 = owns_i(u2 - u1, v2 - v1);
    S.b2 = owns_i(u0 - u2, v0 - v2);
    S.inv = kDepth ? __frcp_rn(__int2float_rn(A2)) : 0.0f;
    S.i0 = i0; S.j0 = j0; S.w = i1 - i0 + 1; S.h = j1 - j0 + 1;
    return kSmall;
}

// Crossings of the pixel box as a bit mask (bit b = pixel (i0 + b % w, j0 + b / w)).
__device__ __forceinline__ unsigned long long hit_mask(const Setup32 &S) {
    int r0, r1, r2;
    S.edges(S.i0, S.j0, r0, r1, r2);
    const int s0 = -(S.v1 - S.v0) * kSubpix, s1 = -(S.v2 - S.v1) * kSubpix, s2 = -(S.v0 - S.v2) * kSubpix;
    const int t0 = (S.u1 - S.u0) * kSubpix, t1 = (S.u2 - S.u1) * kSubpix, t2 = (S.u0 - S.u2) * kSubpix;
    unsigned long long m = 0;
    int bit = 0;
    for (int y = 0; y < S.h; ++y) {
        int e0 = r0, e1 = r1, e2 = r2;
        for (int x = 0; x < S.w; ++x, ++bit) {
            if ((e0 > 0) & (e1 > 0) & (e2 > 0)) m |= 1ull << bit;
            e0 += s0;
            e1 += s1;
            e2 += s2;
        }
        r0 += t0;
        r1 += t1;
        r2 += t2;
    }
    return m;
}

template <class F>
__device__ __forceinline__ void Setup32::for_each_hit(F &&f) const {
    if (w <= 2 && h <= 2) {
        // Edge functions one step beyond the box stay within int32: see kSmallExtent.
        int r0, r1, r2;
        edges(i0, j0, r0, r1, r2);
        const int s0 = -(v1 - v0) * kSubpix, s1 = -(v2 - v1) * kSubpix, s2 = -(v0 - v2) * kSubpix;
        const int t0 = (u1 - u0) * kSubpix, t1 = (u2 - u1) * kSubpix, t2 = (u0 - u2) * kSubpix;
        const unsigned w2 = w == 2, h2 = h == 2;
        const unsigned c00 = (r0 > 0) & (r1 > 0) & (r2 > 0);
        const unsigned c10 = w2 & (r0 + s0 > 0) & (r1 + s1 > 0) & (r2 + s2 > 0);
        const unsigned c01 = h2 & (r0 + t0 > 0) & (r1 + t1 > 0) & (r2 + t2 > 0);
        const unsigned c11 = w2 & h2 & (r0 + s0 + t0 > 0) & (r1 + s1 + t1 > 0) & (r2 + s2 + t2 > 0);
        unsigned m = c00 | (c10 << 1) | (c01 << 2) | (c11 << 3);  // bit x + 2 y
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const int x = b & 1, y = b >> 1;
            f(i0 + x, j0 + y, r0 + x * s0 + y * t0, r1 + x * s1 + y * t1, r2 + x * s2 + y * t2);
        }
        return;
    }
    const unsigned long long m = hit_mask(*this);
    const unsigned long long row_mask = w >= 64 ? ~0ull : ((1ull << w) - 1);
    for (int y = 0; y < h; ++y) {
        unsigned long long r = (m >> (y * w)) & row_mask;
        while (r) {
            const int x = __ffsll((long long)r) - 1;
            r &= r - 1;
            int e0, e1, e2;
            edges(i0 + x, j0 + y, e0, e1, e2);
            f(i0 + x, j0 + y, e0, e1, e2);
        }
    }
}

__device__ __forceinline__ unsigned Setup32::hit_bits() const {
    if (w <= 2 && h <= 2) {  // loop-free, as in for_each_hit
        int r0, r1, r2;
        edges(i0, j0, r0, r1, r2);
        const int s0 = -(v1 - v0) * kSubpix, s1 = -(v2 - v1) * kSubpix, s2 = -(v0 - v2) * kSubpix;
        const int t0 = (u1 - u0) * kSubpix, t1 = (u2 - u1) * kSubpix, t2 = (u0 - u2) * kSubpix;
        const unsigned w2 = w == 2, h2 = h == 2;
        const unsigned c00 = (r0 > 0) & (r1 > 0) & (r2 > 0);
        const unsigned c10 = w2 & (r0 + s0 > 0) & (r1 + s1 > 0) & (r2 + s2 > 0);
        const unsigned c01 = h2 & (r0 + t0 > 0) & (r1 + t1 > 0) & (r2 + t2 > 0);
        const unsigned c11 = w2 & h2 & (r0 + s0 + t0 > 0) & (r1 + s1 + t1 > 0) & (r2 + s2 + t2 > 0);
        return c00 | (c10 << 1) | (c01 << w) | (c11 << (w + 1));  // bit x + w y
    }
    return (unsigned)hit_mask(*this);
}

// 64-bit setup of image a for a queued big triangle; false when parallel.
__device__ __forceinline__ bool setup_big(const TriView &T, int a, int res, Setup64 &S, int &i0, int &i1, int &j0,
                                          int &j1) {
    const int U = (a + 1) % 3, V = (a + 2) % 3;
    long long u0 = T.q[0][U], u1 = T.q[1][U], u2 = T.q[2][U];
    long long v0 = T.q[0][V], v1 = T.q[1][V], v2 = T.q[2][V];
    long long A2 = (u1 - u0) * (v2 - v0) - (v1 - v0) * (u2 - u0);
    if (A2 == 0) return false;
    float a0 = comp(T.p[0], a), a1 = comp(T.p[1], a), a2 = comp(T.p[2], a);
    S.exiting = A2 > 0 ? 1 : 0;
    if (A2 < 0) {
        long long x = u1; u1 = u2; u2 = x;
        x = v1; v1 = v2; v2 = x;
        const float y = a1; a1 = a2; a2 = y;
        A2 = -A2;
    }
    S.u0 = u0; S.v0 = v0; S.u1 = u1; S.v1 = v1; S.u2 = u2; S.v2 = v2;
    S.a0 = a0; S.a1 = a1; S.a2 = a2;
    S.b0 = (v1 - v0 > 0 || (v1 == v0 && u1 - u0 < 0)) ? 1 : 0;
    S.b1 = (v2 - v1 > 0 || (v2 == v1 && u2 - u1 < 0)) ? 1 : 0;
    S.b2 = (v0 - v2 > 0 || (v0 == v2 && u0 - u2 < 0)) ? 1 : 0;
    S.inv = __frcp_rn(__ll2float_rn(A2));
    const long long umin = min(u0, min(u1, u2)), umax = max(u0, max(u1, u2));
    const long long vmin = min(v0, min(v1, v2)), vmax = max(v0, max(v1, v2));
    i0 = (int)max((umin + 127) >> 8, 0ll);
    i1 = (int)min((umax - 128) >> 8, (long long)res - 1);
    j0 = (int)max((vmin + 127) >> 8, 0ll);
    j1 = (int)min((vmax - 128) >> 8, (long long)res - 1);
    return i0 <= i1 && j0 <= j1;
}

// Queue of big (triangle, image) pairs: boxes up to kHugePixels from the
// front (a warp each), larger ones from the back (a block each); n[0], n[1]
// count the two ends.  The queue holds qcap entries.
template <class Code>
__device__ __forceinline__ void enqueue_big(Code *q, long long qcap, int *n, Code code, long long npx) {
    if (npx > kHugePixels)
        q[qcap - 1 - atomicAdd(n + 1, 1)] = code;
    else
        q[atomicAdd(n, 1)] = code;
}

// Visit every queued pair with body(code, first, step), which walks the
// pair's box pixels first, first + step, ...  Blocks blk of nblk: the
// medium pairs a warp each; the huge pairs are shared out to groups of
// nblk / (huge pairs) blocks (at least one), each group sweeping its pairs
// with all its threads, so that a few faces of hundreds of thousands of
// pixels keep every SM busy and many huge faces run side by side.
// huge_blocks is unused (kept for the callers' launch shapes).
template <class Code, class F>
__device__ __forceinline__ void for_each_big(const Code *q, long long qcap, const int *n, int blk, int nblk,
                                             int huge_blocks, F &&body) {
    (void)huge_blocks;
    const int nmed = n[0];
    const int wpb = blockDim.x >> 5;
    for (int e = blk * wpb + (threadIdx.x >> 5); e < nmed; e += nblk * wpb)
        body(q[e], (int)(threadIdx.x & 31), 32);
    const int nh = n[1];
    if (nh <= 0) return;
    const int G = max(1, nblk / nh);  // blocks per huge pair
    const int groups = nblk / G, grp = blk / G, sub = blk - grp * G;
    if (grp >= groups) return;  // the blocks left over when nblk is no multiple of G
    for (int e = grp; e < nh; e += groups)
        body(q[qcap - 1 - e], sub * (int)blockDim.x + (int)threadIdx.x, G * (int)blockDim.x);
}

__device__ __forceinline__ bool key_less(float d0, int t0, float d1, int t1) {
    return d0 < d1 || (d0 == d1 && t0 < t1);
}

// In-place insertion sort of one ray's samples (SoA arrays) by (depth, tri).
// Normals: FP32 in X, Y, Z, or packed 8-bit words in X with Y = Z = nullptr
// (moved as raw bits).
__device__ __forceinline__ void sort_ray_global(long long b, long long e, float *D, int *Tr, float *X, float *Y,
                                                float *Z) {
    const bool three = Y != nullptr;
    for (long long x = b + 1; x < e; ++x) {
        const float d = D[x];
        const int t = Tr[x];
        const float nx = X[x], ny = three ? Y[x] : 0.0f, nz = three ? Z[x] : 0.0f;
        long long y = x - 1;
        while (y >= b && key_less(d, t, D[y], Tr[y])) {
            D[y + 1] = D[y];
            Tr[y + 1] = Tr[y];
            X[y + 1] = X[y];
            if (three) {
                Y[y + 1] = Y[y];
                Z[y + 1] = Z[y];
            }
            --y;
        }
        D[y + 1] = d;
        Tr[y + 1] = t;
        X[y + 1] = nx;
        if (three) {
            Y[y + 1] = ny;
            Z[y + 1] = nz;
        }
    }
}


// ---- ordering by ranks ------------------------------------------------------------
// Sample i of a ray moves to position b + rank(i), the rank counting the
// samples with a smaller key (equal keys, which valid input never has, by
// index).  The key maps the depth's bits to an unsigned order in which -0 and
// +0 are equal, as under key_less, then the triangle index; every key is
// below ~0 because triangle indices are below INT_MAX.

__device__ __forceinline__ unsigned long long sort_key(float d, int t) {
    unsigned u = __float_as_uint(__fadd_rn(d, 0.0f));
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned)(t ^ (int)0x80000000);
}

__device__ __forceinline__ int key_tri(unsigned long long k) { return (int)((unsigned)k ^ 0x80000000u); }

__device__ __forceinline__ int rank_step(unsigned long long kj, unsigned long long ki, int j, int i) {
    return (kj < ki) | ((kj == ki) & (j < i));
}

constexpr int kLanePer = 4;        // a lane orders rays of up to 4 samples by itself
constexpr int kWarpSortMax = 128;  // longest ray a warp stages in shared memory
constexpr int kRankMax = 768;      // longest ray ordered by ranks in place

// one warp's staging area (3 KB): 128 samples, or 4 per lane, or 768 ranks
struct SortStage {
    unsigned long long key[kWarpSortMax];
    float d[kWarpSortMax], x[kWarpSortMax], y[kWarpSortMax], z[kWarpSortMax];
};
static_assert(sizeof(SortStage) >= kRankMax * sizeof(int), "ranks fit the stage");

struct RayOut {
    float *D;
    int *Tr;
    float *X, *Y, *Z;  // FP32 normals, or packed 8-bit normals in X with Y = Z = nullptr
};

// source of a ray's samples that sits where the ordered ray goes
struct InPlace {
    RayOut o;
    long long b;
    __device__ __forceinline__ void operator()(int i, float &d, int &t, float &x, float &y, float &z) const {
        d = o.D[b + i];
        t = o.Tr[b + i];
        x = o.X[b + i];
        y = o.Y ? o.Y[b + i] : 0.0f;
        z = o.Y ? o.Z[b + i] : 0.0f;
    }
};

__device__ __forceinline__ void stage_put(SortStage &st, int s, float d, int t, float x, float y, float z) {
    st.key[s] = sort_key(d, t);
    st.d[s] = d;
    st.x[s] = x;
    st.y[s] = y;
    st.z[s] = z;
}

__device__ __forceinline__ void stage_get(const SortStage &st, int s, const RayOut &o, long long dst) {
    o.D[dst] = st.d[s];
    o.Tr[dst] = key_tri(st.key[s]);
    o.X[dst] = st.x[s];
    if (o.Y) {
        o.Y[dst] = st.y[s];
        o.Z[dst] = st.z[s];
    }
}

// Stages samples [0, n) at slots base + i, then writes each to b + its rank
// among them; every sample is read before the first store.  kWarp: the 32
// lanes share the ray (lane l takes samples l, l + 32, ...); else one lane
// orders it alone.
template <bool kWarp, class Src>
__device__ __forceinline__ void rank_staged(long long b, int n, const Src &src, const RayOut &o, SortStage &st,
                                            int lane, int base) {
    const int first = kWarp ? lane : 0, step = kWarp ? 32 : 1;
    for (int i = first; i < n; i += step) {
        float d, x, y, z;
        int t;
        src(i, d, t, x, y, z);
        stage_put(st, base + i, d, t, x, y, z);
    }
    if (kWarp) __syncwarp();
    for (int i = first; i < n; i += step) {
        const unsigned long long ki = st.key[base + i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += rank_step(st.key[base + j], ki, j, i);
        stage_get(st, base + i, o, b + r);
    }
    if (kWarp) __syncwarp();
}

// In-place ordering of a ray of kWarpSortMax < n <= kRankMax samples by the
// warp: ranks from the keys in global memory, then the permutation applied
// cycle by cycle by the first lane.
__device__ __forceinline__ void rank_long(long long b, int n, const RayOut &o, SortStage &st, int lane) {
    int *rank = reinterpret_cast<int *>(&st);
    for (int i = lane; i < n; i += 32) {
        const unsigned long long ki = sort_key(o.D[b + i], o.Tr[b + i]);
        int r = 0;
        for (int j = 0; j < n; ++j) r += rank_step(sort_key(o.D[b + j], o.Tr[b + j]), ki, j, i);
        rank[i] = r;
    }
    __syncwarp();
    if (lane == 0) {
        const InPlace at{o, b};
        for (int s0 = 0; s0 < n; ++s0) {
            int pos = rank[s0];
            if (pos < 0 || pos == s0) continue;
            rank[s0] = -1;
            float d, x, y, z;
            int t;
            at(s0, d, t, x, y, z);
            while (pos != s0) {  // carry the element to its place, pick up the one there
                const long long q = b + pos;
                float d2, x2, y2, z2;
                int t2;
                at(pos, d2, t2, x2, y2, z2);
                o.D[q] = d;
                o.Tr[q] = t;
                o.X[q] = x;
                if (o.Y) {
                    o.Y[q] = y;
                    o.Z[q] = z;
                }
                const int nxt = rank[pos];
                rank[pos] = -1;
                d = d2, t = t2, x = x2, y = y2, z = z2;
                pos = nxt;
            }
            o.D[b + s0] = d;
            o.Tr[b + s0] = t;
            o.X[b + s0] = x;
            if (o.Y) {
                o.Y[b + s0] = y;
                o.Z[b + s0] = z;
            }
        }
    }
    __syncwarp();
}

__device__ __forceinline__ RayOut shfl_out(const RayOut &o, int src) {
    RayOut r;
    r.D = reinterpret_cast<float *>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(o.D), src));
    r.Tr = reinterpret_cast<int *>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(o.Tr), src));
    r.X = reinterpret_cast<float *>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(o.X), src));
    r.Y = reinterpret_cast<float *>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(o.Y), src));
    r.Z = reinterpret_cast<float *>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(o.Z), src));
    return r;
}

// Orders the rays of the 32 lanes of a warp; every lane calls it, with n = 0
// when it has nothing to order.  Rays of up to kLanePer samples are ordered
// by their own lane, up to kWarpSortMax by the warp from the staged samples,
// up to kRankMax by the warp in place (their samples must already sit at b),
// longer ones by their lane's insertion.  make(sb, b, o) gives the source of
// a ray whose samples are read from sb and go to b in o.  kOneOut: o is the
// same in every lane.
template <bool kOneOut, class Make>
__device__ __forceinline__ void order_warp_rays(long long b, int n, long long sb, const Make &make, const RayOut &o,
                                                SortStage &st, int lane) {
    if (n >= 2 && n <= kLanePer) rank_staged<false>(b, n, make(sb, b, o), o, st, lane, kLanePer * lane);
    if (n > kRankMax) sort_ray_global(b, b + n, o.D, o.Tr, o.X, o.Y, o.Z);
    __syncwarp();
    unsigned deep = __ballot_sync(0xffffffffu, n > kLanePer && n <= kRankMax);
    while (deep) {
        const int src = __ffs(deep) - 1;
        deep &= deep - 1;
        const RayOut oo = kOneOut ? o : shfl_out(o, src);
        const long long bb = __shfl_sync(0xffffffffu, b, src);
        const long long sbb = __shfl_sync(0xffffffffu, sb, src);
        const int nn = __shfl_sync(0xffffffffu, n, src);
        if (nn <= kWarpSortMax)
            rank_staged<true>(bb, nn, make(sbb, bb, oo), oo, st, lane, 0);
        else
            rank_long(bb, nn, oo, st, lane);
    }
}

}  // namespace ldni
