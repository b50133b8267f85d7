// LDNI sampling of a closed triangle mesh, exact two-pass form (Section 3;
// Definitions 1-4).
//
// The paper renders the mesh n_max + 1 times through a stencil-routed
// OpenGL pipeline: pass 1 counts the depth complexity n_p of every pixel,
// passes 2..n_max each capture the n-th fragment, and the host post-sorts
// every pixel (Section 3, Appendix A).  Here the same count-then-fill
// structure runs as CUDA kernels with everything resident on the device:
//
//   count : one thread per triangle snaps its vertices once and, for each
//           requested image, adds 1 to count[p] for every crossed pixel
//           centre (= the stencil pass);
//   scan  : counts -> CSR offsets (scan.cu);
//   fill  : the same traversal; every crossing takes a slot of its ray with
//           an atomic decrement of count[p] and writes depth, normal and
//           triangle id there (= passes 2..n_max);
//   sort  : every ray orders its samples by (depth, tri_id) in place
//           (= the host post-sort).
//
// Triangles whose pixel box is large are handed to a block-per-triangle
// kernel with 64-bit edge functions.
#include "sample_common.cuh"

namespace ldni {
namespace {

constexpr int kThreads = 256;

struct Img {
    int *count[3];          // per-ray counts (count pass), slot cursors (fill pass)
    const int *offsets[3];  // CSR offsets
    float *depth[3];
    float *nx[3];
    float *ny[3];
    float *nz[3];
    int *tri[3];
    long long cap[3];
};

__device__ __forceinline__ int *sel(int *const (&arr)[3], int a) { return a == 0 ? arr[0] : (a == 1 ? arr[1] : arr[2]); }

// One crossing at depth d: count it, or take the next slot of ray p and store the sample.
template <bool kFill>
__device__ __forceinline__ void emit(float d, int a, int t, long long p, const float3 &n, const Img &o,
                                     ldni_info_t *info) {
    int *cnt = sel(o.count, a);
    if (!kFill) {
        atomicAdd(cnt + p, 1);
        return;
    }
    const int k = atomicSub(cnt + p, 1) - 1;
    const int *off = a == 0 ? o.offsets[0] : (a == 1 ? o.offsets[1] : o.offsets[2]);
    const long long cap = a == 0 ? o.cap[0] : (a == 1 ? o.cap[1] : o.cap[2]);
    const long long slot = (long long)off[p] + k;
    if (k < 0 || slot >= cap) {
        set_status(info, LDNI_ST_CAPACITY);
        return;
    }
    float *D = a == 0 ? o.depth[0] : (a == 1 ? o.depth[1] : o.depth[2]);
    float *X = a == 0 ? o.nx[0] : (a == 1 ? o.nx[1] : o.nx[2]);
    float *Y = a == 0 ? o.ny[0] : (a == 1 ? o.ny[1] : o.ny[2]);
    float *Z = a == 0 ? o.nz[0] : (a == 1 ? o.nz[1] : o.nz[2]);
    int *T = a == 0 ? o.tri[0] : (a == 1 ? o.tri[1] : o.tri[2]);
    D[slot] = d;
    T[slot] = t;
    if (Y) {
        X[slot] = n.x;
        Y[slot] = n.y;
        Z[slot] = n.z;
    } else {  // approximate normals (Section 3 item 1)
        X[slot] = __uint_as_float(encode_normal8(n.x, n.y, n.z));
    }
}

// The fill pass over a triangle's box, two crossings at a time: both slot
// claims (returned atomics on the rays' cursors) and both row offsets are in
// flight before either sample is stored.  m: the box's crossings, bit x + w y.
template <int A>
__device__ __forceinline__ void fill_hits(const Setup32 &S, unsigned m, int t, const float3 &n, const Img &o, int res,
                                          ldni_info_t *info) {
    const int wdiv = (256 + S.w - 1) / S.w;  // y = (b * wdiv) >> 8 = b / w for b < 16, w <= 16
    int *cnt = o.count[A];
    const int *off = o.offsets[A];
    const long long cap = o.cap[A];
    while (m) {
        int pr[2], k[2], row[2];
        float d[2];
        bool v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            v[u] = m != 0u;
            const int b = v[u] ? __ffs(m) - 1 : 0;
            m &= m - 1u;
            const int y = (b * wdiv) >> 8, x = b - y * S.w;
            int e0, e1, e2;
            S.edges(S.i0 + x, S.j0 + y, e0, e1, e2);
            pr[u] = (S.j0 + y) * res + S.i0 + x;
            d[u] = S.depth_from(e0, e1, e2);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            k[u] = v[u] ? atomicSub(cnt + pr[u], 1) - 1 : -1;
            row[u] = v[u] ? off[pr[u]] : 0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (!v[u]) continue;
            const long long slot = (long long)row[u] + k[u];
            if (k[u] < 0 || slot >= cap) {
                set_status(info, LDNI_ST_CAPACITY);
                continue;
            }
            o.depth[A][slot] = d[u];
            o.tri[A][slot] = t;
            if (float *Y = o.ny[A]) {
                o.nx[A][slot] = n.x;
                Y[slot] = n.y;
                o.nz[A][slot] = n.z;
            } else {  // approximate normals (Section 3 item 1)
                o.nx[A][slot] = __uint_as_float(encode_normal8(n.x, n.y, n.z));
            }
        }
    }
}

template <bool kFill, int A>
__device__ __forceinline__ void tri_axis(const TriView &T, int t, const float3 &n, const Img &o, int res, int *big_q,
                                         long long qcap, int *big_n, ldni_info_t *info) {
    Setup32 S;
    const int kind = setup_axis<A, kFill>(T, res, S);
    if (kind == kNone) return;
    if (kind == kBig) {
        if (!kFill) enqueue_big(big_q, qcap, big_n, t * 4 + A, (long long)S.w * S.h);  // the fill pass reuses it
        return;
    }
    if (!kFill) {
        S.for_each_hit([&](int i, int j, int, int, int) { atomicAdd(o.count[A] + (long long)j * res + i, 1); });
        return;
    }
    fill_hits<A>(S, S.hit_bits(), t, n, o, res, info);
}

// One thread per triangle; big triangles are queued (count pass) for big_pass.
template <bool kFill>
__global__ void __launch_bounds__(kThreads) tri_pass(const float *__restrict__ verts, const int *__restrict__ tris,
                                                     int nt, int nv, GridDev g, int ax_lo, int ax_hi, Img o,
                                                     int *big_q, long long qcap, int *big_n, ldni_info_t *info) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        TriView T;
        const unsigned bad = load_tri(verts, tris, t, nv, g, T);
        if (bad) {
            if (!kFill) set_status(info, bad);
            continue;
        }
        float3 n = make_float3(0.f, 0.f, 0.f);
        if (kFill) face_normal(T.p[0], T.p[1], T.p[2], n.x, n.y, n.z);
        if (ax_lo <= 0 && 0 <= ax_hi) tri_axis<kFill, 0>(T, t, n, o, g.res, big_q, qcap, big_n, info);
        if (ax_lo <= 1 && 1 <= ax_hi) tri_axis<kFill, 1>(T, t, n, o, g.res, big_q, qcap, big_n, info);
        if (ax_lo <= 2 && 2 <= ax_hi) tri_axis<kFill, 2>(T, t, n, o, g.res, big_q, qcap, big_n, info);
    }
}

// The queued big (triangle, image) pairs, a warp or a block per pair
// (for_each_big); the pair's threads stride over its box pixels.
template <bool kFill>
__global__ void __launch_bounds__(kThreads) big_pass(const float *__restrict__ verts, const int *__restrict__ tris,
                                                     int nv, GridDev g, Img o, const int *big_q, long long qcap,
                                                     const int *big_n, int huge_blocks, ldni_info_t *info) {
    for_each_big(big_q, qcap, big_n, (int)blockIdx.x, (int)gridDim.x, huge_blocks, [&](int code, int first, int step) {
        const int t = code >> 2, a = code & 3;
        TriView T;
        if (load_tri(verts, tris, t, nv, g, T)) return;
        Setup64 S;
        int i0, i1, j0, j1;
        if (!setup_big(T, a, g.res, S, i0, i1, j0, j1)) return;
        float3 n = make_float3(0.f, 0.f, 0.f);
        if (kFill) face_normal(T.p[0], T.p[1], T.p[2], n.x, n.y, n.z);
        const int w = i1 - i0 + 1;
        const long long npx = (long long)w * (j1 - j0 + 1);
        for (long long k = first; k < npx; k += step) {
            const int j = j0 + (int)(k / w), i = i0 + (int)(k % w);
            if (S.inside(i, j)) emit<kFill>(kFill ? S.depth(i, j) : 0.0f, a, t, (long long)j * g.res + i, n, o, info);
        }
    });
}

// Per-ray ordering by (depth, tri_id) in place; also flags odd rays.  A warp
// takes 32 consecutive rays: two samples are ordered by their lane directly,
// longer rays by the rank orderings.
__global__ void __launch_bounds__(kThreads) sort_rays(long long nrays, int ax_lo, Img o, ldni_info_t *info) {
    __shared__ SortStage stage[kThreads / 32];
    const int a = ax_lo + blockIdx.y;
    const int *off = a == 0 ? o.offsets[0] : (a == 1 ? o.offsets[1] : o.offsets[2]);
    RayOut r;
    r.D = a == 0 ? o.depth[0] : (a == 1 ? o.depth[1] : o.depth[2]);
    r.Tr = a == 0 ? o.tri[0] : (a == 1 ? o.tri[1] : o.tri[2]);
    r.X = a == 0 ? o.nx[0] : (a == 1 ? o.nx[1] : o.nx[2]);
    r.Y = a == 0 ? o.ny[0] : (a == 1 ? o.ny[1] : o.ny[2]);
    r.Z = a == 0 ? o.nz[0] : (a == 1 ? o.nz[1] : o.nz[2]);
    const long long cap = a == 0 ? o.cap[0] : (a == 1 ? o.cap[1] : o.cap[2]);
    const int lane = threadIdx.x & 31;
    SortStage &st = stage[threadIdx.x >> 5];
    const auto in_place = [](long long, long long b, const RayOut &o) { return InPlace{o, b}; };
    for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); base < nrays;
         base += (long long)gridDim.x * blockDim.x) {
        const long long p = base + lane;
        long long b = 0;
        int n = 0;
        if (p < nrays) {
            b = off[p];
            long long e = off[p + 1];
            if ((e - b) & 1) {
                atomicAdd(&info->odd_rays, 1u);
                set_status(info, LDNI_ST_ODD);
            }
            if (e > cap) e = cap;
            if (!range_ok(b, max(b, e), cap, info)) e = b;
            if (e - b == 2) {
                const float d0 = r.D[b], d1 = r.D[b + 1];
                const int t0 = r.Tr[b], t1 = r.Tr[b + 1];
                if (key_less(d1, t1, d0, t0)) {
                    r.D[b] = d1; r.D[b + 1] = d0;
                    r.Tr[b] = t1; r.Tr[b + 1] = t0;
                    float s;
                    s = r.X[b]; r.X[b] = r.X[b + 1]; r.X[b + 1] = s;
                    if (r.Y) {
                        s = r.Y[b]; r.Y[b] = r.Y[b + 1]; r.Y[b + 1] = s;
                        s = r.Z[b]; r.Z[b] = r.Z[b + 1]; r.Z[b + 1] = s;
                    }
                }
            } else if (e - b > 2) {
                n = (int)(e - b);
            }
        }
        order_warp_rays<true>(b, n, b, in_place, r, st, lane);
    }
}

// ---- tile binning (exact two-pass, binned) ------------------------------------
//
// The same crossings, counted and placed tile by tile instead of triangle by
// triangle: a counting sort bins every (triangle, image) pair to the 16 x 16
// pixel tiles its pixel box touches; one block per tile then stages the
// exact setup (snapped, oriented edge functions, depths, normal) of its
// triangles in shared memory, 128 at a time, and every thread - one pixel -
// tests them all.  A pixel counts its crossings in a register and, in the
// fill, writes them to its own front slots without any atomic; pairs whose
// box touches more than kMaxBinTiles tiles go to the big-triangle queue of
// the direct form, which takes the back slots.  The per-ray order comes from
// sort_rays, so the output equals the direct form's bit for bit.
constexpr int kBinTile = 16;      // pixels per tile side (one per thread)
constexpr int kMaxBinTiles = 16;  // tiles a binned pair may touch
static_assert(kBinTile * kBinTile == kThreads, "a tile is one pixel per thread");

struct BinImg {
    int *tile_cnt[3];   // pairs per tile (count), then the scatter's cursor
    int *tile_off[3];   // exclusive prefix of tile_cnt, tiles + 1 entries
    int *list[3];       // triangle indices, tile by tile
    int tiles_x;        // tiles per image side
};

// Pixel box of triangle T on image A, with its setup: 0 none, 1 small
// (Setup32 in S), 2 big (Setup64 in L); i0..i1, j0..j1 the pixel box.
template <int A>
__device__ __forceinline__ int classify(const TriView &T, int res, Setup32 &S, Setup64 &L, int &i0, int &i1,
                                        int &j0, int &j1, bool with_depth) {
    const int kind = with_depth ? setup_axis<A, true>(T, res, S) : setup_axis<A, false>(T, res, S);
    if (kind == kNone) return 0;
    if (kind == kSmall) {
        i0 = S.i0;
        j0 = S.j0;
        i1 = S.i0 + S.w - 1;
        j1 = S.j0 + S.h - 1;
        return 1;
    }
    return setup_big(T, A, res, L, i0, i1, j0, j1) ? 2 : 0;
}

__device__ __forceinline__ int tiles_touched(int i0, int i1, int j0, int j1) {
    return ((i1 / kBinTile) - (i0 / kBinTile) + 1) * ((j1 / kBinTile) - (j0 / kBinTile) + 1);
}

// kScatter false: count the pairs of every tile; true: write them into the
// tile lists, and queue the pairs that touch too many tiles.
template <bool kScatter, int A>
__device__ __forceinline__ void bin_axis(const TriView &T, int t, int res, const BinImg &b, int *big_q, long long qcap,
                                         int *big_n) {
    Setup32 S;
    Setup64 L;
    int i0, i1, j0, j1;
    const int kind = classify<A>(T, res, S, L, i0, i1, j0, j1, false);
    if (kind == 0) return;
    if (tiles_touched(i0, i1, j0, j1) > kMaxBinTiles) {
        if (kScatter) enqueue_big(big_q, qcap, big_n, t * 4 + A, (long long)(i1 - i0 + 1) * (j1 - j0 + 1));
        return;
    }
    for (int ty = j0 / kBinTile; ty <= j1 / kBinTile; ++ty)
        for (int tx = i0 / kBinTile; tx <= i1 / kBinTile; ++tx) {
            const int tile = ty * b.tiles_x + tx;
            if (!kScatter) {
                atomicAdd(b.tile_cnt[A] + tile, 1);
            } else {
                const int pos = atomicAdd(b.tile_cnt[A] + tile, 1);
                b.list[A][b.tile_off[A][tile] + pos] = t;
            }
        }
}

template <bool kScatter>
__global__ void __launch_bounds__(kThreads) bin_pass(const float *__restrict__ verts, const int *__restrict__ tris,
                                                     int nt, int nv, GridDev g, int ax_lo, int ax_hi, BinImg b,
                                                     int *big_q, long long qcap, int *big_n, ldni_info_t *info) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        TriView T;
        const unsigned bad = load_tri(verts, tris, t, nv, g, T);
        if (bad) {
            if (!kScatter) set_status(info, bad);
            continue;
        }
        if (ax_lo <= 0 && 0 <= ax_hi) bin_axis<kScatter, 0>(T, t, g.res, b, big_q, qcap, big_n);
        if (ax_lo <= 1 && 1 <= ax_hi) bin_axis<kScatter, 1>(T, t, g.res, b, big_q, qcap, big_n);
        if (ax_lo <= 2 && 2 <= ax_hi) bin_axis<kScatter, 2>(T, t, g.res, b, big_q, qcap, big_n);
    }
}

// One staged triangle of a tile: its setup (small: Setup32, big: Setup64),
// pixel box, id and normal.
struct TileTri {
    Setup64 L;
    Setup32 S;
    int kind;  // 0 none, 1 small, 2 big
    int t;
    int i0, i1, j0, j1;
    float nx, ny, nz;
};

template <int A>
__device__ __forceinline__ void stage_tri(const float *__restrict__ verts, const int *__restrict__ tris, int nv,
                                          const GridDev &g, int t, bool fill, TileTri &R) {
    TriView T;
    R.kind = 0;
    R.t = t;
    if (load_tri(verts, tris, t, nv, g, T)) return;
    R.kind = classify<A>(T, g.res, R.S, R.L, R.i0, R.i1, R.j0, R.j1, fill);
    if (fill && R.kind) face_normal(T.p[0], T.p[1], T.p[2], R.nx, R.ny, R.nz);
}

// Block = tile (blockIdx.x) of image ax_lo + blockIdx.y; thread = pixel.
// Count pass: counts[p] = the pixel's binned crossings (before the big pairs
// add theirs).  Fill pass: the crossings go to the ray's first slots.
constexpr int kTileStage = 128;  // triangles staged per round (26 KB of shared memory)

template <bool kFill>
__global__ void __launch_bounds__(kThreads) tile_pass(const float *__restrict__ verts, const int *__restrict__ tris,
                                                      int nv, GridDev g, int ax_lo, BinImg b, Img o,
                                                      ldni_info_t *info) {
    __shared__ TileTri st[kTileStage];
    const int a = ax_lo + blockIdx.y;
    const int tile = blockIdx.x;
    const int tx = tile % b.tiles_x, ty = tile / b.tiles_x;
    const int i = tx * kBinTile + (threadIdx.x % kBinTile), j = ty * kBinTile + (threadIdx.x / kBinTile);
    const bool mine = i < g.res && j < g.res;
    const int *lst = sel(b.list, a) + sel(b.tile_off, a)[tile];
    const int n = sel(b.tile_off, a)[tile + 1] - sel(b.tile_off, a)[tile];
    const long long p = (long long)j * g.res + i;
    int found = 0;
    long long slot_end = 0;  // fill: the pixel's crossings take its last slots, downwards from here
    long long cap = 0;
    if (kFill && mine) {
        slot_end = (long long)(a == 0 ? o.offsets[0] : (a == 1 ? o.offsets[1] : o.offsets[2]))[p] +
                   sel(o.count, a)[p];
        cap = a == 0 ? o.cap[0] : (a == 1 ? o.cap[1] : o.cap[2]);
    }
    for (int k0 = 0; k0 < n; k0 += kTileStage) {
        const int k = k0 + threadIdx.x;
        if (threadIdx.x < kTileStage && k < n) {
            if (a == 0) stage_tri<0>(verts, tris, nv, g, lst[k], kFill, st[threadIdx.x]);
            else if (a == 1) stage_tri<1>(verts, tris, nv, g, lst[k], kFill, st[threadIdx.x]);
            else stage_tri<2>(verts, tris, nv, g, lst[k], kFill, st[threadIdx.x]);
        }
        __syncthreads();
        const int m = min(kTileStage, n - k0);
        for (int r = 0; r < m && mine; ++r) {
            const TileTri &R = st[r];
            if (R.kind == 0 || i < R.i0 || i > R.i1 || j < R.j0 || j > R.j1) continue;
            float d = 0.0f;
            bool hit;
            if (R.kind == 1) {
                int e0, e1, e2;
                R.S.edges(i, j, e0, e1, e2);
                hit = (e0 > 0) & (e1 > 0) & (e2 > 0);
                if (kFill && hit) d = R.S.depth_from(e0, e1, e2);
            } else {
                hit = R.L.inside(i, j);
                if (kFill && hit) d = R.L.depth(i, j);
            }
            if (!hit) continue;
            if (kFill) {
                const long long at = slot_end - 1 - found;
                if (at >= cap || at < 0) {
                    set_status(info, LDNI_ST_CAPACITY);
                } else {
                    (a == 0 ? o.depth[0] : (a == 1 ? o.depth[1] : o.depth[2]))[at] = d;
                    (a == 0 ? o.tri[0] : (a == 1 ? o.tri[1] : o.tri[2]))[at] = R.t;
                    float *X = a == 0 ? o.nx[0] : (a == 1 ? o.nx[1] : o.nx[2]);
                    float *Y = a == 0 ? o.ny[0] : (a == 1 ? o.ny[1] : o.ny[2]);
                    float *Z = a == 0 ? o.nz[0] : (a == 1 ? o.nz[1] : o.nz[2]);
                    if (Y) {
                        X[at] = R.nx;
                        Y[at] = R.ny;
                        Z[at] = R.nz;
                    } else {  // approximate normals (Section 3 item 1)
                        X[at] = __uint_as_float(encode_normal8(R.nx, R.ny, R.nz));
                    }
                }
            }
            ++found;
        }
        __syncthreads();
    }
    if (!mine) return;
    int *cnt = sel(o.count, a) + p;
    if (!kFill)
        *cnt = found;  // the big pairs add theirs afterwards
    else
        *cnt -= found;  // the big pairs take the remaining (first) slots
}

struct SampleWs {
    int *count[3];
    int *big_n;          // two queue counts right after the counts: one memset clears all
    long long qcap;
    size_t clear_bytes;
    long long *scan_words;
    int *big_q;
};

SampleWs carve_sample_ws(Carver &c, long long nt, int res, int naxes) {
    SampleWs w{};
    const long long N = (long long)res * res;
    const long long stride = (N + 63) / 64 * 64;  // every image's counts start 256-byte aligned
    int *block = c.take<int>((size_t)(stride * naxes + 2));
    for (int a = 0; a < naxes; ++a) w.count[a] = block ? block + (size_t)a * stride : nullptr;
    w.big_n = block ? block + (size_t)stride * naxes : nullptr;
    w.clear_bytes = sizeof(int) * (size_t)(stride * naxes + 2);
    w.scan_words = c.take<long long>(csr_scan_partials(N) * naxes);
    w.qcap = nt * naxes > 0 ? nt * naxes : 1;
    w.big_q = c.take<int>((size_t)w.qcap);
    return w;
}

struct Call {
    GridDev g;
    int ax_lo, ax_hi, naxes;
    long long nrays;
    Img o;
    SampleWs w;
    cudaStream_t s;
};

int prepare(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid, int32_t axis,
            ldni_layers_t *out, ldni_info_t *info, void *ws, size_t ws_bytes, void *stream, bool need_samples,
            Call &C) {
    if (!grid_valid(grid) || !out || !info || !ws || axis < 0 || axis > LDNI_AXIS_ALL || nv <= 0 || nt < 0 ||
        (nt > 0 && (!verts || !tris)))
        return LDNI_EINVAL;
    if (nt > (INT_MAX / 4) || nv > INT_MAX) return LDNI_ETOOLARGE;
    C.ax_lo = axis == LDNI_AXIS_ALL ? 0 : axis;
    C.ax_hi = axis == LDNI_AXIS_ALL ? 2 : axis;
    C.naxes = C.ax_hi - C.ax_lo + 1;
    C.g = make_grid(grid);
    C.nrays = (long long)grid->res * grid->res;
    C.s = static_cast<cudaStream_t>(stream);
    Carver c(ws, ws_bytes);
    SampleWs w = carve_sample_ws(c, nt, grid->res, C.naxes);
    if (!c.fits()) return LDNI_EWORKSPACE;
    C.w = w;
    C.o = Img{};
    for (int k = 0; k < C.naxes; ++k) {
        const int a = C.ax_lo + k;
        const ldni_layers_t &L = out[k];
        if (!L.offsets) return LDNI_EINVAL;
        if (need_samples && !samples_ok(L)) return LDNI_EINVAL;
        if (L.capacity < 0) return LDNI_EINVAL;
        C.o.count[a] = w.count[k];
        C.o.offsets[a] = L.offsets;
        C.o.depth[a] = L.depth;
        normal_arrays(L, C.o.nx[a], C.o.ny[a], C.o.nz[a]);
        C.o.tri[a] = L.tri_id;
        C.o.cap[a] = L.capacity;
    }
    return LDNI_OK;
}

int grid_blocks(long long work) {
    long long b = (work + kThreads - 1) / kThreads;
    const long long lim = (long long)num_sms() * current_tuning().tri_blocks_per_sm;
    if (b > lim) b = lim;
    return (int)(b > 0 ? b : 1);
}

int run_count(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const Call &C, ldni_info_t *info) {
    if (int rc_ = cuda_check(cudaMemsetAsync(C.w.count[0], 0, C.w.clear_bytes, C.s))) return rc_;
    if (nt > 0) {
        LDNI_LAUNCH(K_COUNT_TRI, C.s,
                    tri_pass<false><<<grid_blocks(nt), kThreads, 0, C.s>>>(verts, tris, (int)nt, (int)nv, C.g,
                                                                          C.ax_lo, C.ax_hi, C.o, C.w.big_q,
                                                                          C.w.qcap, C.w.big_n, info));
        LDNI_LAUNCH(K_COUNT_BIG, C.s,
                    big_pass<false><<<5 * num_sms(), kThreads, 0, C.s>>>(verts, tris, (int)nv, C.g, C.o, C.w.big_q,
                                                                        C.w.qcap, C.w.big_n, num_sms(), info));
    }
    const int *cnt[3];
    int *off[3];
    for (int k = 0; k < C.naxes; ++k) {
        cnt[k] = C.w.count[k];
        off[k] = const_cast<int *>(C.o.offsets[C.ax_lo + k]);
    }
    int rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    return csr_scan(cnt, off, C.naxes, C.nrays, C.w.scan_words, info, C.ax_lo, C.s);
}

int run_fill(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const Call &C, ldni_info_t *info) {
    if (nt > 0) {
        LDNI_LAUNCH(K_FILL_TRI, C.s,
                    tri_pass<true><<<grid_blocks(nt), kThreads, 0, C.s>>>(verts, tris, (int)nt, (int)nv, C.g,
                                                                         C.ax_lo, C.ax_hi, C.o, C.w.big_q,
                                                                         C.w.qcap, C.w.big_n, info));
        LDNI_LAUNCH(K_FILL_BIG, C.s,
                    big_pass<true><<<5 * num_sms(), kThreads, 0, C.s>>>(verts, tris, (int)nv, C.g, C.o, C.w.big_q,
                                                                       C.w.qcap, C.w.big_n, num_sms(), info));
    }
    LDNI_LAUNCH(K_SORT, C.s,
                sort_rays<<<dim3(grid_blocks(C.nrays), C.naxes), kThreads, 0, C.s>>>(C.nrays, C.ax_lo, C.o, info));
    return cuda_status();
}

// ---- binned form: workspace and launches --------------------------------------

struct BinWs {
    BinImg b;
    int *tile_cnt0;           // every image's tile counts (one clear)
    size_t tile_bytes;
    long long *tile_words;    // scan partials of the tile counts
    ldni_info_t *tile_info;   // the tile scan's report (not the caller's)
    int ntiles;
};

BinWs carve_bin_ws(Carver &c, long long nt, int res, int naxes) {
    BinWs w{};
    w.b.tiles_x = (res + kBinTile - 1) / kBinTile;
    w.ntiles = w.b.tiles_x * w.b.tiles_x;
    const long long stride = ((long long)w.ntiles + 1 + 63) / 64 * 64;
    int *cnt = c.take<int>((size_t)(stride * naxes));
    int *off = c.take<int>((size_t)(stride * naxes));
    const long long lcap = (long long)kMaxBinTiles * (nt > 0 ? nt : 1);
    int *lst = c.take<int>((size_t)(lcap * naxes));
    for (int a = 0; a < naxes; ++a) {
        w.b.tile_cnt[a] = cnt ? cnt + (size_t)a * stride : nullptr;
        w.b.tile_off[a] = off ? off + (size_t)a * stride : nullptr;
        w.b.list[a] = lst ? lst + (size_t)a * lcap : nullptr;
    }
    w.tile_cnt0 = cnt;
    w.tile_bytes = sizeof(int) * (size_t)(stride * naxes);
    w.tile_words = c.take<long long>(csr_scan_partials(w.ntiles) * naxes);
    w.tile_info = c.take<ldni_info_t>(1);
    return w;
}

// The binned image arrays indexed by image (a = ax_lo + k).
BinImg bin_view(const BinWs &w, const Call &C) {
    BinImg b{};
    b.tiles_x = w.b.tiles_x;
    for (int k = 0; k < C.naxes; ++k) {
        b.tile_cnt[C.ax_lo + k] = w.b.tile_cnt[k];
        b.tile_off[C.ax_lo + k] = w.b.tile_off[k];
        b.list[C.ax_lo + k] = w.b.list[k];
    }
    return b;
}

int run_binned_count(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const Call &C, const BinWs &w,
                     ldni_info_t *info) {
    if (int rc_ = cuda_check(cudaMemsetAsync(C.w.count[0], 0, C.w.clear_bytes, C.s))) return rc_;
    if (int rc_ = cuda_check(cudaMemsetAsync(w.tile_cnt0, 0, w.tile_bytes, C.s))) return rc_;
    const BinImg b = bin_view(w, C);
    if (nt > 0)
        LDNI_LAUNCH(K_BIN, C.s,
                    bin_pass<false><<<grid_blocks(nt), kThreads, 0, C.s>>>(verts, tris, (int)nt, (int)nv, C.g, C.ax_lo,
                                                                          C.ax_hi, b, C.w.big_q, C.w.qcap, C.w.big_n,
                                                                          info));
    const int *tc[3];
    int *to[3];
    for (int k = 0; k < C.naxes; ++k) {
        tc[k] = w.b.tile_cnt[k];
        to[k] = w.b.tile_off[k];
    }
    int rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    rc = csr_scan(tc, to, C.naxes, w.ntiles, w.tile_words, w.tile_info, 0, C.s);
    if (rc != LDNI_OK) return rc;
    if (int rc_ = cuda_check(cudaMemsetAsync(w.tile_cnt0, 0, w.tile_bytes, C.s))) return rc_;  // the scatter's cursors
    if (nt > 0)
        LDNI_LAUNCH(K_BIN, C.s,
                    bin_pass<true><<<grid_blocks(nt), kThreads, 0, C.s>>>(verts, tris, (int)nt, (int)nv, C.g, C.ax_lo,
                                                                         C.ax_hi, b, C.w.big_q, C.w.qcap, C.w.big_n,
                                                                         info));
    LDNI_LAUNCH(K_TILE, C.s,
                tile_pass<false><<<dim3(w.ntiles, C.naxes), kThreads, 0, C.s>>>(verts, tris, (int)nv, C.g, C.ax_lo, b,
                                                                               C.o, info));
    if (nt > 0)
        LDNI_LAUNCH(K_COUNT_BIG, C.s,
                    big_pass<false><<<5 * num_sms(), kThreads, 0, C.s>>>(verts, tris, (int)nv, C.g, C.o, C.w.big_q,
                                                                        C.w.qcap, C.w.big_n, num_sms(), info));
    const int *cnt[3];
    int *off[3];
    for (int k = 0; k < C.naxes; ++k) {
        cnt[k] = C.w.count[k];
        off[k] = const_cast<int *>(C.o.offsets[C.ax_lo + k]);
    }
    rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    return csr_scan(cnt, off, C.naxes, C.nrays, C.w.scan_words, info, C.ax_lo, C.s);
}

int run_binned_fill(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const Call &C, const BinWs &w,
                    ldni_info_t *info) {
    const BinImg b = bin_view(w, C);
    LDNI_LAUNCH(K_TILE, C.s,
                tile_pass<true><<<dim3(w.ntiles, C.naxes), kThreads, 0, C.s>>>(verts, tris, (int)nv, C.g, C.ax_lo, b,
                                                                              C.o, info));
    if (nt > 0)
        LDNI_LAUNCH(K_FILL_BIG, C.s,
                    big_pass<true><<<5 * num_sms(), kThreads, 0, C.s>>>(verts, tris, (int)nv, C.g, C.o, C.w.big_q,
                                                                       C.w.qcap, C.w.big_n, num_sms(), info));
    LDNI_LAUNCH(K_SORT, C.s,
                sort_rays<<<dim3(grid_blocks(C.nrays), C.naxes), kThreads, 0, C.s>>>(C.nrays, C.ax_lo, C.o, info));
    return cuda_status();
}

// prepare() plus the binned part of the workspace (after the direct form's).
int prepare_binned(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                   int32_t axis, ldni_layers_t *out, ldni_info_t *info, void *ws, size_t ws_bytes, void *stream,
                   bool need_samples, Call &C, BinWs &w) {
    int rc = prepare(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes, stream, need_samples, C);
    if (rc != LDNI_OK) return rc;
    Carver c(ws, ws_bytes);
    carve_sample_ws(c, nt, grid->res, C.naxes);
    w = carve_bin_ws(c, nt, grid->res, C.naxes);
    return c.fits() ? LDNI_OK : LDNI_EWORKSPACE;
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_sample_workspace_size(int64_t nv, int64_t nt, int32_t res, int32_t axis, size_t *bytes) {
    if (!bytes || res < 1 || res > 8192 || nt < 0 || nv < 0 || axis < 0 || axis > LDNI_AXIS_ALL) return LDNI_EINVAL;
    Carver c(nullptr, 0);
    carve_sample_ws(c, nt, res, axis == LDNI_AXIS_ALL ? 3 : 1);
    *bytes = align_up(c.off);
    return LDNI_OK;
}

extern "C" int ldni_sample_count(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                                 const ldni_grid_t *grid, int32_t axis, ldni_layers_t *out, ldni_info_t *info,
                                 void *ws, size_t ws_bytes, void *stream) {
    Call C;
    int rc = prepare(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes, stream, false, C);
    if (rc != LDNI_OK) return rc;
    return run_count(verts, nv, tris, nt, C, info);
}

extern "C" int ldni_sample_fill(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                                const ldni_grid_t *grid, int32_t axis, ldni_layers_t *out, ldni_info_t *info,
                                void *ws, size_t ws_bytes, void *stream) {
    Call C;
    int rc = prepare(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes, stream, true, C);
    if (rc != LDNI_OK) return rc;
    return run_fill(verts, nv, tris, nt, C, info);
}

static int ldni_sample_exact2(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                       int32_t axis, ldni_layers_t *out, ldni_info_t *info, void *ws, size_t ws_bytes, void *stream) {
    Call C;
    int rc = prepare(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes, stream, true, C);
    if (rc != LDNI_OK) return rc;
    rc = run_count(verts, nv, tris, nt, C, info);
    if (rc != LDNI_OK) return rc;
    return run_fill(verts, nv, tris, nt, C, info);
}

extern "C" int ldni_sample_binned_workspace_size(int64_t nv, int64_t nt, int32_t res, int32_t axis, size_t *bytes) {
    if (!bytes || res < 1 || res > 8192 || nt < 0 || nv < 0 || axis < 0 || axis > LDNI_AXIS_ALL) return LDNI_EINVAL;
    if (nt > (INT_MAX / (4 * kMaxBinTiles))) return LDNI_ETOOLARGE;
    Carver c(nullptr, 0);
    const int naxes = axis == LDNI_AXIS_ALL ? 3 : 1;
    carve_sample_ws(c, nt, res, naxes);
    carve_bin_ws(c, nt, res, naxes);
    *bytes = align_up(c.off);
    return LDNI_OK;
}

extern "C" int ldni_sample_binned_count(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                                        const ldni_grid_t *grid, int32_t axis, ldni_layers_t *out, ldni_info_t *info,
                                        void *ws, size_t ws_bytes, void *stream) {
    if (nt > (INT_MAX / (4 * kMaxBinTiles))) return LDNI_ETOOLARGE;
    Call C;
    BinWs w;
    int rc = prepare_binned(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes, stream, false, C, w);
    if (rc != LDNI_OK) return rc;
    return run_binned_count(verts, nv, tris, nt, C, w, info);
}

extern "C" int ldni_sample_binned_fill(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                                       const ldni_grid_t *grid, int32_t axis, ldni_layers_t *out, ldni_info_t *info,
                                       void *ws, size_t ws_bytes, void *stream) {
    if (nt > (INT_MAX / (4 * kMaxBinTiles))) return LDNI_ETOOLARGE;
    Call C;
    BinWs w;
    int rc = prepare_binned(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes, stream, true, C, w);
    if (rc != LDNI_OK) return rc;
    return run_binned_fill(verts, nv, tris, nt, C, w, info);
}

extern "C" int ldni_sample(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                           int32_t axis, int32_t mode, ldni_layers_t *out, ldni_info_t *info, void *ws,
                           size_t ws_bytes, void *stream) {
    if (mode == LDNI_MODE_EXACT2) return ldni_sample_exact2(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes,
                                                            stream);
    if (mode != LDNI_MODE_BINNED2) return LDNI_EINVAL;  // the learned one-pass form is ldni_sample_learned
    int rc = ldni_sample_binned_count(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes, stream);
    if (rc != LDNI_OK) return rc;
    return ldni_sample_binned_fill(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes, stream);
}
