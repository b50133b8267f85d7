// LDNI sampling of a closed triangle mesh (Section 3; Definitions 1-4).
//
// The paper renders the mesh n_max + 1 times through a stencil-routed
// OpenGL pipeline: pass 1 counts the depth complexity n_p of every pixel,
// passes 2..n_max each capture the n-th fragment, and the host post-sorts
// every pixel (Section 3, Appendix A).  Here the same exact two-pass
// structure runs as CUDA kernels with everything resident on the device:
//
//   count : one thread per triangle snaps its vertices once, then for each
//           requested image tests the pixel centres of its bounding box and
//           adds 1 to count[p] per crossing (= the stencil pass);
//   scan  : counts -> CSR row offsets (scan.cu);
//   fill  : the same traversal; every crossing takes a slot of its ray with
//           an atomic decrement of count[p] (leaving the counts at zero) and
//           writes depth, normal and triangle id there (= passes 2..n_max);
//   sort  : every ray orders its samples by (depth, tri_id) in place
//           (= the host post-sort).
//
// Triangles whose pixel box holds more than kBigPixels centres are handed to
// a CTA-per-triangle kernel so that a few large faces do not serialise a warp.
#include <climits>

#include "ldni_host.h"

namespace ldni {
namespace {

constexpr int kThreads = 256;
constexpr int kBigPixels = 64;

struct ImgPtrs {
    int *count[3];
    const int *offsets[3];
    float *depth[3];
    float *nx[3];
    float *ny[3];
    float *nz[3];
    int *tri[3];
    long long cap[3];
};

template <class T>
__device__ __forceinline__ T pick(T const (&arr)[3], int a) {
    return a == 0 ? arr[0] : (a == 1 ? arr[1] : arr[2]);
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

template <int A>
__device__ __forceinline__ bool project_axis(const TriView &T, int res, ProjTri &P) {
    constexpr int U = (A + 1) % 3, V = (A + 2) % 3;
    const int qu[3] = {T.q[0][U], T.q[1][U], T.q[2][U]};
    const int qv[3] = {T.q[0][V], T.q[1][V], T.q[2][V]};
    const float a[3] = {comp(T.p[0], A), comp(T.p[1], A), comp(T.p[2], A)};
    return project_tri(qu, qv, a, res, P);
}

__device__ __forceinline__ bool project_axis_rt(const TriView &T, int a, int res, ProjTri &P) {
    if (a == 0) return project_axis<0>(T, res, P);
    if (a == 1) return project_axis<1>(T, res, P);
    return project_axis<2>(T, res, P);
}

struct Normal {
    float x, y, z;
};

// Test one pixel centre; on a crossing either count it or store the sample.
template <bool kFill>
__device__ __forceinline__ void visit_pixel(const ProjTri &P, const EdgeBias &B, int i, int j, int a, int t,
                                            const Normal &n, const ImgPtrs &o, int res, ldni_info_t *info) {
    const EdgeEval E = edges_at(P, i * kSubpix + kHalfSubpix, j * kSubpix + kHalfSubpix);
    if (!inside(E, B)) return;
    const long long p = (long long)j * res + i;
    int *cnt = pick(o.count, a);
    if (!kFill) {
        atomicAdd(cnt + p, 1);
        return;
    }
    const int k = atomicSub(cnt + p, 1) - 1;
    const long long slot = (long long)pick(o.offsets, a)[p] + k;
    if (k < 0 || slot >= pick(o.cap, a)) {
        set_status(info, LDNI_ST_CAPACITY);
        return;
    }
    pick(o.depth, a)[slot] = crossing_depth(P, E);
    pick(o.tri, a)[slot] = t;
    pick(o.nx, a)[slot] = n.x;
    pick(o.ny, a)[slot] = n.y;
    pick(o.nz, a)[slot] = n.z;
}

template <bool kFill, int A>
__device__ __forceinline__ void small_tri_axis(const TriView &T, int t, const Normal &n, const ImgPtrs &o, int res,
                                               int *big_q, int *big_n, ldni_info_t *info) {
    ProjTri P;
    if (!project_axis<A>(T, res, P)) return;
    const long long npx = (long long)(P.i1 - P.i0 + 1) * (P.j1 - P.j0 + 1);
    if (npx > kBigPixels) {
        const int k = atomicAdd(big_n, 1);
        big_q[k] = t * 4 + A;
        return;
    }
    const EdgeBias B = edge_bias(P);
    for (int j = P.j0; j <= P.j1; ++j)
        for (int i = P.i0; i <= P.i1; ++i) visit_pixel<kFill>(P, B, i, j, A, t, n, o, res, info);
}

// One thread per triangle; big triangles are queued for big_tri_pass.
template <bool kFill>
__global__ void __launch_bounds__(kThreads) tri_pass(const float *__restrict__ verts, const int *__restrict__ tris,
                                                     int nt, int nv, GridDev g, int ax_lo, int ax_hi,
                                                     ImgPtrs o, int *big_q, int *big_n, ldni_info_t *info) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        TriView T;
        const unsigned bad = load_tri(verts, tris, t, nv, g, T);
        if (bad) {
            set_status(info, bad);
            continue;
        }
        Normal n{0.f, 0.f, 0.f};
        if (kFill) face_normal(T.p[0], T.p[1], T.p[2], n.x, n.y, n.z);
        if (ax_lo <= 0 && 0 <= ax_hi) small_tri_axis<kFill, 0>(T, t, n, o, g.res, big_q, big_n, info);
        if (ax_lo <= 1 && 1 <= ax_hi) small_tri_axis<kFill, 1>(T, t, n, o, g.res, big_q, big_n, info);
        if (ax_lo <= 2 && 2 <= ax_hi) small_tri_axis<kFill, 2>(T, t, n, o, g.res, big_q, big_n, info);
    }
}

// One CTA per queued (triangle, image) pair; threads stride over its pixels.
template <bool kFill>
__global__ void __launch_bounds__(kThreads) big_tri_pass(const float *__restrict__ verts,
                                                         const int *__restrict__ tris, int nv, GridDev g,
                                                         ImgPtrs o, const int *big_q, const int *big_n,
                                                         ldni_info_t *info) {
    const int nq = *big_n;
    for (int e = blockIdx.x; e < nq; e += gridDim.x) {
        const int code = big_q[e];
        const int t = code >> 2, a = code & 3;
        TriView T;
        if (load_tri(verts, tris, t, nv, g, T)) continue;
        ProjTri P;
        if (!project_axis_rt(T, a, g.res, P)) continue;
        Normal n{0.f, 0.f, 0.f};
        if (kFill) face_normal(T.p[0], T.p[1], T.p[2], n.x, n.y, n.z);
        const EdgeBias B = edge_bias(P);
        const int w = P.i1 - P.i0 + 1;
        const long long npx = (long long)w * (P.j1 - P.j0 + 1);
        for (long long k = threadIdx.x; k < npx; k += blockDim.x) {
            const int j = P.j0 + (int)(k / w), i = P.i0 + (int)(k % w);
            visit_pixel<kFill>(P, B, i, j, a, t, n, o, g.res, info);
        }
    }
}

__device__ __forceinline__ bool key_less(float d0, int t0, float d1, int t1) {
    return d0 < d1 || (d0 == d1 && t0 < t1);
}

// Per-ray ordering by (depth, tri_id) in place; also flags odd rays.
__global__ void __launch_bounds__(kThreads) sort_rays(long long nrays, int ax_lo, ImgPtrs o, ldni_info_t *info) {
    const int a = ax_lo + blockIdx.y;
    const int *off = pick(o.offsets, a);
    float *D = pick(o.depth, a);
    int *Tr = pick(o.tri, a);
    float *X = pick(o.nx, a);
    float *Y = pick(o.ny, a);
    float *Z = pick(o.nz, a);
    const long long cap = pick(o.cap, a);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nrays;
         p += (long long)gridDim.x * blockDim.x) {
        const long long b = off[p];
        long long e = off[p + 1];
        if ((e - b) & 1) {
            atomicAdd(&info->odd_rays, 1u);
            set_status(info, LDNI_ST_ODD);
        }
        if (e > cap) e = cap;
        if (e - b < 2) continue;
        if (e - b == 2) {
            const float d0 = D[b], d1 = D[b + 1];
            const int t0 = Tr[b], t1 = Tr[b + 1];
            if (key_less(d1, t1, d0, t0)) {
                D[b] = d1; D[b + 1] = d0;
                Tr[b] = t1; Tr[b + 1] = t0;
                float s;
                s = X[b]; X[b] = X[b + 1]; X[b + 1] = s;
                s = Y[b]; Y[b] = Y[b + 1]; Y[b + 1] = s;
                s = Z[b]; Z[b] = Z[b + 1]; Z[b + 1] = s;
            }
            continue;
        }
        for (long long x = b + 1; x < e; ++x) {
            const float d = D[x];
            const int t = Tr[x];
            const float nx = X[x], ny = Y[x], nz = Z[x];
            long long y = x - 1;
            while (y >= b && key_less(d, t, D[y], Tr[y])) {
                D[y + 1] = D[y];
                Tr[y + 1] = Tr[y];
                X[y + 1] = X[y];
                Y[y + 1] = Y[y];
                Z[y + 1] = Z[y];
                --y;
            }
            D[y + 1] = d;
            Tr[y + 1] = t;
            X[y + 1] = nx;
            Y[y + 1] = ny;
            Z[y + 1] = nz;
        }
    }
}

struct SampleWs {
    int *count[3];
    long long *partials;
    int *big_q;
    int *big_n;
};

SampleWs carve_sample_ws(Carver &c, long long nt, int res, int naxes) {
    SampleWs w{};
    const long long N = (long long)res * res;
    for (int a = 0; a < naxes; ++a) w.count[a] = c.take<int>((size_t)N);
    w.partials = c.take<long long>(csr_scan_partials(N) * naxes);
    w.big_q = c.take<int>((size_t)(nt * naxes > 0 ? nt * naxes : 1));
    w.big_n = c.take<int>(1);
    return w;
}

struct Call {
    GridDev g;
    int ax_lo, ax_hi, naxes;
    long long nrays;
    ImgPtrs o;
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
    C.o = ImgPtrs{};
    for (int k = 0; k < C.naxes; ++k) {
        const int a = C.ax_lo + k;
        const ldni_layers_t &L = out[k];
        if (!L.offsets) return LDNI_EINVAL;
        if (need_samples && L.capacity > 0 && (!L.depth || !L.nx || !L.ny || !L.nz || !L.tri_id)) return LDNI_EINVAL;
        if (L.capacity < 0) return LDNI_EINVAL;
        C.o.count[a] = w.count[k];
        C.o.offsets[a] = L.offsets;
        C.o.depth[a] = L.depth;
        C.o.nx[a] = L.nx;
        C.o.ny[a] = L.ny;
        C.o.nz[a] = L.nz;
        C.o.tri[a] = L.tri_id;
        C.o.cap[a] = L.capacity;
    }
    return LDNI_OK;
}

int grid_blocks(long long work) {
    long long b = (work + kThreads - 1) / kThreads;
    const long long lim = (long long)num_sms() * 16;
    if (b > lim) b = lim;
    return (int)(b > 0 ? b : 1);
}

int run_count(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const Call &C, ldni_info_t *info) {
    for (int k = 0; k < C.naxes; ++k)
        if (cudaMemsetAsync(C.w.count[k], 0, sizeof(int) * (size_t)C.nrays, C.s) != cudaSuccess) return LDNI_ECUDA;
    if (cudaMemsetAsync(C.w.big_n, 0, sizeof(int), C.s) != cudaSuccess) return LDNI_ECUDA;
    if (nt > 0) {
        LDNI_LAUNCH(K_COUNT_TRI, C.s,
                    tri_pass<false><<<grid_blocks(nt), kThreads, 0, C.s>>>(
                        verts, tris, (int)nt, (int)nv, C.g, C.ax_lo, C.ax_hi, C.o, C.w.big_q, C.w.big_n, info));
        LDNI_LAUNCH(K_COUNT_BIG, C.s,
                    big_tri_pass<false><<<num_sms() * 4, kThreads, 0, C.s>>>(verts, tris, (int)nv, C.g, C.o,
                                                                            C.w.big_q, C.w.big_n, info));
    }
    const int *cnt[3];
    int *off[3];
    for (int k = 0; k < C.naxes; ++k) {
        cnt[k] = C.w.count[k];
        off[k] = const_cast<int *>(C.o.offsets[C.ax_lo + k]);
    }
    int rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    return csr_scan(cnt, off, C.naxes, C.nrays, C.w.partials, info, C.ax_lo, C.s);
}

int run_fill(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const Call &C, ldni_info_t *info) {
    if (cudaMemsetAsync(C.w.big_n, 0, sizeof(int), C.s) != cudaSuccess) return LDNI_ECUDA;
    if (nt > 0) {
        LDNI_LAUNCH(K_FILL_TRI, C.s,
                    tri_pass<true><<<grid_blocks(nt), kThreads, 0, C.s>>>(
                        verts, tris, (int)nt, (int)nv, C.g, C.ax_lo, C.ax_hi, C.o, C.w.big_q, C.w.big_n, info));
        LDNI_LAUNCH(K_FILL_BIG, C.s,
                    big_tri_pass<true><<<num_sms() * 4, kThreads, 0, C.s>>>(verts, tris, (int)nv, C.g, C.o,
                                                                           C.w.big_q, C.w.big_n, info));
    }
    LDNI_LAUNCH(K_SORT, C.s,
                sort_rays<<<dim3(grid_blocks(C.nrays), C.naxes), kThreads, 0, C.s>>>(C.nrays, C.ax_lo, C.o, info));
    return cuda_status();
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

extern "C" int ldni_sample(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                           int32_t axis, int32_t mode, ldni_layers_t *out, ldni_info_t *info, void *ws,
                           size_t ws_bytes, void *stream) {
    if (mode != LDNI_MODE_EXACT2) return LDNI_EINVAL;
    Call C;
    int rc = prepare(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes, stream, true, C);
    if (rc != LDNI_OK) return rc;
    rc = run_count(verts, nv, tris, nt, C, info);
    if (rc != LDNI_OK) return rc;
    return run_fill(verts, nv, tris, nt, C, info);
}
