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
    S.for_each_hit([&](int i, int j, int e0, int e1, int e2) {
        emit<true>(S.depth_from(e0, e1, e2), A, t, (long long)j * res + i, n, o, info);
    });
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

extern "C" int ldni_sample(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                           int32_t axis, int32_t mode, ldni_layers_t *out, ldni_info_t *info, void *ws,
                           size_t ws_bytes, void *stream) {
    if (mode != LDNI_MODE_EXACT2) return LDNI_EINVAL;  // the learned one-pass form is ldni_sample_learned
    return ldni_sample_exact2(verts, nv, tris, nt, grid, axis, out, info, ws, ws_bytes, stream);
}
