// Many meshes, of uneven size and resolution, sampled by ONE launch per stage
// (count, scan, fill, sort) for the whole batch - the exact two-pass form of
// sample.cu spread over every triangle, chunk and ray of the batch at once.
// Each thread finds its mesh by a binary search over prefix tables that a
// setup kernel builds on the device from the caller's device array of item
// descriptors, so a batch call needs no host synchronisation and can be
// captured in a CUDA graph.
#include "lookback.cuh"
#include "sample_common.cuh"

namespace ldni {
namespace {

constexpr int kThreads = 256;

struct Tables {
    long long *tri_prefix;    // [count + 1]
    long long *ray_prefix;    // [3 count + 1]  rays of image (m, a) at 3 m + a
    long long *chunk_prefix;  // [3 count + 1]  scan chunks
    long long *count_base;    // [3 count]      start of the image's counts
    long long *big;           // queued big (item, triangle, image): item << 34 | tri << 2 | a
    long long qcap;
    int *big_n;               // counts of the queue's two ends
};

__device__ __forceinline__ int find(const long long *prefix, int n, long long x) {  // prefix[k] <= x < prefix[k+1]
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= x)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ GridDev grid_dev(const ldni_grid_t &g) {
    GridDev d;
    d.o[0] = g.origin[0];
    d.o[1] = g.origin[1];
    d.o[2] = g.origin[2];
    d.s = (float)((double)g.res * (double)kSubpix / (double)g.width);  // as the host computes it
    d.res = g.res;
    return d;
}

// One block builds the prefix tables of the batch, kThreads items at a time:
// per item its triangles, and per image its rays, scan chunks and counts
// (padded to 64 ints); the images of an item have the same size.
__global__ void __launch_bounds__(kThreads) setup_kernel(const ldni_batch_item_t *items, int count, Tables T) {
    __shared__ long long sh[4][kThreads / 32 + 1];
    __shared__ long long carry[4];
    if (threadIdx.x < 4) carry[threadIdx.x] = 0;
    __syncthreads();
    for (int m0 = 0; m0 < count; m0 += kThreads) {
        const int m = m0 + threadIdx.x;
        long long v[4] = {0, 0, 0, 0};  // triangles, rays, chunks, count ints of one image
        if (m < count) {
            const long long N = (long long)items[m].grid.res * items[m].grid.res;
            v[0] = items[m].nt;
            v[1] = N;
            v[2] = (N + kScanChunk - 1) / kScanChunk;
            v[3] = (N + 63) / 64 * 64;
        }
        long long ex[4], tot[4];
        ex[0] = block_exclusive_scan<kThreads>(v[0], sh[0], &tot[0]);
#pragma unroll
        for (int q = 1; q < 4; ++q) ex[q] = block_exclusive_scan<kThreads>(3 * v[q], sh[q], &tot[q]);
        if (m < count) {
            T.tri_prefix[m] = carry[0] + ex[0];
            for (int a = 0; a < 3; ++a) {
                T.ray_prefix[3 * m + a] = carry[1] + ex[1] + a * v[1];
                T.chunk_prefix[3 * m + a] = carry[2] + ex[2] + a * v[2];
                T.count_base[3 * m + a] = carry[3] + ex[3] + a * v[3];
            }
        }
        __syncthreads();  // every thread has read the carries
        if (threadIdx.x < 4) carry[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        T.tri_prefix[count] = carry[0];
        T.ray_prefix[3 * count] = carry[1];
        T.chunk_prefix[3 * count] = carry[2];
    }
}

template <bool kFill>
__device__ __forceinline__ void batch_emit(const ldni_batch_item_t &it, int a, long long p, float d, int t,
                                           const float3 &n, int *cnt, ldni_info_t *info) {
    if (!kFill) {
        atomicAdd(cnt + p, 1);
        return;
    }
    const ldni_layers_t &L = it.out[a];
    const int k = atomicSub(cnt + p, 1) - 1;
    const long long slot = (long long)L.offsets[p] + k;
    if (k < 0 || slot >= L.capacity) {
        set_status(info, LDNI_ST_CAPACITY);
        return;
    }
    L.depth[slot] = d;
    L.tri_id[slot] = t;
    if (L.nrm8) {  // approximate normals (Section 3 item 1)
        L.nrm8[slot] = encode_normal8(n.x, n.y, n.z);
    } else {
        L.nx[slot] = n.x;
        L.ny[slot] = n.y;
        L.nz[slot] = n.z;
    }
}

// The fill pass over a triangle's box, two crossings at a time: both slot
// claims and both row offsets are in flight before either sample is stored
// (as the single-mesh fill).  mk: the box's crossings, bit x + w y.
template <int A>
__device__ __forceinline__ void batch_fill_hits(const ldni_batch_item_t &it, const Setup32 &S, unsigned mk, int t,
                                                const float3 &n, int *cnt, int res, ldni_info_t *info) {
    const ldni_layers_t &L = it.out[A];
    const int *off = L.offsets;
    const long long cap = L.capacity;
    const int wdiv = (256 + S.w - 1) / S.w;  // y = (b * wdiv) >> 8 = b / w for b < 16, w <= 16
    while (mk) {
        int pr[2], k[2], row[2];
        float d[2];
        bool v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            v[u] = mk != 0u;
            const int b = v[u] ? __ffs(mk) - 1 : 0;
            mk &= mk - 1u;
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
            L.depth[slot] = d[u];
            L.tri_id[slot] = t;
            if (L.nrm8) {  // approximate normals (Section 3 item 1)
                L.nrm8[slot] = encode_normal8(n.x, n.y, n.z);
            } else {
                L.nx[slot] = n.x;
                L.ny[slot] = n.y;
                L.nz[slot] = n.z;
            }
        }
    }
}

template <bool kFill, int A>
__device__ __forceinline__ void batch_axis(const ldni_batch_item_t &it, int m, const TriView &Tv, int t,
                                           const float3 &n, int res, int *counts, const Tables &T, ldni_info_t *info) {
    Setup32 S;
    const int kind = setup_axis<A, kFill>(Tv, res, S);
    if (kind == kNone) return;
    if (kind == kBig) {
        if (!kFill)
            enqueue_big(T.big, T.qcap, T.big_n, ((long long)m << 34) | ((long long)t << 2) | A, (long long)S.w * S.h);
        return;
    }
    int *cnt = counts + T.count_base[3 * m + A];
    if (!kFill) {
        S.for_each_hit([&](int i, int j, int, int, int) { atomicAdd(cnt + (long long)j * res + i, 1); });
        return;
    }
    batch_fill_hits<A>(it, S, S.hit_bits(), t, n, cnt, res, info);
}

template <bool kFill>
__global__ void __launch_bounds__(kThreads) batch_tri_pass(const ldni_batch_item_t *items, int count, Tables T,
                                                           int *counts, ldni_info_t *infos) {
    const long long total = T.tri_prefix[count];
    for (long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x; gt < total;
         gt += (long long)gridDim.x * blockDim.x) {
        const int m = find(T.tri_prefix, count, gt);
        const ldni_batch_item_t &it = items[m];
        const int t = (int)(gt - T.tri_prefix[m]);
        const GridDev g = grid_dev(it.grid);
        TriView Tv;
        const unsigned bad = load_tri(it.verts, it.tris, t, (int)it.nv, g, Tv);
        if (bad) {
            if (!kFill) set_status(infos + m, bad);
            continue;
        }
        float3 n = make_float3(0.f, 0.f, 0.f);
        if (kFill) face_normal(Tv.p[0], Tv.p[1], Tv.p[2], n.x, n.y, n.z);
        batch_axis<kFill, 0>(it, m, Tv, t, n, g.res, counts, T, infos + m);
        batch_axis<kFill, 1>(it, m, Tv, t, n, g.res, counts, T, infos + m);
        batch_axis<kFill, 2>(it, m, Tv, t, n, g.res, counts, T, infos + m);
    }
}

template <bool kFill>
__global__ void __launch_bounds__(kThreads) batch_big(const ldni_batch_item_t *items, Tables T, int *counts,
                                                      int huge_blocks, ldni_info_t *infos) {
    for_each_big(T.big, T.qcap, T.big_n, (int)blockIdx.x, (int)gridDim.x, huge_blocks,
                 [&](long long code, int first, int step) {
        const int m = (int)(code >> 34), t = (int)((code >> 2) & 0xFFFFFFFF), a = (int)(code & 3);
        const ldni_batch_item_t &it = items[m];
        const GridDev g = grid_dev(it.grid);
        TriView Tv;
        if (load_tri(it.verts, it.tris, t, (int)it.nv, g, Tv)) return;
        Setup64 S;
        int i0, i1, j0, j1;
        if (!setup_big(Tv, a, g.res, S, i0, i1, j0, j1)) return;
        float3 n = make_float3(0.f, 0.f, 0.f);
        if (kFill) face_normal(Tv.p[0], Tv.p[1], Tv.p[2], n.x, n.y, n.z);
        int *cnt = counts + T.count_base[3 * m + a];
        const int w = i1 - i0 + 1;
        const long long npx = (long long)w * (j1 - j0 + 1);
        for (long long k = first; k < npx; k += step) {
            const int j = j0 + (int)(k / w), i = i0 + (int)(k % w);
            if (S.inside(i, j))
                batch_emit<kFill>(it, a, (long long)j * g.res + i, kFill ? S.depth(i, j) : 0.0f, t, n, cnt, infos + m);
        }
    });
}

// Scan of every image's counts: chunks of all images in one launch; the
// look-back of a chunk stops at the first chunk of its own image.
__global__ void __launch_bounds__(kThreads) batch_scan(const ldni_batch_item_t *items, int count, Tables T,
                                                       const int *counts, unsigned long long *words,
                                                       ldni_info_t *infos, int spin_limit) {
    __shared__ long long sh[kThreads / 32 + 1];
    __shared__ long long s_chunk, s_base;
    const long long nchunks = T.chunk_prefix[3 * count];
    if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(words + nchunks, 1ull);
    __syncthreads();
    const long long c = s_chunk;
    const int img = find(T.chunk_prefix, 3 * count, c);
    const int m = img / 3, a = img % 3;
    const long long local = c - T.chunk_prefix[img];
    const long long N = (long long)items[m].grid.res * items[m].grid.res;
    const int *cnt = counts + T.count_base[img];
    int *out = items[m].out[a].offsets;
    const long long base = local * kScanChunk;
    constexpr int kPer = kScanChunk / kThreads;  // 16 counts per thread
    int v[kPer];
    long long mine = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const long long e = base + (long long)threadIdx.x * kPer + k;
        v[k] = e < N ? cnt[e] : 0;
        mine += v[k];
    }
    long long total;
    const long long excl = block_exclusive_scan<kThreads>(mine, sh, &total);
    if (threadIdx.x < 32) {
        // image-local status words: chunk 0 of the image starts at prefix 0
        const long long b = lookback_warp(words + T.chunk_prefix[img], (int)local, total, infos + m, spin_limit);
        if (threadIdx.x == 0) s_base = b;
    }
    __syncthreads();
    long long run = s_base + excl;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const long long e = base + (long long)threadIdx.x * kPer + k;
        if (e < N) out[e] = (int)min(run, (long long)INT_MAX);
        run += v[k];
    }
    if (local == T.chunk_prefix[img + 1] - T.chunk_prefix[img] - 1 && threadIdx.x == 0) {
        const long long n_img = s_base + total;
        out[N] = (int)min(n_img, (long long)INT_MAX);
        infos[m].n[a] = n_img;
        if (n_img > INT_MAX) set_status(infos + m, LDNI_ST_TOOLARGE);
    }
}

// Ordering of every ray of the batch as in the single-mesh sampling: a warp
// takes 32 consecutive rays of the batch; its first lane finds the image of
// the first ray, and the others step forward from there.
__global__ void __launch_bounds__(kThreads) batch_sort(const ldni_batch_item_t *items, int count, Tables T,
                                                       ldni_info_t *infos) {
    __shared__ SortStage stage[kThreads / 32];
    const long long total = T.ray_prefix[3 * count];
    const int lane = threadIdx.x & 31;
    SortStage &st = stage[threadIdx.x >> 5];
    const auto in_place = [](long long, long long b, const RayOut &o) { return InPlace{o, b}; };
    for (long long wb = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); wb < total;
         wb += (long long)gridDim.x * blockDim.x) {
        int img = lane == 0 ? find(T.ray_prefix, 3 * count, wb) : 0;
        img = __shfl_sync(0xffffffffu, img, 0);
        const long long gr = wb + lane;
        const bool act = gr < total;
        if (act)
            while (gr >= T.ray_prefix[img + 1]) ++img;
        const int m = img / 3, a = img % 3;
        RayOut r{};
        long long b = 0;
        int n = 0;
        if (act) {
            const ldni_layers_t &L = items[m].out[a];
            r = L.nrm8 ? RayOut{L.depth, L.tri_id, reinterpret_cast<float *>(L.nrm8), nullptr, nullptr}
                       : RayOut{L.depth, L.tri_id, L.nx, L.ny, L.nz};
            const long long p = gr - T.ray_prefix[img];
            b = L.offsets[p];
            long long e = L.offsets[p + 1];
            if ((e - b) & 1) {
                atomicAdd(&infos[m].odd_rays, 1u);
                set_status(infos + m, LDNI_ST_ODD);
            }
            if (e > L.capacity) e = L.capacity;
            if (e - b >= 2) n = (int)(e - b);
        }
        // the rays of a warp may belong to two or more images: each is
        // ordered with the arrays of its own lane
        order_warp_rays<false>(b, n, b, in_place, r, st, lane);
    }
}

struct BatchWs {
    Tables T;
    int *counts;
    size_t counts_bytes;  // counts and big_n are cleared by one memset
    unsigned long long *words;
    size_t words_bytes;
};

BatchWs carve_batch(Carver &c, const ldni_batch_item_t *items_host, int count) {
    BatchWs w{};
    long long cints = 0, chunks = 0, tris = 0;
    for (int m = 0; m < count; ++m) {
        const long long N = (long long)items_host[m].grid.res * items_host[m].grid.res;
        cints += 3 * ((N + 63) / 64 * 64);
        chunks += 3 * ((N + kScanChunk - 1) / kScanChunk);
        tris += items_host[m].nt;
    }
    w.counts = c.take<int>((size_t)cints + 64);
    w.T.big_n = w.counts ? w.counts + cints : nullptr;
    w.counts_bytes = sizeof(int) * ((size_t)cints + 64);
    w.words = c.take<unsigned long long>((size_t)chunks + 1);
    w.words_bytes = sizeof(unsigned long long) * ((size_t)chunks + 1);
    w.T.tri_prefix = c.take<long long>((size_t)count + 1);
    w.T.ray_prefix = c.take<long long>(3 * (size_t)count + 1);
    w.T.chunk_prefix = c.take<long long>(3 * (size_t)count + 1);
    w.T.count_base = c.take<long long>(3 * (size_t)count);
    w.T.qcap = 3 * tris > 0 ? 3 * tris : 1;
    w.T.big = c.take<long long>((size_t)w.T.qcap);
    return w;
}

bool items_ok(const ldni_batch_item_t *items, int count) {
    for (int m = 0; m < count; ++m) {
        const ldni_batch_item_t &it = items[m];
        if (!grid_valid(&it.grid) || it.nv <= 0 || it.nt < 0 || (it.nt > 0 && (!it.verts || !it.tris)) ||
            it.nt > (1ll << 31) - 1 || it.nv > INT_MAX)
            return false;
        for (int a = 0; a < 3; ++a) {
            const ldni_layers_t &L = it.out[a];
            if (!L.offsets || L.capacity < 0 || !samples_ok(L))
                return false;
        }
    }
    return count < (1 << 29);
}

int blocks_for(long long work) {
    long long b = (work + kThreads - 1) / kThreads;
    const long long lim = (long long)num_sms() * 16;
    return (int)(b < 1 ? 1 : (b > lim ? lim : b));
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_sample_batch_workspace_size(const ldni_batch_item_t *items_host, int32_t count, size_t *bytes) {
    if (!items_host || count < 1 || !bytes || !items_ok(items_host, count)) return LDNI_EINVAL;
    Carver c(nullptr, 0);
    carve_batch(c, items_host, count);
    *bytes = align_up(c.off);
    return LDNI_OK;
}

extern "C" int ldni_sample_batch(const ldni_batch_item_t *items_dev, const ldni_batch_item_t *items_host,
                                 int32_t count, ldni_info_t *infos, void *ws, size_t ws_bytes, void *stream) {
    if (!items_dev || !items_host || count < 1 || !infos || !ws || !items_ok(items_host, count)) return LDNI_EINVAL;
    Carver c(ws, ws_bytes);
    BatchWs w = carve_batch(c, items_host, count);
    if (!c.fits()) return LDNI_EWORKSPACE;
    long long tris = 0, rays = 0, chunks = 0;
    for (int m = 0; m < count; ++m) {
        const long long N = (long long)items_host[m].grid.res * items_host[m].grid.res;
        tris += items_host[m].nt;
        rays += 3 * N;
        chunks += 3 * ((N + kScanChunk - 1) / kScanChunk);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc_ = cuda_check(cudaMemsetAsync(w.counts, 0, w.counts_bytes, s))) return rc_;
    if (int rc_ = cuda_check(cudaMemsetAsync(w.words, 0, w.words_bytes, s))) return rc_;
    if (int rc_ = cuda_check(cudaMemsetAsync(infos, 0, sizeof(ldni_info_t) * (size_t)count, s))) return rc_;
    LDNI_LAUNCH(K_BATCH, s, setup_kernel<<<1, kThreads, 0, s>>>(items_dev, count, w.T));
    if (tris > 0) {
        LDNI_LAUNCH(K_BATCH, s, batch_tri_pass<false><<<blocks_for(tris), kThreads, 0, s>>>(items_dev, count, w.T,
                                                                                             w.counts, infos));
        LDNI_LAUNCH(K_BATCH, s,
                    batch_big<false><<<5 * num_sms(), kThreads, 0, s>>>(items_dev, w.T, w.counts, num_sms(), infos));
    }
    LDNI_LAUNCH(K_BATCH, s,
                batch_scan<<<(unsigned)chunks, kThreads, 0, s>>>(items_dev, count, w.T, w.counts, w.words, infos,
                                                                  wait_limit()));
    if (tris > 0) {
        LDNI_LAUNCH(K_BATCH, s, batch_tri_pass<true><<<blocks_for(tris), kThreads, 0, s>>>(items_dev, count, w.T,
                                                                                            w.counts, infos));
        LDNI_LAUNCH(K_BATCH, s,
                    batch_big<true><<<5 * num_sms(), kThreads, 0, s>>>(items_dev, w.T, w.counts, num_sms(), infos));
    }
    LDNI_LAUNCH(K_BATCH, s, batch_sort<<<blocks_for(rays), kThreads, 0, s>>>(items_dev, count, w.T, infos));
    return cuda_status();
}
