// A chain of unions on one grid: out = P0 u P1 u ... u P(n-1), evaluated left
// to right with the Boolean of Section 4.1 at every step and the small-
// interval removal of Section 4.1.1 after every step - the repeated
// operation of offsetting and sweeps (Section 4.2: one union per sphere) and
// of any sequence of Booleans on one grid (Section 4.1.1 keeps such chains
// exact because every operand shares the grid).
//
// Every step treats each ray on its own, so the whole chain is a fold along
// each ray: a thread carries its ray's accumulated samples from step to step
// and never waits for another ray or another step.  Two passes over the
// rays (count, then write, with the CSR scan between them) replace the n - 1
// Booleans of the step-by-step evaluation, whose intermediate images would
// each be written to and read back from memory.
//
// The result equals the step-by-step chain bit for bit: each step is the
// same merge (merge.cuh) with the accumulated solid as the first operand, so
// at a shared depth the accumulated sample is kept, and a sample that first
// enters through part k >= 1 carries the second-operand mark (tri_id bit 31)
// from then on.
#include <climits>

#include "ldni_host.h"
#include "merge.cuh"

namespace ldni {
namespace {

constexpr int kThreads = 128;
// Samples a ray's accumulated result may hold at any step.  A ray that needs
// more is left empty and reported (LDNI_ST_EVENTS).
constexpr int kChainMaxLayers = 64;

struct Entry {
    float d;
    int part;  // source part
    int idx;   // source sample in that part
};

// The fold of ray p of image img: the accumulated samples in acc (returns
// their number), or -1 when a step needed more than kChainMaxLayers.
__device__ __forceinline__ int fold_ray(const ldni_layers_t *__restrict__ parts, int count, long long p, float eps,
                                        Entry (&acc)[2][kChainMaxLayers], int &cur) {
    cur = 0;
    int na = 0;
    {
        const ldni_layers_t &P = parts[0];
        const long long b = min((long long)P.offsets[p], (long long)P.capacity);
        const long long e = min((long long)P.offsets[p + 1], (long long)P.capacity);
        if (e - b > kChainMaxLayers) return -1;
        for (long long x = b; x < e; ++x) acc[0][na++] = Entry{P.depth[x], 0, (int)x};
    }
    for (int k = 1; k < count; ++k) {
        const ldni_layers_t &P = parts[k];
        const long long b = min((long long)P.offsets[p], (long long)P.capacity);
        const long long e = min((long long)P.offsets[p + 1], (long long)P.capacity);
        // uniting a merged result (strictly ascending, no empty interval) with nothing, and no thin
        // pieces to remove, changes nothing
        if (e == b && eps == 0.0f && k > 1) continue;
        const Entry *A = acc[cur];
        Entry *O = acc[cur ^ 1];
        bool over = false;
        struct AccDepth {
            const Entry *a;
            __device__ __forceinline__ float operator[](int i) const { return a[i].d; }
        };
        const float *dB = P.depth + b;
        const int m = merge_core<int>(AccDepth{A}, 0, na, dB, 0, (int)(e - b), LDNI_OP_UNION, eps,
                                      [&](bool pb, int pi, bool cb, int ci, int mm) {
                                          if (mm + 2 > kChainMaxLayers) {
                                              over = true;
                                              return;
                                          }
                                          O[mm] = pb ? Entry{dB[pi], k, (int)(b + pi)} : A[pi];
                                          O[mm + 1] = cb ? Entry{dB[ci], k, (int)(b + ci)} : A[ci];
                                      });
        if (over) return -1;
        na = m;
        cur ^= 1;
    }
    return na;
}

// Pass 1 (kWrite false): every ray's result count into counts.  Pass 2: the
// samples at the offsets of out.  blockIdx.y = image; parts of image j are
// parts[j * count ..].
struct Counts {
    int *c[3];
};

template <bool kWrite>
__global__ void __launch_bounds__(kThreads) chain_pass(long long N, const ldni_layers_t *__restrict__ parts_all,
                                                       int count, float eps, Counts counts, ldni_layers_t o0,
                                                       ldni_layers_t o1, ldni_layers_t o2, ldni_info_t *info) {
    const int img = blockIdx.y;
    const ldni_layers_t *parts = parts_all + (size_t)img * count;
    const ldni_layers_t &o = img == 0 ? o0 : (img == 1 ? o1 : o2);
    Entry acc[2][kChainMaxLayers];
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        if (!kWrite) {
            for (int k = 0; k < count; ++k) {  // Definition 4 on the inputs
                const int c = parts[k].offsets[p + 1] - parts[k].offsets[p];
                if (c & 1) {
                    atomicAdd(&info->odd_rays, 1u);
                    set_status(info, LDNI_ST_ODD);
                }
            }
        }
        int cur;
        int n = fold_ray(parts, count, p, eps, acc, cur);
        if (n < 0) {
            if (!kWrite) set_status(info, LDNI_ST_EVENTS);
            n = 0;
        }
        if (!kWrite) {
            counts.c[img][p] = n;
            continue;
        }
        const long long base = o.offsets[p];
        for (int x = 0; x < n; ++x) {
            const Entry &E = acc[cur][x];
            const long long at = base + x;
            if (at >= o.capacity) {
                set_status(info, LDNI_ST_CAPACITY);
                break;
            }
            const ldni_layers_t &P = parts[E.part];
            o.depth[at] = E.d;
            if (o.nrm8) {
                o.nrm8[at] = P.nrm8[E.idx];
            } else {
                o.nx[at] = P.nx[E.idx];
                o.ny[at] = P.ny[E.idx];
                o.nz[at] = P.nz[E.idx];
            }
            o.tri_id[at] = E.part == 0 ? P.tri_id[E.idx] : (int)((unsigned)P.tri_id[E.idx] | 0x80000000u);
        }
    }
}

struct ChainWs {
    int *counts[3];
    long long *partials;
};

ChainWs carve_chain_ws(Carver &c, int res, int nimg) {
    ChainWs w{};
    const long long N = (long long)res * res;
    for (int j = 0; j < nimg; ++j) w.counts[j] = c.take<int>((size_t)N);
    w.partials = c.take<long long>(csr_scan_partials(N) * nimg);
    return w;
}

int grid_for(long long N) {
    long long b = (N + kThreads - 1) / kThreads;
    const long long lim = (long long)num_sms() * 16;
    return (int)(b < 1 ? 1 : (b > lim ? lim : b));
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_union_chain_workspace_size(int32_t res, int32_t nimg, size_t *bytes) {
    if (!bytes || res < 1 || res > 8192 || nimg < 1 || nimg > 3) return LDNI_EINVAL;
    Carver c(nullptr, 0);
    carve_chain_ws(c, res, nimg);
    *bytes = align_up(c.off);
    return LDNI_OK;
}

extern "C" int ldni_union_chain(const ldni_layers_t *parts_dev, const ldni_layers_t *parts_host, int32_t count,
                                int32_t nimg, const ldni_grid_t *grid, float eps, ldni_layers_t *out,
                                ldni_info_t *info, void *ws, size_t ws_bytes, void *stream) {
    if (!parts_dev || !parts_host || count < 1 || nimg < 1 || nimg > 3 || !grid_valid(grid) || !out || !info ||
        !ws || !(eps >= 0.0f))
        return LDNI_EINVAL;
    for (int j = 0; j < nimg; ++j) {
        const ldni_layers_t &o = out[j];
        if (!o.offsets || o.capacity < 0 || !samples_ok(o)) return LDNI_EINVAL;
        const ldni_layers_t *fmt[2] = {&o, nullptr};
        bool packed = false, pk = false;
        if (!same_format(fmt, 1, &packed)) return LDNI_EINVAL;
        for (int k = 0; k < count; ++k) {
            const ldni_layers_t &P = parts_host[(size_t)j * count + k];
            fmt[1] = &P;
            if (!P.offsets || P.capacity < 0 || !samples_ok(P) || !same_format(fmt, 2, &pk)) return LDNI_EINVAL;
        }
    }
    Carver c(ws, ws_bytes);
    ChainWs w = carve_chain_ws(c, grid->res, nimg);
    if (!c.fits()) return LDNI_EWORKSPACE;
    const long long N = (long long)grid->res * grid->res;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ldni_layers_t o[3] = {out[0], nimg > 1 ? out[1] : out[0], nimg > 2 ? out[2] : out[0]};
    const dim3 g((unsigned)grid_for(N), (unsigned)nimg);
    const Counts cn{{w.counts[0], w.counts[1], w.counts[2]}};
    LDNI_LAUNCH(K_CHAIN, s,
                chain_pass<false><<<g, kThreads, 0, s>>>(N, parts_dev, count, eps, cn, o[0], o[1], o[2], info));
    int rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    const int *cnt[3] = {w.counts[0], w.counts[1], w.counts[2]};
    int *off[3] = {out[0].offsets, nimg > 1 ? out[1].offsets : nullptr, nimg > 2 ? out[2].offsets : nullptr};
    rc = csr_scan(cnt, off, nimg, N, w.partials, info, 0, s);
    if (rc != LDNI_OK) return rc;
    LDNI_LAUNCH(K_CHAIN, s,
                chain_pass<true><<<g, kThreads, 0, s>>>(N, parts_dev, count, eps, cn, o[0], o[1], o[2], info));
    return cuda_status();
}
