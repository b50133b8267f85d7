// Enclosed volume seen by one LDNI: h^2 times the summed lengths of the
// inside ranges d[2k] .. d[2k+1] of every ray (odd-to-even ranges are inside,
// Section 2 after Proposition 1).
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the per-ray
// work stays in FP32: each difference d[2k+1] - d[2k] is split exactly into
// a rounded FP32 value and its FP32 rounding error (TwoSum, Knuth, TAOCP
// vol. 2, 4.2.2), and the per-thread and per-block sums are kept as unevaluated
// FP32 pairs (double-float arithmetic, Dekker 1971).  Each block's pair is
// widened to FP64 once; the last block to finish adds the block partials in
// a fixed order.  The result is deterministic for a given device and within
// about 1e-13 relative of the exact sum.
#include "dfloat.cuh"
#include "ldni_host.h"

namespace ldni {
namespace {

constexpr int kThreads = 256;
constexpr int kRaysPerThread = 4;

// The images of one call (blockIdx.y = image), all at one resolution.
struct VolJobs {
    const int *off[LDNI_MAX_IMAGES];
    const float *d[LDNI_MAX_IMAGES];
    long long cap[LDNI_MAX_IMAGES];
    double *vol[LDNI_MAX_IMAGES];
    ldni_info_t *info[LDNI_MAX_IMAGES];
};

__global__ void __launch_bounds__(kThreads) volume_kernel(long long nrays, const __grid_constant__ VolJobs J,
                                                          double *partials_all, unsigned *done_all, double h2) {
    const int job = blockIdx.y;
    const int *__restrict__ off = J.off[job];
    const float *__restrict__ d = J.d[job];
    const long long cap = J.cap[job];
    double *partials = partials_all + (size_t)job * gridDim.x;
    unsigned *done = done_all + job;
    ldni_info_t *info = J.info[job];
    __shared__ DF sh[kThreads / 32];
    __shared__ bool s_last;
    DF acc{0.0f, 0.0f};
    const long long span = (long long)kThreads * kRaysPerThread;
    for (long long p0 = blockIdx.x * span + threadIdx.x; p0 < nrays; p0 += (long long)gridDim.x * span) {
        // kRaysPerThread independent rays: their loads are all in flight together
        long long b[kRaysPerThread], e[kRaysPerThread];
#pragma unroll
        for (int r = 0; r < kRaysPerThread; ++r) {
            const long long p = p0 + (long long)r * kThreads;
            b[r] = p < nrays ? off[p] : 0;
            e[r] = p < nrays ? off[p + 1] : 0;
        }
#pragma unroll
        for (int r = 0; r < kRaysPerThread; ++r) {
            if ((e[r] - b[r]) & 1) {
                atomicAdd(&info->odd_rays, 1u);
                set_status(info, LDNI_ST_ODD);
                e[r] = b[r];
            }
            if (e[r] > cap) e[r] = cap;
        }
        float lo[kRaysPerThread], hi[kRaysPerThread];
#pragma unroll
        for (int r = 0; r < kRaysPerThread; ++r) {  // first inside range of every ray
            const bool has = e[r] - b[r] >= 2;
            lo[r] = has ? d[b[r]] : 0.0f;
            hi[r] = has ? d[b[r] + 1] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < kRaysPerThread; ++r) {
            DF diff;
            two_sum(hi[r], -lo[r], diff.hi, diff.lo);
            acc = df_add(acc, diff);
            for (long long k = b[r] + 2; k + 1 < e[r]; k += 2) {  // further ranges (multi-layer rays)
                two_sum(d[k + 1], -d[k], diff.hi, diff.lo);
                acc = df_add(acc, diff);
            }
        }
    }
    const DF t = df_block_sum<kThreads>(acc, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = (double)t.hi + (double)t.lo;
        __threadfence();
        s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // last block: FP64 sum of the block partials in a fixed order
    __threadfence();
    __shared__ double shd[kThreads];
    const double sum = fixed_order_sum<kThreads>(partials, (int)gridDim.x, shd);
    if (threadIdx.x == 0) *J.vol[job] = sum * h2;
}

int volume_blocks(long long nrays) {
    long long b = (nrays + (long long)kThreads * kRaysPerThread - 1) / ((long long)kThreads * kRaysPerThread);
    const long long lim = (long long)num_sms() * 2;  // few blocks: each ends with a reduction and a fence
    if (b > lim) b = lim;
    return (int)(b > 0 ? b : 1);
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_volume_many_workspace_size(int32_t res, int32_t count, size_t *bytes) {
    if (!bytes || res < 1 || res > 8192 || count < 1 || count > LDNI_MAX_IMAGES) return LDNI_EINVAL;
    *bytes = align_up((sizeof(double) * (size_t)volume_blocks((long long)res * res) + sizeof(unsigned)) * count);
    return LDNI_OK;
}

extern "C" int ldni_volume_workspace_size(int32_t res, size_t *bytes) {
    return ldni_volume_many_workspace_size(res, 1, bytes);
}

extern "C" int ldni_volume_many(int32_t count, const ldni_layers_t *L, const ldni_grid_t *grid, double *vols,
                                ldni_info_t *infos, void *ws, size_t ws_bytes, void *stream) {
    if (count < 1 || count > LDNI_MAX_IMAGES || !L || !grid_valid(grid) || !vols || !infos || !ws)
        return LDNI_EINVAL;
    VolJobs J{};
    for (int j = 0; j < count; ++j) {
        if (!L[j].offsets || (L[j].capacity > 0 && !L[j].depth) || L[j].capacity < 0) return LDNI_EINVAL;
        J.off[j] = L[j].offsets;
        J.d[j] = L[j].depth;
        J.cap[j] = L[j].capacity;
        J.vol[j] = vols + j;
        J.info[j] = infos + j;
    }
    const long long N = (long long)grid->res * grid->res;
    const int nb = volume_blocks(N);
    size_t need = 0;
    ldni_volume_many_workspace_size(grid->res, count, &need);
    if (ws_bytes < need) return LDNI_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *partials = static_cast<double *>(ws);
    unsigned *done = reinterpret_cast<unsigned *>(partials + (size_t)nb * count);
    if (cudaMemsetAsync(done, 0, sizeof(unsigned) * count, s) != cudaSuccess) return LDNI_ECUDA;
    const double h = (double)grid->width / (double)grid->res;
    LDNI_LAUNCH(K_VOL_PARTIAL, s, volume_kernel<<<dim3(nb, count), kThreads, 0, s>>>(N, J, partials, done, h * h));
    return cuda_status();
}

extern "C" int ldni_volume(const ldni_layers_t *L, const ldni_grid_t *grid, double *vol, ldni_info_t *info, void *ws,
                           size_t ws_bytes, void *stream) {
    return ldni_volume_many(1, L, grid, vol, info, ws, ws_bytes, stream);
}
