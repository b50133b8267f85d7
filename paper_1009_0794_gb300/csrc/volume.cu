// Enclosed volume seen by one LDNI: h^2 times the summed lengths of the
// inside ranges d[2k] .. d[2k+1] of every ray (odd-to-even ranges are inside,
// Section 2 after Proposition 1).  FP32 samples, exact FP64 differences, FP64
// sums in a fixed order, so the result is deterministic for a given device.
#include "ldni_host.h"

namespace ldni {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum_d(double v, double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

__global__ void __launch_bounds__(kThreads) volume_partial(long long nrays, const int *__restrict__ off,
                                                           const float *__restrict__ d, long long cap,
                                                           double *partials, ldni_info_t *info) {
    __shared__ double sh[kThreads / 32];
    double acc = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nrays;
         p += (long long)gridDim.x * blockDim.x) {
        const long long b = off[p];
        long long e = off[p + 1];
        if ((e - b) & 1) {
            atomicAdd(&info->odd_rays, 1u);
            set_status(info, LDNI_ST_ODD);
            continue;
        }
        if (e > cap) e = cap;
        for (long long k = b; k + 1 < e; k += 2) acc += (double)d[k + 1] - (double)d[k];
    }
    acc = block_sum_d(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) volume_final(const double *partials, int nblocks, double h2,
                                                         double *vol) {
    __shared__ double sh[kThreads / 32];
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) acc += partials[k];
    acc = block_sum_d(acc, sh);
    if (threadIdx.x == 0) *vol = acc * h2;
}

int volume_blocks(long long nrays) {
    long long b = (nrays + kThreads - 1) / kThreads;
    const long long lim = (long long)num_sms() * 8;
    if (b > lim) b = lim;
    return (int)(b > 0 ? b : 1);
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_volume_workspace_size(int32_t res, size_t *bytes) {
    if (!bytes || res < 1 || res > 8192) return LDNI_EINVAL;
    *bytes = align_up(sizeof(double) * (size_t)volume_blocks((long long)res * res));
    return LDNI_OK;
}

extern "C" int ldni_volume(const ldni_layers_t *L, const ldni_grid_t *grid, double *vol, ldni_info_t *info, void *ws,
                           size_t ws_bytes, void *stream) {
    if (!L || !L->offsets || (L->capacity > 0 && !L->depth) || L->capacity < 0 || !grid_valid(grid) || !vol ||
        !info || !ws)
        return LDNI_EINVAL;
    const long long N = (long long)grid->res * grid->res;
    const int nb = volume_blocks(N);
    if (ws_bytes < sizeof(double) * (size_t)nb) return LDNI_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *partials = static_cast<double *>(ws);
    const double h = (double)grid->width / (double)grid->res;
    LDNI_LAUNCH(K_VOL_PARTIAL, s, volume_partial<<<nb, kThreads, 0, s>>>(N, L->offsets, L->depth, L->capacity, partials, info));
    LDNI_LAUNCH(K_VOL_FINAL, s, volume_final<<<1, kThreads, 0, s>>>(partials, nb, h * h, vol));
    return cuda_status();
}
