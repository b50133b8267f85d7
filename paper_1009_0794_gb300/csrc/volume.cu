// Enclosed volume seen by one LDNI: h^2 times the summed lengths of the
// inside ranges d[2k] .. d[2k+1] of every ray (odd-to-even ranges are inside,
// Section 2 after Proposition 1).  Rays with an odd count are skipped.
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
constexpr int kBlockRays = 4096;                      // rays per block

// The images of one call (blockIdx.y = image), all at one resolution.
struct VolJobs {
    const int *off[LDNI_MAX_IMAGES];
    const float *d[LDNI_MAX_IMAGES];
    long long cap[LDNI_MAX_IMAGES];
    double *vol[LDNI_MAX_IMAGES];
    ldni_info_t *info[LDNI_MAX_IMAGES];
};

// One block per kBlockRays rays.  When all of its rays are even, their
// samples [off[R0], off[R1]) are whole inside ranges one after another (a
// ray's ranges start at even positions from its first sample), so the block
// reads them as a contiguous run of (d[2m], d[2m + 1]) pairs, 8-byte loads,
// with no per-ray bookkeeping.  A block with an odd ray walks its rays one by
// one and skips the odd ones.
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
    __shared__ int s_odd;
    if (threadIdx.x == 0) s_odd = 0;
    __syncthreads();
    const long long R0 = (long long)blockIdx.x * kBlockRays, R1 = min(R0 + kBlockRays, nrays);
    // parity of every ray of the block: all its offsets even or odd alike
    int odd = 0;
    for (long long p = R0 + threadIdx.x; p <= R1; p += kThreads) odd |= (off[p] ^ off[R0]) & 1;
    if (odd) s_odd = 1;
    __syncthreads();
    DF acc{0.0f, 0.0f};
    if (!s_odd) {
        long long s0 = off[R0], s1 = min((long long)off[R1], cap);
        if (!range_ok(s0, max(s0, s1), cap, info)) s1 = s0;  // (checked builds)
        const bool aligned = (s0 & 1) == 0;  // 8-byte pairs when the run starts on an even sample
        for (long long k = s0 + 2LL * threadIdx.x; k + 1 < s1; k += 2LL * kThreads) {
            float lo, hi;
            if (aligned) {
                const float2 v = *reinterpret_cast<const float2 *>(d + k);
                lo = v.x;
                hi = v.y;
            } else {
                lo = d[k];
                hi = d[k + 1];
            }
            DF diff;
            two_sum(hi, -lo, diff.hi, diff.lo);
            acc = df_add(acc, diff);
        }
    } else {
        for (long long p = R0 + threadIdx.x; p < R1; p += kThreads) {
            const long long b = off[p];
            long long e = off[p + 1];
            if ((e - b) & 1) {
                atomicAdd(&info->odd_rays, 1u);
                set_status(info, LDNI_ST_ODD);
                continue;
            }
            if (e > cap) e = cap;
            if (!range_ok(b, max(b, e), cap, info)) continue;  // (checked builds)
            for (long long k = b; k + 1 < e; k += 2) {
                DF diff;
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
    const long long b = (nrays + kBlockRays - 1) / kBlockRays;
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
    if (int rc_ = cuda_check(cudaMemsetAsync(done, 0, sizeof(unsigned) * count, s))) return rc_;
    const double h = (double)grid->width / (double)grid->res;
    LDNI_LAUNCH(K_VOL_PARTIAL, s, volume_kernel<<<dim3(nb, count), kThreads, 0, s>>>(N, J, partials, done, h * h));
    return cuda_status();
}

extern "C" int ldni_volume(const ldni_layers_t *L, const ldni_grid_t *grid, double *vol, ldni_info_t *info, void *ws,
                           size_t ws_bytes, void *stream) {
    return ldni_volume_many(1, L, grid, vol, info, ws, ws_bytes, stream);
}
