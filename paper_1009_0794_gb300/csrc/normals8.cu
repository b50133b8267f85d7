// Approximate (8-bit) surface normals, Section 3 item 1: the paper reads the
// three components of the unit normal back from an 8-bit-per-channel colour
// buffer, 256 levels on [-1, 1], and normalises the decoded vector.  The
// sampling, Boolean and gather kernels write and move the packed words
// directly (ldni_layers_t.nrm8); these two entry points convert between the
// packed words and FP32 normals.
#include "ldni_host.h"

namespace ldni {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) encode8_kernel(const float *nx, const float *ny, const float *nz,
                                                           long long n, unsigned *w) {
    for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
        w[i] = encode_normal8(nx[i], ny[i], nz[i]);
}

// c = fl32(fl32(q / 127.5) - 1) per component, then c / sqrt(fl32(fl32(cx^2
// + cy^2) + cz^2)), every operation rounded to nearest
__global__ void __launch_bounds__(kThreads) decode8_kernel(const unsigned *w, long long n, float *nx, float *ny,
                                                           float *nz) {
    for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
        const unsigned v = w[i];
        const float cx = __fsub_rn(__fdiv_rn((float)(v & 255u), 127.5f), 1.0f);
        const float cy = __fsub_rn(__fdiv_rn((float)((v >> 8) & 255u), 127.5f), 1.0f);
        const float cz = __fsub_rn(__fdiv_rn((float)((v >> 16) & 255u), 127.5f), 1.0f);
        const float len = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy)), __fmul_rn(cz, cz)));
        nx[i] = __fdiv_rn(cx, len);
        ny[i] = __fdiv_rn(cy, len);
        nz[i] = __fdiv_rn(cz, len);
    }
}

unsigned blocks_for(long long n) {
    const long long b = (n + kThreads - 1) / kThreads, lim = 8LL * num_sms();
    return (unsigned)(b < 1 ? 1 : (b > lim ? lim : b));
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_normals_encode8(const float *nx, const float *ny, const float *nz, int64_t n, uint32_t *w,
                                    void *stream) {
    if (n < 0 || (n > 0 && (!nx || !ny || !nz || !w))) return LDNI_EINVAL;
    if (n == 0) return LDNI_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LDNI_LAUNCH(K_CODEC, s, encode8_kernel<<<blocks_for(n), kThreads, 0, s>>>(nx, ny, nz, n, w));
    return cuda_status();
}

extern "C" int ldni_normals_decode8(const uint32_t *w, int64_t n, float *nx, float *ny, float *nz, void *stream) {
    if (n < 0 || (n > 0 && (!nx || !ny || !nz || !w))) return LDNI_EINVAL;
    if (n == 0) return LDNI_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LDNI_LAUNCH(K_CODEC, s, decode8_kernel<<<blocks_for(n), kThreads, 0, s>>>(w, n, nx, ny, nz));
    return cuda_status();
}
