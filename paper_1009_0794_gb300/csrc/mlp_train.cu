// Inference and training of the per-tile capacity network (mlp.cuh) with
// hand-written kernels: dense layers, an asymmetric squared loss, the
// backward pass and Adam (Kingma & Ba, 2015).  The forward pass uses the BF16
// weights with FP32 accumulation in the same order as the sampler's
// inference, so trained outputs and sampler predictions agree bit for bit.
#include <cuda_bf16.h>

#include "ldni_host.h"
#include "mlp.cuh"

namespace ldni {
namespace {

constexpr int kThreads = 256;

// thread per row: the whole network (used by ldni_mlp_forward)
__global__ void __launch_bounds__(128) mlp_rows(const __nv_bfloat16 *__restrict__ W, const float *__restrict__ b,
                                                const float *__restrict__ X, long long n, float *y) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[kMlpIn];
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) x[i] = X[r * kMlpIn + i];
    y[r] = mlp_forward_row(W, b, x);
}

// Z = Ain W^T + b, Aout = relu(Z) (identity for the output layer)
__global__ void __launch_bounds__(kThreads) dense_fwd(const float *__restrict__ Ain, int in,
                                                      const __nv_bfloat16 *__restrict__ W,
                                                      const float *__restrict__ b, int out, long long n, float *Z,
                                                      float *Aout, int relu) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n * out) return;
    const long long r = idx / out;
    const int o = (int)(idx % out);
    float s = b[o];
    for (int i = 0; i < in; ++i) s = fmaf(__bfloat162float(W[o * in + i]), Ain[r * in + i], s);
    Z[idx] = s;
    Aout[idx] = relu ? fmaxf(s, 0.0f) : s;
}

// dy = dL/dy for L = mean_r w_r (y_r - t_r)^2, w_r = uw if y_r < t_r else 1
__global__ void __launch_bounds__(kThreads) loss_grad(const float *__restrict__ y, const float *__restrict__ t,
                                                      long long n, float uw, float *dy, float *loss) {
    __shared__ float sh[kThreads / 32];
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (r < n) {
        const float d = y[r] - t[r];
        const float w = d < 0.0f ? uw : 1.0f;
        dy[r] = 2.0f * w * d / (float)n;
        l = w * d * d / (float)n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) s += sh[w];
        atomicAdd(loss, s);
    }
}

// dA <- dA * relu'(Z)
__global__ void __launch_bounds__(kThreads) relu_bwd(float *dA, const float *__restrict__ Z, long long cnt) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < cnt && Z[k] <= 0.0f) dA[k] = 0.0f;
}

// gW[o][i] = sum_r dZ[r][o] Ain[r][i], gb[o] = sum_r dZ[r][o]; block (o, 32 inputs),
// 8 row groups reduced in a fixed order
__global__ void __launch_bounds__(kThreads) dense_wgrad(const float *__restrict__ dZ, const float *__restrict__ Ain,
                                                        long long n, int in, int out, float *gW, float *gb) {
    __shared__ float sh[8][33];
    const int o = blockIdx.x;
    const int il = threadIdx.x & 31, rg = threadIdx.x >> 5;
    const int i = blockIdx.y * 32 + il;  // i == in is the bias
    float s = 0.0f;
    if (i <= in) {
        for (long long r = rg; r < n; r += 8) {
            const float a = i < in ? Ain[r * in + i] : 1.0f;
            s = fmaf(dZ[r * out + o], a, s);
        }
    }
    sh[rg][il] = s;
    __syncthreads();
    if (rg == 0 && i <= in) {
        float t = 0.0f;
        for (int g = 0; g < 8; ++g) t += sh[g][il];
        if (i < in)
            gW[o * in + i] = t;
        else
            gb[o] = t;
    }
}

// dAin[r][i] = sum_o W[o][i] dZ[r][o]
__global__ void __launch_bounds__(kThreads) dense_dgrad(const float *__restrict__ dZ,
                                                        const __nv_bfloat16 *__restrict__ W, long long n, int in,
                                                        int out, float *dAin) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n * in) return;
    const long long r = idx / in;
    const int i = (int)(idx % in);
    float s = 0.0f;
    for (int o = 0; o < out; ++o) s = fmaf(__bfloat162float(W[o * in + i]), dZ[r * out + o], s);
    dAin[idx] = s;
}

__global__ void __launch_bounds__(kThreads) adam_kernel(float *p, const float *__restrict__ g, float *m, float *v,
                                                        int cnt, float lr, float b1, float b2, float eps, float c1,
                                                        float c2, __nv_bfloat16 *bf) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    p[k] = pk;
    if (bf) bf[k] = __float2bfloat16_rn(pk);
}

struct TrainWs {
    float *Z[4], *A[4];   // per layer pre- and post-activation
    float *dA0, *dA1;     // gradients w.r.t. layer inputs (ping-pong, [n][64])
    float *g;             // weights then biases
};

TrainWs carve_train(Carver &c, long long n) {
    TrainWs w{};
    for (int l = 0; l < 3; ++l) {
        w.Z[l] = c.take<float>((size_t)n * kMlpHidden);
        w.A[l] = c.take<float>((size_t)n * kMlpHidden);
    }
    w.Z[3] = c.take<float>((size_t)n);
    w.A[3] = c.take<float>((size_t)n);
    w.dA0 = c.take<float>((size_t)n * kMlpHidden);
    w.dA1 = c.take<float>((size_t)n * kMlpHidden);
    w.g = c.take<float>((size_t)(kMlpWeights + kMlpBiases));
    return w;
}

inline unsigned blocks_for(long long cnt, int th = kThreads) { return (unsigned)((cnt + th - 1) / th); }

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_mlp_forward(const ldni_mlp_t *mlp, const float *X, int64_t n, float *y, void *stream) {
    if (!mlp || !mlp->w || !mlp->b || !X || !y || n < 0) return LDNI_EINVAL;
    if (n == 0) return LDNI_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LDNI_LAUNCH(K_MLP, s,
                mlp_rows<<<blocks_for(n, 128), 128, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(mlp->w), mlp->b,
                                                             X, n, y));
    return cuda_status();
}

extern "C" int ldni_mlp_train_workspace_size(int64_t n, size_t *bytes) {
    if (!bytes || n < 1) return LDNI_EINVAL;
    Carver c(nullptr, 0);
    carve_train(c, n);
    *bytes = align_up(c.off);
    return LDNI_OK;
}

extern "C" int ldni_mlp_train_step(float *master_w, float *b, uint16_t *w_bf16, float *m, float *v, const float *X,
                                   const float *label, int64_t n, float lr, int32_t step, float under_weight,
                                   float *loss, float *grad, void *ws, size_t ws_bytes, void *stream) {
    if (!master_w || !b || !w_bf16 || !m || !v || !X || !label || n < 1 || step < 1 || !loss || !ws ||
        !(lr > 0.0f) || !(under_weight > 0.0f))
        return LDNI_EINVAL;
    Carver c(ws, ws_bytes);
    TrainWs w = carve_train(c, n);
    if (!c.fits()) return LDNI_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const __nv_bfloat16 *W = reinterpret_cast<const __nv_bfloat16 *>(w_bf16);
    const int H = kMlpHidden;
    const int ins[4] = {kMlpIn, H, H, H};
    const int outs[4] = {H, H, H, 1};
    const int woff[4] = {kW0, kW1, kW2, kW3};
    const int boff[4] = {kB0, kB1, kB2, kB3};
    if (int rc_ = cuda_check(cudaMemsetAsync(loss, 0, sizeof(float), s))) return rc_;
    // forward
    const float *Ain = X;
    for (int l = 0; l < 4; ++l) {
        LDNI_LAUNCH(K_MLP, s,
                    dense_fwd<<<blocks_for(n * outs[l]), kThreads, 0, s>>>(Ain, ins[l], W + woff[l], b + boff[l],
                                                                          outs[l], n, w.Z[l], w.A[l], l < 3));
        Ain = w.A[l];
    }
    // loss and dL/dy (dZ of the output layer, stored in A[3])
    float *gw = w.g, *gb = w.g + kMlpWeights;
    LDNI_LAUNCH(K_MLP, s, loss_grad<<<blocks_for(n), kThreads, 0, s>>>(w.Z[3], label, n, under_weight, w.A[3], loss));
    float *dZ = w.A[3];
    float *bufs[2] = {w.dA0, w.dA1};
    for (int l = 3; l >= 0; --l) {
        const float *A_in = l > 0 ? w.A[l - 1] : X;
        LDNI_LAUNCH(K_MLP, s,
                    dense_wgrad<<<dim3(outs[l], (ins[l] + 1 + 31) / 32), kThreads, 0, s>>>(dZ, A_in, n, ins[l],
                                                                                          outs[l], gw + woff[l],
                                                                                          gb + boff[l]));
        if (l > 0) {
            float *dA = bufs[l & 1];
            LDNI_LAUNCH(K_MLP, s,
                        dense_dgrad<<<blocks_for(n * ins[l]), kThreads, 0, s>>>(dZ, W + woff[l], n, ins[l], outs[l],
                                                                               dA));
            LDNI_LAUNCH(K_MLP, s, relu_bwd<<<blocks_for(n * ins[l]), kThreads, 0, s>>>(dA, w.Z[l - 1], n * ins[l]));
            dZ = dA;
        }
    }
    if (grad)
        if (int rc_ = cuda_check(
                cudaMemcpyAsync(grad, w.g, sizeof(float) * (kMlpWeights + kMlpBiases), cudaMemcpyDeviceToDevice, s)))
            return rc_;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    LDNI_LAUNCH(K_MLP, s,
                adam_kernel<<<blocks_for(kMlpWeights), kThreads, 0, s>>>(master_w, gw, m, v, kMlpWeights, lr, b1, b2,
                                                                         eps, c1, c2,
                                                                         reinterpret_cast<__nv_bfloat16 *>(w_bf16)));
    LDNI_LAUNCH(K_MLP, s,
                adam_kernel<<<blocks_for(kMlpBiases), kThreads, 0, s>>>(b, gb, m + kMlpWeights, v + kMlpWeights,
                                                                        kMlpBiases, lr, b1, b2, eps, c1, c2,
                                                                        nullptr));
    return cuda_status();
}
