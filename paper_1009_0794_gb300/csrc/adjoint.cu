// Adjoint of LDNI sample depths and LDNI volume with respect to the mesh
// vertices.
//
// A sample of ray (u, v) on triangle t sits where the ray meets t's plane:
// d = sum_k lambda_k a_k with lambda_k the barycentrics of (u, v) in t's
// (unsnapped) projection and a_k the vertex a-coordinates.  Moving vertex j by
// delta moves the surface point under the ray by lambda_j delta, so
//     d(d) / d(V_j) = lambda_j * n / n_a          (n: the face normal)
// and, since odd-to-even ranges are inside (Section 2 after Proposition 1),
// the volume h^2 sum_rays sum_k (d_{2k+1} - d_{2k}) has
//     d(V_a) / d(V_j) = h^2 sum_samples sigma_s lambda_j n / n_a,
// sigma = -1 for even positions (entering), +1 for odd (leaving).  The set of
// crossings is held fixed: where a vertex move would add or remove a
// crossing the volume changes by a boundary term this derivative leaves out.
#include "ldni_host.h"

namespace ldni {
namespace {

constexpr int kThreads = 256;

// The geometry runs in FP32 with error-free steps where cancellation would
// hurt (this GPU's FP64 rate is a small fraction of its FP32 rate):
//  - edge vectors are differences of nearby FP32 coordinates (exact, or
//    within an ulp of their size);
//  - every 2 x 2 determinant a d - b c comes from Kahan's fused form, within
//    about 1.5 ulp of the exact value even when the two products nearly cancel
//    (a face seen edge-on, a ray near an edge);
//  - the ray centre o + (i + 1/2) h is kept as an unevaluated pair of floats,
//    so its offset from a vertex has the accuracy of the offset, not of 1.
__device__ __forceinline__ float det2(float a, float b, float c, float d) {  // a d - b c
    const float w = b * c;
    const float e = fmaf(-b, c, w);  // w - b c, exactly
    const float f = fmaf(a, d, -w);
    return f + e;
}

__device__ __forceinline__ float comp3(const float (&v)[3], int a) { return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]); }

struct Pair {  // hi + lo, |lo| <= ulp(hi) / 2
    float hi, lo;
};

// o + t h, with h = h_hi + h_lo, to about 2^-44 relative
__device__ __forceinline__ Pair centre(float o, float t, float h_hi, float h_lo) {
    const float p = t * h_hi;
    const float p_err = fmaf(t, h_hi, -p) + t * h_lo;
    const float s = o + p;  // TwoSum(o, p)
    const float bp = s - o;
    const float s_err = (o - (s - bp)) + (p - bp);
    return Pair{s, s_err + p_err};
}

__global__ void __launch_bounds__(kThreads) depth_vjp_kernel(const float *__restrict__ verts,
                                                             const int *__restrict__ tris, int nv, int nt, GridDev g,
                                                             float h_hi, float h_lo, int axis,
                                                             const int *__restrict__ off,
                                                             const int *__restrict__ tri_id, long long cap,
                                                             const float *__restrict__ wsample, float vol_weight,
                                                             float *grad, ldni_info_t *info) {
    const long long nrays = (long long)g.res * g.res;
    const int U = (axis + 1) % 3, V = (axis + 2) % 3;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nrays;
         p += (long long)gridDim.x * blockDim.x) {
        const long long b = off[p];
        long long e = off[p + 1];
        if (e > cap) e = cap;
        if (e <= b) continue;
        const int i = (int)(p % g.res), j = (int)(p / g.res);
        const Pair cu = centre(g.o[U], (float)i + 0.5f, h_hi, h_lo);  // i + 1/2 exact for res < 2^23
        const Pair cv = centre(g.o[V], (float)j + 0.5f, h_hi, h_lo);
        for (long long s = b; s < e; ++s) {
            const int t = tri_id[s];
            if (t < 0 || t >= nt) {  // not a sample of this mesh (e.g. a Boolean's B side)
                set_status(info, LDNI_ST_INDEX);
                continue;
            }
            float w = vol_weight * (((s - b) & 1) ? 1.0f : -1.0f);
            if (wsample) w += wsample[s];
            if (w == 0.0f) continue;
            const int id[3] = {tris[3 * (long long)t], tris[3 * (long long)t + 1], tris[3 * (long long)t + 2]};
            if ((unsigned)id[0] >= (unsigned)nv || (unsigned)id[1] >= (unsigned)nv || (unsigned)id[2] >= (unsigned)nv) {
                set_status(info, LDNI_ST_INDEX);
                continue;
            }
            float P[3][3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) P[k][c] = __ldg(verts + 3 * (long long)id[k] + c);
            const float e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
            const float e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
            const float n[3] = {det2(e1[1], e1[2], e2[1], e2[2]), det2(e1[2], e1[0], e2[2], e2[0]),
                                det2(e1[0], e1[1], e2[0], e2[1])};
            // n_a is also the determinant of the projected edges (u1 v2 - v1 u2)
            const float na = comp3(n, axis);
            if (na == 0.0f) continue;
            // continuous barycentrics of the centre, relative to vertex 0
            const float u1 = comp3(e1, U), v1 = comp3(e1, V), u2 = comp3(e2, U), v2 = comp3(e2, V);
            const float xu = (cu.hi - comp3(P[0], U)) + cu.lo, xv = (cv.hi - comp3(P[0], V)) + cv.lo;
            const float l1 = det2(xu, u2, xv, v2) / na;  // (xu v2 - u2 xv) / na
            const float l2 = det2(u1, v1, xu, xv) / na;  // (u1 xv - v1 xu) / na
            const float l[3] = {1.0f - l1 - l2, l1, l2};
            const float sw = w / na;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float *gk = grad + 3 * (long long)id[k];
                const float c = sw * l[k];
                atomicAdd(gk + 0, c * n[0]);
                atomicAdd(gk + 1, c * n[1]);
                atomicAdd(gk + 2, c * n[2]);
            }
        }
    }
}

int launch(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid, int32_t axis,
           const ldni_layers_t *L, const float *wsample, float vol_weight, float *grad, ldni_info_t *info,
           void *stream) {
    if (!grid_valid(grid) || !L || !L->offsets || (L->capacity > 0 && !L->tri_id) || axis < 0 || axis > 2 || nv <= 0 ||
        nt < 0 || (nt > 0 && (!verts || !tris)) || !grad || !info)
        return LDNI_EINVAL;
    if (nt > INT_MAX || nv > INT_MAX) return LDNI_ETOOLARGE;
    const long long N = (long long)grid->res * grid->res;
    long long blocks = (N + kThreads - 1) / kThreads;
    if (blocks > (long long)num_sms() * 16) blocks = (long long)num_sms() * 16;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double h = (double)grid->width / (double)grid->res;  // the pitch as an unevaluated float pair
    const float h_hi = (float)h, h_lo = (float)(h - (double)h_hi);
    LDNI_LAUNCH(K_GRAD, s,
                depth_vjp_kernel<<<(int)blocks, kThreads, 0, s>>>(verts, tris, (int)nv, (int)nt, make_grid(grid), h_hi,
                                                                  h_lo, axis, L->offsets, L->tri_id, L->capacity,
                                                                  wsample, vol_weight, grad, info));
    return cuda_status();
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_depth_vjp(const float *verts, int64_t nv, const int32_t *tris, int64_t nt, const ldni_grid_t *grid,
                              int32_t axis, const ldni_layers_t *L, const float *grad_depth, float *grad_verts,
                              ldni_info_t *info, void *stream) {
    if (!grad_depth) return LDNI_EINVAL;
    return launch(verts, nv, tris, nt, grid, axis, L, grad_depth, 0.0f, grad_verts, info, stream);
}

extern "C" int ldni_volume_grad(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                                const ldni_grid_t *grid, int32_t axis, const ldni_layers_t *L, double grad_volume,
                                float *grad_verts, ldni_info_t *info, void *stream) {
    if (!grid_valid(grid)) return LDNI_EINVAL;
    const double h = (double)grid->width / (double)grid->res;
    return launch(verts, nv, tris, nt, grid, axis, L, nullptr, (float)(grad_volume * h * h), grad_verts, info,
                  stream);
}
