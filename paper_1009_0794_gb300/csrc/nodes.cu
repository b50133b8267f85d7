// Grid-node classification from the three LDNIs (Section 5.1, Step 1): the
// rays of the x-, y- and z-LDNI meet at the res^3 nodes of the grid
// (Definition 3); a node is inside the solid when it lies in the solid
// volume of at least two of the three images, which settles the images'
// disagreements near the surface.
//
// Node (i, j, k) sits at (c_x(i), c_y(j), c_z(k)) with
// c_a(t) = fl32(o_a + fl32((t + 1/2) * h)), h = fl32(W / res): the pixel
// centres of the images.  Image a puts the node inside when an odd number of
// the samples of its ray through the node lie strictly below c_a (the
// odd-to-even ranges are inside, Section 2 after Proposition 1).
//
// Ray kernels write one bit volume per image, the bits of a word running
// along that image's rays, laid out so that the stores are coalesced; a vote
// kernel then takes 32 x 32 x 32 node cubes, transposes the y and z bits
// through shared memory and writes the majority in the x-fastest output
// layout.
#include "ldni_host.h"

namespace ldni {
namespace {

constexpr int kRayWarps = 8;

__device__ __forceinline__ float node_c(int t, float o, float h) {
    return __fadd_rn(o, __fmul_rn((float)t + 0.5f, h));
}

// First node t in [0, res] with c(t) > d (c increases with t): a float
// estimate, then corrected with the exact node positions.
__device__ __forceinline__ int first_above(float d, int res, float o, float h) {
    float est = (d - o) / h - 0.5f;
    int t = !(est > 0.0f) ? 0 : (est >= (float)res ? res : (int)est);
    while (t > 0 && node_c(t - 1, o, h) > d) --t;
    while (t < res && !(node_c(t, o, h) > d)) ++t;
    return t;
}

// Bits t = 32 w .. 32 w + 31 of one ray: node t is inside iff an odd number
// of the ray's sorted depths [d, d + n) are < c(t), i.e. iff c(t) lies in
// some (d[2m], d[2m+1]] (or above the last depth of an odd ray).
__device__ __forceinline__ unsigned ray_word(const float *__restrict__ d, int n, int w, int res, float o, float h) {
    const int t0 = 32 * w, t1 = min(t0 + 32, res);  // nodes [t0, t1)
    unsigned word = 0;
    for (int m = 0; m < n; m += 2) {
        const int lo = first_above(d[m], res, o, h);                           // c(t) > d[2m]
        const int hi = m + 1 < n ? first_above(d[m + 1], res, o, h) : res;     // c(t) > d[2m+1] from here on
        const int a = max(lo, t0), b = min(hi, t1);
        if (a < b) {
            const int len = b - a;
            word |= (len >= 32 ? 0xffffffffu : ((1u << len) - 1u)) << (a - t0);
        }
    }
    return word;
}

__device__ __forceinline__ void ray_range(const int *__restrict__ off, long long cap, long long p, long long &b,
                                          long long &e, ldni_info_t *info, bool report) {
    b = off[p];
    e = off[p + 1];
    if (((e - b) & 1) && report) {
        atomicAdd(&info->odd_rays, 1u);
        set_status(info, LDNI_ST_ODD);
    }
    if (e > cap) {
        if (report) set_status(info, LDNI_ST_CAPACITY);
        e = cap;
        b = min(b, e);
    }
}

// x-image: one warp per ray p = k res + j, lane l writing word l of row
// (k, j) of Vx: Vx[(k res + j) W + w] holds nodes i = 32 w .. 32 w + 31.
__global__ void __launch_bounds__(kRayWarps * 32) node_rays_x(const int *__restrict__ off,
                                                               const float *__restrict__ depth, long long cap, int res,
                                                               int W, float o, float h, unsigned *V,
                                                               ldni_info_t *info) {
    const long long p = (long long)blockIdx.x * kRayWarps + (threadIdx.x >> 5);
    if (p >= (long long)res * res) return;
    const int lane = threadIdx.x & 31;
    long long b, e;
    ray_range(off, cap, p, b, e, info, lane == 0);
    for (int w = lane; w < W; w += 32) V[p * W + w] = ray_word(depth + b, (int)(e - b), w, res, o, h);
}

// y- and z-images: one thread per ray, consecutive threads = consecutive
// node index i, so every word store is coalesced:
//   y-image ray p = i res + k: word w (nodes j) at Vy[(w res + k) res + i]
//   z-image ray p = j res + i: word w (nodes k) at Vz[(w res + j) res + i]
__global__ void __launch_bounds__(256) node_rays_yz(const int *__restrict__ off, const float *__restrict__ depth,
                                                     long long cap, int res, int W, float o, float h, int is_y,
                                                     unsigned *V, ldni_info_t *info) {
    const long long q = blockIdx.x * 256LL + threadIdx.x;  // = r res + i, r = k (y) or j (z)
    if (q >= (long long)res * res) return;
    const long long i = q % res, r = q / res;
    const long long p = is_y ? i * res + r : r * res + i;
    long long b, e;
    ray_range(off, cap, p, b, e, info, true);
    const long long plane = (long long)res * res;
    for (int w = 0; w < W; ++w) V[w * plane + q] = ray_word(depth + b, (int)(e - b), w, res, o, h);
}

// One block per cube of 32 (i) x 32 (j) x 32 (k) nodes; thread (kk, jj)
// writes the output word of row (k, j), i-block ib.  The y and z words of
// the cube are contiguous rows of 32 i (coalesced) and are transposed
// through shared memory.
__global__ void __launch_bounds__(1024) node_vote(const unsigned *__restrict__ Vx, const unsigned *__restrict__ Vy,
                                                  const unsigned *__restrict__ Vz, int res, int W, unsigned *out) {
    __shared__ unsigned sy[32][33];  // [kk][ii]: y-image word jb of ray (k, i)
    __shared__ unsigned sz[32][33];  // [jj][ii]: z-image word kb of ray (i, j)
    const int ib = blockIdx.x, jb = blockIdx.y, kb = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    {
        const long long plane = (long long)res * res;
        const int k = kb * 32 + ty, i = ib * 32 + tx, j = jb * 32 + ty;
        sy[ty][tx] = (k < res && i < res) ? Vy[jb * plane + (long long)k * res + i] : 0u;
        sz[ty][tx] = (j < res && i < res) ? Vz[kb * plane + (long long)j * res + i] : 0u;
    }
    __syncthreads();
    const int kk = ty, jj = tx;  // thread = output row (k, j)
    const int k = kb * 32 + kk, j = jb * 32 + jj;
    if (k >= res || j >= res) return;
    const long long idx = ((long long)k * res + j) * W + ib;
    const unsigned x = Vx[idx];
    unsigned y = 0, z = 0;
#pragma unroll
    for (int ii = 0; ii < 32; ++ii) {
        y |= ((sy[kk][ii] >> jj) & 1u) << ii;
        z |= ((sz[jj][ii] >> kk) & 1u) << ii;
    }
    out[idx] = (x & y) | (z & (x | y));  // at least two of three
}

bool image_ok(const ldni_layers_t &L) {
    return L.offsets && L.capacity >= 0 && (L.capacity == 0 || L.depth);
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_classify_nodes_workspace_size(int32_t res, size_t *bytes) {
    if (!bytes || res < 1 || res > 4096) return LDNI_EINVAL;
    const size_t W = ((size_t)res + 31) / 32;
    *bytes = align_up(3 * sizeof(unsigned) * (size_t)res * res * W + 2 * kAlign);
    return LDNI_OK;
}

extern "C" int ldni_classify_nodes(const ldni_layers_t *L, const ldni_grid_t *grid, uint32_t *inside,
                                   ldni_info_t *info, void *ws, size_t ws_bytes, void *stream) {
    if (!L || !grid_valid(grid) || !inside || !info || !ws) return LDNI_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!image_ok(L[a])) return LDNI_EINVAL;
    const int res = grid->res;
    size_t need = 0;
    int rc = ldni_classify_nodes_workspace_size(res, &need);
    if (rc != LDNI_OK) return rc;
    if (ws_bytes < need) return LDNI_EWORKSPACE;
    const int W = (res + 31) / 32;
    const size_t vol = (size_t)res * res * W;
    Carver c(ws, ws_bytes);
    unsigned *V[3];
    for (int a = 0; a < 3; ++a) V[a] = c.take<unsigned>(vol);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float hh = (float)grid->width / (float)res;  // FP32 division, as the node positions are defined
    const long long nrays = (long long)res * res;
    LDNI_LAUNCH(K_NODES, s,
                node_rays_x<<<(unsigned)((nrays + kRayWarps - 1) / kRayWarps), kRayWarps * 32, 0, s>>>(
                    L[0].offsets, L[0].depth, L[0].capacity, res, W, grid->origin[0], hh, V[0], info));
    for (int a = 1; a < 3; ++a)
        LDNI_LAUNCH(K_NODES, s,
                    node_rays_yz<<<(unsigned)((nrays + 255) / 256), 256, 0, s>>>(
                        L[a].offsets, L[a].depth, L[a].capacity, res, W, grid->origin[a], hh, a == 1, V[a], info));
    const int nb = (res + 31) / 32;
    LDNI_LAUNCH(K_NODES, s, node_vote<<<dim3(W, nb, nb), 1024, 0, s>>>(V[0], V[1], V[2], res, W, inside));
    return cuda_status();
}
