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
// A ray kernel writes one bit volume per image, the bits of a word running
// along that image's rays, laid out so that the stores are coalesced; a vote
// kernel then takes 32 x 32 x 32 node cubes, transposes the y and z bits
// with warp shuffles and writes the majority in the x-fastest output layout.
#include "ldni_host.h"

namespace ldni {
namespace {


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

// Node t of a ray is inside iff an odd number of the ray's depths lie below
// c(t), i.e. iff an odd number of the boundaries b_m = first_above(d_m) are
// <= t.  So the ray's bits are the XOR of one step per sample: the bits
// t >= b_m.  step_word gives the bits of word w (nodes 32 w .. 32 w + 31) of
// one step; bits of nodes t >= res are cleared by live_bits.
__device__ __forceinline__ unsigned step_word(int b, int w) {
    const int t0 = 32 * w;
    if (b <= t0) return 0xffffffffu;
    if (b >= t0 + 32) return 0u;
    return 0xffffffffu << (b - t0);
}

__device__ __forceinline__ unsigned live_bits(int w, int res) {
    const int left = res - 32 * w;
    return left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
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

// One thread per ray of image a, consecutive threads = consecutive rays of
// one node row, so that every word store is coalesced: word w of the ray
// holds its nodes 32 w .. 32 w + 31 and sits at V[w res^2 + q], with
//   x-image ray p = k res + j:  q = k res + j (nodes i)
//   y-image ray p = i res + k:  q = k res + i (nodes j)
//   z-image ray p = j res + i:  q = j res + i (nodes k)
// The thread walks its ray's boundaries once, in order, while it writes the
// words.
__global__ void __launch_bounds__(256) node_rays(const int *__restrict__ off, const float *__restrict__ depth,
                                                 long long cap, int res, int W, float o, float h, int axis,
                                                 unsigned *V, ldni_info_t *info) {
    const long long q = blockIdx.x * 256LL + threadIdx.x;
    if (q >= (long long)res * res) return;
    const long long p = axis == 1 ? (q % res) * res + q / res : q;
    long long b, e;
    ray_range(off, cap, p, b, e, info, true);
    const long long plane = (long long)res * res;
    const int n = (int)(e - b);
    int m = 0;
    int bm = n > 0 ? first_above(depth[b], res, o, h) : res;
    unsigned after = 0;  // all ones once an odd number of boundaries lie before the current word
    for (int w = 0; w < W; ++w) {
        unsigned word = after;
        while (m < n && bm < 32 * w + 32) {  // boundaries that reach into this word
            word ^= step_word(bm, w);
            after = ~after;
            if (++m < n) bm = first_above(depth[b + m], res, o, h);
        }
        V[w * plane + q] = word & live_bits(w, res);
    }
}

// Transpose of the 32 x 32 bit matrix held by a warp, one row per lane (bit c
// of lane r = element (r, c)): afterwards lane r holds column r.  Five
// stages swap the off-diagonal blocks of width 16, 8, 4, 2, 1 between lanes
// r and r ^ j.
__device__ __forceinline__ unsigned warp_transpose32(unsigned x, int lane) {
    const unsigned lows[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int j = 16 >> s;
        const unsigned low = lows[s];
        const unsigned other = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~low) | ((other & ~low) >> j)) : ((x & low) | ((other & low) << j));
    }
    return x;
}

// One block per kVoteCubes cubes of 32 (i) x 32 (j) x 32 (k) nodes along i;
// warp w and lane l produce the output words of row (k = 32 kb + w,
// j = 32 jb + l) for i-words ib0 .. ib0 + kVoteCubes - 1 and store them
// together (one 32-byte sector per lane).  For each cube ib:
//   x: word ib of x-ray (k, j) as stored;
//   y: warp w loads word jb of the y-rays (k, i = 32 ib + l) and transposes:
//      lane l then holds the bits over i of row (k, j = 32 jb + l);
//   z: warp w loads word kb of the z-rays (j = 32 jb + w, i = 32 ib + l) and
//      transposes: lane l holds the bits over i of row (k = 32 kb + l,
//      j = 32 jb + w), which reach their row's warp through shared memory.
constexpr int kVoteCubes = 8;

__global__ void __launch_bounds__(1024, 2) node_vote(const unsigned *__restrict__ Vx, const unsigned *__restrict__ Vy,
                                                  const unsigned *__restrict__ Vz, int res, int W, unsigned *out) {
    __shared__ unsigned zt[2][32][33];  // [cube parity][k in cube][j in cube]
    const int ib0 = blockIdx.x * kVoteCubes, jb = blockIdx.y, kb = blockIdx.z;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long plane = (long long)res * res;
    const int k = kb * 32 + w, j = jb * 32 + lane, jz = jb * 32 + w;
    unsigned word[kVoteCubes];
#pragma unroll
    for (int c = 0; c < kVoteCubes; ++c) {
        const int ib = ib0 + c;
        const int i = ib * 32 + lane;
        const bool live = ib < W && i < res;
        const unsigned zw = (live && jz < res) ? Vz[kb * plane + (long long)jz * res + i] : 0u;
        const unsigned yw = (live && k < res) ? Vy[jb * plane + (long long)k * res + i] : 0u;
        const unsigned x = (ib < W && k < res && j < res) ? Vx[ib * plane + (long long)k * res + j] : 0u;
        zt[c & 1][lane][w] = warp_transpose32(zw, lane);  // row (k = 32 kb + lane, j = 32 jb + w)
        const unsigned y = warp_transpose32(yw, lane);     // row (k, j)
        __syncthreads();  // zt[c & 1] complete; the read of zt[c & 1] two cubes back is done
        const unsigned z = zt[c & 1][w][lane];
        word[c] = (x & y) | (z & (x | y));  // at least two of three
    }
    if (k >= res || j >= res) return;
    unsigned *row = out + ((long long)k * res + j) * W;
    if ((W & 3) == 0 && ib0 + kVoteCubes <= W && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {  // aligned runs
#pragma unroll
        for (int c = 0; c < kVoteCubes; c += 4)
            *reinterpret_cast<uint4 *>(row + ib0 + c) = make_uint4(word[c], word[c + 1], word[c + 2], word[c + 3]);
    } else {
#pragma unroll
        for (int c = 0; c < kVoteCubes; ++c)
            if (ib0 + c < W) row[ib0 + c] = word[c];
    }
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
    for (int a = 0; a < 3; ++a)
        LDNI_LAUNCH(K_NODES, s,
                    node_rays<<<(unsigned)((nrays + 255) / 256), 256, 0, s>>>(
                        L[a].offsets, L[a].depth, L[a].capacity, res, W, grid->origin[a], hh, a, V[a], info));
    const int nb = (res + 31) / 32;
    LDNI_LAUNCH(K_NODES, s,
                node_vote<<<dim3((W + kVoteCubes - 1) / kVoteCubes, nb, nb), 1024, 0, s>>>(V[0], V[1], V[2], res, W,
                                                                                         inside));
    return cuda_status();
}
