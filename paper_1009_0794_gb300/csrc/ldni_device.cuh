// Device-side building blocks shared by the LDNI kernels: the grid, the
// fixed-point snap and the face normal.  (The exact crossing test itself is
// in sample_common.cuh.)
//
// A ray of image a passes through the centre of pixel (i, j); in fixed point
// (8 subpixel bits) that centre is (256 i + 128, 256 j + 128).  A triangle's
// vertices are snapped to the same lattice, so "does the ray cross the
// triangle" becomes an exact integer question (Definition 1; the pixel-centre
// convention of Section 3).  The top-left rule (an edge d owns the lattice
// points on it iff d_v > 0, or d_v == 0 and d_u < 0) gives a shared
// non-silhouette edge to exactly one of its two faces and a silhouette edge
// to both or neither, which is Remark 1's one / zero-or-two crossing rule and
// makes every ray of a closed mesh even (Definition 4).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ldni.h"

namespace ldni {

constexpr int kSubpix = 256;      // 2^LDNI_SUBPIX_BITS
constexpr int kHalfSubpix = 128;
constexpr float kSnapLimit = 16777216.0f;  // |q| < 2^24 keeps edge products in int64

struct GridDev {
    float o[3];  // cube origin
    float s;     // fixed-point units per world unit: fl32(res * 256 / W)
    int res;
};

// q = round-half-even(fl32(fl32(x - o) * s)); false if out of the snappable range.
__device__ __forceinline__ bool snap(float x, float o, float s, int &q) {
    const float y = __fmul_rn(__fsub_rn(x, o), s);
    if (!(y > -kSnapLimit && y < kSnapLimit)) return false;
    q = __float2int_rn(y);
    return true;
}

// unit face normal from the stored winding (accurate normal sampling, Section 3 item 2)
__device__ __forceinline__ void face_normal(const float3 &p0, const float3 &p1, const float3 &p2, float &nx,
                                            float &ny, float &nz) {
    const float ex = p1.x - p0.x, ey = p1.y - p0.y, ez = p1.z - p0.z;
    const float fx = p2.x - p0.x, fy = p2.y - p0.y, fz = p2.z - p0.z;
    nx = ey * fz - ez * fy;
    ny = ez * fx - ex * fz;
    nz = ex * fy - ey * fx;
    const float len2 = nx * nx + ny * ny + nz * nz;
    if (len2 > 0.0f) {
        const float r = rsqrtf(len2);  // a few ulp; the normal tolerance is 1e-5
        nx *= r;
        ny *= r;
        nz *= r;
    }
}

// Packed approximate normal (Section 3 item 1): three 8-bit codes
// q = rint(fl32(fl32(n + 1) * 127.5)), half to even, clamped to [0, 255].
__device__ __forceinline__ unsigned normal_code8(float n) {
    const float v = __fmul_rn(__fadd_rn(n, 1.0f), 127.5f);
    return v >= 255.0f ? 255u : (v > 0.0f ? (unsigned)__float2int_rn(v) : 0u);
}
__device__ __forceinline__ unsigned encode_normal8(float x, float y, float z) {
    return normal_code8(x) | (normal_code8(y) << 8) | (normal_code8(z) << 16);
}
constexpr unsigned kInvert8 = 0x00FFFFFFu;  // q -> 255 - q in every code (an inverted normal)

__device__ __forceinline__ float comp(const float3 &p, int k) { return k == 0 ? p.x : (k == 1 ? p.y : p.z); }

__device__ __forceinline__ void set_status(ldni_info_t *info, unsigned bits) {
    if (info) atomicOr(&info->status, bits);
}

// Checked builds (-DLDNI_CHECKS, a debugging aid in place of a memory
// checker): every CSR and slab range a kernel is about to touch is tested
// against its array; a range outside it is reported as LDNI_ST_BOUNDS and
// the access skipped, so the kernel neither faults nor traps.  Release builds
// compile the test away (the ranges are then guaranteed by construction).
#ifdef LDNI_CHECKS
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
// [i0, i1) within [0, n)
__device__ __forceinline__ bool range_ok(long long i0, long long i1, long long n, ldni_info_t *info) {
    if (!kChecked || (0 <= i0 && i0 <= i1 && i1 <= n)) return true;
    set_status(info, LDNI_ST_BOUNDS);
    return false;
}

}  // namespace ldni
