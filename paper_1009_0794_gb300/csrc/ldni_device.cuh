// Device-side building blocks shared by the LDNI kernels: the fixed-point
// snap, the projected-triangle setup and the exact top-left crossing test.
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

__device__ __forceinline__ int floor_div256(int x) { return x >> 8; }  // arithmetic shift = floor

// Projection of one triangle onto image `axis`, turned counter-clockwise.
struct ProjTri {
    int u0, v0, u1, v1, u2, v2;  // snapped in-plane vertices, CCW
    float a0, a1, a2;            // matching world a-coordinates
    long long area2;             // twice the signed area, > 0
    int i0, i1, j0, j1;          // pixel-centre bounding box, clamped to the image
};

// Build the CCW projection; false when the projection has zero area (the face
// is parallel to the ray, Definition 1 note) or covers no pixel centre.
__device__ __forceinline__ bool project_tri(const int (&qu)[3], const int (&qv)[3], const float (&a)[3], int res,
                                            ProjTri &P) {
    long long A2 = (long long)(qu[1] - qu[0]) * (qv[2] - qv[0]) - (long long)(qv[1] - qv[0]) * (qu[2] - qu[0]);
    if (A2 == 0) return false;
    P.u0 = qu[0];
    P.v0 = qv[0];
    P.a0 = a[0];
    if (A2 > 0) {
        P.u1 = qu[1]; P.v1 = qv[1]; P.a1 = a[1];
        P.u2 = qu[2]; P.v2 = qv[2]; P.a2 = a[2];
    } else {
        P.u1 = qu[2]; P.v1 = qv[2]; P.a1 = a[2];
        P.u2 = qu[1]; P.v2 = qv[1]; P.a2 = a[1];
        A2 = -A2;
    }
    P.area2 = A2;
    const int umin = min(P.u0, min(P.u1, P.u2)), umax = max(P.u0, max(P.u1, P.u2));
    const int vmin = min(P.v0, min(P.v1, P.v2)), vmax = max(P.v0, max(P.v1, P.v2));
    // smallest i with 256 i + 128 >= umin, largest with 256 i + 128 <= umax
    P.i0 = max(0, -floor_div256(kHalfSubpix - umin));
    P.i1 = min(res - 1, floor_div256(umax - kHalfSubpix));
    P.j0 = max(0, -floor_div256(kHalfSubpix - vmin));
    P.j1 = min(res - 1, floor_div256(vmax - kHalfSubpix));
    return P.i0 <= P.i1 && P.j0 <= P.j1;
}

__device__ __forceinline__ long long owns_bias(int du, int dv) {
    // 1 when the edge owns its zero set (top-left rule), else 0
    return (dv > 0 || (dv == 0 && du < 0)) ? 1 : 0;
}

// Edge functions E_k at the lattice point (cu, cv) for the CCW triangle:
// E_k = d_k x (c - P_k), d_k = P_{k+1} - P_k.  E_k is twice the area of the
// sub-triangle opposite vertex k+2, so lambda_{k+2} = E_k / area2.
struct EdgeEval {
    long long e0, e1, e2;
};

__device__ __forceinline__ EdgeEval edges_at(const ProjTri &P, int cu, int cv) {
    EdgeEval E;
    E.e0 = (long long)(P.u1 - P.u0) * (cv - P.v0) - (long long)(P.v1 - P.v0) * (cu - P.u0);
    E.e1 = (long long)(P.u2 - P.u1) * (cv - P.v1) - (long long)(P.v2 - P.v1) * (cu - P.u1);
    E.e2 = (long long)(P.u0 - P.u2) * (cv - P.v2) - (long long)(P.v0 - P.v2) * (cu - P.u2);
    return E;
}

struct EdgeBias {
    long long b0, b1, b2;
};

__device__ __forceinline__ EdgeBias edge_bias(const ProjTri &P) {
    EdgeBias B;
    B.b0 = owns_bias(P.u1 - P.u0, P.v1 - P.v0);
    B.b1 = owns_bias(P.u2 - P.u1, P.v2 - P.v1);
    B.b2 = owns_bias(P.u0 - P.u2, P.v0 - P.v2);
    return B;
}

// inside iff every E_k > 0, or E_k == 0 on an owned edge
__device__ __forceinline__ bool inside(const EdgeEval &E, const EdgeBias &B) {
    return (E.e0 + B.b0 > 0) && (E.e1 + B.b1 > 0) && (E.e2 + B.b2 > 0);
}

// depth = sum_k lambda_k a_k, FP32 from the exact integer weights
__device__ __forceinline__ float crossing_depth(const ProjTri &P, const EdgeEval &E) {
    const float inv = 1.0f / (float)P.area2;
    const float l0 = (float)E.e1 * inv;  // weight of vertex 0
    const float l1 = (float)E.e2 * inv;  // weight of vertex 1
    const float l2 = (float)E.e0 * inv;  // weight of vertex 2
    return l0 * P.a0 + l1 * P.a1 + l2 * P.a2;
}

// unit face normal from the stored winding (accurate normal sampling, Section 3 item 2)
__device__ __forceinline__ void face_normal(const float3 &p0, const float3 &p1, const float3 &p2, float &nx,
                                            float &ny, float &nz) {
    const float ex = p1.x - p0.x, ey = p1.y - p0.y, ez = p1.z - p0.z;
    const float fx = p2.x - p0.x, fy = p2.y - p0.y, fz = p2.z - p0.z;
    nx = ey * fz - ez * fy;
    ny = ez * fx - ex * fz;
    nz = ex * fy - ey * fx;
    const float len = sqrtf(nx * nx + ny * ny + nz * nz);
    if (len > 0.0f) {
        nx = nx / len;
        ny = ny / len;
        nz = nz / len;
    }
}

__device__ __forceinline__ float comp(const float3 &p, int k) { return k == 0 ? p.x : (k == 1 ? p.y : p.z); }

__device__ __forceinline__ void set_status(ldni_info_t *info, unsigned bits) {
    if (info) atomicOr(&info->status, bits);
}

}  // namespace ldni
