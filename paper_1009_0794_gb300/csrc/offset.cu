// Offsetting by sphere unions (Section 4.2): the solid H united with (inner
// offset: minus) one sphere of radius r about every sample of its three
// LDNIs, each sphere given by its own LDNIs on H's grid.
//
// The paper applies one Boolean per sphere.  Here every ray is answered once:
// the ray's samples of H and of every sphere that meets it are ordered by
// depth and swept in one pass.  The result is the one the step-by-step
// Booleans give (without small-interval removal, which follows once):
//  - the solid is {t : H(t) or some sphere holds t} (inner: H(t) and no
//    sphere), by associativity of the set operations;
//  - where it changes state at depth d, the step-by-step Booleans keep the
//    sample of the first source in the order H, sphere 0, sphere 1, ... whose
//    own state changes at d (each Boolean keeps the accumulated solid's
//    sample at a tie), so the sweep takes that one.
//
// A sample of image a at pixel (i, j) with depth d sits at the point with
// a-coordinate d and in-plane coordinates c_u(i), c_v(j),
// c(t) = fl32(o + fl32((t + 1/2) h)), h = fl32(W / res); spheres are numbered
// in sample order (image x, y, z, each in CSR order).  The sphere about C
// meets the ray through (P_u, P_v) of image b iff q < fl32(r r) with
// q = fl32(fl32(du du) + fl32(dv dv)), du = fl32(P_u - C_u), dv likewise; its
// samples are fl32(C_b -+ t), t = sqrt(fl32(r r - q)) rounded, with outward
// normals (du / r, dv / r, -+t / r), each operation rounded to nearest.
//
// Stages: sphere centres; per image, sphere lists of 8 x 8-pixel tiles
// (count, scan, fill); per ray (a warp each) a count pass, the scan of the
// counts into the output offsets, and the write pass.  A ray merges its
// spheres 64 at a time into the solid accumulated so far; since the first
// changing source wins at every depth, merging in batches gives the result of
// merging all at once.
#include <algorithm>
#include <climits>
#include <cmath>

#include "ldni_host.h"
#include "sample_common.cuh"

namespace ldni {
namespace {

constexpr int kOffWarps = 4;      // rays per block, a warp each
constexpr int kOffEvents = 512;   // samples one ray can order: H's plus two per sphere
constexpr int kTile = 8;          // pixels per side of a sphere-list tile
constexpr int kThreads = 256;

struct OffArgs {
    // H
    const int *hoff[3];
    const float *hd[3], *hx[3], *hy[3], *hz[3];
    const int *ht[3];
    long long base[3];  // first sphere of each image
    long long n[3];     // samples of each image
    long long S;        // spheres
    // grid
    float o[3];
    float h;
    int res;
    float r, r2, eps;
    int inner;
    // sphere centres and tile lists
    float4 *C;
    int *tcnt[3];   // per tile: spheres binned (count pass), then the fill cursor
    int *toff[3];   // tile list offsets [ntiles + 1]
    int *tlist[3];  // sphere indices
    int ntx;        // tiles per side
    // output
    int *cnt[3];    // per-ray output counts
    int *ooff[3];
    float *od[3], *ox[3], *oy[3], *oz[3];
    int *ot[3];
    long long ocap[3];
};

__device__ __forceinline__ float pix(long long t, float o, float h) {
    return __fadd_rn(o, __fmul_rn((float)t + 0.5f, h));
}

__device__ __forceinline__ float c4(const float4 &c, int k) { return k == 0 ? c.x : (k == 1 ? c.y : c.z); }

template <class T>
__device__ __forceinline__ T pick(T const (&arr)[3], int a) {
    return a == 0 ? arr[0] : (a == 1 ? arr[1] : arr[2]);
}

// the sphere about c on the ray (pu, pv) of image b
__device__ __forceinline__ bool sphere_hit(const float4 &c, int b, float pu, float pv, float r2, float &e, float &x,
                                           float &t, float &du, float &dv) {
    du = __fsub_rn(pu, c4(c, b == 2 ? 0 : b + 1));
    dv = __fsub_rn(pv, c4(c, b == 0 ? 2 : b - 1));
    const float q = __fadd_rn(__fmul_rn(du, du), __fmul_rn(dv, dv));
    if (!(q < r2)) return false;
    t = __fsqrt_rn(__fsub_rn(r2, q));
    e = __fsub_rn(c4(c, b), t);
    x = __fadd_rn(c4(c, b), t);
    return true;
}

// sphere centres in sample order: a thread per ray of image blockIdx.y
__global__ void __launch_bounds__(kThreads) off_centres(OffArgs A) {
    const int a = blockIdx.y;
    const long long N = (long long)A.res * A.res;
    const long long p = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (p >= N) return;
    const int *off = pick(A.hoff, a);
    const float *D = pick(A.hd, a);
    const int iu = a == 2 ? 0 : a + 1, iv = a == 0 ? 2 : a - 1;
    const float cu = pix(p % A.res, A.o[iu], A.h), cv = pix(p / A.res, A.o[iv], A.h);
    const long long b0 = pick(A.base, a), na = pick(A.n, a);
    for (long long k = max(off[p], 0); k < min((long long)off[p + 1], na); ++k) {
        float v[3];
        v[a] = D[k];
        v[iu] = cu;
        v[iv] = cv;
        A.C[b0 + k] = make_float4(v[0], v[1], v[2], 0.0f);
    }
}

// Sphere s into the lists of the tiles of image blockIdx.y that its shadow
// (widened by a pixel) touches: count (kFill = false) or fill.
template <bool kFill>
__global__ void __launch_bounds__(kThreads) off_bin(OffArgs A) {
    const int b = blockIdx.y;
    const long long s = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (s >= A.S) return;
    const float4 c = A.C[s];
    const int bu = b == 2 ? 0 : b + 1, bv = b == 0 ? 2 : b - 1;
    const double hh = A.h;
    const double lo_u = ((double)c4(c, bu) - A.r - A.o[bu]) / hh - 0.5, hi_u = ((double)c4(c, bu) + A.r - A.o[bu]) / hh - 0.5;
    const double lo_v = ((double)c4(c, bv) - A.r - A.o[bv]) / hh - 0.5, hi_v = ((double)c4(c, bv) + A.r - A.o[bv]) / hh - 0.5;
    if (!(isfinite(lo_u) && isfinite(hi_u) && isfinite(lo_v) && isfinite(hi_v))) return;  // a sample at infinity
    const double last = A.res - 1;
    const double i0 = fmax(floor(lo_u) - 1.0, 0.0), i1 = fmin(ceil(hi_u) + 1.0, last);
    const double j0 = fmax(floor(lo_v) - 1.0, 0.0), j1 = fmin(ceil(hi_v) + 1.0, last);
    if (!(i0 <= i1 && j0 <= j1)) return;  // the shadow misses the image (or a coordinate is NaN)
    int *tc = pick(A.tcnt, b);
    const int ti0 = (int)i0 / kTile, ti1 = (int)i1 / kTile, tj0 = (int)j0 / kTile, tj1 = (int)j1 / kTile;
    for (int tj = tj0; tj <= tj1; ++tj)
        for (int ti = ti0; ti <= ti1; ++ti) {
            const int tile = tj * A.ntx + ti;
            if (!kFill) {
                atomicAdd(tc + tile, 1);
            } else {
                const int slot = pick(A.toff, b)[tile] + atomicAdd(tc + tile, 1);
                pick(A.tlist, b)[slot] = (int)s;
            }
        }
}

__device__ __forceinline__ unsigned long long ev_key(float d, unsigned low) {
    unsigned u = __float_as_uint(__fadd_rn(d, 0.0f));
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | low;
}

// Low word of an event: kNew marks a sample of a sphere being merged (else a
// boundary of the solid accumulated so far); kSph marks a sphere's sample
// (payload 2 s + 0 entering / 1 leaving), else H's sample (payload: its index
// in the ray).  Ordered by depth, then accumulated boundaries before new
// samples, H before spheres, spheres by index.
constexpr unsigned kNew = 0x80000000u, kSph = 0x40000000u, kPay = 0x3fffffffu;
constexpr unsigned kNone = 0xffffffffu;

__device__ __forceinline__ bool first_wins(unsigned a, unsigned b) {  // a before b in the order H, sphere 0, 1, ...
    if (!(a & kSph)) return true;
    if (!(b & kSph)) return false;
    return ((a & kPay) >> 1) < ((b & kPay) >> 1);
}

// Merges the sorted events ev[0, n) of the accumulated solid and of new
// spheres into the accumulated solid's boundaries ev[0, returned): a sweep
// from below every sample, where the accumulated state flips at each of its
// boundaries (parity) and each new sphere adds one cover between its two
// samples.  Where the combined state changes, the boundary takes the source
// that comes first among those whose own state changes there.  One lane.
__device__ int sweep_merge(unsigned long long *ev, int n, int inner) {
    int ain = 0, cover = 0, w = 0;
    for (int k = 0; k < n;) {
        const unsigned hi32 = (unsigned)(ev[k] >> 32);
        int acnt = 0, delta = 0;
        unsigned atag = kNone, btag = kNone;
        while (k < n && (unsigned)(ev[k] >> 32) == hi32) {
            const unsigned low = (unsigned)ev[k];
            if (!(low & kNew)) {
                if (acnt++ == 0) atag = low;
                ++k;
            } else {
                delta += (low & 1u) ? -1 : 1;
                if (btag == kNone) btag = low;
                ++k;
            }
        }
        const int before = inner ? (ain && cover == 0) : (ain || cover > 0);
        ain ^= acnt & 1;
        cover += delta;
        const int after = inner ? (ain && cover == 0) : (ain || cover > 0);
        if (before == after) continue;
        // a new sphere whose two samples share this depth was not kept, so a
        // new sample here always changes its sphere's state
        unsigned tag;
        if ((acnt & 1) && btag != kNone)
            tag = first_wins(atag, btag) ? atag : btag;
        else
            tag = (acnt & 1) ? atag : btag;
        ev[w++] = ((unsigned long long)hi32 << 32) | (tag & ~kNew);
    }
    return w;
}

// One warp per ray p of image blockIdx.y.  The accumulated solid starts as
// H's samples; the spheres that meet the ray and can change the result are
// gathered, kBatch samples at a time, and merged into it.
constexpr int kBatch = 128;  // new sphere samples per merge

template <bool kWrite>
__global__ void __launch_bounds__(kOffWarps * 32) off_rays(OffArgs A, ldni_info_t *info) {
    __shared__ unsigned long long sev[kOffWarps][kOffEvents];
    __shared__ unsigned long long snew[kOffWarps][kBatch];
    const int b = blockIdx.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long N = (long long)A.res * A.res;
    const long long p = (long long)blockIdx.x * kOffWarps + w;
    if (p >= N) return;  // the same for the whole warp
    unsigned long long *ev = sev[w], *nev = snew[w];
    const int *hoff = pick(A.hoff, b);
    const float *HD = pick(A.hd, b);
    long long hb = hoff[p], he = hoff[p + 1];
    if (hb < 0 || he < hb || he > pick(A.n, b)) {  // offsets that do not fit the stated sample count
        if (lane == 0) set_status(info, LDNI_ST_CAPACITY);
        hb = he = 0;
    }
    const int nh = (int)(he - hb);
    if ((nh & 1) && lane == 0 && !kWrite) {
        atomicAdd(&info->odd_rays, 1u);
        set_status(info, LDNI_ST_ODD);
    }
    bool over = nh > kOffEvents - kBatch;
    int na = over ? 0 : nh, nn = 0;
    for (int k = lane; k < na; k += 32) ev[k] = ev_key(HD[hb + k], (unsigned)k);
    const int bu = b == 2 ? 0 : b + 1, bv = b == 0 ? 2 : b - 1;
    const int i = (int)(p % A.res), j = (int)(p / A.res);
    const float pu = pix(i, A.o[bu], A.h), pv = pix(j, A.o[bv], A.h);
    const int tile = (j / kTile) * A.ntx + i / kTile;
    const int l0 = pick(A.toff, b)[tile], l1 = pick(A.toff, b)[tile + 1];
    const int *lst = pick(A.tlist, b);
    // merge the gathered samples into the accumulated solid (whole warp)
    bool merged = false, met = false;
    auto merge = [&]() {
        merged = true;
        __syncwarp();
        if (na + nn > kOffEvents) {
            over = true;
            return;
        }
        for (int k = lane; k < nn; k += 32) ev[na + k] = nev[k];
        int np2 = 1;
        while (np2 < na + nn) np2 <<= 1;
        for (int k = na + nn + lane; k < np2; k += 32) ev[k] = ~0ull;
        __syncwarp();
        for (int size = 2; size <= np2; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = lane; t < (np2 >> 1); t += 32) {
                    const int lo = 2 * stride * (t / stride) + (t % stride), hi = lo + stride;
                    const unsigned long long u = ev[lo], v = ev[hi];
                    if ((u > v) == ((lo & size) == 0)) {
                        ev[lo] = v;
                        ev[hi] = u;
                    }
                }
                __syncwarp();
            }
        int m = 0;
        if (lane == 0) m = sweep_merge(ev, na + nn, A.inner);
        na = __shfl_sync(0xffffffffu, m, 0);
        nn = 0;
        __syncwarp();
    };
    for (int base = l0; base < l1 && !over; base += 32) {
        const int idx = base + lane;
        bool keep = false;
        float e = 0.0f, x = 0.0f;
        int s = 0;
        if (idx < l1) {
            s = lst[idx];
            float t, du, dv;
            keep = sphere_hit(A.C[s], b, pu, pv, A.r2, e, x, t, du, dv);
            met = met || keep;
            keep = keep && e < x;  // e == x: no change of state
            // a sphere's samples strictly inside one of H's solid intervals
            // (inner offset: one of its gaps) change nothing
            for (int k = 0; keep && k <= nh; k += 2) {
                const float lo = A.inner ? (k == 0 ? -INFINITY : HD[hb + k - 1]) : (k < nh ? HD[hb + k] : INFINITY);
                const float hi = A.inner ? (k < nh ? HD[hb + k] : INFINITY) : (k + 1 < nh ? HD[hb + k + 1] : -INFINITY);
                if (e > lo && x < hi) keep = false;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (nn + 2 * __popc(m) > kBatch) merge();
        if (over) break;
        const int at = nn + 2 * __popc(m & ((1u << lane) - 1u));
        if (keep) {
            nev[at] = ev_key(e, kNew | kSph | ((unsigned)s << 1));
            nev[at + 1] = ev_key(x, kNew | kSph | ((unsigned)s << 1) | 1u);
        }
        nn += 2 * __popc(m);
    }
    // A sphere met the ray: the step-by-step Booleans then also merge H's
    // touching intervals and drop its empty ones, so the ray is swept even
    // when every sphere was set aside.
    met = __any_sync(0xffffffffu, met);
    if (!over && (nn > 0 || (met && !merged))) merge();
    if (over) {  // more than one warp orders: leave the ray empty and say so
        if (lane == 0) {
            set_status(info, LDNI_ST_EVENTS);
            if (!kWrite) pick(A.cnt, b)[p] = 0;
        }
        return;
    }
    __syncwarp();
    if (lane != 0) return;
    // the accumulated boundaries alternate entering / leaving; small-interval
    // removal, then the samples
    const long long oslot = kWrite ? (long long)pick(A.ooff, b)[p] : 0;
    const long long cap = pick(A.ocap, b);
    int nout = 0;
    for (int q = 0; q + 1 < na; q += 2) {
        float dd[2], nb3[2], nu3[2], nv3[2];
        int id[2];
        for (int z = 0; z < 2; ++z) {
            const unsigned low = (unsigned)ev[q + z];
            if (!(low & kSph)) {
                const long long k2 = hb + (low & kPay);
                dd[z] = HD[k2];
                if (kWrite) {
                    const float hx = pick(A.hx, b)[k2], hy = pick(A.hy, b)[k2], hz = pick(A.hz, b)[k2];
                    nb3[z] = b == 0 ? hx : (b == 1 ? hy : hz);
                    nu3[z] = bu == 0 ? hx : (bu == 1 ? hy : hz);
                    nv3[z] = bv == 0 ? hx : (bv == 1 ? hy : hz);
                    id[z] = pick(A.ht, b)[k2];
                }
            } else {
                const long long sid = (low & kPay) >> 1;
                float e, x, t, du, dv;
                sphere_hit(A.C[sid], b, pu, pv, A.r2, e, x, t, du, dv);
                const bool leaving = low & 1u;
                dd[z] = leaving ? x : e;
                if (kWrite) {
                    const float na3 = __fdiv_rn(t, A.r);
                    float n0 = leaving ? na3 : -na3, n1 = __fdiv_rn(du, A.r), n2 = __fdiv_rn(dv, A.r);
                    if (A.inner) {  // the spheres are subtracted: inverted normals (Section 4.1)
                        n0 = -n0;
                        n1 = -n1;
                        n2 = -n2;
                    }
                    nb3[z] = n0;
                    nu3[z] = n1;
                    nv3[z] = n2;
                    id[z] = (int)(0x80000000u | (unsigned)sid);
                }
            }
        }
        if (__fsub_rn(dd[1], dd[0]) < A.eps) continue;  // a solid interval thinner than eps
        if (kWrite) {
            for (int z = 0; z < 2; ++z) {
                const long long slot = oslot + nout + z;
                if (slot >= cap) {
                    set_status(info, LDNI_ST_CAPACITY);
                    continue;
                }
                float n3[3];
                n3[b] = nb3[z];
                n3[bu] = nu3[z];
                n3[bv] = nv3[z];
                pick(A.od, b)[slot] = dd[z];
                pick(A.ox, b)[slot] = n3[0];
                pick(A.oy, b)[slot] = n3[1];
                pick(A.oz, b)[slot] = n3[2];
                pick(A.ot, b)[slot] = id[z];
            }
        }
        nout += 2;
    }
    if (!kWrite) pick(A.cnt, b)[p] = nout;
}

struct OffWs {
    float4 *C;
    int *tcnt[3], *toff[3], *tlist[3], *cnt[3];
    long long *partials;
    ldni_info_t *tinfo;
    size_t clear_bytes;  // tile counts and tinfo: one memset from tcnt[0]
};

long long tiles_per_sphere(double r_pixels) {
    const double span = std::ceil(2.0 * r_pixels) + 6.0;  // pixel centres a widened shadow can hold, and one more
    const long long per_side = (long long)std::ceil(span / kTile) + 1;
    return per_side * per_side;
}

bool carve_offset(Carver &c, long long S, int res, double r_pixels, OffWs &w) {
    const long long N = (long long)res * res;
    const long long ntx = (res + kTile - 1) / kTile, ntiles = ntx * ntx;
    const double pairs = (double)S * (double)tiles_per_sphere(r_pixels);
    if (pairs > (double)INT_MAX) return false;
    const long long tstride = (ntiles + 63) / 64 * 64;
    int *block = c.take<int>((size_t)(3 * tstride) + sizeof(ldni_info_t) / sizeof(int) + 16);
    for (int a = 0; a < 3; ++a) w.tcnt[a] = block ? block + a * tstride : nullptr;
    w.tinfo = block ? reinterpret_cast<ldni_info_t *>(block + 3 * tstride) : nullptr;
    w.clear_bytes = sizeof(int) * ((size_t)(3 * tstride) + sizeof(ldni_info_t) / sizeof(int) + 16);
    w.C = c.take<float4>((size_t)(S > 0 ? S : 1));
    for (int a = 0; a < 3; ++a) {
        w.toff[a] = c.take<int>((size_t)ntiles + 1);
        w.tlist[a] = c.take<int>((size_t)(pairs > 0 ? pairs : 1));
        w.cnt[a] = c.take<int>((size_t)N);
    }
    const size_t parts = std::max(csr_scan_partials(N), csr_scan_partials(ntiles));
    w.partials = c.take<long long>(parts * 3);
    return true;
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_offset_workspace_size(const int64_t *n, int32_t res, float r, float width, size_t *bytes) {
    if (!n || !bytes || res < 1 || res > 8192 || !(r > 0.0f) || !(width > 0.0f)) return LDNI_EINVAL;
    const long long S = (long long)n[0] + n[1] + n[2];
    if (n[0] < 0 || n[1] < 0 || n[2] < 0 || S >= (1ll << 29)) return LDNI_ETOOLARGE;
    Carver c(nullptr, 0);
    OffWs w{};
    const float h = width / (float)res;
    if (!carve_offset(c, S, res, (double)r / (double)h, w)) return LDNI_ETOOLARGE;
    *bytes = align_up(c.off);
    return LDNI_OK;
}

extern "C" int ldni_offset(const ldni_layers_t *H, const int64_t *n, const ldni_grid_t *grid, float r, int32_t inner,
                           float eps, ldni_layers_t *out, ldni_info_t *info, void *ws, size_t ws_bytes,
                           void *stream) {
    if (!H || !n || !grid_valid(grid) || !(r > 0.0f) || !(r < 3.0e38f) || (inner != 0 && inner != 1) || !out ||
        !info || !ws || !(eps >= 0.0f))
        return LDNI_EINVAL;
    const long long S = (long long)n[0] + n[1] + n[2];
    if (n[0] < 0 || n[1] < 0 || n[2] < 0 || S >= (1ll << 29)) return LDNI_ETOOLARGE;
    for (int a = 0; a < 3; ++a) {
        if (!H[a].offsets || (n[a] > 0 && (!H[a].depth || !H[a].nx || !H[a].ny || !H[a].nz || !H[a].tri_id)) ||
            H[a].capacity < n[a] || H[a].nrm8 || out[a].nrm8)  // FP32 normals only
            return LDNI_EINVAL;
        if (!out[a].offsets || out[a].capacity < 0 ||
            (out[a].capacity > 0 && (!out[a].depth || !out[a].nx || !out[a].ny || !out[a].nz || !out[a].tri_id)))
            return LDNI_EINVAL;
    }
    const int res = grid->res;
    const long long N = (long long)res * res;
    const float h = grid->width / (float)res;
    Carver c(ws, ws_bytes);
    OffWs w{};
    if (!carve_offset(c, S, res, (double)r / (double)h, w)) return LDNI_ETOOLARGE;
    if (!c.fits()) return LDNI_EWORKSPACE;
    OffArgs A{};
    long long acc = 0;
    for (int a = 0; a < 3; ++a) {
        A.hoff[a] = H[a].offsets;
        A.hd[a] = H[a].depth;
        A.hx[a] = H[a].nx;
        A.hy[a] = H[a].ny;
        A.hz[a] = H[a].nz;
        A.ht[a] = H[a].tri_id;
        A.base[a] = acc;
        A.n[a] = n[a];
        acc += n[a];
        A.tcnt[a] = w.tcnt[a];
        A.toff[a] = w.toff[a];
        A.tlist[a] = w.tlist[a];
        A.cnt[a] = w.cnt[a];
        A.ooff[a] = out[a].offsets;
        A.od[a] = out[a].depth;
        A.ox[a] = out[a].nx;
        A.oy[a] = out[a].ny;
        A.oz[a] = out[a].nz;
        A.ot[a] = out[a].tri_id;
        A.ocap[a] = out[a].capacity;
        A.o[a] = grid->origin[a];
    }
    A.S = S;
    A.h = h;
    A.res = res;
    A.r = r;
    A.r2 = r * r;
    A.eps = eps;
    A.inner = inner;
    A.C = w.C;
    A.ntx = (res + kTile - 1) / kTile;
    const long long ntiles = (long long)A.ntx * A.ntx;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc_ = cuda_check(cudaMemsetAsync(w.tcnt[0], 0, w.clear_bytes, s))) return rc_;
    const unsigned rblocks = (unsigned)((N + kThreads - 1) / kThreads);
    const unsigned sblocks = (unsigned)((S + kThreads - 1) / kThreads);
    LDNI_LAUNCH(K_OFFSET, s, off_centres<<<dim3(rblocks, 3), kThreads, 0, s>>>(A));
    if (S > 0) LDNI_LAUNCH(K_OFFSET, s, off_bin<false><<<dim3(sblocks, 3), kThreads, 0, s>>>(A));
    int rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    {
        const int *cnts[3] = {w.tcnt[0], w.tcnt[1], w.tcnt[2]};
        int *offs[3] = {w.toff[0], w.toff[1], w.toff[2]};
        rc = csr_scan(cnts, offs, 3, ntiles, w.partials, w.tinfo, 0, s);
        if (rc != LDNI_OK) return rc;
    }
    // the counts become the fill cursors
    if (int rc_ = cuda_check(cudaMemsetAsync(w.tcnt[0], 0, w.clear_bytes, s))) return rc_;
    if (S > 0) LDNI_LAUNCH(K_OFFSET, s, off_bin<true><<<dim3(sblocks, 3), kThreads, 0, s>>>(A));
    const unsigned wblocks = (unsigned)((N + kOffWarps - 1) / kOffWarps);
    LDNI_LAUNCH(K_OFFSET, s, off_rays<false><<<dim3(wblocks, 3), kOffWarps * 32, 0, s>>>(A, info));
    rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    {
        const int *cnts[3] = {w.cnt[0], w.cnt[1], w.cnt[2]};
        int *offs[3] = {out[0].offsets, out[1].offsets, out[2].offsets};
        rc = csr_scan(cnts, offs, 3, N, w.partials, info, 0, s);
        if (rc != LDNI_OK) return rc;
    }
    LDNI_LAUNCH(K_OFFSET, s, off_rays<true><<<dim3(wblocks, 3), kOffWarps * 32, 0, s>>>(A, info));
    return cuda_status();
}
