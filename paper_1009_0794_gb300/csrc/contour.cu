// Contouring, Steps 2 and 3 (Section 5.1): cell edges typed and regularised
// (Rules 1 and 2), the outside corners of every cell flooded through its
// empty edges into clusters, and one vertex per cluster at the minimum of
// the quadratic error function of its Hermite data (dual contouring).
//
// Grid nodes and their signs come from Step 1 (nodes.cu): node t of axis a
// at c_a(t) = fl32(o_a + fl32((t + 1/2) h)).  The edge (t, t + 1) along a
// lies on the ray of image a through its two other node indices and holds
// the ray's samples with c_a(t) <= d < c_a(t + 1), the samples that change
// Step 1's parity count between its end nodes.
//
// Readings the kernels follow (the paper leaves them open):
//  - Rule 1 keeps the first and last samples of a complex edge; Rule 2 keeps,
//    of an intersect edge's samples whose normal's a-component points from
//    the inside end to the outside end, the one nearest the midpoint (the
//    earlier on a tie; all samples compete when none points that way);
//  - a cluster takes the kept sample of each intersect edge at one of its
//    corners and, of a complex edge between outside corners, the sample
//    nearer each corner (a single one goes to the nearer corner); complex
//    edges between inside corners join no cluster;
//  - clusters are numbered by their lowest corner (di + 2 dj + 4 dk); every
//    cluster of a cell that meets an intersect, none-intersect or complex
//    edge yields a vertex;
//  - x = m + (A^T A)^+ (A^T b - A^T A m), m the points' mean, eigenvalues of
//    A^T A below 0.01 of the largest dropped (singular values below 0.1),
//    in FP64 with a cyclic Jacobi eigensolver; a cluster with no Hermite
//    data sits at the mean of its corners with no points.
//
// Stages: active-cell marks (edges with samples, from the samples; edges
// whose end signs differ, word-parallel from the node bits), their
// compaction, one thread per active cell writing its record to a dense
// scratch, and the compaction of the cells that yield a vertex.
#include "ldni_host.h"

namespace ldni {
namespace {

constexpr int kThreads = 256;

struct CImg {
    const int *off[3];
    const float *d[3];
    const float *nx[3], *ny[3], *nz[3];
    long long cap[3];
};

__device__ __forceinline__ float node_c(int t, float o, float h) {
    return __fadd_rn(o, __fmul_rn((float)t + 0.5f, h));
}

// first node t in [0, res] with c(t) > d
__device__ __forceinline__ int first_above(float d, int res, float o, float h) {
    const float est = (d - o) / h - 0.5f;
    int t = !(est > 0.0f) ? 0 : (est >= (float)res ? res : (int)est);
    while (t > 0 && node_c(t - 1, o, h) > d) --t;
    while (t < res && !(node_c(t, o, h) > d)) ++t;
    return t;
}

template <class T>
__device__ __forceinline__ T pick(T const (&arr)[3], int a) {
    return a == 0 ? arr[0] : (a == 1 ? arr[1] : arr[2]);
}

__device__ __forceinline__ void mark(unsigned *act, int n, int Wc, int i, int j, int k) {
    if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return;
    atomicOr(act + ((long long)k * n + j) * Wc + (i >> 5), 1u << (i & 31));
}

// Cells around every edge that holds a sample: a thread per ray of image
// blockIdx.y.
__global__ void __launch_bounds__(kThreads) mark_samples(CImg I, int res, float o0, float o1, float o2, float h,
                                                         unsigned *act, int Wc) {
    const int a = blockIdx.y;
    const long long p = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (p >= (long long)res * res) return;
    const int n = res - 1;
    const int *off = pick(I.off, a);
    const float *D = pick(I.d, a);
    const long long cap = pick(I.cap, a);
    const float oa = a == 0 ? o0 : (a == 1 ? o1 : o2);
    const int iu = (int)(p % res), iv = (int)(p / res);
    const long long e = min((long long)off[p + 1], cap);
    for (long long s = off[p]; s < e; ++s) {
        const int t = first_above(D[s], res, oa, h) - 1;  // c(t) <= d < c(t + 1)
        if (t < 0 || t >= n) continue;
        for (int du = 0; du < 2; ++du)
            for (int dv = 0; dv < 2; ++dv) {
                const int cu = iu - du, cv = iv - dv;
                if (a == 0) mark(act, n, Wc, t, cu, cv);
                else if (a == 1) mark(act, n, Wc, cv, t, cu);
                else mark(act, n, Wc, cu, cv, t);
            }
    }
}

// bits i of node row (j, k) where nodes i and i + 1 differ along x
__device__ __forceinline__ unsigned xdiff(const unsigned *node, int W, int res, int j, int k, int w) {
    const unsigned *row = node + ((long long)k * res + j) * W;
    const unsigned lo = row[w], hi = w + 1 < W ? row[w + 1] : 0u;
    return lo ^ ((lo >> 1) | (hi << 31));
}

__device__ __forceinline__ unsigned row_word(const unsigned *node, int W, int res, int j, int k, int w) {
    return (w < W) ? node[((long long)k * res + j) * W + w] : 0u;
}

// cell bit i from node-column bits i and i + 1
__device__ __forceinline__ unsigned spread(unsigned lo, unsigned hi) { return lo | (lo >> 1) | (hi << 31); }

// Cells around every edge whose end nodes differ: a thread per word of a
// cell row (j, k).  The cell and node bit volumes share the word width.
__global__ void __launch_bounds__(kThreads) mark_signs(const unsigned *node, int res, int W, unsigned *act, int Wc) {
    const int n = res - 1;
    const long long q = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (q >= (long long)n * n * Wc) return;
    const int w = (int)(q % Wc);
    const int j = (int)((q / Wc) % n), k = (int)(q / ((long long)Wc * n));
    // x-edges of the four node rows around cell row (j, k)
    unsigned m = xdiff(node, W, res, j, k, w) | xdiff(node, W, res, j + 1, k, w) | xdiff(node, W, res, j, k + 1, w) |
                 xdiff(node, W, res, j + 1, k + 1, w);
    // y-edges (node rows (j, k') and (j + 1, k'), k' = k, k + 1) and z-edges
    // (rows (j', k) and (j', k + 1), j' = j, j + 1), at node columns i, i + 1
    unsigned ylo = 0, yhi = 0, zlo = 0, zhi = 0;
    for (int dk = 0; dk < 2; ++dk) {
        ylo |= row_word(node, W, res, j, k + dk, w) ^ row_word(node, W, res, j + 1, k + dk, w);
        yhi |= row_word(node, W, res, j, k + dk, w + 1) ^ row_word(node, W, res, j + 1, k + dk, w + 1);
    }
    for (int dj = 0; dj < 2; ++dj) {
        zlo |= row_word(node, W, res, j + dj, k, w) ^ row_word(node, W, res, j + dj, k + 1, w);
        zhi |= row_word(node, W, res, j + dj, k, w + 1) ^ row_word(node, W, res, j + dj, k + 1, w + 1);
    }
    m |= spread(ylo, yhi) | spread(zlo, zhi);
    const int valid = n - 32 * w;  // cells i < n
    if (valid < 32) m &= (1u << valid) - 1u;
    if (m) atomicOr(act + ((long long)k * n + j) * Wc + w, m);
}

__global__ void __launch_bounds__(kThreads) count_words(const unsigned *act, long long nw, int *cnt) {
    const long long q = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (q < nw) cnt[q] = __popc(act[q]);
}

__global__ void __launch_bounds__(kThreads) list_cells(const unsigned *act, long long nw, const int *woff, int n,
                                                       int Wc, long long *cells, long long max_active,
                                                       ldni_info_t *info) {
    const long long q = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (q >= nw) return;
    unsigned m = act[q];
    long long at = woff[q];
    const long long row = q / Wc;  // k * n + j
    const int w = (int)(q % Wc);
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        if (at >= max_active) {
            set_status(info, LDNI_ST_CAPACITY);
            return;
        }
        cells[at++] = row * n + 32 * w + b;  // i + n (j + n k)
    }
}

// ---- one cell --------------------------------------------------------------------

struct Edge {
    int a, q0, q1;  // axis, lower and upper corner
    int iu, iv, t;  // ray node indices, edge index along a
};

__device__ __forceinline__ Edge cell_edge(int e, int i, int j, int k) {
    Edge E;
    const int x = e & 1, y = (e >> 1) & 1;
    if (e < 4) {  // x-edges at (j + x, k + y)
        E = Edge{0, 0 + 2 * x + 4 * y, 1 + 2 * x + 4 * y, j + x, k + y, i};
    } else if (e < 8) {  // y-edges at (i + x, k + y): ray (u, v) = (z, x)
        E = Edge{1, x + 4 * y, x + 2 + 4 * y, k + y, i + x, j};
    } else {  // z-edges at (i + x, j + y)
        E = Edge{2, x + 2 * y, x + 2 * y + 4, i + x, j + y, k};
    }
    return E;
}

struct Kept {
    unsigned char type;  // 0 empty, 1 none-intersect, 2 intersect, 3 complex
    unsigned char nk;    // kept samples
    int s0, s1;          // kept sample indices (ascending depth)
};

struct Sym3 {  // A^T A, A^T b, sum of points, count
    double xx, xy, xz, yy, yz, zz, bx, by, bz, px, py, pz;
    int n;
};

__device__ __forceinline__ void add_point(Sym3 &Q, double P[3], double N[3]) {
    Q.xx += N[0] * N[0];
    Q.xy += N[0] * N[1];
    Q.xz += N[0] * N[2];
    Q.yy += N[1] * N[1];
    Q.yz += N[1] * N[2];
    Q.zz += N[2] * N[2];
    const double nb = N[0] * P[0] + N[1] * P[1] + N[2] * P[2];
    Q.bx += N[0] * nb;
    Q.by += N[1] * nb;
    Q.bz += N[2] * nb;
    Q.px += P[0];
    Q.py += P[1];
    Q.pz += P[2];
    Q.n += 1;
}

// Cyclic Jacobi rotations on a symmetric 3 x 3 matrix: eigenvalues on the
// diagonal of S, eigenvectors in the columns of V.  The sweeps stop once the
// off-diagonal sum is below 1e-12 of the diagonal's: the eigenvalues are then
// exact to second order (about 1e-24 relative) and the eigenvectors to about
// 1e-12, while FP64 rounding keeps the off-diagonal near 1e-16 of the
// diagonal, so a stricter bound would only spend sweeps.
__device__ void jacobi3(double S[3][3], double V[3][3]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) V[r][c] = r == c ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 32; ++sweep) {
        const double off = fabs(S[0][1]) + fabs(S[0][2]) + fabs(S[1][2]);
        const double dia = fabs(S[0][0]) + fabs(S[1][1]) + fabs(S[2][2]);
        if (!(off > 1e-300) || off <= 1e-12 * dia) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const double apq = S[p][q];
                if (fabs(apq) <= 1e-300) continue;
                const double theta = (S[q][q] - S[p][p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < 3; ++r) {  // S <- J^T S J
                    const double srp = S[r][p], srq = S[r][q];
                    S[r][p] = c * srp - s * srq;
                    S[r][q] = s * srp + c * srq;
                }
                for (int r = 0; r < 3; ++r) {
                    const double spr = S[p][r], sqr = S[q][r];
                    S[p][r] = c * spr - s * sqr;
                    S[q][r] = s * spr + c * sqr;
                }
                S[p][q] = S[q][p] = 0.0;
                for (int r = 0; r < 3; ++r) {
                    const double vrp = V[r][p], vrq = V[r][q];
                    V[r][p] = c * vrp - s * vrq;
                    V[r][q] = s * vrp + c * vrq;
                }
            }
    }
}

__device__ void qef_solve(const Sym3 &Q, double x[3]) {
    const double m[3] = {Q.px / Q.n, Q.py / Q.n, Q.pz / Q.n};
    double S[3][3] = {{Q.xx, Q.xy, Q.xz}, {Q.xy, Q.yy, Q.yz}, {Q.xz, Q.yz, Q.zz}};
    const double AtA[3][3] = {{Q.xx, Q.xy, Q.xz}, {Q.xy, Q.yy, Q.yz}, {Q.xz, Q.yz, Q.zz}};
    double r[3] = {Q.bx, Q.by, Q.bz};
    for (int a = 0; a < 3; ++a) r[a] -= AtA[a][0] * m[0] + AtA[a][1] * m[1] + AtA[a][2] * m[2];
    double V[3][3];
    jacobi3(S, V);
    const double lam[3] = {S[0][0], S[1][1], S[2][2]};
    const double top = fmax(lam[0], fmax(lam[1], lam[2]));
    double y[3];
    for (int c = 0; c < 3; ++c) {
        const double vr = V[0][c] * r[0] + V[1][c] * r[1] + V[2][c] * r[2];
        y[c] = (top > 0.0 && lam[c] >= 0.01 * top) ? vr / lam[c] : 0.0;
    }
    for (int a = 0; a < 3; ++a) x[a] = m[a] + V[a][0] * y[0] + V[a][1] * y[1] + V[a][2] * y[2];
}

__device__ __forceinline__ void hermite(const CImg &I, int a, int s, int iu, int iv, float o[3], float h,
                                        double P[3], double N[3]) {
    const int u = a == 2 ? 0 : a + 1, v = a == 0 ? 2 : a - 1;
    P[a] = (double)pick(I.d, a)[s];
    P[u] = (double)node_c(iu, o[u], h);
    P[v] = (double)node_c(iv, o[v], h);
    double n3[3] = {(double)pick(I.nx, a)[s], (double)pick(I.ny, a)[s], (double)pick(I.nz, a)[s]};
    N[0] = n3[0];
    N[1] = n3[1];
    N[2] = n3[2];
}

// One thread per active cell (the first *nact of the list).
__global__ void __launch_bounds__(128) cell_kernel(CImg I, const unsigned *node, int res, int W, float o0, float o1,
                                                   float o2, float h, const long long *cells, const int *nact,
                                                   long long max_active, ldni_cell_t *rec) {
    const long long q = blockIdx.x * 128LL + threadIdx.x;
    if (q >= min((long long)*nact, max_active)) return;
    const int n = res - 1;
    const long long ci = cells[q];
    const int i = (int)(ci % n), j = (int)((ci / n) % n), k = (int)(ci / ((long long)n * n));
    float o[3] = {o0, o1, o2};
    unsigned sgn = 0;  // bit c: corner c inside
    for (int c = 0; c < 8; ++c) {
        const int ii = i + (c & 1), jj = j + ((c >> 1) & 1), kk = k + (c >> 2);
        const unsigned wd = node[((long long)kk * res + jj) * W + (ii >> 5)];
        sgn |= ((wd >> (ii & 31)) & 1u) << c;
    }
    Kept K[12];
    for (int e = 0; e < 12; ++e) {
        const Edge E = cell_edge(e, i, j, k);
        const int *off = pick(I.off, E.a);
        const float *D = pick(I.d, E.a);
        const long long p = (long long)E.iv * res + E.iu;
        const long long b0 = off[p], e0 = min((long long)off[p + 1], pick(I.cap, E.a));
        const float lo = node_c(E.t, o[E.a], h), hi = node_c(E.t + 1, o[E.a], h);
        const bool in0 = (sgn >> E.q0) & 1u, in1 = (sgn >> E.q1) & 1u;
        const double mid = ((double)lo + (double)hi) / 2.0;
        const float want = in0 ? 1.0f : -1.0f;
        int cnt = 0, first = -1, last = -1, best = -1, bestc = -1;
        double bd = 0.0, bdc = 0.0;
        const float *NA = E.a == 0 ? pick(I.nx, 0) : (E.a == 1 ? pick(I.ny, 1) : pick(I.nz, 2));
        for (long long s = b0; s < e0; ++s) {
            const float d = D[s];
            if (d < lo) continue;
            if (!(d < hi)) break;  // ascending depths
            ++cnt;
            if (first < 0) first = (int)s;
            last = (int)s;
            const double dist = fabs((double)d - mid);
            if (best < 0 || dist < bd) {
                best = (int)s;
                bd = dist;
            }
            if (NA[s] * want > 0.0f && (bestc < 0 || dist < bdc)) {
                bestc = (int)s;
                bdc = dist;
            }
        }
        Kept &k2 = K[e];
        if (in0 != in1) {
            k2.type = cnt ? 2 : 1;
            k2.nk = cnt ? 1 : 0;
            k2.s0 = bestc >= 0 ? bestc : best;
            k2.s1 = -1;
        } else {
            k2.type = cnt ? 3 : 0;
            k2.nk = cnt >= 2 ? 2 : cnt;
            k2.s0 = first;
            k2.s1 = cnt >= 2 ? last : -1;
        }
    }
    // flood the outside corners through empty edges
    unsigned char lab[8];
    for (int c = 0; c < 8; ++c) lab[c] = 0xff;
    int ncl = 0;
    for (int c = 0; c < 8; ++c) {
        if (((sgn >> c) & 1u) || lab[c] != 0xff) continue;
        unsigned comp = 1u << c, grow = comp;
        while (grow) {  // breadth-first over empty edges between outside corners
            unsigned next = 0;
            for (int e = 0; e < 12; ++e) {
                if (K[e].type != 0) continue;
                const Edge E = cell_edge(e, 0, 0, 0);
                const unsigned m0 = 1u << E.q0, m1 = 1u << E.q1;
                if ((sgn & (m0 | m1)) != 0) continue;
                if ((grow & m0) && !(comp & m1)) next |= m1;
                if ((grow & m1) && !(comp & m0)) next |= m0;
            }
            comp |= next;
            grow = next;
        }
        for (int d = 0; d < 8; ++d)
            if ((comp >> d) & 1u) lab[d] = (unsigned char)ncl;
        ++ncl;
    }
    ldni_cell_t R;
    R.cell = ci;
    R.nvert = 0;
    R.labels = 0;
    R.npts = 0;
    R.pad_ = 0;
    for (int c = 0; c < 8; ++c) R.labels |= (unsigned)(lab[c] == 0xff ? 0xf : lab[c]) << (4 * c);
    for (int v = 0; v < 12; ++v) R.v[v] = 0.0f;
    if (ncl == 0) {
        rec[q] = R;
        return;
    }
    // Hermite data and the surface clusters
    bool surf[4] = {false, false, false, false};
    Sym3 Q[4];
    for (int g = 0; g < 4; ++g) Q[g] = Sym3{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int e = 0; e < 12; ++e) {
        const Edge E = cell_edge(e, i, j, k);
        const Kept &k2 = K[e];
        const bool in0 = (sgn >> E.q0) & 1u;
        double P[3], N[3];
        if (k2.type == 2) {
            const int g = lab[in0 ? E.q1 : E.q0];
            surf[g] = true;
            hermite(I, E.a, k2.s0, E.iu, E.iv, o, h, P, N);
            add_point(Q[g], P, N);
        } else if (k2.type == 1) {
            surf[lab[in0 ? E.q1 : E.q0]] = true;
        } else if (k2.type == 3 && !in0) {
            const int g0 = lab[E.q0], g1 = lab[E.q1];
            surf[g0] = surf[g1] = true;
            if (k2.nk == 2) {
                hermite(I, E.a, k2.s0, E.iu, E.iv, o, h, P, N);
                add_point(Q[g0], P, N);
                hermite(I, E.a, k2.s1, E.iu, E.iv, o, h, P, N);
                add_point(Q[g1], P, N);
            } else {
                const float lo = node_c(E.t, o[E.a], h), hi = node_c(E.t + 1, o[E.a], h);
                const double mid = ((double)lo + (double)hi) / 2.0;
                hermite(I, E.a, k2.s0, E.iu, E.iv, o, h, P, N);
                add_point(Q[P[E.a] < mid ? g0 : g1], P, N);
            }
        }
    }
    bool any = false;
    for (int g = 0; g < ncl; ++g) any = any || surf[g];
    if (!any) {
        rec[q] = R;
        return;
    }
    R.nvert = ncl;
    for (int g = 0; g < ncl; ++g) {
        double x[3];
        if (Q[g].n > 0) {
            qef_solve(Q[g], x);
        } else {  // no Hermite data: the mean of the cluster's corners
            double s3[3] = {0.0, 0.0, 0.0};
            int m = 0;
            for (int c = 0; c < 8; ++c) {
                if (lab[c] != g) continue;
                s3[0] += (double)node_c(i + (c & 1), o[0], h);
                s3[1] += (double)node_c(j + ((c >> 1) & 1), o[1], h);
                s3[2] += (double)node_c(k + (c >> 2), o[2], h);
                ++m;
            }
            x[0] = s3[0] / m;
            x[1] = s3[1] / m;
            x[2] = s3[2] / m;
        }
        R.v[3 * g] = (float)x[0];
        R.v[3 * g + 1] = (float)x[1];
        R.v[3 * g + 2] = (float)x[2];
        R.npts |= (unsigned)min(Q[g].n, 255) << (8 * g);
    }
    rec[q] = R;
}

__global__ void __launch_bounds__(kThreads) has_vertex(const ldni_cell_t *rec, const int *nact, long long n,
                                                       int *flag) {
    const long long q = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (q < n) flag[q] = (q < *nact && rec[q].nvert > 0) ? 1 : 0;
}

__global__ void __launch_bounds__(kThreads) compact_cells(const ldni_cell_t *rec, const int *nact, long long n,
                                                          const int *at, ldni_cell_t *out, long long cap,
                                                          ldni_info_t *info) {
    const long long q = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (q >= n || q >= *nact || rec[q].nvert == 0) return;
    const long long slot = at[q];
    if (slot >= cap) {
        set_status(info, LDNI_ST_CAPACITY);
        return;
    }
    out[slot] = rec[q];
}

struct ContourWs {
    unsigned *act;
    size_t act_bytes;
    int *wcnt, *woff;
    long long *cells;
    ldni_cell_t *rec;
    int *flag, *at;
    long long *partials;
    ldni_info_t *tinfo;
};

ContourWs carve_contour(Carver &c, int res, long long max_active) {
    ContourWs w{};
    const long long n = res - 1, Wc = (n + 31) / 32, nw = n * n * Wc;
    w.act = c.take<unsigned>((size_t)nw);
    w.act_bytes = sizeof(unsigned) * (size_t)nw;
    w.wcnt = c.take<int>((size_t)nw);
    w.woff = c.take<int>((size_t)nw + 1);
    w.cells = c.take<long long>((size_t)max_active);
    w.rec = c.take<ldni_cell_t>((size_t)max_active);
    w.flag = c.take<int>((size_t)max_active);
    w.at = c.take<int>((size_t)max_active + 1);
    w.partials = c.take<long long>(std::max(csr_scan_partials(nw), csr_scan_partials(max_active)));
    w.tinfo = c.take<ldni_info_t>(1);
    return w;
}

}  // namespace
}  // namespace ldni

using namespace ldni;

extern "C" int ldni_contour_workspace_size(int32_t res, int64_t max_active, size_t *bytes) {
    if (!bytes || res < 2 || res > 2048 || max_active < 1 || max_active > INT_MAX) return LDNI_EINVAL;
    Carver c(nullptr, 0);
    carve_contour(c, res, max_active);
    *bytes = align_up(c.off);
    return LDNI_OK;
}

extern "C" int ldni_contour_cells(const ldni_layers_t *L, const ldni_grid_t *grid, const uint32_t *inside,
                                  int64_t max_active, ldni_cell_t *cells, int64_t capacity, ldni_info_t *info,
                                  void *ws, size_t ws_bytes, void *stream) {
    if (!L || !grid_valid(grid) || !inside || !info || !ws || (capacity > 0 && !cells) || capacity < 0 ||
        max_active < 1 || max_active > INT_MAX)
        return LDNI_EINVAL;
    const int res = grid->res;
    if (res < 2 || res > 2048) return LDNI_EINVAL;
    CImg I{};
    for (int a = 0; a < 3; ++a) {
        if (!L[a].offsets || L[a].capacity < 0 || !samples_ok(L[a]) || L[a].nrm8) return LDNI_EINVAL;
        I.off[a] = L[a].offsets;
        I.d[a] = L[a].depth;
        I.nx[a] = L[a].nx;
        I.ny[a] = L[a].ny;
        I.nz[a] = L[a].nz;
        I.cap[a] = L[a].capacity;
    }
    Carver c(ws, ws_bytes);
    ContourWs w = carve_contour(c, res, max_active);
    if (!c.fits()) return LDNI_EWORKSPACE;
    const int n = res - 1, W = (res + 31) / 32, Wc = (n + 31) / 32;
    const long long nw = (long long)n * n * Wc;
    const float h = grid->width / (float)res;
    const float *o = grid->origin;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc_ = cuda_check(cudaMemsetAsync(w.act, 0, w.act_bytes, s))) return rc_;
    if (int rc_ = cuda_check(cudaMemsetAsync(w.tinfo, 0, sizeof(ldni_info_t), s))) return rc_;
    const long long N = (long long)res * res;
    LDNI_LAUNCH(K_CONTOUR, s,
                mark_signs<<<(unsigned)((nw + kThreads - 1) / kThreads), kThreads, 0, s>>>(inside, res, W, w.act, Wc));
    LDNI_LAUNCH(K_CONTOUR, s,
                mark_samples<<<dim3((unsigned)((N + kThreads - 1) / kThreads), 3), kThreads, 0, s>>>(
                    I, res, o[0], o[1], o[2], h, w.act, Wc));
    LDNI_LAUNCH(K_CONTOUR, s,
                count_words<<<(unsigned)((nw + kThreads - 1) / kThreads), kThreads, 0, s>>>(w.act, nw, w.wcnt));
    int rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    {
        const int *cn[1] = {w.wcnt};
        int *of[1] = {w.woff};
        rc = csr_scan(cn, of, 1, nw, w.partials, w.tinfo, 0, s);
        if (rc != LDNI_OK) return rc;
    }
    // every later launch covers max_active cells and reads the active count
    // on the device, so the call needs no host synchronisation
    const int *nact = w.woff + nw;
    const unsigned ablocks = (unsigned)((max_active + kThreads - 1) / kThreads);
    LDNI_LAUNCH(K_CONTOUR, s,
                list_cells<<<(unsigned)((nw + kThreads - 1) / kThreads), kThreads, 0, s>>>(
                    w.act, nw, w.woff, n, Wc, w.cells, max_active, info));
    LDNI_LAUNCH(K_CONTOUR, s,
                cell_kernel<<<(unsigned)((max_active + 127) / 128), 128, 0, s>>>(I, inside, res, W, o[0], o[1], o[2],
                                                                                   h, w.cells, nact, max_active,
                                                                                   w.rec));
    LDNI_LAUNCH(K_CONTOUR, s, has_vertex<<<ablocks, kThreads, 0, s>>>(w.rec, nact, max_active, w.flag));
    rc = cuda_status();
    if (rc != LDNI_OK) return rc;
    {
        const int *cn[1] = {w.flag};
        int *of[1] = {w.at};
        rc = csr_scan(cn, of, 1, max_active, w.partials, info, 0, s);
        if (rc != LDNI_OK) return rc;
    }
    LDNI_LAUNCH(K_CONTOUR, s,
                compact_cells<<<ablocks, kThreads, 0, s>>>(w.rec, nact, max_active, w.at, cells, capacity, info));
    return cuda_status();
}
