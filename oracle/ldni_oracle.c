/*
 * LDNI oracle: a plain, slow, obviously correct CPU statement of what the
 * LDNI hot path computes.  TEST INFRASTRUCTURE ONLY: it is called by the
 * tests, by __graft_entry__.smoke() and by the CPU-baseline leg of bench.py,
 * never by the library.  It shares no code with the CUDA path.
 *
 * Floating point is FP64 except where the method makes an integer decision
 * from floating point (the fixed-point snap of vertex coordinates and the
 * small-interval test of the Boolean): those are taken in FP32, the precision
 * of the paper's depth buffer and vertex pipeline (Section 3, "Balance between
 * time and accuracy": 32-bit float depth buffer).
 *
 * Conventions (readings of the paper; the paper states none of them):
 *  - axis a in {0:x, 1:y, 2:z}; in-plane (u, v) = (y, z), (z, x), (x, y).
 *  - cube origin o, width W, resolution res; pixel (i, j) -> p = j*res + i.
 *  - rays pass through pixel centres (Section 3, pixel-centre convention),
 *    run along +a; depth = world a-coordinate of the crossing, ascending
 *    (Definition 1).
 *  - snap: q = nearbyint(fl32(fl32(x - o) * s)), s = fl32(res * 2^8 / W), so
 *    a pixel centre is the integer 256*i + 128.
 *  - a crossing of ray c with triangle t: t's snapped projection, turned
 *    counter-clockwise, contains c under the top-left rule (an edge d owns
 *    the points on it iff d_v > 0, or d_v == 0 and d_u < 0).  Zero projected
 *    area = face parallel to the ray = no crossing (Definition 1 note).  A
 *    shared non-silhouette edge is then crossed once, a silhouette edge 0 or
 *    2 times (Remark 1), and every ray of a closed mesh has an even count
 *    (Definition 4).
 *  - depth = sum_k lambda_k * a_k with lambda_k = E_k / A2 from the exact
 *    integer edge functions and a_k the vertex a-coordinates.
 *  - normal = unit face normal from the vertex winding ("accurate normal
 *    sampling", Section 3 item 2), the sample keeps the triangle id.
 *  - samples of one ray are ordered by (depth, tri_id).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -5
#define OR_ERANGE -8
#define OR_EODD -3

#define SUBPIX_BITS 8
#define SNAP_LIMIT 16777216.0f /* |q| < 2^24 keeps every edge product in int64 */

/* ------------------------------------------------------------------ */
/* grid and snapping                                                    */
/* ------------------------------------------------------------------ */

static void plane_axes(int axis, int *iu, int *iv) {
    /* cyclic in-plane axes: x-LDNI -> (y,z), y-LDNI -> (z,x), z-LDNI -> (x,y) */
    *iu = (axis + 1) % 3;
    *iv = (axis + 2) % 3;
}

static float snap_scale(int32_t res, float width) {
    return (float)((double)res * (double)(1 << SUBPIX_BITS) / (double)width);
}

/* fixed-point coordinate of one vertex component, decided in FP32 */
static int snap_coord(float x, float o, float s, int64_t *q) {
    float t = x - o;
    float y = t * s;
    if (!(y > -SNAP_LIMIT && y < SNAP_LIMIT)) return OR_ERANGE;
    *q = (int64_t)nearbyintf(y);
    return OR_OK;
}

static int64_t floor_div(int64_t a, int64_t b) { /* b > 0 */
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

static int64_t ceil_div(int64_t a, int64_t b) { /* b > 0 */
    return -floor_div(-a, b);
}

/* ------------------------------------------------------------------ */
/* the crossing predicate                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t pu[3], pv[3]; /* snapped projected vertices, counter-clockwise */
    double a[3];          /* vertex a-coordinates in the same order */
    int64_t area2;        /* > 0 */
} proj_tri;

/* Build the counter-clockwise projected triangle; returns 0 when the
 * projection has zero area (the face is parallel to the ray). */
static int project_tri(const int64_t *qv, const float *verts, const int32_t *t, int axis, proj_tri *P) {
    int iu, iv;
    plane_axes(axis, &iu, &iv);
    int64_t u[3], v[3];
    double a[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = qv[3 * (int64_t)t[k] + iu];
        v[k] = qv[3 * (int64_t)t[k] + iv];
        a[k] = (double)verts[3 * (int64_t)t[k] + axis];
    }
    int64_t A2 = (u[1] - u[0]) * (v[2] - v[0]) - (v[1] - v[0]) * (u[2] - u[0]);
    if (A2 == 0) return 0;
    int ord[3] = {0, 1, 2};
    if (A2 < 0) { ord[1] = 2; ord[2] = 1; A2 = -A2; }
    for (int k = 0; k < 3; ++k) {
        P->pu[k] = u[ord[k]];
        P->pv[k] = v[ord[k]];
        P->a[k] = a[ord[k]];
    }
    P->area2 = A2;
    return 1;
}

/* top-left ownership of the zero set of edge direction (du, dv) */
static int owns(int64_t du, int64_t dv) { return dv > 0 || (dv == 0 && du < 0); }

/* Does the ray through fixed-point centre (cu, cv) cross P?  On success the
 * crossing depth is written to *depth. */
static int crosses(const proj_tri *P, int64_t cu, int64_t cv, double *depth) {
    int64_t E[3];
    for (int k = 0; k < 3; ++k) {
        int k1 = (k + 1) % 3;
        int64_t du = P->pu[k1] - P->pu[k];
        int64_t dv = P->pv[k1] - P->pv[k];
        E[k] = du * (cv - P->pv[k]) - dv * (cu - P->pu[k]);
        if (E[k] < 0) return 0;
        if (E[k] == 0 && !owns(du, dv)) return 0;
    }
    /* E[k] is twice the area opposite vertex k+2: barycentric lambda_{k+2} */
    double A = (double)P->area2;
    *depth = ((double)E[1] / A) * P->a[0] + ((double)E[2] / A) * P->a[1] + ((double)E[0] / A) * P->a[2];
    return 1;
}

static void face_normal(const float *verts, const int32_t *t, double n[3]) {
    const float *p0 = verts + 3 * (int64_t)t[0];
    const float *p1 = verts + 3 * (int64_t)t[1];
    const float *p2 = verts + 3 * (int64_t)t[2];
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = (double)p1[k] - (double)p0[k];
        e2[k] = (double)p2[k] - (double)p0[k];
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (len > 0) { n[0] /= len; n[1] /= len; n[2] /= len; }
}

/* ------------------------------------------------------------------ */
/* sampling                                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;        /* total samples */
    int64_t nrays;    /* res*res */
    int64_t *offsets; /* [nrays+1] */
    double *depth;    /* [n] */
    double *nrm;      /* [n][3] */
    int32_t *tri;     /* [n] */
} oracle_ldni;

typedef struct {
    int64_t ray;
    double depth;
    int32_t tri;
} crossing;

static int cmp_crossing(const void *x, const void *y) {
    const crossing *A = (const crossing *)x, *B = (const crossing *)y;
    if (A->ray != B->ray) return A->ray < B->ray ? -1 : 1;
    if (A->depth != B->depth) return A->depth < B->depth ? -1 : 1;
    if (A->tri != B->tri) return A->tri < B->tri ? -1 : 1;
    return 0;
}

typedef struct {
    crossing *c;
    int64_t n, cap;
} crossing_list;

static int push(crossing_list *L, int64_t ray, double depth, int32_t tri) {
    if (L->n == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 1024;
        crossing *q = (crossing *)realloc(L->c, (size_t)nc * sizeof(crossing));
        if (!q) return OR_ENOMEM;
        L->c = q;
        L->cap = nc;
    }
    L->c[L->n].ray = ray;
    L->c[L->n].depth = depth;
    L->c[L->n].tri = tri;
    L->n++;
    return OR_OK;
}

void oracle_free(oracle_ldni *L) {
    if (!L) return;
    free(L->offsets);
    free(L->depth);
    free(L->nrm);
    free(L->tri);
    free(L);
}

/*
 * Sample one LDNI (Definitions 1-2).
 *   mode 0 = brute force: every pixel-centre ray against every triangle
 *            (the definition itself);
 *   mode 1 = scan: every triangle against the pixel centres inside its
 *            snapped bounding box (same predicate, fewer candidates).
 * Returns NULL and sets *err on failure.
 */
oracle_ldni *oracle_sample(const float *verts, int64_t nv, const int32_t *tris, int64_t nt,
                           const float *origin, float width, int32_t res, int32_t axis,
                           int32_t mode, int32_t *err) {
    *err = OR_OK;
    if (!verts || !tris || !origin || nv <= 0 || nt < 0 || res <= 0 || axis < 0 || axis > 2 ||
        !(width > 0) || (int64_t)res * 256 + 256 > (1LL << 24)) {
        *err = OR_EINVAL;
        return NULL;
    }
    for (int64_t t = 0; t < 3 * nt; ++t)
        if (tris[t] < 0 || tris[t] >= nv) { *err = OR_EINVAL; return NULL; }
    float s = snap_scale(res, width);
    int64_t *qv = (int64_t *)malloc((size_t)nv * 3 * sizeof(int64_t));
    if (!qv) { *err = OR_ENOMEM; return NULL; }
    for (int64_t i = 0; i < nv; ++i)
        for (int k = 0; k < 3; ++k)
            if (snap_coord(verts[3 * i + k], origin[k], s, &qv[3 * i + k]) != OR_OK) {
                free(qv);
                *err = OR_ERANGE;
                return NULL;
            }
    int64_t nrays = (int64_t)res * res;
    crossing_list L = {0, 0, 0};
    int rc = OR_OK;
    if (mode == 0) {
        proj_tri *PT = (proj_tri *)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(proj_tri));
        char *ok = (char *)malloc((size_t)(nt > 0 ? nt : 1));
        if (!PT || !ok) { free(PT); free(ok); free(qv); *err = OR_ENOMEM; return NULL; }
        for (int64_t t = 0; t < nt; ++t) ok[t] = (char)project_tri(qv, verts, tris + 3 * t, axis, &PT[t]);
        for (int64_t j = 0; j < res && rc == OR_OK; ++j)
            for (int64_t i = 0; i < res && rc == OR_OK; ++i) {
                int64_t cu = 256 * i + 128, cv = 256 * j + 128;
                for (int64_t t = 0; t < nt; ++t) {
                    double d;
                    if (ok[t] && crosses(&PT[t], cu, cv, &d)) {
                        rc = push(&L, j * res + i, d, (int32_t)t);
                        if (rc != OR_OK) break;
                    }
                }
            }
        free(PT);
        free(ok);
    } else {
        for (int64_t t = 0; t < nt && rc == OR_OK; ++t) {
            proj_tri P;
            if (!project_tri(qv, verts, tris + 3 * t, axis, &P)) continue;
            int64_t umin = P.pu[0], umax = P.pu[0], vmin = P.pv[0], vmax = P.pv[0];
            for (int k = 1; k < 3; ++k) {
                if (P.pu[k] < umin) umin = P.pu[k];
                if (P.pu[k] > umax) umax = P.pu[k];
                if (P.pv[k] < vmin) vmin = P.pv[k];
                if (P.pv[k] > vmax) vmax = P.pv[k];
            }
            int64_t i0 = ceil_div(umin - 128, 256), i1 = floor_div(umax - 128, 256);
            int64_t j0 = ceil_div(vmin - 128, 256), j1 = floor_div(vmax - 128, 256);
            if (i0 < 0) i0 = 0;
            if (j0 < 0) j0 = 0;
            if (i1 > res - 1) i1 = res - 1;
            if (j1 > res - 1) j1 = res - 1;
            for (int64_t j = j0; j <= j1 && rc == OR_OK; ++j)
                for (int64_t i = i0; i <= i1; ++i) {
                    double d;
                    if (crosses(&P, 256 * i + 128, 256 * j + 128, &d)) {
                        rc = push(&L, j * res + i, d, (int32_t)t);
                        if (rc != OR_OK) break;
                    }
                }
        }
    }
    free(qv);
    if (rc != OR_OK) { free(L.c); *err = rc; return NULL; }
    if (L.n > 0) qsort(L.c, (size_t)L.n, sizeof(crossing), cmp_crossing);

    oracle_ldni *out = (oracle_ldni *)calloc(1, sizeof(oracle_ldni));
    if (!out) { free(L.c); *err = OR_ENOMEM; return NULL; }
    out->n = L.n;
    out->nrays = nrays;
    out->offsets = (int64_t *)calloc((size_t)nrays + 1, sizeof(int64_t));
    out->depth = (double *)malloc((size_t)(L.n > 0 ? L.n : 1) * sizeof(double));
    out->nrm = (double *)malloc((size_t)(L.n > 0 ? L.n : 1) * 3 * sizeof(double));
    out->tri = (int32_t *)malloc((size_t)(L.n > 0 ? L.n : 1) * sizeof(int32_t));
    if (!out->offsets || !out->depth || !out->nrm || !out->tri) {
        free(L.c);
        oracle_free(out);
        *err = OR_ENOMEM;
        return NULL;
    }
    for (int64_t k = 0; k < L.n; ++k) {
        out->offsets[L.c[k].ray + 1]++;
        out->depth[k] = L.c[k].depth;
        out->tri[k] = L.c[k].tri;
        face_normal(verts, tris + 3 * (int64_t)L.c[k].tri, out->nrm + 3 * k);
    }
    for (int64_t p = 0; p < nrays; ++p) out->offsets[p + 1] += out->offsets[p];
    free(L.c);
    return out;
}

/* ------------------------------------------------------------------ */
/* Boolean (Section 4.1) and small-interval removal (Section 4.1.1)    */
/* ------------------------------------------------------------------ */

#define OP_UNION 0
#define OP_INTER 1
#define OP_DIFF 2

typedef struct {
    int64_t n;
    int64_t nrays;
    int64_t *offsets; /* [nrays+1] */
    float *depth;     /* [n] */
    float *nrm;       /* [n][3] */
    int32_t *tri;     /* [n]; bit 31 set = sample came from B */
} oracle_bool;

void oracle_bool_free(oracle_bool *R) {
    if (!R) return;
    free(R->offsets);
    free(R->depth);
    free(R->nrm);
    free(R->tri);
    free(R);
}

static int op_apply(int op, int a, int b) {
    if (op == OP_UNION) return a || b;
    if (op == OP_INTER) return a && b;
    return a && !b;
}

/* parity of #{x in list : x < d} (strict) and of #{x <= d} */
static void parity_around(const float *x, int64_t n, float d, int *before, int *after) {
    int64_t lt = 0, le = 0;
    for (int64_t k = 0; k < n; ++k) {
        if (x[k] < d) lt++;
        if (x[k] <= d) le++;
    }
    *before = (int)(lt & 1);
    *after = (int)(le & 1);
}

static int cmp_float(const void *x, const void *y) {
    float a = *(const float *)x, b = *(const float *)y;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* One ray.  The result is the boundary of the regularised 1D set
 * {t : op(in_A(t), in_B(t))}, where in_X(t) = odd number of X samples below t
 * (odd-to-even ranges are inside, Section 2).  Every depth where the state
 * just below differs from the state just above is one output sample; its
 * normal and id come from A if A's state flips there, else from B (normal
 * inverted for a difference, Section 4.1).  Then solid intervals thinner than
 * eps (FP32 difference) are removed. */
static int64_t bool_ray(const float *dA, const float *nA, const int32_t *tA, int64_t na,
                        const float *dB, const float *nB, const int32_t *tB, int64_t nb, int op, float eps,
                        float *od, float *on, int32_t *ot, float *cand) {
    int64_t nc = 0;
    for (int64_t k = 0; k < na; ++k) cand[nc++] = dA[k];
    for (int64_t k = 0; k < nb; ++k) cand[nc++] = dB[k];
    qsort(cand, (size_t)nc, sizeof(float), cmp_float);
    int64_t m = 0;
    for (int64_t k = 0; k < nc; ++k) {
        if (k > 0 && cand[k] == cand[k - 1]) continue;
        float d = cand[k];
        int a0, a1, b0, b1;
        parity_around(dA, na, d, &a0, &a1);
        parity_around(dB, nb, d, &b0, &b1);
        if (op_apply(op, a0, b0) == op_apply(op, a1, b1)) continue;
        int from_a = (a0 != a1);
        const float *dl = from_a ? dA : dB;
        int64_t nl = from_a ? na : nb, s = -1;
        for (int64_t q = 0; q < nl; ++q)
            if (dl[q] == d) { s = q; break; }
        od[m] = d;
        if (from_a) {
            for (int c = 0; c < 3; ++c) on[3 * m + c] = nA[3 * s + c];
            ot[m] = tA[s];
        } else {
            float sg = (op == OP_DIFF) ? -1.0f : 1.0f;
            for (int c = 0; c < 3; ++c) on[3 * m + c] = sg * nB[3 * s + c];
            ot[m] = (int32_t)((uint32_t)tB[s] | 0x80000000u);
        }
        m++;
    }
    /* small-interval removal on solid intervals (d_{2k}, d_{2k+1}) */
    int64_t w = 0;
    for (int64_t k = 0; k + 1 < m; k += 2) {
        float th = od[k + 1] - od[k];
        if (th < eps) continue;
        for (int q = 0; q < 2; ++q) {
            od[w] = od[k + q];
            for (int c = 0; c < 3; ++c) on[3 * w + c] = on[3 * (k + q) + c];
            ot[w] = ot[k + q];
            w++;
        }
    }
    return w;
}

/*
 * Boolean of two LDNIs on the same grid (Section 4.1; both operands must be
 * sampled with the same origin and rate, Section 4.1.1).  Inputs are CSR
 * with FP32 depth, FP32 normals [n][3] and int32 ids; each ray ascending.
 */
oracle_bool *oracle_boolean(int64_t nrays, const int64_t *offA, const float *dA, const float *nA,
                            const int32_t *tA, const int64_t *offB, const float *dB, const float *nB,
                            const int32_t *tB, int32_t op, float eps, int32_t *err) {
    *err = OR_OK;
    if (nrays < 0 || op < 0 || op > 2 || !offA || !offB) { *err = OR_EINVAL; return NULL; }
    int64_t maxc = 0;
    for (int64_t p = 0; p < nrays; ++p) {
        int64_t ca = offA[p + 1] - offA[p], cb = offB[p + 1] - offB[p];
        if (ca < 0 || cb < 0) { *err = OR_EINVAL; return NULL; }
        if ((ca & 1) || (cb & 1)) { *err = OR_EODD; return NULL; }
        if (ca + cb > maxc) maxc = ca + cb;
    }
    int64_t cap = offA[nrays] - offA[0] + offB[nrays] - offB[0];
    oracle_bool *R = (oracle_bool *)calloc(1, sizeof(oracle_bool));
    float *cand = (float *)malloc((size_t)(maxc > 0 ? maxc : 1) * sizeof(float));
    if (!R || !cand) { free(R); free(cand); *err = OR_ENOMEM; return NULL; }
    R->nrays = nrays;
    R->offsets = (int64_t *)calloc((size_t)nrays + 1, sizeof(int64_t));
    R->depth = (float *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(float));
    R->nrm = (float *)malloc((size_t)(cap > 0 ? cap : 1) * 3 * sizeof(float));
    R->tri = (int32_t *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
    if (!R->offsets || !R->depth || !R->nrm || !R->tri) {
        free(cand);
        oracle_bool_free(R);
        *err = OR_ENOMEM;
        return NULL;
    }
    int64_t w = 0;
    for (int64_t p = 0; p < nrays; ++p) {
        int64_t a0 = offA[p], na = offA[p + 1] - offA[p];
        int64_t b0 = offB[p], nb = offB[p + 1] - offB[p];
        int64_t m = bool_ray(dA + a0, nA + 3 * a0, tA + a0, na, dB + b0, nB + 3 * b0, tB + b0, nb, op, eps,
                             R->depth + w, R->nrm + 3 * w, R->tri + w, cand);
        w += m;
        R->offsets[p + 1] = w;
    }
    R->n = w;
    free(cand);
    return R;
}

/* ------------------------------------------------------------------ */
/* volume                                                               */
/* ------------------------------------------------------------------ */

/*
 * Enclosed volume seen by one LDNI: each ray contributes the lengths of its
 * inside ranges, sample 2k to sample 2k+1 (odd-to-even depth ranges are
 * inside, Section 2 after Proposition 1), times the pixel area h^2.
 */
int32_t oracle_volume(int64_t nrays, const int64_t *off, const float *depth, double h, double *vol) {
    double acc = 0.0;
    for (int64_t p = 0; p < nrays; ++p) {
        int64_t c = off[p + 1] - off[p];
        if (c & 1) return OR_EODD;
        for (int64_t k = off[p]; k + 1 < off[p + 1]; k += 2) acc += (double)depth[k + 1] - (double)depth[k];
    }
    *vol = acc * h * h;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* offsetting (Section 4.2)                                             */
/* ------------------------------------------------------------------ */

/*
 * Offsetting of a solid H by r (Section 4.2): one sphere of radius r is
 * placed at every depth-normal sample of H's three LDNIs, and H is united
 * with the spheres one after another (outer offset), or the spheres are
 * subtracted one after another (inner offset), each sphere itself given by
 * its LDNIs on H's grid.
 *
 * Readings (the paper gives no arithmetic for the sphere's samples):
 *  - a sample of image a at pixel (i, j) with depth d sits at the point with
 *    a-coordinate d and in-plane coordinates c_u(i), c_v(j), where
 *    c(t) = fl32(o + fl32((t + 1/2) * h)), h = fl32(W / res);
 *  - the spheres are taken in the order of the samples: image x, y, z, each
 *    in CSR order; sphere s is the s-th sample in that order;
 *  - the sphere about C meets the ray through (P_u, P_v) of image b iff
 *    q < fl32(r * r), q = fl32(fl32(du * du) + fl32(dv * dv)),
 *    du = fl32(P_u - C_u), dv = fl32(P_v - C_v); its two samples are
 *    fl32(C_b -+ t), t = sqrt(fl32(r * r - q)) rounded to FP32, with the
 *    outward normals (du, dv, -+t) / r (each component rounded to FP32) and
 *    id s;
 *  - each step is the Boolean of Section 4.1 with no small-interval removal;
 *    the removal (eps) is applied once, to the final result, so that the
 *    result does not depend on the order of the spheres.
 * All sphere arithmetic is single precision, each operation rounded to
 * nearest, so the samples are exact functions of the inputs.
 */

static float pixel_coord(int64_t t, float o, float h) {
    float x = ((float)t + 0.5f) * h;
    return o + x;
}

/* The sphere about c on the ray (pu, pv) of image b: 1 and its two samples
 * (entering, leaving), or 0 when it misses the ray. */
static int sphere_on_ray(const float c[3], int b, float pu, float pv, float r, float r2, float d[2], float n[6]) {
    int iu, iv;
    plane_axes(b, &iu, &iv);
    float du = pu - c[iu];
    float dv = pv - c[iv];
    float du2 = du * du;
    float dv2 = dv * dv;
    float q = du2 + dv2;
    if (!(q < r2)) return 0;
    float t = sqrtf(r2 - q);
    d[0] = c[b] - t;
    d[1] = c[b] + t;
    float nu = du / r, nv = dv / r, na = t / r;
    n[b] = -na;
    n[iu] = nu;
    n[iv] = nv;
    n[3 + b] = na;
    n[3 + iu] = nu;
    n[3 + iv] = nv;
    return 1;
}

/*
 * Image b of the offset of H.  off: the three images' offsets one after
 * another (3 (res^2 + 1) values, each image's starting at 0); depth, nrm
 * ([n][3]) and tri: the three images' samples one after another, n[a] each.
 * op: OP_UNION (outer offset) or OP_DIFF (inner offset).
 */
oracle_bool *oracle_offset(int32_t res, const float *origin, float width, const int64_t *off, const float *depth,
                           const float *nrm, const int32_t *tri, const int64_t *n, int32_t b, float r, int32_t op,
                           float eps, int32_t *err) {
    *err = OR_OK;
    if (res < 1 || b < 0 || b > 2 || !(r > 0.0f) || (op != OP_UNION && op != OP_DIFF)) {
        *err = OR_EINVAL;
        return NULL;
    }
    const int64_t nrays = (int64_t)res * res;
    const float h = width / (float)res;
    const float r2 = r * r;
    int64_t S = n[0] + n[1] + n[2], base[3] = {0, n[0], n[0] + n[1]};
    /* sphere centres, in sample order */
    float *C = (float *)malloc((size_t)(S > 0 ? S : 1) * 3 * sizeof(float));
    int64_t *cnt = (int64_t *)calloc((size_t)nrays + 1, sizeof(int64_t));
    if (!C || !cnt) { free(C); free(cnt); *err = OR_ENOMEM; return NULL; }
    for (int a = 0; a < 3; ++a) {
        int iu, iv;
        plane_axes(a, &iu, &iv);
        const int64_t *oa = off + (int64_t)a * (nrays + 1);
        for (int64_t p = 0; p < nrays; ++p) {
            float cu = pixel_coord(p % res, origin[iu], h), cv = pixel_coord(p / res, origin[iv], h);
            for (int64_t k = oa[p]; k < oa[p + 1]; ++k) {
                float *c = C + 3 * (base[a] + k);
                c[a] = depth[base[a] + k];
                c[iu] = cu;
                c[iv] = cv;
            }
        }
    }
    /* the spheres that may meet each ray of image b (a box of pixel centres
     * one pixel wider than the sphere's shadow), in sphere order */
    int bu, bv;
    plane_axes(b, &bu, &bv);
    int64_t *box = (int64_t *)malloc((size_t)(S > 0 ? S : 1) * 4 * sizeof(int64_t));
    if (!box) { free(C); free(cnt); *err = OR_ENOMEM; return NULL; }
    for (int64_t s = 0; s < S; ++s) {
        const float *c = C + 3 * s;
        double lo_u = ((double)c[bu] - r - origin[bu]) / h - 0.5, hi_u = ((double)c[bu] + r - origin[bu]) / h - 0.5;
        double lo_v = ((double)c[bv] - r - origin[bv]) / h - 0.5, hi_v = ((double)c[bv] + r - origin[bv]) / h - 0.5;
        int64_t i0 = (int64_t)floor(lo_u) - 1, i1 = (int64_t)ceil(hi_u) + 1;
        int64_t j0 = (int64_t)floor(lo_v) - 1, j1 = (int64_t)ceil(hi_v) + 1;
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (i1 > res - 1) i1 = res - 1;
        if (j1 > res - 1) j1 = res - 1;
        box[4 * s] = i0, box[4 * s + 1] = i1, box[4 * s + 2] = j0, box[4 * s + 3] = j1;
        for (int64_t j = j0; j <= j1; ++j)
            for (int64_t i = i0; i <= i1; ++i) cnt[j * res + i + 1]++;
    }
    for (int64_t p = 0; p < nrays; ++p) cnt[p + 1] += cnt[p];
    int64_t *lst = (int64_t *)malloc((size_t)(cnt[nrays] > 0 ? cnt[nrays] : 1) * sizeof(int64_t));
    int64_t *fillp = (int64_t *)malloc((size_t)nrays * sizeof(int64_t));
    if (!lst || !fillp) { free(C); free(cnt); free(box); free(lst); free(fillp); *err = OR_ENOMEM; return NULL; }
    memcpy(fillp, cnt, (size_t)nrays * sizeof(int64_t));
    for (int64_t s = 0; s < S; ++s)
        for (int64_t j = box[4 * s + 2]; j <= box[4 * s + 3]; ++j)
            for (int64_t i = box[4 * s]; i <= box[4 * s + 1]; ++i) lst[fillp[j * res + i]++] = s;
    free(box);
    free(fillp);

    /* ray by ray: H's samples, then one Boolean per sphere that meets the ray */
    const int64_t *ob = off + (int64_t)b * (nrays + 1);
    const float *db = depth + base[b];
    const float *nb = nrm + 3 * base[b];
    const int32_t *tb = tri + base[b];
    int64_t maxlen = 0, total_cap = 0;
    for (int64_t p = 0; p < nrays; ++p) {
        int64_t len = (ob[p + 1] - ob[p]) + 2 * (cnt[p + 1] - cnt[p]) + 2;
        if ((ob[p + 1] - ob[p]) & 1) { *err = OR_EODD; }
        if (len > maxlen) maxlen = len;
        total_cap += len;
    }
    if (*err != OR_OK) { free(C); free(cnt); free(lst); return NULL; }
    oracle_bool *R = (oracle_bool *)calloc(1, sizeof(oracle_bool));
    float *bd[2], *bn[2], *cand = (float *)malloc((size_t)maxlen * sizeof(float));
    int32_t *bt[2];
    int ok = R && cand;
    for (int q = 0; q < 2; ++q) {
        bd[q] = (float *)malloc((size_t)maxlen * sizeof(float));
        bn[q] = (float *)malloc((size_t)maxlen * 3 * sizeof(float));
        bt[q] = (int32_t *)malloc((size_t)maxlen * sizeof(int32_t));
        ok = ok && bd[q] && bn[q] && bt[q];
    }
    if (ok) {
        R->nrays = nrays;
        R->offsets = (int64_t *)calloc((size_t)nrays + 1, sizeof(int64_t));
        R->depth = (float *)malloc((size_t)(total_cap > 0 ? total_cap : 1) * sizeof(float));
        R->nrm = (float *)malloc((size_t)(total_cap > 0 ? total_cap : 1) * 3 * sizeof(float));
        R->tri = (int32_t *)malloc((size_t)(total_cap > 0 ? total_cap : 1) * sizeof(int32_t));
        ok = R->offsets && R->depth && R->nrm && R->tri;
    }
    int64_t w = 0;
    for (int64_t p = 0; ok && p < nrays; ++p) {
        float pu = pixel_coord(p % res, origin[bu], h), pv = pixel_coord(p / res, origin[bv], h);
        int cur = 0;
        int64_t m = ob[p + 1] - ob[p];
        for (int64_t k = 0; k < m; ++k) {
            bd[cur][k] = db[ob[p] + k];
            for (int c = 0; c < 3; ++c) bn[cur][3 * k + c] = nb[3 * (ob[p] + k) + c];
            bt[cur][k] = tb[ob[p] + k];
        }
        for (int64_t e = cnt[p]; e < cnt[p + 1]; ++e) {
            int64_t s = lst[e];
            float sd[2], sn[6];
            int32_t st[2] = {(int32_t)s, (int32_t)s};
            if (!sphere_on_ray(C + 3 * s, b, pu, pv, r, r2, sd, sn)) continue;
            m = bool_ray(bd[cur], bn[cur], bt[cur], m, sd, sn, st, 2, op, 0.0f, bd[1 - cur], bn[1 - cur],
                         bt[1 - cur], cand);
            cur = 1 - cur;
        }
        /* small-interval removal, once */
        for (int64_t k = 0; k + 1 < m; k += 2) {
            float th = bd[cur][k + 1] - bd[cur][k];
            if (th < eps) continue;
            for (int q = 0; q < 2; ++q) {
                R->depth[w] = bd[cur][k + q];
                for (int c = 0; c < 3; ++c) R->nrm[3 * w + c] = bn[cur][3 * (k + q) + c];
                R->tri[w] = bt[cur][k + q];
                w++;
            }
        }
        R->offsets[p + 1] = w;
    }
    if (R) R->n = w;
    free(C);
    free(cnt);
    free(lst);
    free(cand);
    for (int q = 0; q < 2; ++q) { free(bd[q]); free(bn[q]); free(bt[q]); }
    if (!ok) {
        oracle_bool_free(R);
        *err = OR_ENOMEM;
        return NULL;
    }
    return R;
}
