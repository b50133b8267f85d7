"""Contouring, Steps 2 and 3 (TEST INFRASTRUCTURE ONLY): Section 5.1.
Written from the paper's description in plain NumPy/Python; shares no code
with the CUDA library.

Step 2 builds the cell edges between neighbouring grid nodes (the res^3
nodes where the three images' rays meet, Definition 3) from the samples of
the ray the edge lies on, types them by the signs of their end nodes (from
the 2-of-3 vote of Step 1) and the samples on them, and regularises them by
Rules 1 and 2.  Step 3 floods the outside nodes of every cell through its
empty edges into clusters and places one vertex per cluster at the minimum
of the quadratic error function of the Hermite data (point and normal) on
the cluster's edges.

Readings (the paper leaves these open):
  - node t of axis a sits at c_a(t) = fl32(o_a + fl32((t + 1/2) h)); the
    edge (t, t + 1) along a holds the samples of its ray with
    c_a(t) <= d < c_a(t + 1), the samples that change the parity count of
    Step 1 between its end nodes;
  - edge types: intersect (signs differ, samples), none-intersect (signs
    differ, none), empty (same sign, none), complex (same sign, samples);
  - Rule 1 keeps the first and the last sample of a complex edge with more
    than two; Rule 2 keeps, of an intersect edge's samples whose normal's
    a-component points from its inside end to its outside end, the one
    nearest the edge's midpoint (the earlier one on a tie; all samples when
    none points that way);
  - a cell's outside corners joined by empty edges form a cluster; a
    cluster takes the kept sample of each intersect edge at one of its
    corners, and of each complex edge between two outside corners the
    sample nearer each corner (a single sample goes to the nearer corner);
    complex edges between two inside corners join no cluster;
  - clusters are numbered by their lowest corner (corner index
    di + 2 dj + 4 dk); a cell yields a vertex for every cluster that meets
    an intersect, none-intersect or complex edge;
  - QEF as in dual contouring: x = m + (A^T A)^+ (A^T b - A^T A m), m the
    mean of the points, eigenvalues of A^T A below 0.01 of the largest
    (singular values below 0.1 of the largest) dropped from the inverse, all
    in FP64; a cluster without Hermite data (only none-intersect edges) is
    placed at the mean of its corner nodes and reported with no points (the
    paper smooths it after Step 4).
"""
from __future__ import annotations

import numpy as np

from .nodes import node_coords

QEF_TRUNC = 0.01  # eigenvalue ratio (0.1 in singular values)


def _coords(origin, width, res):
    return [node_coords(origin[a], width, res).astype(np.float32) for a in range(3)]


def _edge_samples(L, a, c, res, iu, iv, t):
    """Indices (into the image's arrays) of the samples on edge t of the ray
    through node indices (iu, iv) of image a."""
    p = iv * res + iu
    off = L["offsets"]
    d = np.asarray(L["depth"], np.float32)[off[p]:off[p + 1]]
    lo, hi = c[a][t], c[a][t + 1]
    k = np.nonzero((d >= lo) & (d < hi))[0]
    return [int(off[p] + x) for x in k]


def _regularise(L, a, idx, s_lo, s_hi, c, t):
    """Rules 1 and 2 on the samples idx of an edge with end signs s_lo
    (node t) and s_hi (node t + 1); returns (type, kept indices)."""
    if s_lo != s_hi:
        if not idx:
            return "none", []
        if len(idx) == 1:
            return "intersect", idx
        mid = (np.float64(c[a][t]) + np.float64(c[a][t + 1])) / 2
        want = 1.0 if s_lo else -1.0  # inside at t: the normal points to +a
        nrm = np.asarray(L["nrm"], np.float64).reshape(-1, 3)
        ok = [x for x in idx if nrm[x, a] * want > 0] or idx
        d = np.asarray(L["depth"], np.float64)
        best = min(ok, key=lambda x: (abs(d[x] - mid), d[x]))
        return "intersect", [best]
    if not idx:
        return "empty", []
    if len(idx) > 2:
        return "complex", [idx[0], idx[-1]]
    return "complex", idx


def _qef(P, N, ratios=None):
    """The QEF minimum; ratios, if a list, receives the eigenvalues of A^T A
    over the largest (how near each is to the 0.01 cut)."""
    P = np.asarray(P, np.float64)
    N = np.asarray(N, np.float64)
    m = P.mean(0)
    AtA = N.T @ N
    Atb = N.T @ np.einsum("ij,ij->i", N, P)
    lam, V = np.linalg.eigh(AtA)
    top = lam.max()
    if ratios is not None:
        ratios.extend((lam / top).tolist() if top > 0 else [0.0, 0.0, 0.0])
    inv = np.where(lam >= QEF_TRUNC * top, 1.0 / np.where(lam > 0, lam, 1.0), 0.0) if top > 0 else np.zeros(3)
    return m + V @ (inv * (V.T @ (Atb - AtA @ m)))


CORNER_OF = {(di, dj, dk): di + 2 * dj + 4 * dk for di in (0, 1) for dj in (0, 1) for dk in (0, 1)}


def cell(Ls, inside, c, res, i, j, k):
    """One cell (i, j, k): None when it yields no vertex, else a dict with
    labels (cluster per corner, -1 inside), vertices [nv, 3] (FP64) and
    points (Hermite points per vertex)."""
    s = np.zeros(8, bool)
    for (di, dj, dk), q in CORNER_OF.items():
        s[q] = inside[k + dk, j + dj, i + di]
    # the 12 edges: (axis, lower corner, upper corner, ray node indices, t)
    edges = []
    for dj in (0, 1):
        for dk in (0, 1):
            edges.append((0, CORNER_OF[0, dj, dk], CORNER_OF[1, dj, dk], j + dj, k + dk, i))
    for di in (0, 1):
        for dk in (0, 1):
            edges.append((1, CORNER_OF[di, 0, dk], CORNER_OF[di, 1, dk], k + dk, i + di, j))
    for di in (0, 1):
        for dj in (0, 1):
            edges.append((2, CORNER_OF[di, dj, 0], CORNER_OF[di, dj, 1], i + di, j + dj, k))
    typed = []
    for a, q0, q1, iu, iv, t in edges:
        idx = _edge_samples(Ls[a], a, c, res, iu, iv, t)
        ty, kept = _regularise(Ls[a], a, idx, s[q0], s[q1], c, t)
        typed.append((a, q0, q1, iu, iv, t, ty, kept))
    # flood the outside corners through empty edges (union-find)
    parent = list(range(8))

    def root(x):
        while parent[x] != x:
            x = parent[x]
        return x

    for a, q0, q1, iu, iv, t, ty, kept in typed:
        if ty == "empty" and not s[q0] and not s[q1]:
            r0, r1 = root(q0), root(q1)
            if r0 != r1:
                parent[max(r0, r1)] = min(r0, r1)
    labels = [-1] * 8
    roots = []
    for q in range(8):
        if not s[q]:
            r = root(q)
            if r not in roots:
                roots.append(r)
            labels[q] = roots.index(r)
    if not roots:
        return None
    pts = [[] for _ in roots]
    surface = [False] * len(roots)

    def point(a, x, iu, iv):
        L = Ls[a]
        P = np.zeros(3)
        P[a] = np.float64(np.float32(L["depth"][x]))
        P[(a + 1) % 3] = np.float64(c[(a + 1) % 3][iu])
        P[(a + 2) % 3] = np.float64(c[(a + 2) % 3][iv])
        return P, np.asarray(L["nrm"], np.float64).reshape(-1, 3)[x]

    for a, q0, q1, iu, iv, t, ty, kept in typed:
        if ty == "intersect":
            qo = q1 if s[q0] else q0
            surface[labels[qo]] = True
            pts[labels[qo]].append(point(a, kept[0], iu, iv))
        elif ty == "none":
            surface[labels[q1 if s[q0] else q0]] = True
        elif ty == "complex" and not s[q0]:
            surface[labels[q0]] = surface[labels[q1]] = True
            if len(kept) == 2:
                pts[labels[q0]].append(point(a, kept[0], iu, iv))
                pts[labels[q1]].append(point(a, kept[1], iu, iv))
            else:
                d = np.float64(Ls[a]["depth"][kept[0]])
                mid = (np.float64(c[a][t]) + np.float64(c[a][t + 1])) / 2
                q = q0 if d < mid else q1
                pts[labels[q]].append(point(a, kept[0], iu, iv))
    if not any(surface):
        return None
    verts, npts, rat = [], [], []
    for g in range(len(roots)):
        rat.append([])
        if pts[g]:
            P = [p for p, _ in pts[g]]
            N = [n for _, n in pts[g]]
            verts.append(_qef(P, N, rat[-1]))
        else:
            cs = [q for q in range(8) if labels[q] == g]
            verts.append(np.mean([[c[0][i + (q & 1)], c[1][j + ((q >> 1) & 1)], c[2][k + (q >> 2)]]
                                  for q in cs], axis=0).astype(np.float64))
        npts.append(len(pts[g]))
    return {"labels": labels, "vertices": np.array(verts), "points": npts, "ratios": rat}


def contour(Ls, inside, origin, width, res, cells=None):
    """Steps 2-3 over the cells (all (res-1)^3, or the listed (i, j, k)):
    {cell index i + (res-1) (j + (res-1) k): cell(...)} for the cells that
    yield a vertex.  inside: bool [k, j, i] node signs (Step 1)."""
    c = _coords(origin, width, res)
    out = {}
    n = res - 1
    it = cells if cells is not None else ((i, j, k) for k in range(n) for j in range(n) for i in range(n))
    for i, j, k in it:
        r = cell(Ls, inside, c, res, i, j, k)
        if r is not None:
            out[i + n * (j + n * k)] = r
    return out
