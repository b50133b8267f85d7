"""Pins of the sampling oracle against facts fixed by the paper and by
geometry, independent of the oracle's own code.

Definitions 1-4 and Remark 1 (Section 2); pixel-centre rays (Section 3).
"""
from fractions import Fraction

import numpy as np
import pytest

import meshgen as M
import oracle

O3 = [-0.5, -0.5, -0.5]


def uv_axes(axis):
    return (axis + 1) % 3, (axis + 2) % 3


def centres(res, width=1.0, o=-0.5):
    return o + (np.arange(res) + 0.5) * (width / res)


# ---------------------------------------------------------------- box ----
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_box_closed_form(axis):
    """Axis-aligned box with faces between pixel centres: every ray whose
    centre projects inside crosses exactly two faces, at the face
    coordinates, with normals -e_a then +e_a; no other ray crosses."""
    lo = np.array([-0.3, -0.2, -0.1])
    hi = np.array([0.2, 0.3, 0.4])
    v, t = M.box(lo, hi)
    res = 32
    L = oracle.sample(v, t, O3, 1.0, res, axis, "scan")
    iu, iv = uv_axes(axis)
    c = centres(res)
    inu = (c > lo[iu]) & (c < hi[iu])
    inv = (c > lo[iv]) & (c < hi[iv])
    expect = (inv[:, None] & inu[None, :]).astype(np.int64).reshape(-1) * 2  # row p = j*res + i
    counts = np.diff(L["offsets"])
    assert np.array_equal(counts, expect)
    d = L["depth"].reshape(-1, 2)
    assert np.allclose(d[:, 0], np.float32(lo[axis]), rtol=0, atol=1e-12)
    assert np.allclose(d[:, 1], np.float32(hi[axis]), rtol=0, atol=1e-12)
    n = L["nrm"].reshape(-1, 2, 3)
    e = np.zeros(3)
    e[axis] = 1.0
    assert np.array_equal(n[:, 0], np.tile(-e, (n.shape[0], 1)))
    assert np.array_equal(n[:, 1], np.tile(e, (n.shape[0], 1)))
    vol = oracle.volume(oracle.as_f32(L), 1.0 / res)
    ext = float(np.float32(hi[axis])) - float(np.float32(lo[axis]))
    assert vol == pytest.approx(expect.sum() / 2 * ext / res**2, rel=1e-14)


# --------------------------------------------------------- octahedron ----
def _perturbed_inside(di, dj, c):
    """Is (di - eps, dj - eps^2) inside the open diamond |x| + |y| < c for
    infinitesimal eps > 0?  (The top-left rule is exactly coverage at this
    symbolically shifted point.)"""
    s = abs(di) + abs(dj) - c
    if s != 0:
        return s < 0
    # first-order term in eps: d|di - eps| = -sign(di) (or +1 at di == 0)
    t1 = -np.sign(di) if di != 0 else 1
    if t1 != 0:
        return t1 < 0
    return False


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_octahedron_on_pixel_centres(axis):
    """Octahedron whose vertices and edges pass exactly through pixel
    centres.  Shared non-silhouette edges are crossed once per face pair and
    silhouette edges 0 or 2 times (Remark 1); the count map is the coverage of
    the projected diamond at the perturbed point, derived here by hand; depths
    are the analytic face planes."""
    res = 32
    h = 1.0 / res
    ci = 16
    cc = -0.5 + (ci + 0.5) * h
    c_pix = 8
    v, t = M.octahedron([cc, cc, cc], c_pix * h)
    L = oracle.sample(v, t, O3, 1.0, res, axis, "brute")
    counts = np.diff(L["offsets"]).reshape(res, res)  # [j, i]
    for j in range(res):
        for i in range(res):
            inside = _perturbed_inside(i - ci, j - ci, c_pix)
            assert counts[j, i] == (2 if inside else 0), (i, j)
    off = L["offsets"]
    for j in range(res):
        for i in range(res):
            p = j * res + i
            if counts[j, i] == 0:
                continue
            half = (c_pix - abs(i - ci) - abs(j - ci)) * h
            d = L["depth"][off[p]:off[p + 1]]
            assert d[0] == pytest.approx(cc - half, abs=1e-12)
            assert d[1] == pytest.approx(cc + half, abs=1e-12)


# -------------------------------------------------------- tetrahedron ----
def test_tetrahedron_depth_is_ray_plane_intersection():
    """Vertices on the fixed-point lattice (snap is exact), so each crossing
    depth must equal the exact ray-plane intersection of its face."""
    rng = np.random.default_rng(5)
    res = 16
    unit = 1.0 / (res * 256)
    for trial in range(6):
        pts = rng.integers(-1500, 1500, size=(4, 3)) * unit
        if abs(np.linalg.det(np.c_[pts[1:] - pts[0]])) < 1e-3:
            continue
        v, t = M.tetrahedron(pts)
        for axis in range(3):
            L = oracle.sample(v, t, O3, 1.0, res, axis, "brute")
            iu, iv = uv_axes(axis)
            off = L["offsets"]
            c = centres(res)
            for p in np.nonzero(np.diff(off))[0]:
                j, i = divmod(p, res)
                for k in range(off[p], off[p + 1]):
                    tri = t[L["tri"][k]].astype(np.int64)
                    P = v[tri].astype(np.float64)
                    nrm = np.cross(P[1] - P[0], P[2] - P[0])
                    # plane: nrm . (x - P0) = 0, solve for x_axis at (u, v)
                    x = np.zeros(3)
                    x[iu], x[iv] = c[i], c[j]
                    rest = nrm[iu] * (x[iu] - P[0, iu]) + nrm[iv] * (x[iv] - P[0, iv])
                    da = P[0, axis] - rest / nrm[axis]
                    assert L["depth"][k] == pytest.approx(da, abs=1e-12)
                    assert np.allclose(L["nrm"][k], nrm / np.linalg.norm(nrm), atol=1e-12)


# ------------------------------------------------ brute force == scan ----
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_scan_equals_brute_force(seed):
    meshes = [M.icosphere(2, r=0.3, noise=0.05, seed=seed),
              M.torus(0.25, 0.1, 8, 4, center=(0.05 * seed, 0, 0)),
              M.box([-0.25, -0.125, -0.3], [0.25, 0.375, 0.0625])]
    for v, t in meshes:
        for axis in range(3):
            for res in (7, 16, 32):
                B = oracle.sample(v, t, O3, 1.0, res, axis, "brute")
                S = oracle.sample(v, t, O3, 1.0, res, axis, "scan")
                assert np.array_equal(B["offsets"], S["offsets"])
                assert np.array_equal(B["tri"], S["tri"])
                assert np.array_equal(B["depth"], S["depth"])
                assert np.array_equal(B["nrm"], S["nrm"])


# ------------------------------------------------------ even counts ----
def test_even_counts_and_alternating_normals_pr1():
    """Definition 4: closed meshes give even counts on every ray; the sorted
    samples alternate entering (n_a < 0) and leaving (n_a > 0) faces, because
    odd-to-even ranges are inside."""
    A, B = M.pr1_pair()
    for mesh in (A, B):
        for axis in range(3):
            L = oracle.sample(*mesh, O3, 1.0, 128, axis, "scan")
            cnt = np.diff(L["offsets"])
            assert np.all(cnt % 2 == 0)
            assert cnt.sum() > 0
            k = np.arange(L["depth"].size) - np.repeat(L["offsets"][:-1], cnt)
            na = L["nrm"][:, axis]
            assert np.all(na[k % 2 == 0] < 0)
            assert np.all(na[k % 2 == 1] > 0)


# ------------------------------------------------------ sagitta bound ----
def test_icosphere_crossings_between_inscribed_and_circumscribed():
    """Crossings of a noise-free geodesic sphere of radius r lie between the
    smallest face-plane distance and r (up to the fixed-point snap shift of
    at most h/512 per in-plane coordinate); normals point outward."""
    r = 0.35
    v, t = M.icosphere(6, r=r)
    P = v[t].astype(np.float64)
    nrm = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r_in = np.min(np.einsum("ij,ij->i", nrm, P[:, 0]))
    res = 64
    h = 1.0 / res
    slack = 2 * np.sqrt(2) * h / 512
    c = centres(res)
    for axis in range(3):
        L = oracle.sample(v, t, O3, 1.0, res, axis, "scan")
        iu, iv = uv_axes(axis)
        cnt = np.diff(L["offsets"])
        p = np.repeat(np.arange(res * res), cnt)
        j, i = np.divmod(p, res)
        X = np.zeros((p.size, 3))
        X[:, iu], X[:, iv], X[:, axis] = c[i], c[j], L["depth"]
        rad = np.linalg.norm(X, axis=1)
        assert np.all(rad <= r + slack) and np.all(rad >= r_in - slack)
        assert np.all(np.einsum("ij,ij->i", L["nrm"], X) > 0)
        assert set(np.unique(cnt)) <= {0, 2}


# ------------------------------------------- exact unsnapped predicate ----
def _exact_inside(P, cu, cv):
    """Top-left coverage on exact rationals (no snapping)."""
    (u0, v0), (u1, v1), (u2, v2) = P
    A2 = (u1 - u0) * (v2 - v0) - (v1 - v0) * (u2 - u0)
    if A2 == 0:
        return False, None
    if A2 < 0:
        P = [P[0], P[2], P[1]]
    E = []
    for k in range(3):
        (au, av), (bu, bv) = P[k], P[(k + 1) % 3]
        du, dv = bu - au, bv - av
        e = du * (cv - av) - dv * (cu - au)
        if e < 0 or (e == 0 and not (dv > 0 or (dv == 0 and du < 0))):
            return False, None
        E.append((e, (du * du + dv * dv)))
    dist = min(float(abs(e)) / float(ln) ** 0.5 for e, ln in E)
    return True, dist


def test_snapped_predicate_agrees_with_exact_except_near_edges():
    """Snapping moves projected vertices by at most half a fixed-point unit
    (h/512 per coordinate), so the snapped and exact predicates may disagree
    only for rays within that distance of a triangle edge."""
    rng = np.random.default_rng(9)
    v, t = M.icosphere(3, r=0.3, noise=0.05, seed=4)
    res = 24
    h = Fraction(1, res)
    bound = 1.5 * np.sqrt(2) / (512 * res)
    for axis in range(3):
        iu, iv = uv_axes(axis)
        L = oracle.sample(v, t, O3, 1.0, res, axis, "brute")
        got = set()
        for p in range(res * res):
            for k in range(L["offsets"][p], L["offsets"][p + 1]):
                got.add((p, int(L["tri"][k])))
        for ti, tri in enumerate(t):
            P = [(Fraction(float(v[q, iu])), Fraction(float(v[q, iv]))) for q in tri]
            umin = min(x[0] for x in P)
            umax = max(x[0] for x in P)
            vmin = min(x[1] for x in P)
            vmax = max(x[1] for x in P)
            for j in range(res):
                cv = Fraction(-1, 2) + (j + Fraction(1, 2)) * h
                if cv < vmin - h or cv > vmax + h:
                    continue
                for i in range(res):
                    cu = Fraction(-1, 2) + (i + Fraction(1, 2)) * h
                    if cu < umin - h or cu > umax + h:
                        continue
                    ins, dist = _exact_inside(P, cu, cv)
                    key = (j * res + i, ti)
                    if ins != (key in got):
                        if ins:
                            assert dist <= bound, (axis, key, dist)
                        else:
                            # recompute the distance to the nearest edge line
                            dmin = min(
                                abs(float((P[(k + 1) % 3][0] - P[k][0]) * (cv - P[k][1])
                                          - (P[(k + 1) % 3][1] - P[k][1]) * (cu - P[k][0])))
                                / float((P[(k + 1) % 3][0] - P[k][0]) ** 2 + (P[(k + 1) % 3][1] - P[k][1]) ** 2) ** 0.5
                                for k in range(3))
                            assert dmin <= bound, (axis, key, dmin)
        _ = rng


# ---------------------------------------------------------- volume ----
def test_volume_converges_to_mesh_volume():
    """The LDNI volume (odd-to-even ranges inside) tends to the exact mesh
    volume (divergence theorem) as the resolution grows, on every axis, and
    the three axes agree with each other ever more closely."""
    A, _ = M.pr1_pair()
    vm = M.signed_volume(*A)
    errs = []
    for res in (32, 64, 128, 256, 512):
        vs = []
        for axis in range(3):
            L = oracle.sample(*A, O3, 1.0, res, axis, "scan")
            vs.append(oracle.volume(oracle.as_f32(L), 1.0 / res))
        errs.append(max(abs(x - vm) for x in vs))
    assert errs[-1] < 2e-4 * vm
    assert errs[-1] < errs[0] / 8


def test_parallel_faces_excluded():
    """Faces parallel to the ray are not sampled (Definition 1 note): the box
    side faces are parallel to the view axis and contribute no samples even
    for rays lying in their planes."""
    res = 16
    h = 1.0 / res
    lo = -0.5 + 4.5 * h
    hi = -0.5 + 9.5 * h  # side faces pass exactly through pixel centres
    v, t = M.box([lo, lo, -0.2], [hi, hi, 0.3])
    L = oracle.sample(v, t, O3, 1.0, res, 2, "brute")
    ids = set(L["tri"].tolist())
    P = v[t].astype(np.float64)
    nz = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])[:, 2]
    assert all(abs(nz[i]) > 0 for i in ids)
    assert np.all(np.diff(L["offsets"]) % 2 == 0)
