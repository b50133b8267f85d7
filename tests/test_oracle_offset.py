"""Offsetting oracle (Section 4.2) against what geometry fixes: the offset of
a box lies within distance r of the box and contains it, its point
membership equals "in the box, or within r of a sample" away from the
boundary, a tiny radius only lengthens every ray's own intervals by r, and
the inner offset is the mirror image of the outer one."""
import numpy as np
import pytest

import meshgen as M
import oracle

O3 = (-0.5, -0.5, -0.5)
LO, HI = np.array([-0.31, -0.22, -0.13]), np.array([0.27, 0.36, 0.19])


def _images(mesh, res):
    return [oracle.as_f32(oracle.sample(*mesh, O3, 1.0, res, a, "scan")) for a in range(3)]


def _pix(t, res):
    """Pixel-centre coordinates, FP32: fl32(o + fl32((t + 1/2) h))."""
    h = np.float32(1.0) / np.float32(res)
    return (np.float32(-0.5) + (np.asarray(t, dtype=np.float32) + np.float32(0.5)) * h).astype(np.float32)


def _centres(Ls, res):
    """Sphere centres in sample order (x-, y-, z-image, each in CSR order)."""
    out = []
    for a, L in enumerate(Ls):
        off = L["offsets"]
        p = np.repeat(np.arange(res * res), np.diff(off))
        C = np.zeros((len(p), 3))
        C[:, a] = L["depth"]
        C[:, (a + 1) % 3] = _pix(p % res, res)
        C[:, (a + 2) % 3] = _pix(p // res, res)
        out.append(C)
    return np.concatenate(out)


def _ray_points(L, b, res):
    """(pixel index, 3D point) of every sample of image b, FP64."""
    off = L["offsets"]
    p = np.repeat(np.arange(res * res), np.diff(off))
    P = np.zeros((len(p), 3))
    P[:, b] = L["depth"]
    P[:, (b + 1) % 3] = _pix(p % res, res)
    P[:, (b + 2) % 3] = _pix(p // res, res)
    return p, P


def _dist_box(P):
    d = np.maximum(np.maximum(LO - P, P - HI), 0.0)
    return np.linalg.norm(d, axis=1)


def _min_dist(P, C):
    out = np.empty(len(P))
    for k in range(0, len(P), 512):
        out[k:k + 512] = np.sqrt(((P[k:k + 512, None, :] - C[None]) ** 2).sum(-1)).min(1)
    return out


@pytest.mark.parametrize("inner", [False, True])
def test_box_offset_geometry(inner):
    res = 24
    h = 1.0 / res
    r = 2.5 * h
    H = _images(M.box(LO, HI), res)
    C = _centres(H, res)
    for b, R in enumerate(oracle.offset(H, O3, 1.0, res, r, inner=inner)):
        assert np.all(np.diff(R["offsets"]) % 2 == 0)
        p, P = _ray_points(R, b, res)
        dist = _min_dist(P, C)
        if not inner:
            # every boundary point is within r of the box, and is either on
            # the box or exactly r from its nearest sample
            assert np.all(_dist_box(P) <= r * (1 + 1e-5))
            on_sphere = np.abs(dist - r) <= 1e-5
            on_box = _dist_box(P) <= 1e-7
            assert np.all(on_sphere | on_box)
        else:
            # the inner offset's boundary points are in the box and at least
            # r from every sample (r exactly on a sphere)
            assert np.all(_dist_box(P) <= 1e-7)
            assert np.all(dist >= r * (1 - 1e-5))
        # a sphere sample carries its sphere's id and the sphere's outward
        # normal at the point (inverted in the inner offset)
        sph = R["tri"] < 0
        sid = (R["tri"][sph].view(np.uint32) & 0x7FFFFFFF).astype(np.int64)
        want_n = (P[sph] - C[sid]) / r * (-1 if inner else 1)
        assert np.abs(R["nrm"][sph] - want_n).max(initial=0) < 1e-5
        assert np.allclose(np.linalg.norm(P[sph] - C[sid], axis=1), r, rtol=1e-5)
        # point membership along every ray, away from the boundary
        off = R["offsets"]
        for q in range(0, res * res, 7):
            t = np.linspace(-0.5, 0.5, 61)
            d = R["depth"][off[q]:off[q + 1]].astype(np.float64)
            if d.size and np.min(np.abs(t[:, None] - d[None])) < 1e-4:
                t = t[np.min(np.abs(t[:, None] - d[None]), axis=1) >= 1e-4]
            X = np.zeros((len(t), 3))
            X[:, b] = t
            X[:, (b + 1) % 3] = _pix(q % res, res)
            X[:, (b + 2) % 3] = _pix(q // res, res)
            in_box = np.all((X > LO) & (X < HI), axis=1)
            near = _min_dist(X, C) < r
            want = (in_box & ~near) if inner else (in_box | near)
            got = (np.searchsorted(d, t, side="left") % 2) == 1
            ok = np.abs(_min_dist(X, C) - r) > 1e-4  # not on a sphere's surface
            assert np.array_equal(got[ok], want[ok]), (b, q)


@pytest.mark.parametrize("inner", [False, True])
def test_tiny_radius_moves_own_ray_ends(inner):
    """With r far below the distance from any sample to another image's
    rays, each sphere meets only its own ray: every interval [d0, d1] becomes
    [d0 - t, d1 + t] (inner: [d0 + t, d1 - t]) with t = sqrt(fl32(r r)), the
    ends taken from the spheres of the end samples, ids s | 2^31, normals
    along the ray pointing out of the result."""
    res = 16
    H = _images(M.box(LO, HI), res)
    r = np.float32(1e-4 / res)
    t = np.sqrt(r * r, dtype=np.float32)
    R = oracle.offset(H, O3, 1.0, res, float(r), inner=inner)
    base = np.cumsum([0] + [L["depth"].size for L in H])
    for b in range(3):
        L, G = H[b], R[b]
        assert np.array_equal(L["offsets"], G["offsets"])
        s = base[b] + np.arange(L["depth"].size)
        d = L["depth"]
        enter = np.arange(d.size) % 2 == 0
        sign = -1 if inner else 1
        want = np.where(enter, d - sign * t, d + sign * t).astype(np.float32)
        assert np.array_equal(G["depth"], want)
        assert np.array_equal(G["tri"], (s | (1 << 31)).astype(np.uint32).view(np.int32))
        na = np.float32(t / r)
        nb = np.where(enter, -na, na)  # inner: an inverted leaving (entering) sphere normal
        assert np.array_equal(G["nrm"][:, b], nb.astype(np.float32))
        assert np.all(G["nrm"][:, (b + 1) % 3] == 0) and np.all(G["nrm"][:, (b + 2) % 3] == 0)


def test_empty_solid_and_eps():
    res = 12
    empty = {"offsets": np.zeros(res * res + 1, np.int64), "depth": np.zeros(0, np.float32),
             "nrm": np.zeros((0, 3), np.float32), "tri": np.zeros(0, np.int32)}
    for R in oracle.offset([empty] * 3, O3, 1.0, res, 0.1):
        assert R["depth"].size == 0
    H = _images(M.box(LO, HI), res)
    # eps above every interval's thickness removes everything; eps = 0 nothing
    assert all(R["depth"].size == 0 for R in oracle.offset(H, O3, 1.0, res, 0.05, eps=2.0))
    R0 = oracle.offset(H, O3, 1.0, res, 0.05, eps=0.0)
    assert all(R["depth"].size > 0 for R in R0)


def test_union_then_difference_bounds():
    """H is inside its outer offset and contains its inner offset, ray by
    ray (interval containment)."""
    res = 20
    H = _images(M.icosphere(3, r=0.3, noise=0.02, seed=2), res)
    outer = oracle.offset(H, O3, 1.0, res, 0.06)
    inner = oracle.offset(H, O3, 1.0, res, 0.06, inner=True)

    def inside(L, q, x):
        d = L["depth"][L["offsets"][q]:L["offsets"][q + 1]]
        return (np.searchsorted(d, x, side="left") % 2) == 1

    x = np.linspace(-0.5, 0.5, 97)
    for b in range(3):
        for q in range(res * res):
            h_in, o_in, i_in = inside(H[b], q, x), inside(outer[b], q, x), inside(inner[b], q, x)
            assert not np.any(h_in & ~o_in)
            assert not np.any(i_in & ~h_in)


def test_tie_goes_to_earliest_sphere():
    """Two spheres whose samples on a ray coincide (centres mirrored about
    the ray, exactly representable pixel centres): the result takes the
    sample of the sphere that comes first in sample order, as the step-by-step
    union of Section 4.2 does (each step keeps the accumulated solid's sample
    at a tie, Section 4.1)."""
    res, i, j = 16, 7, 5
    h = 1.0 / res
    d0, d1 = np.float32(-0.2), np.float32(0.1)
    off = np.zeros(res * res + 1, np.int64)
    rows = [j * res + i - 1, j * res + i + 1]
    for p in rows:
        off[p + 1:] += 2
    L0 = {"offsets": off, "depth": np.array([d0, d1, d0, d1], np.float32),
          "nrm": np.tile(np.array([[-1, 0, 0], [1, 0, 0]], np.float32), (2, 1)),
          "tri": np.array([10, 11, 12, 13], np.int32)}
    empty = {"offsets": np.zeros(res * res + 1, np.int64), "depth": np.zeros(0, np.float32),
             "nrm": np.zeros((0, 3), np.float32), "tri": np.zeros(0, np.int32)}
    R = oracle.offset([L0, empty, empty], O3, 1.0, res, 1.5 * h, axes=(0,))[0]
    q = j * res + i
    got = R["tri"][R["offsets"][q]:R["offsets"][q + 1]].view(np.uint32) & 0x7FFFFFFF
    # spheres 0, 1 (ray i-1) come before 2, 3 (ray i+1); 0 and 2 coincide on
    # the ray, as do 1 and 3
    assert got.tolist() == [0, 0, 1, 1]
    dep = R["depth"][R["offsets"][q]:R["offsets"][q + 1]]
    t = np.sqrt(np.float32(1.5 * h) ** 2 - np.float32(h) ** 2, dtype=np.float32)
    assert dep[0] == np.float32(d0 - t) and dep[-1] == np.float32(d1 + t)
