"""Grid-node classification oracle (Section 5.1, Step 1) against closed
forms, an independent point-in-mesh test and the 2-of-3 rule itself."""
import numpy as np
import pytest

import meshgen as M
import oracle
from oracle import nodes

O3 = (-0.5, -0.5, -0.5)


def _images(mesh, res):
    return [oracle.as_f32(oracle.sample(*mesh, O3, 1.0, res, a, "scan")) for a in range(3)]


def _coords(res):
    c = nodes.node_coords(-0.5, 1.0, res).astype(np.float64)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    return X, Y, Z


@pytest.mark.parametrize("res", [16, 23])
def test_box_closed_form(res):
    lo, hi = np.array([-0.31, -0.22, -0.13]), np.array([0.27, 0.36, 0.19])
    got = nodes.classify(_images(M.box(lo, hi), res), O3, 1.0, res)
    X, Y, Z = _coords(res)
    ref = (X > lo[0]) & (X < hi[0]) & (Y > lo[1]) & (Y < hi[1]) & (Z > lo[2]) & (Z < hi[2])
    assert np.array_equal(got, ref)
    # every image alone agrees on a box (no silhouettes at nodes)
    for a, L in enumerate(_images(M.box(lo, hi), res)):
        assert np.array_equal(nodes.image_votes(L, a, O3, 1.0, res), ref)


def _winding(points, verts, tris):
    """Generalised winding number of a closed mesh at points (solid angles,
    Van Oosterom and Strackee), FP64: an independent inside test."""
    V = verts.astype(np.float64)[tris]  # [T, 3, 3]
    w = np.zeros(len(points))
    for n0 in range(0, len(points), 256):
        P = points[n0:n0 + 256, None, None, :]
        R = V[None] - P  # [n, T, 3, 3]
        a, b, c = R[:, :, 0], R[:, :, 1], R[:, :, 2]
        la, lb, lc = (np.linalg.norm(x, axis=-1) for x in (a, b, c))
        num = np.einsum("ntk,ntk->nt", a, np.cross(b, c))
        den = la * lb * lc + np.einsum("ntk,ntk->nt", a, b) * lc + np.einsum("ntk,ntk->nt", b, c) * la \
            + np.einsum("ntk,ntk->nt", c, a) * lb
        w[n0:n0 + 256] = (2 * np.arctan2(num, den)).sum(1) / (4 * np.pi)
    return w


@pytest.mark.parametrize("which", ["sphere", "torus"])
def test_matches_point_in_mesh(which):
    """Away from the surface (winding number within 0.05 of 0 or 1) the
    2-of-3 vote equals the inside test of the mesh itself."""
    A, B = M.pr1_pair()
    mesh = A if which == "sphere" else B
    res = 16
    got = nodes.classify(_images(mesh, res), O3, 1.0, res)
    X, Y, Z = _coords(res)
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    w = _winding(pts, *mesh).reshape(res, res, res)
    clear = (np.abs(w) < 0.05) | (np.abs(w - 1) < 0.05)
    assert clear.mean() > 0.9
    assert np.array_equal(got[clear], (w > 0.5)[clear])


def test_two_of_three_rule():
    """With one image emptied the vote follows the other two where they
    agree; with two emptied no node is inside."""
    res = 16
    L = _images(M.icosphere(6, r=0.33, noise=0.03, seed=3), res)
    empty = {"offsets": np.zeros(res * res + 1, np.int64), "depth": np.zeros(0, np.float32),
             "nrm": np.zeros((0, 3), np.float32), "tri": np.zeros(0, np.int32)}
    vy = nodes.image_votes(L[1], 1, O3, 1.0, res)
    vz = nodes.image_votes(L[2], 2, O3, 1.0, res)
    got = nodes.classify([empty, L[1], L[2]], O3, 1.0, res)
    assert np.array_equal(got, vy & vz)
    assert not nodes.classify([empty, empty, L[2]], O3, 1.0, res).any()
    full = nodes.classify(L, O3, 1.0, res)
    vx = nodes.image_votes(L[0], 0, O3, 1.0, res)
    assert np.array_equal(full, (vx & vy) | (vy & vz) | (vx & vz))


def test_node_coordinates_are_pixel_centres():
    c = nodes.node_coords(-0.5, 1.0, 8)
    assert c.dtype == np.float32
    assert np.allclose(c, -0.5 + (np.arange(8) + 0.5) / 8, atol=1e-7)
