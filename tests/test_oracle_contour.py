"""Contouring oracle, Steps 2-3 (Section 5.1) against closed forms: the QEF
of one, two and three planes, Rules 1 and 2 on hand-made edges, the vertex
positions of a box (corners, edges, faces exactly), a slab thinner than a
cell (two vertices, one on each face: the thin-structure case), and the
distance of a sphere's vertices to the sphere."""
import numpy as np
import pytest

import meshgen as M
import oracle
from oracle import contour as C
from oracle import nodes

O3 = (-0.5, -0.5, -0.5)


def _solid(mesh, res):
    Ls = [oracle.as_f32(oracle.sample(*mesh, O3, 1.0, res, a, "scan")) for a in range(3)]
    return Ls, nodes.classify(Ls, O3, 1.0, res)


def test_qef_planes():
    p = np.array([0.1, -0.2, 0.3])
    e = np.eye(3)
    # three planes through p (each given by a point of its own) meet at p
    assert np.allclose(C._qef([p + [0, 5, 7], p + [3, 0, 1], p + [1, 2, 0]], e), p, atol=1e-12)
    # two planes: the point of their line nearest the points' mean
    P = [p + [0, 0.5, 0], p + [0.4, 0, 0]]
    x = C._qef(P, [[1, 0, 0], [0, 0, 1]])
    assert np.allclose(x, [p[0], np.mean([q[1] for q in P]), p[2]], atol=1e-12)
    # one plane: the mean projected onto it
    x = C._qef([p, p + [0, 1, 1]], [[1, 0, 0], [1, 0, 0]])
    assert np.allclose(x, [p[0], p[1] + 0.5, p[2] + 0.5], atol=1e-12)
    # nearly parallel planes: the weak direction (singular value below 0.1 of
    # the largest) keeps the mean's coordinate; without the cut the vertex
    # would run off to the planes' intersection at y = p_y + 3
    x = C._qef([p, p, p + [0, 3, 0]], [[1, 0, 0], [1, 0, 0], [0.999, 0.0447, 0]])
    assert abs(x[1] - (p[1] + 1.0)) < 0.01


def test_rules_on_hand_made_edges():
    c = [np.array([0.0, 1.0], np.float32)] * 3
    L = {"offsets": np.array([0, 4]), "depth": np.array([0.1, 0.3, 0.55, 0.9], np.float32),
         "nrm": np.array([[1, 0, 0], [-1, 0, 0], [1, 0, 0], [-1, 0, 0]], np.float32)}
    idx = [0, 1, 2, 3]
    # Rule 1: a complex edge keeps its first and last samples
    assert C._regularise(L, 0, idx, False, False, c, 0) == ("complex", [0, 3])
    # Rule 2: inside at the lower node -> normals along +x; nearest the midpoint 0.5
    assert C._regularise(L, 0, idx, True, False, c, 0) == ("intersect", [2])
    # inside at the upper node -> normals along -x: 0.3 (0.2 away) beats 0.9 (0.4 away)
    assert C._regularise(L, 0, idx, False, True, c, 0) == ("intersect", [1])
    assert C._regularise(L, 0, [], False, True, c, 0) == ("none", [])
    assert C._regularise(L, 0, [], True, True, c, 0) == ("empty", [])


def test_box_vertices_exact():
    res = 16
    lo, hi = np.array([-0.31, -0.22, -0.13]), np.array([0.27, 0.36, 0.19])
    Ls, ins = _solid(M.box(lo, hi), res)
    out = C.contour(Ls, ins, O3, 1.0, res)
    assert out
    c = nodes.node_coords(-0.5, 1.0, res).astype(np.float64)
    for idx, r in out.items():
        assert len(r["vertices"]) == 1 and r["points"][0] > 0
        v = r["vertices"][0]
        i, j, k = idx % 15, (idx // 15) % 15, idx // 225
        cube_lo = np.array([c[i], c[j], c[k]])
        # which box planes cross this cell
        on = [(a, w) for a in range(3) for w in (lo[a], hi[a]) if cube_lo[a] <= w < cube_lo[a] + 1.0 / res]
        assert on
        for a, w in on:
            assert abs(v[a] - np.float32(w)) < 1e-6, (idx, a)


def test_thin_slab_two_vertices():
    """A slab 0.3 cells thick between two node planes: the cells it passes
    through have outside corners on both sides, joined by no empty edge,
    and get one vertex on each face (Figure 7's thin structure)."""
    res = 16
    h = 1.0 / res
    c = nodes.node_coords(-0.5, 1.0, res).astype(np.float64)
    x0 = c[7] + 0.35 * h
    x1 = x0 + 0.3 * h
    Ls, ins = _solid(M.box([x0, -0.3, -0.25], [x1, 0.3, 0.25]), res)
    assert not ins.any()  # no node inside: Step 1 alone loses the slab
    out = C.contour(Ls, ins, O3, 1.0, res)
    interior = [r for idx, r in out.items() if idx % 15 == 7 and 3 <= (idx // 15) % 15 <= 11
                and 4 <= idx // 225 <= 10]
    assert interior
    for r in interior:
        assert len(r["vertices"]) == 2 and r["points"] == [4, 4]
        # cluster 0 holds the corners below the slab, cluster 1 those above
        assert r["labels"] == [0, 1, 0, 1, 0, 1, 0, 1]
        assert abs(r["vertices"][0][0] - np.float32(x0)) < 1e-6
        assert abs(r["vertices"][1][0] - np.float32(x1)) < 1e-6


def test_sphere_vertices_near_surface():
    res = 20
    r0 = 0.3
    Ls, ins = _solid(M.icosphere(8, r=r0), res)
    out = C.contour(Ls, ins, O3, 1.0, res)
    V = np.concatenate([r["vertices"] for r in out.values()])
    dist = np.abs(np.linalg.norm(V, axis=1) - r0)
    assert dist.max() < 0.5 / res  # within half a cell of the (inscribed) sphere
    # every cell yields one vertex here (no thin parts)
    assert all(len(r["vertices"]) == 1 for r in out.values())
