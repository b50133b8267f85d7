"""Contouring Steps 2-3 (ldni_contour_cells, Section 5.1) through the C ABI
against the oracle.

Inputs are the oracle's samplings rounded to FP32 and the oracle's node
signs, uploaded as they are.  The set of cells, their vertex counts, corner
labels and Hermite point counts agree exactly; vertex positions (FP64 QEF,
stored in FP32) within 2e-6 of the cube, except where an eigenvalue ratio of
the oracle's QEF lies within 1e-6 of the 0.01 cut (none so far).
"""
import numpy as np
import pytest

import meshgen as M
import oracle
from oracle import contour as C
from oracle import nodes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

O3 = (-0.5, -0.5, -0.5)


@pytest.fixture(scope="module")
def ldni():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1009_0794_gb300 as pkg
    pkg._lib.load()
    return pkg


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _upload(ldni, grid, a, L):
    nrm = np.asarray(L["nrm"], np.float32).reshape(-1, 3)
    return ldni.LDNI(grid, a, _t(np.asarray(L["offsets"], np.int32)), _t(np.asarray(L["depth"], np.float32)),
                     _t(nrm[:, 0]), _t(nrm[:, 1]), _t(nrm[:, 2]), _t(np.asarray(L["tri"], np.int32)),
                     int(L["offsets"][-1]))


def _bits(inside):
    """bool [k, j, i] -> uint32 words [k][j][ceil(res / 32)], bit i % 32."""
    res = inside.shape[2]
    W = (res + 31) // 32
    pad = np.zeros(inside.shape[:2] + (W * 32,), bool)
    pad[:, :, :res] = inside
    return np.packbits(pad, axis=2, bitorder="little").view(np.uint32)


def _compare(ldni, mesh, res, origin=O3, width=1.0):
    grid = ldni.Grid.cube(origin, width, res)
    ref = [oracle.as_f32(oracle.sample(*mesh, origin, width, res, a, "scan")) for a in range(3)]
    ins = nodes.classify(ref, origin, width, res)
    H = [_upload(ldni, grid, a, L) for a, L in enumerate(ref)]
    got = ldni.contour_cells(H, inside=_t(_bits(ins).view(np.int32)))
    want = C.contour(ref, ins, origin, width, res)
    keys = sorted(want)
    assert got["cell"].tolist() == keys
    for rec, key in zip(got, keys):
        w = want[key]
        nv = len(w["vertices"])
        assert rec["nvert"] == nv, key
        lab = [(int(rec["labels"]) >> (4 * c)) & 15 for c in range(8)]
        assert lab == [15 if x < 0 else x for x in w["labels"]], key
        assert [(int(rec["npts"]) >> (8 * g)) & 255 for g in range(nv)] == w["points"], key
        near_cut = any(abs(r - C.QEF_TRUNC) < 1e-6 for rs in w["ratios"] for r in rs)
        if not near_cut:
            assert np.abs(rec["v"][:nv] - w["vertices"]).max() <= 2e-6 * width, key
    return got, want


def test_box_and_sphere(ldni):
    _compare(ldni, M.box([-0.31, -0.22, -0.13], [0.27, 0.36, 0.19]), 16)
    _compare(ldni, M.box([-0.31, -0.22, -0.13], [0.27, 0.36, 0.19]), 21)
    _compare(ldni, M.pr1_pair()[0], 24)


def test_thin_structures_and_multilayer(ldni):
    """A slab thinner than a cell (two vertices per cell), flower petals and
    knot strands (many samples per edge, Rules 1 and 2)."""
    res = 16
    c = nodes.node_coords(-0.5, 1.0, res).astype(np.float64)
    x0 = c[7] + 0.35 / res
    got, _ = _compare(ldni, M.box([x0, -0.3, -0.25], [x0 + 0.3 / res, 0.3, 0.25]), res)
    assert (got["nvert"] == 2).sum() > 0
    _compare(ldni, M.flower(64, 64), 28)
    _compare(ldni, M.torus_knot(n_ring=128, n_side=16), 30)


def test_offset_grid_and_pr1_torus(ldni):
    v, t = M.icosphere(6, r=0.3, noise=0.02, seed=8)
    v2 = (v.astype(np.float64) * 3.0 + np.array([10.0, -4.0, 2.5])).astype(np.float32)
    _compare(ldni, (v2, t), 19, origin=(8.7, -5.3, 1.2), width=2.6)
    _compare(ldni, M.pr1_pair()[1], 26)


def test_inside_from_classify_nodes(ldni):
    """The same result when the node signs come from ldni_classify_nodes."""
    A = M.pr1_pair()[0]
    res = 24
    grid = ldni.Grid.cube(O3, 1.0, res)
    ref = [oracle.as_f32(oracle.sample(*A, O3, 1.0, res, a, "scan")) for a in range(3)]
    H = [_upload(ldni, grid, a, L) for a, L in enumerate(ref)]
    ins = nodes.classify(ref, O3, 1.0, res)
    a = ldni.contour_cells(H, inside=_t(_bits(ins).view(np.int32)))
    b = ldni.contour_cells(H)
    assert a.tobytes() == b.tobytes()
