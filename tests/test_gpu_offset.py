"""Offsetting by sphere unions (ldni_offset, Section 4.2) through the C ABI
against the step-by-step oracle.

The input LDNIs are the oracle's samplings rounded to FP32 (the storage
precision), uploaded as they are; the sphere samples are single-precision
functions of those inputs, so the results agree bit for bit: counts, depths,
normals and ids (sphere s | 2^31).
"""
import numpy as np
import pytest

import meshgen as M
import oracle
from ldni_compare import bit_equal

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


def _upload(ldni, grid, a, L):
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    nrm = np.asarray(L["nrm"], np.float32).reshape(-1, 3)
    return ldni.LDNI(grid, a, t(np.asarray(L["offsets"], np.int32)), t(np.asarray(L["depth"], np.float32)),
                     t(nrm[:, 0]), t(nrm[:, 1]), t(nrm[:, 2]), t(np.asarray(L["tri"], np.int32)),
                     int(L["offsets"][-1]))


def _solid(ldni, mesh, res, origin=O3, width=1.0):
    grid = ldni.Grid.cube(origin, width, res)
    ref = [oracle.as_f32(oracle.sample(*mesh, origin, width, res, a, "scan")) for a in range(3)]
    return grid, ref, [_upload(ldni, grid, a, L) for a, L in enumerate(ref)]


def _check(ldni, grid, ref, H, r, inner, eps=0.0, **kw):
    got = ldni.offset(H, r, inner=inner, eps=eps, **kw)
    want = oracle.offset(ref, grid.origin, grid.width, grid.res, r, inner=inner, eps=eps)
    for a in range(3):
        g = got[a].numpy()
        assert got[a].n == int(want[a]["offsets"][-1]), a
        assert bit_equal(g, want[a]), a
    return got


@pytest.mark.parametrize("inner", [False, True])
@pytest.mark.parametrize("rpix", [1.5, 3.0])
def test_pr1_parity(ldni, inner, rpix):
    A, B = M.pr1_pair()
    res = 48
    for mesh in (A, B):
        grid, ref, H = _solid(ldni, mesh, res)
        _check(ldni, grid, ref, H, rpix / res, inner)


def test_box_ragged_resolution_and_eps(ldni):
    """A box at a resolution that is no multiple of the 8-pixel tiles, with
    and without small-interval removal."""
    grid, ref, H = _solid(ldni, M.box([-0.31, -0.22, -0.13], [0.27, 0.36, 0.19]), 37)
    for eps in (0.0, 0.02):
        _check(ldni, grid, ref, H, 2.2 / 37, False, eps=eps)
        _check(ldni, grid, ref, H, 2.2 / 37, True, eps=eps)


def test_multilayer_and_offset_grid(ldni):
    """Many layers per ray (flower petals, knot strands), a non-unit cube
    with a shifted origin, spheres reaching past the cube."""
    for mesh, res in ((M.flower(48, 48), 40), (M.torus_knot(n_ring=96, n_side=12), 44)):
        grid, ref, H = _solid(ldni, mesh, res)
        _check(ldni, grid, ref, H, 2.0 / res, False)
        _check(ldni, grid, ref, H, 2.0 / res, True)
    v, t = M.icosphere(4, r=0.3, noise=0.02, seed=8)
    v2 = (v.astype(np.float64) * 3.0 + np.array([10.0, -4.0, 2.5])).astype(np.float32)
    grid, ref, H = _solid(ldni, (v2, t), 33, origin=(8.7, -5.3, 1.2), width=2.6)
    _check(ldni, grid, ref, H, 0.2, False)


def test_empty_solid_and_capacity_retry(ldni):
    res = 24
    grid = ldni.Grid.cube(O3, 1.0, res)
    empty = {"offsets": np.zeros(res * res + 1, np.int64), "depth": np.zeros(0, np.float32),
             "nrm": np.zeros((0, 3), np.float32), "tri": np.zeros(0, np.int32)}
    H = [_upload(ldni, grid, a, empty) for a in range(3)]
    for inner in (False, True):
        out = ldni.offset(H, 0.1, inner=inner)
        assert all(L.n == 0 for L in out)
    # a first capacity far too small: one retry with the exact sizes
    grid, ref, H = _solid(ldni, M.pr1_pair()[0], 32)
    _check(ldni, grid, ref, H, 2.0 / 32, False, capacity=1)


def test_large_radius_and_deep_rays(ldni):
    """A radius of a third of the cube (hundreds of spheres on every ray,
    merged 64 at a time) agrees with the oracle; a solid whose rays hold more
    samples than one warp orders is reported instead of answered wrongly."""
    grid, ref, H = _solid(ldni, M.box([-0.31, -0.22, -0.13], [0.27, 0.36, 0.19]), 24)
    _check(ldni, grid, ref, H, 0.3, False)
    _check(ldni, grid, ref, H, 0.1, True)
    grid, ref, H = _solid(ldni, M.slab_stack(200, axis=0, seed=1), 16)
    assert max(np.diff(ref[0]["offsets"])) > 384
    with pytest.raises(ldni.LDNIError):
        ldni.offset(H, 0.5 / 16)


def test_table4_style_flower_sizes(ldni):
    """Offsets of the flower at 128^2 (the resolution of the paper's
    offsetting examples, Table 4) by +-2.5 and +-5 pixels, every ray against
    the oracle."""
    res = 128
    grid, ref, H = _solid(ldni, M.flower(128, 128), res)
    for rpix in (2.5, 5.0):
        for inner in (False, True):
            got = ldni.offset(H, rpix / res, inner=inner)
            want = oracle.offset(ref, O3, 1.0, res, rpix / res, inner=inner)
            for a in range(3):
                assert bit_equal(got[a].numpy(), want[a]), (rpix, inner, a)
