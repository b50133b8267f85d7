"""Exact two-pass sampling with tile binning (LDNI_MODE_BINNED2) through the C
ABI: the same LDNIs as the direct traversal, bit for bit, on meshes whose
triangles cover many pixels (the regime binning is for), on the flower and
knot at their stated 512^2 size (every ray also against the oracle), on the
sub-pixel triangles of the 1.31 M-triangle sphere, on deep rays, with packed
normals, single images, ragged resolutions and an empty mesh."""
import numpy as np
import pytest

import meshgen as M
import oracle
from ldni_compare import compare_ldni

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

O3 = (-0.5, -0.5, -0.5)
DIAG = 3 ** 0.5


@pytest.fixture(scope="module")
def ldni():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1009_0794_gb300 as pkg
    pkg._lib.load()
    return pkg


def _same(ldni, mesh, res, axis="all", packed=False, origin=O3, width=1.0):
    grid = ldni.Grid.cube(origin, width, res)
    a = ldni.sample(*mesh, grid, axis, packed=packed)
    b = ldni.sample(*mesh, grid, axis, mode="binned2", packed=packed)
    a = a if isinstance(a, list) else [a]
    b = b if isinstance(b, list) else [b]
    for x, y in zip(a, b):
        assert ldni.identical(x, y), x.axis
    return b


@pytest.mark.parametrize("res", [128, 77, 300])
def test_pr1_meshes(ldni, res):
    A, B = M.pr1_pair()
    _same(ldni, A, res)
    _same(ldni, B, res)


def test_big_triangles_and_closed_forms(ldni):
    """Boxes and octahedra whose faces span many tiles (some beyond four:
    the big-triangle path), vertices on pixel centres, a shifted cube."""
    _same(ldni, M.box([-0.31, -0.22, -0.13], [0.27, 0.36, 0.19]), 64)
    _same(ldni, M.box([-0.31, -0.22, -0.13], [0.27, 0.36, 0.19]), 512)
    res = 32
    h = 1.0 / res
    cc = -0.5 + 16.5 * h  # a pixel centre: vertices and edges on pixel centres (the top-left rule decides)
    _same(ldni, M.octahedron([cc, cc, cc], 11 * h), res)
    v, t = M.icosphere(3, r=0.3, noise=0.02, seed=8)
    v2 = (v.astype(np.float64) * 3.0 + np.array([10.0, -4.0, 2.5])).astype(np.float32)
    _same(ldni, (v2, t), 203, origin=(8.7, -5.3, 1.2), width=2.6)


def test_flower_and_knot_at_512(ldni):
    grid_res = 512
    fl = M.flower(512, 512)
    kn = M.torus_knot(2, 3, 0.25, 0.1, 0.035, 256, 32)
    for mesh in (fl, kn):
        got = _same(ldni, mesh, grid_res)
        for a in range(3):
            ref = oracle.sample(*mesh, O3, 1.0, grid_res, a, "scan")
            compare_ldni(got[a].numpy(), ref, DIAG)


def test_tiny_triangles_and_deep_rays(ldni):
    _same(ldni, M.scale_sphere(), 1024)
    _same(ldni, M.slab_stack(60, axis=0, seed=1), 40)
    _same(ldni, M.slab_stack(60, axis=2, seed=2), 40)


def test_packed_single_axis_and_empty(ldni):
    A, _ = M.pr1_pair()
    _same(ldni, A, 128, packed=True)
    for axis in (0, 1, 2):
        _same(ldni, A, 96, axis=axis)
    grid = ldni.Grid.cube(O3, 1.0, 64)
    E = ldni.sample(np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32), grid, "all", mode="binned2")
    assert all(L.n == 0 for L in E)


def test_plan_capacity_overflow_flagged(ldni):
    A, _ = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, 64)
    caps = [L.n for L in ldni.sample(*A, grid, "all")]
    vt, tt = torch.from_numpy(A[0]).cuda(), torch.from_numpy(A[1]).cuda()
    plan = ldni.SamplePlan(len(A[0]), len(A[1]), grid, [c // 2 for c in caps], mode="binned2")
    plan.run(vt, tt)
    with pytest.raises(ldni.LDNIError):
        plan.finish()
    plan = ldni.SamplePlan(len(A[0]), len(A[1]), grid, caps, mode="binned2")
    plan.run(vt, tt)
    outs = plan.finish()
    ref = ldni.sample(*A, grid, "all")
    assert all(ldni.identical(x, y) for x, y in zip(outs, ref))


def test_tuner_picks_a_traversal(ldni, tmp_path, monkeypatch):
    """The tuner times both traversals of a mesh and returns the faster; the
    choice is cached, and sampling with it gives the same bits."""
    from paper_1009_0794_gb300 import tune
    monkeypatch.setenv(tune.CACHE_ENV, str(tmp_path / "tune.json"))
    A, _ = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, 128)
    r = tune.choose_sampling_mode(*A, grid, reps=3)
    assert r["mode"] in ("exact2", "binned2") and not r["cached"]
    assert r["ms"][r["mode"]] == min(r["ms"].values())
    again = tune.choose_sampling_mode(*A, grid)
    assert again["cached"] and again["mode"] == r["mode"]
    got = ldni.sample(*A, grid, "all", mode=r["mode"])
    ref = ldni.sample(*A, grid, "all")
    assert all(ldni.identical(x, y) for x, y in zip(got, ref))
