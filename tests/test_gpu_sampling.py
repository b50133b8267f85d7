"""CUDA sampling through the C ABI against the FP64 oracle (Definitions 1-4,
Remark 1, Section 3).  Counts and triangle ids bit-exact, depths within
1e-5 of the cube diagonal, normals within 1e-5."""
import ctypes

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


def _check_all_axes(ldni, mesh, res, origin=O3, width=1.0):
    v, t = mesh
    grid = ldni.Grid.cube(origin, width, res)
    got = ldni.sample(v, t, grid, "all", check_odd=True)
    stats = []
    for a in range(3):
        ref = oracle.sample(v, t, grid.origin, grid.width, res, a, "scan")
        stats.append(compare_ldni(got[a].numpy(), ref, DIAG * grid.width))
    return got, stats


@pytest.mark.parametrize("res", [128, 100, 37])
def test_pr1_parity(ldni, res):
    A, B = M.pr1_pair()
    for mesh in (A, B):
        _check_all_axes(ldni, mesh, res)


def test_single_axis_calls_match_fused(ldni):
    A, _ = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, 96)
    fused = ldni.sample(*A, grid, "all")
    for a in range(3):
        one = ldni.sample(*A, grid, a).numpy()
        ref = oracle.sample(*A, grid.origin, 1.0, 96, a, "scan")
        compare_ldni(one, ref, DIAG)
        assert np.array_equal(one["offsets"], fused[a].numpy()["offsets"])


def test_octahedron_on_pixel_centres(ldni):
    """Edges and vertices exactly on ray lattice points (Remark 1)."""
    res = 64
    h = 1.0 / res
    cc = -0.5 + 32.5 * h
    mesh = M.octahedron([cc, cc, cc], 11 * h)
    got, _ = _check_all_axes(ldni, mesh, res)
    for a in range(3):
        assert set(np.unique(got[a].counts().cpu().numpy())) <= {0, 2}


def test_big_triangles_and_partial_cover(ldni):
    """Faces spanning thousands of pixels (CTA-per-triangle path), a mesh
    sticking out of the cube (clamped boxes), a ragged resolution."""
    _check_all_axes(ldni, M.box([-0.45, -0.3, -0.41], [0.37, 0.44, 0.33]), 201)
    _check_all_axes(ldni, M.box([-0.7, -0.2, -0.1], [0.3, 0.9, 0.2]), 130)
    _check_all_axes(ldni, M.icosphere(3, r=0.6, noise=0.05, seed=3), 150)


def test_flower_and_knot_multilayer(ldni):
    """Multi-layer rays (petals, knot strands) at a moderate resolution."""
    _check_all_axes(ldni, M.flower(96, 96), 160)
    _check_all_axes(ldni, M.torus_knot(n_ring=128, n_side=16), 160)


@pytest.mark.parametrize("k", [3, 40, 100, 450])
def test_deep_rays_ordered(ldni, k):
    """Stacked boxes give rays of up to 2k samples, so every way of ordering
    a ray is taken: by its lane (up to 4), by a warp from shared memory (up to
    128), by ranks in place (up to 768) and by insertion beyond."""
    mesh = M.slab_stack(k, axis=k % 3, seed=k)
    got, _ = _check_all_axes(ldni, mesh, 48)
    assert int(got[k % 3].counts().max()) > {3: 4, 40: 64, 100: 128, 450: 768}[k]


def test_grid_offset_and_scale(ldni):
    """A non-unit cube with a non-trivial origin."""
    v, t = M.icosphere(6, r=0.3, noise=0.02, seed=8)
    v2 = (v.astype(np.float64) * 3.0 + np.array([10.0, -4.0, 2.5])).astype(np.float32)
    _check_all_axes(ldni, (v2, t), 90, origin=(8.7, -5.3, 1.2), width=2.6)


def test_empty_mesh_and_outside_mesh(ldni):
    grid = ldni.Grid.cube(O3, 1.0, 32)
    v = np.zeros((3, 3), np.float32)
    t = np.zeros((0, 3), np.int32)
    out = ldni.sample(v, t, grid, "all")
    for L in out:
        assert L.n == 0 and int(L.offsets[-1]) == 0 and int(L.counts().abs().sum()) == 0
    far = M.translate(M.icosphere(2, r=0.2), (3.0, 0.0, 0.0))
    out = ldni.sample(*far, grid, "all")
    assert out[0].n > 0 and out[1].n == 0 and out[2].n == 0


def test_open_mesh_reports_odd_rays(ldni):
    """Definition 4 violated on purpose (a face removed): the odd rays are
    reported, and the count map still equals the oracle's."""
    v, t = M.icosphere(4, r=0.35)
    t_open = t[1:]
    grid = ldni.Grid.cube(O3, 1.0, 64)
    got = ldni.sample(v, t_open, grid, 2)
    ref = oracle.sample(v, t_open, grid.origin, 1.0, 64, 2, "scan")
    assert np.array_equal(got.numpy()["offsets"], ref["offsets"])
    assert np.any(np.diff(ref["offsets"]) % 2 == 1)
    with pytest.raises(ldni.LDNIError):
        ldni.sample(v, t_open, grid, 2, check_odd=True)


def _guarded_layers(ldni, grid, axis, cap, guard, fill):
    """Output arrays of one image carved from a single allocation, with
    `guard` words of `fill` before, between and after them."""
    N = grid.res * grid.res
    sizes = [N + 1, cap, cap, cap, cap, cap]  # offsets, depth, nx, ny, nz, tri
    backing = torch.full((sum(sizes) + guard * (len(sizes) + 1),), fill, dtype=torch.int32, device="cuda")
    views, guards, at = [], [backing[:guard]], guard
    for k in sizes:
        views.append(backing[at:at + k])
        guards.append(backing[at + k:at + k + guard])
        at += k + guard
    f = lambda t: t.view(torch.float32)
    L = ldni.LDNI(grid, axis, views[0], f(views[1]), f(views[2]), f(views[3]), f(views[4]), views[5], 0)
    return L, guards


def test_capacity_overflow_flagged_not_written(ldni):
    """Outputs of half the needed size, each array fenced by guard words in
    the same allocation: the overflow is reported and no write lands outside
    the arrays."""
    A, _ = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, 64)
    exact = ldni.sample(*A, grid, "all")
    caps = [L.n for L in exact]
    lib = ldni._lib.load()
    vt = torch.from_numpy(A[0]).cuda()
    tt = torch.from_numpy(A[1]).cuda()
    fill = 0x7F5A5A5A
    outs, guards = zip(*[_guarded_layers(ldni, grid, a, caps[a] // 2, 1024, fill) for a in range(3)])
    arr = (ldni._CLayers * 3)(*[o.c() for o in outs])
    ws = torch.empty(ldni.sample_workspace_size(len(A[0]), len(A[1]), 64), dtype=torch.uint8, device="cuda")
    info = ldni.new_info()
    g = grid.c()
    rc = lib.ldni_sample(vt.data_ptr(), vt.shape[0], tt.data_ptr(), tt.shape[0], ctypes.byref(g), 3, 0, arr,
                         info.data_ptr(), ws.data_ptr(), ws.numel(), None)
    assert rc == 0
    meta = ldni.info_decode(info)
    assert meta["status"] & ldni._lib.ST_CAPACITY
    assert [meta["n"][a] for a in range(3)] == caps  # the sizes needed
    for gs in guards:
        for gd in gs:
            assert bool((gd == fill).all())
    plan2 = ldni.SamplePlan(len(A[0]), len(A[1]), grid, caps)
    plan2.run(vt, tt)
    outs = plan2.finish()
    for a in range(3):
        ref = oracle.sample(*A, grid.origin, 1.0, 64, a, "scan")
        compare_ldni(outs[a].numpy(), ref, DIAG)


def test_repeatable_bitwise(ldni):
    """Two calls give bit-identical LDNIs (slot order is atomic, but the
    per-ray sort fixes the final order)."""
    A, _ = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, 128)
    x = [L.numpy() for L in ldni.sample(*A, grid, "all")]
    y = [L.numpy() for L in ldni.sample(*A, grid, "all")]
    for a in range(3):
        for k in ("offsets", "depth", "nrm", "tri"):
            assert np.array_equal(x[a][k], y[a][k])


@pytest.mark.parametrize("res", [1024, 2048])
def test_scale_sphere_full_size(ldni, res):
    """The 1,310,720-triangle noisy icosphere at both resolutions of the
    sampling-throughput workload, every ray compared with the oracle; the
    one-pass form with fixed two-layer capacity gives the same bits."""
    got, _ = _check_all_axes(ldni, M.scale_sphere(), res)
    grid = ldni.Grid.cube(O3, 1.0, res)
    one = ldni.sample_learned(*M.scale_sphere(), grid, "all", net=None, layers=2)
    assert all(ldni.identical(x, y) for x, y in zip(one, got))


def test_max_resolution_sampled_rays(ldni):
    """res 8192, the largest grid the library accepts: every ray's count."""
    v, t = M.icosphere(16, r=0.4, noise=0.03, seed=2)
    res = 8192
    grid = ldni.Grid.cube(O3, 1.0, res)
    L = ldni.sample(v, t, grid, 1)
    off = L.offsets.cpu().numpy().astype(np.int64)
    assert np.all(np.diff(off) % 2 == 0)
    ref = oracle.sample(v, t, grid.origin, 1.0, res, 1, "scan")
    assert np.array_equal(off, ref["offsets"])
