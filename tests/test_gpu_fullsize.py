"""Parity at the sizes the benchmark runs, through the C ABI.

* The step's Boolean: the three 1024^2 images of the 1,310,720-triangle
  noisy sphere against the resident (2,3) torus-knot images, in the same
  three-image call and launch form the benchmark uses, for all three
  operations of Section 4.1, with and without the small-interval removal of
  Section 4.1.1.  Both sides read the same FP32 images, so every count,
  depth, normal and id must match the oracle bit for bit.
* The flower-and-knot workload at its stated size: the 523,264-triangle
  flower (512 x 512 (theta, phi) grid) and the 16,384-triangle knot sampled
  at 512^2 (every ray against the oracle's scan mode), then union,
  intersection and difference of the sampled images.
* Grid-node classification (Section 5.1, Step 1) of a 256^2 union, every
  node against the oracle.
* Offsetting (Section 4.2) of the benchmark's flower at 128^2 by +-2.5
  pixels, every ray against the step-by-step oracle.
* Contouring Steps 2-3 (Section 5.1) of a 256^2 union: a seeded sample of
  10,000 cells with vertices, and 10,000 cells drawn from the whole grid,
  against the oracle.
* One-pass sampling with the trained capacity network at 1024^2 equals the
  exact two-pass output bit for bit.
"""
import numpy as np
import pytest

import meshgen as M
import oracle
from ldni_compare import bit_equal, compare_ldni
from oracle import contour as C
from oracle import nodes

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


@pytest.fixture(scope="module")
def bench_images(ldni):
    """The benchmark's operands at 1024^2: the sphere's and the knot's three
    images, sampled on the device (exact two-pass)."""
    grid = ldni.Grid.cube(O3, 1.0, 1024)
    S = ldni.sample(*M.scale_sphere(), grid, "all", check_odd=True)
    K = ldni.sample(*M.torus_knot(2, 3, 0.25, 0.1, 0.035, 256, 32), grid, "all", check_odd=True)
    return grid, S, K, [L.numpy() for L in S], [L.numpy() for L in K]


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _upload(ldni, grid, a, L):
    nrm = np.asarray(L["nrm"], np.float32).reshape(-1, 3)
    return ldni.LDNI(grid, a, _t(np.asarray(L["offsets"], np.int32)), _t(np.asarray(L["depth"], np.float32)),
                     _t(nrm[:, 0]), _t(nrm[:, 1]), _t(nrm[:, 2]), _t(np.asarray(L["tri"], np.int32)),
                     int(L["offsets"][-1]))


@pytest.mark.parametrize("op", ["union", "inter", "diff"])
@pytest.mark.parametrize("eps", [0.0, 1e-5])
def test_bench_boolean_1024_bit_exact(ldni, bench_images, op, eps):
    """The benchmark's three-image call (default launch form at this size:
    count and write passes, with the volumes finished in the write pass)."""
    grid, S, K, Sn, Kn = bench_images
    vols = torch.zeros(3, dtype=torch.float64, device="cuda")
    got = ldni.boolean_many(S, K, op, eps=eps, vols=vols)
    for a in range(3):
        ref = oracle.boolean(Sn[a], Kn[a], op, eps=eps)
        g = got[a].numpy()
        assert got[a].n == int(ref["offsets"][-1]), a
        assert bit_equal(g, ref), a
        v_ref = oracle.volume(ref, grid.h)
        assert abs(float(vols[a]) - v_ref) <= 1e-12 * max(abs(v_ref), 1e-30), a


@pytest.fixture(scope="module")
def flower_knot_512(ldni):
    grid = ldni.Grid.cube(O3, 1.0, 512)
    fl = M.flower(512, 512)
    kn = M.torus_knot(2, 3, 0.25, 0.1, 0.035, 256, 32)
    assert len(fl[1]) == 523264 and len(kn[1]) == 16384
    return grid, fl, kn


def test_flower_knot_512_sampling_every_ray(ldni, flower_knot_512):
    grid, fl, kn = flower_knot_512
    for mesh in (fl, kn):
        got = ldni.sample(*mesh, grid, "all", check_odd=True)
        one = ldni.sample_learned(*mesh, grid, "all", net=None, layers=2)
        for a in range(3):
            ref = oracle.sample(*mesh, O3, 1.0, 512, a, "scan")
            compare_ldni(got[a].numpy(), ref, DIAG)
            assert ldni.identical(one[a], got[a]), a


@pytest.mark.parametrize("eps", [0.0, 1e-5])
def test_flower_knot_512_booleans_bit_exact(ldni, flower_knot_512, eps):
    grid, fl, kn = flower_knot_512
    A = ldni.sample(*fl, grid, "all")
    B = ldni.sample(*kn, grid, "all")
    An, Bn = [L.numpy() for L in A], [L.numpy() for L in B]
    for op in ("union", "inter", "diff"):
        got = ldni.boolean_many(A, B, op, eps=eps)
        for a in range(3):
            ref = oracle.boolean(An[a], Bn[a], op, eps=eps)
            assert bit_equal(got[a].numpy(), ref), (op, a)


@pytest.fixture(scope="module")
def union_256():
    """The oracle's FP32 images of the sphere-knot union at 256^2 and the
    oracle's node signs."""
    res = 256
    S = [oracle.as_f32(oracle.sample(*M.scale_sphere(), O3, 1.0, res, a, "scan")) for a in range(3)]
    K = [oracle.as_f32(oracle.sample(*M.torus_knot(2, 3, 0.25, 0.1, 0.035, 256, 32), O3, 1.0, res, a, "scan"))
         for a in range(3)]
    U = [oracle.boolean(S[a], K[a], "union") for a in range(3)]
    return res, U, nodes.classify(U, O3, 1.0, res)


def _bits(inside):
    res = inside.shape[2]
    W = (res + 31) // 32
    pad = np.zeros(inside.shape[:2] + (W * 32,), bool)
    pad[:, :, :res] = inside
    return np.packbits(pad, axis=2, bitorder="little").view(np.uint32)


def test_nodes_256_every_node(ldni, union_256):
    res, U, ins = union_256
    grid = ldni.Grid.cube(O3, 1.0, res)
    H = [_upload(ldni, grid, a, L) for a, L in enumerate(U)]
    got = ldni.classify_nodes(H).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, _bits(ins))


def test_contour_256_sampled_cells(ldni, union_256):
    res, U, ins = union_256
    grid = ldni.Grid.cube(O3, 1.0, res)
    H = [_upload(ldni, grid, a, L) for a, L in enumerate(U)]
    got = ldni.contour_cells(H, inside=_t(_bits(ins).view(np.int32)))
    n = res - 1
    rng = np.random.default_rng(2024)
    keys = got["cell"].astype(np.int64)
    assert keys.size > 10000
    pick = np.sort(rng.choice(keys.size, 10000, replace=False))
    cells = [(int(c % n), int((c // n) % n), int(c // (n * n))) for c in keys[pick]]
    want = C.contour(U, ins, O3, 1.0, res, cells=cells)
    assert sorted(want) == keys[pick].tolist()
    for rec in got[pick]:
        w = want[int(rec["cell"])]
        nv = len(w["vertices"])
        assert rec["nvert"] == nv
        lab = [(int(rec["labels"]) >> (4 * c)) & 15 for c in range(8)]
        assert lab == [15 if x < 0 else x for x in w["labels"]]
        assert [(int(rec["npts"]) >> (8 * g)) & 255 for g in range(nv)] == w["points"]
        near_cut = any(abs(r - C.QEF_TRUNC) < 1e-6 for rs in w["ratios"] for r in rs)
        if not near_cut:
            assert np.abs(rec["v"][:nv] - w["vertices"]).max() <= 2e-6
    # cells drawn from the whole grid: a vertex exactly where the oracle gives one
    flat = rng.integers(0, n ** 3, size=10000)
    cells = [(int(c % n), int((c // n) % n), int(c // (n * n))) for c in flat]
    want = C.contour(U, ins, O3, 1.0, res, cells=cells)
    listed = set(keys.tolist())
    for c in flat.tolist():
        assert (c in want) == (c in listed), c


@pytest.mark.parametrize("inner", [False, True])
def test_offset_bench_flower_128(ldni, inner):
    """The benchmark's offsetting workload: the 523,264-triangle flower at
    128^2 by 2.5 pixels (the paper's offsetting examples, Table 4)."""
    res = 128
    grid = ldni.Grid.cube(O3, 1.0, res)
    fl = M.flower(512, 512)
    ref = [oracle.as_f32(oracle.sample(*fl, O3, 1.0, res, a, "scan")) for a in range(3)]
    H = [_upload(ldni, grid, a, L) for a, L in enumerate(ref)]
    got = ldni.offset(H, 2.5 / res, inner=inner)
    want = oracle.offset(ref, O3, 1.0, res, 2.5 / res, inner=inner)
    for a in range(3):
        assert got[a].n == int(want[a]["offsets"][-1]), a
        assert bit_equal(got[a].numpy(), want[a]), a


def test_learned_trained_net_1024_identical(ldni, bench_images):
    """The benchmark's one-pass sampling with the network trained as the
    benchmark trains it (200 seeded noisy spheres at 512^2) equals the exact
    two-pass images bit for bit."""
    from paper_1009_0794_gb300 import capacity
    grid, S, K, Sn, Kn = bench_images
    net, meta = capacity.train_default(count=200, res=512, steps=1500)
    assert meta["loss_last"] < meta["loss_first"]
    v, t = M.scale_sphere()
    vt, tt = _t(v), _t(t)
    plan = ldni.LearnedPlan(len(v), len(t), grid, [L.n for L in S], slab_samples=8 * 3 * 1024 * 1024, net=net,
                            margin=0.25, feature_stride=32)
    for _ in range(2):  # twice: the second run starts from the first run's workspace
        plan.run(vt, tt)
        outs = plan.finish()
        assert all(ldni.identical(x, y) for x, y in zip(outs, S))
