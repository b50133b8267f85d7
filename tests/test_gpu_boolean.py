"""CUDA Boolean and volume through the C ABI against the oracle
(Section 4.1, 4.1.1; odd-to-even volume).  Both sides read the same FP32
LDNIs, so the Boolean must match bit for bit: counts, depths, normals, ids."""
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


def _pairs(ldni, meshA, meshB, res):
    grid = ldni.Grid.cube(O3, 1.0, res)
    return ldni.sample(*meshA, grid, "all"), ldni.sample(*meshB, grid, "all")


@pytest.mark.parametrize("res", [128, 77])
@pytest.mark.parametrize("op", ["union", "inter", "diff"])
@pytest.mark.parametrize("eps", [0.0, 1e-5])
def test_pr1_boolean_bit_exact(ldni, res, op, eps):
    A, B = M.pr1_pair()
    LA, LB = _pairs(ldni, A, B, res)
    for a in range(3):
        got = ldni.boolean(LA[a], LB[a], op, eps=eps).numpy()
        ref = oracle.boolean(LA[a].numpy(), LB[a].numpy(), op, eps=eps)
        assert bit_equal(got, ref)


def test_flower_knot_boolean_bit_exact(ldni):
    (fv, ft), (kv, kt) = M.flower(128, 128), M.torus_knot(n_ring=128, n_side=16)
    LA, LB = _pairs(ldni, (fv, ft), (kv, kt), 192)
    for a in range(3):
        for op in ("union", "inter", "diff"):
            got = ldni.boolean(LA[a], LB[a], op, eps=1e-5).numpy()
            ref = oracle.boolean(LA[a].numpy(), LB[a].numpy(), op, eps=1e-5)
            assert bit_equal(got, ref)


def test_identities_on_gpu(ldni):
    """A u A = A, A \\ A = empty, (A n B) \\ A = empty (Figure 6), and
    (A \\ B) u (A n B) = A in depths, all on the device."""
    A, B = M.pr1_pair()
    LA, LB = _pairs(ldni, A, B, 128)
    for a in range(3):
        X = LA[a].numpy()
        assert bit_equal(ldni.boolean(LA[a], LA[a], "union").numpy(), X)
        assert ldni.boolean(LA[a], LA[a], "diff").n == 0
        I = ldni.boolean(LA[a], LB[a], "inter")
        assert ldni.boolean(I, LA[a], "diff").n == 0
        D = ldni.boolean(LA[a], LB[a], "diff")
        R = ldni.boolean(D, I, "union").numpy()
        assert np.array_equal(R["offsets"], X["offsets"]) and np.array_equal(R["depth"], X["depth"])


def test_empty_operands(ldni):
    A, _ = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, 64)
    LA = ldni.sample(*A, grid, 0)
    E = ldni.sample(np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32), grid, 0)
    assert bit_equal(ldni.boolean(LA, E, "union").numpy(), LA.numpy())
    assert ldni.boolean(LA, E, "inter").n == 0
    assert bit_equal(ldni.boolean(LA, E, "diff").numpy(), LA.numpy())
    assert ldni.boolean(E, E, "union").n == 0
    # an empty first operand (no sample arrays at all): the result's normals still come from B
    from paper_1009_0794_gb300 import tune
    for op in ("union", "inter", "diff"):
        for split in (0, 1):
            prev = tune.set(bool_split=split)
            try:
                got = ldni.boolean(E, LA, op).numpy()
            finally:
                tune.set(**prev)
            assert bit_equal(got, oracle.boolean(E.numpy(), LA.numpy(), op)), (op, split)


def test_grid_mismatch_rejected(ldni):
    A, _ = M.pr1_pair()
    L1 = ldni.sample(*A, ldni.Grid.cube(O3, 1.0, 64), 0)
    L2 = ldni.sample(*A, ldni.Grid.cube((-0.5, -0.5, -0.25), 1.0, 64), 0)
    with pytest.raises(ldni.LDNIError) as e:
        ldni.boolean(L1, L2, "union")
    assert e.value.code == -2


@pytest.mark.parametrize("res", [64, 128, 333])
def test_volume_matches_oracle(ldni, res):
    A, B = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, res)
    for mesh in (A, B):
        for L in ldni.sample(*mesh, grid, "all"):
            v = ldni.volume(L)
            ref = oracle.volume(L.numpy(), grid.h)
            assert v == pytest.approx(ref, rel=1e-12)


def test_volume_deterministic_and_inclusion_exclusion(ldni):
    A, B = M.pr1_pair()
    LA, LB = _pairs(ldni, A, B, 128)
    for a in range(3):
        vA, vB = ldni.volume(LA[a]), ldni.volume(LB[a])
        assert ldni.volume(LA[a]) == vA
        vU = ldni.volume(ldni.boolean(LA[a], LB[a], "union"))
        vI = ldni.volume(ldni.boolean(LA[a], LB[a], "inter"))
        assert vU + vI == pytest.approx(vA + vB, rel=1e-12)


def test_volume_multilayer_and_odd_rays_skipped(ldni):
    """Multi-layer rays, and an open mesh whose odd rays the volume skips
    (their blocks take the ray-by-ray path): the value equals the oracle's
    on the same image with the odd rays emptied."""
    grid = ldni.Grid.cube(O3, 1.0, 150)
    for mesh in (M.flower(96, 96), M.torus_knot(n_ring=128, n_side=16)):
        for L in ldni.sample(*mesh, grid, "all"):
            assert ldni.volume(L) == pytest.approx(oracle.volume(L.numpy(), grid.h), rel=1e-12)
    v, t = M.icosphere(6, r=0.35)
    for a in range(3):
        L = ldni.sample(v, t[7:], grid, a)
        got = float(ldni.volume(L, sync=False).item())
        X = L.numpy()
        cnt = np.diff(X["offsets"])
        assert (cnt % 2).sum() > 0
        keep = np.repeat(cnt % 2 == 0, cnt)
        cnt2 = np.where(cnt % 2 == 0, cnt, 0)
        Y = {"offsets": np.concatenate([[0], np.cumsum(cnt2)]), "depth": X["depth"][keep]}
        assert got == pytest.approx(oracle.volume(Y, grid.h), rel=1e-12)


def test_odd_operand_rejected(ldni):
    v, t = M.icosphere(4, r=0.35)
    grid = ldni.Grid.cube(O3, 1.0, 64)
    L = ldni.sample(v, t[1:], grid, 2)
    with pytest.raises(ldni.LDNIError):
        ldni.boolean(L, L, "union")
    with pytest.raises(ldni.LDNIError):
        ldni.volume(L)


@pytest.mark.parametrize("tile", [256, 512, 1024, 2048])
@pytest.mark.parametrize("stage", [0, 64, 4096, 16384])
@pytest.mark.parametrize("split", [0, 1])
def test_tuning_does_not_change_results(ldni, tile, stage, split):
    """Every launch shape of the Boolean (tile rays, samples staged in shared
    memory; 64 forces a mix of staged and unstaged tiles) gives the oracle's
    bits, on a ragged grid and on multi-layer rays."""
    from paper_1009_0794_gb300 import tune
    prev = tune.set(bool_tile_rays=tile, bool_stage_samples=stage, bool_split=split)
    try:
        A, B = M.pr1_pair()
        for (ma, mb), res in (((A, B), 77), ((M.flower(64, 64), M.torus_knot(n_ring=96, n_side=12)), 150)):
            LA, LB = _pairs(ldni, ma, mb, res)
            for a in range(3):
                for op in ("union", "inter", "diff"):
                    got = ldni.boolean(LA[a], LB[a], op, eps=1e-5).numpy()
                    ref = oracle.boolean(LA[a].numpy(), LB[a].numpy(), op, eps=1e-5)
                    assert bit_equal(got, ref), (op, a)
    finally:
        tune.set(**prev)


def test_tuner_picks_a_valid_choice(ldni, tmp_path, monkeypatch):
    from paper_1009_0794_gb300 import tune
    monkeypatch.setenv(tune.CACHE_ENV, str(tmp_path / "tune.json"))
    prev = tune.get()
    try:
        A, B = M.pr1_pair()
        LA, LB = _pairs(ldni, A, B, 128)
        r = tune.tune_boolean(LA[0], LB[0], "union", reps=3, candidates=[(256, 0, 0), (1024, 4096, 1)])
        assert not r["cached"] and set(r["ms"]) == {"256/0/0", "1024/4096/1"}
        assert tune.get()["bool_tile_rays"] == r["choice"]["bool_tile_rays"]
        again = tune.tune_boolean(LA[0], LB[0], "union")
        assert again["cached"] and again["choice"] == r["choice"]
        s = tune.tune_sampling(*A, ldni.Grid.cube(O3, 1.0, 64), reps=2, candidates=[4, 16])
        assert s["choice"]["tri_blocks_per_sm"] in (4, 16)
    finally:
        tune.set(**prev)


@pytest.mark.parametrize("split,res", [(0, 130), (1, 130), (1, 24)])
def test_many_images_in_one_call(ldni, split, res):
    """ldni_boolean_many and ldni_volume_many over the three images equal
    the one-image calls bit for bit.  At 24^2 the two-launch form has two
    512-ray write tiles for three images, so one block finishes two of the
    three volumes."""
    from paper_1009_0794_gb300 import tune
    prev = tune.set(bool_split=split)
    try:
        (fv, ft), (kv, kt) = M.flower(96, 96), M.torus_knot(n_ring=128, n_side=16)
        LA, LB = _pairs(ldni, (fv, ft), (kv, kt), res)
        for op in ("union", "inter", "diff"):
            many = ldni.boolean_many(LA, LB, op, eps=1e-5)
            for a in range(3):
                one = ldni.boolean(LA[a], LB[a], op, eps=1e-5)
                assert bit_equal(many[a].numpy(), one.numpy())
            vols = ldni.volume_many(many)
            assert vols == [ldni.volume(U) for U in many]
            fused = torch.zeros(3, dtype=torch.float64, device="cuda")
            ldni.boolean_many(LA, LB, op, eps=1e-5, vols=fused)
            for v, f in zip(vols, fused.cpu().numpy()):
                assert f == pytest.approx(v, rel=1e-12, abs=1e-15)
    finally:
        tune.set(**prev)


def test_results_in_one_allocation(ldni):
    """Outputs carved from one allocation (empty_layers_flat) hold the same
    bits as separately allocated ones, and one copy of the allocation brings
    all of them to the host."""
    (fv, ft), (kv, kt) = M.flower(64, 64), M.torus_knot(n_ring=96, n_side=12)
    LA, LB = _pairs(ldni, (fv, ft), (kv, kt), 96)
    outs, flat = ldni.empty_layers_flat(LA[0].grid, range(3), [A.n + B.n for A, B in zip(LA, LB)])
    assert flat.data_ptr() % 256 == 0
    for X in outs:
        for t in (X.offsets, X.depth, X.nx, X.ny, X.nz, X.tri):
            assert t.data_ptr() % 256 == 0
            assert flat.data_ptr() <= t.data_ptr() and t.data_ptr() + 4 * t.numel() <= flat.data_ptr() + flat.numel()
    got = ldni.boolean_many(LA, LB, "union", outs=outs)
    host = flat.cpu()  # every image with one copy
    for a in range(3):
        ref = ldni.boolean(LA[a], LB[a], "union").numpy()
        assert bit_equal(got[a].numpy(), ref)
        off = (got[a].offsets.data_ptr() - flat.data_ptr())
        assert np.array_equal(host[off:off + 4 * got[a].offsets.numel()].view(torch.int32).numpy(), ref["offsets"])


def _ldni_from_rays(ldni, grid, rays, seed):
    """An LDNI whose ray p holds the sorted depths rays[p] (other rays empty),
    with seeded unit normals and distinct triangle ids."""
    N = grid.res * grid.res
    counts = np.zeros(N, np.int64)
    counts[:len(rays)] = [len(r) for r in rays]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    depth = np.concatenate([np.asarray(r, np.float32) for r in rays] + [np.zeros(0, np.float32)])
    n = depth.size
    rng = np.random.default_rng(seed)
    nrm = rng.normal(size=(n, 3)).astype(np.float32)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    tri = np.arange(n, dtype=np.int32) + 1000 * (seed + 1)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    L = ldni.LDNI(grid, 0, t(off), t(depth), t(nrm[:, 0]), t(nrm[:, 1]), t(nrm[:, 2]), t(tri), n)
    return L, {"offsets": off.astype(np.int64), "depth": depth, "nrm": nrm, "tri": tri}


def _tie_cases(rng):
    """Every pair of intervals with endpoints in {0, 1, 2, 3} (ties, touching,
    nested, zero-length), single intervals against nothing, and random
    multi-interval rays with shared depths."""
    iv = [(x, y) for x in range(4) for y in range(x, 4)]
    A, B = [], []
    for a in iv:
        for b in iv:
            A.append([0.25 * a[0], 0.25 * a[1]])
            B.append([0.25 * b[0], 0.25 * b[1]])
    for a in iv:
        A.append([0.25 * a[0], 0.25 * a[1]]); B.append([])
        A.append([]); B.append([0.25 * a[0], 0.25 * a[1]])
    A.append([]); B.append([])
    for _ in range(300):
        na, nb = 2 * rng.integers(0, 4), 2 * rng.integers(0, 4)
        A.append(sorted(0.25 * rng.integers(0, 6, na)))
        B.append(sorted(0.25 * rng.integers(0, 6, nb)))
    return A, B


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("tile", [256, 1024])
def test_interval_ties_against_oracle(ldni, split, tile):
    """All tie and touching configurations of one interval per operand (the
    closed-form path) and random multi-interval rays (the general merge),
    every operation, eps 0 and 0.3, against the oracle bit for bit."""
    from paper_1009_0794_gb300 import tune
    prev = tune.set(bool_split=split, bool_tile_rays=tile, bool_stage_samples=4096)
    try:
        ra, rb = _tie_cases(np.random.default_rng(5))
        grid = ldni.Grid.cube(O3, 1.0, 24)
        LA, hA = _ldni_from_rays(ldni, grid, ra, 1)
        LB, hB = _ldni_from_rays(ldni, grid, rb, 2)
        for op in ("union", "inter", "diff"):
            for eps in (0.0, 0.3):
                got = ldni.boolean(LA, LB, op, eps=eps).numpy()
                ref = oracle.boolean(hA, hB, op, eps=eps)
                assert bit_equal(got, ref), (op, eps)
    finally:
        tune.set(**prev)


def test_hand_worked_cases(ldni):
    """The CUDA Boolean (both launch forms) on the hand-worked cases of
    tests/golden/boolean_segments.txt, each case on its own ray."""
    from golden_cases import cases, expected, ray
    from paper_1009_0794_gb300 import tune
    cs = cases()
    grid = ldni.Grid.cube(O3, 1.0, 1)
    for split in (0, 1):
        prev = tune.set(bool_split=split)
        try:
            for c in cs:
                A, B = ray(c["A"], 1, 1), ray(c["B"], 100, 2)
                LA, _ = _ldni_from_rays(ldni, grid, [c["A"]], 1)
                LB, _ = _ldni_from_rays(ldni, grid, [c["B"]], 2)
                # same normals and ids as the dicts
                for L, H in ((LA, A), (LB, B)):
                    if H["depth"].size:
                        L.nx.copy_(torch.from_numpy(H["nrm"][:, 0]))
                        L.ny.copy_(torch.from_numpy(H["nrm"][:, 1]))
                        L.nz.copy_(torch.from_numpy(H["nrm"][:, 2]))
                        L.tri.copy_(torch.from_numpy(H["tri"]))
                got = ldni.boolean(LA, LB, c["op"], eps=c["eps"]).numpy()
                assert bit_equal(got, expected(c, A, B)), c["name"]
        finally:
            tune.set(**prev)


@pytest.mark.parametrize("split,tile", [(0, 256), (1, 256), (1, 512), (1, 2048)])
def test_truncated_operand_reported(ldni, split, tile):
    """An operand whose offsets run past its capacity (its samples were cut
    off) is reported, nothing past its capacity is read, and every ray before
    the first cut-off ray is answered as with the whole operand."""
    from paper_1009_0794_gb300 import tune
    A, B = M.pr1_pair()
    LA, LB = _pairs(ldni, A, B, 77)
    prev = tune.set(bool_split=split, bool_tile_rays=tile)
    try:
        for a in range(3):
            X = LA[a]
            cap = X.n // 2
            T = ldni.LDNI(X.grid, X.axis, X.offsets, X.depth[:cap].clone(), X.nx[:cap].clone(), X.ny[:cap].clone(),
                          X.nz[:cap].clone(), X.tri[:cap].clone(), X.n)
            full = ldni.boolean(X, LB[a], "union").numpy()
            info = ldni.new_info()
            out = ldni.boolean(T, LB[a], "union", info=info, sync=False)
            torch.cuda.synchronize()
            assert ldni.info_decode(info)["status"] & ldni._lib.ST_CAPACITY, a
            offs = X.offsets.cpu().numpy()
            first = int(np.argmax(offs[1:] > cap))  # the first ray that runs past the capacity
            got_off = out.offsets.cpu().numpy()[:first + 1]
            assert np.array_equal(got_off, full["offsets"][:first + 1]), a
            m = int(full["offsets"][first])
            for k in ("depth", "tri"):
                assert np.array_equal(getattr(out, k)[:m].cpu().numpy(), full[k][:m]), (a, k)
    finally:
        tune.set(**prev)
