"""One-pass sampling with learned per-tile capacity (ldni_sample_learned).

* Its LDNIs equal the exact two-pass LDNIs bit for bit whatever the
  capacities are: the network's, too small (every tile redone exactly),
  zero, or a slab too short for the layout.
* The network's CUDA forward pass and gradient agree with the FP64 oracle.
* Training lowers the loss, and the trained network needs fewer exact redos
  than a fixed two-layer capacity and less slab than a fixed capacity that
  never overflows.
"""
import numpy as np
import pytest

import meshgen as M
from ldni_compare import bit_equal
from oracle import mlp as MLPO

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


@pytest.fixture(scope="module")
def cap():
    from paper_1009_0794_gb300 import capacity
    return capacity


@pytest.fixture(scope="module")
def small_net(ldni, cap):
    X, L = cap.build_dataset(cap.training_meshes(24, seed=5), res=256)
    net = cap.CapacityNet(seed=1)
    losses = net.fit(X, L, steps=400, batch=1024)
    return net, losses


def _exact(ldni, mesh, grid):
    return [L.numpy() for L in ldni.sample(*mesh, grid, "all")]


def _learned(ldni, mesh, grid, **kw):
    v = torch.from_numpy(mesh[0]).cuda()
    t = torch.from_numpy(mesh[1]).cuda()
    ex = ldni.sample(v, t, grid, "all")
    plan = ldni.LearnedPlan(v.shape[0], t.shape[0], grid, [L.n for L in ex], kw.pop("slab", 4 * 3 * grid.res ** 2),
                            **kw)
    plan.run(v, t)
    outs = plan.finish()
    return [L.numpy() for L in outs], plan.overflow_tiles()


@pytest.mark.parametrize("res", [128, 100])
def test_fixed_capacities_equal_exact(ldni, res):
    A, B = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, res)
    for mesh in (A, B):
        ref = _exact(ldni, mesh, grid)
        for layers in (0, 2, 4, 64):
            got, n_over = _learned(ldni, mesh, grid, layers=layers)
            for a in range(3):
                assert bit_equal(got[a], ref[a]), (layers, a)
            if layers == 0:
                assert n_over > 0


def test_slab_too_short_still_exact(ldni):
    A, _ = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, 128)
    ref = _exact(ldni, A, grid)
    got, n_over = _learned(ldni, A, grid, layers=4, slab=5000)
    assert n_over > 0
    for a in range(3):
        assert bit_equal(got[a], ref[a])


def test_multilayer_and_big_triangles_equal_exact(ldni):
    grid = ldni.Grid.cube(O3, 1.0, 160)
    for mesh in (M.flower(96, 96), M.torus_knot(n_ring=128, n_side=16),
                 M.box([-0.45, -0.3, -0.41], [0.37, 0.44, 0.33])):
        ref = _exact(ldni, mesh, grid)
        for layers in (2, 6):
            got, _ = _learned(ldni, mesh, grid, layers=layers)
            for a in range(3):
                assert bit_equal(got[a], ref[a])


@pytest.mark.parametrize("k", [3, 40, 100, 450])
def test_deep_rays_equal_exact(ldni, k):
    """Rays of up to 2k samples: read from the slab when the tile's capacity
    holds them, redone exactly and ordered in place when it does not."""
    mesh = M.slab_stack(k, axis=k % 3, seed=k)
    grid = ldni.Grid.cube(O3, 1.0, 48)
    ref = _exact(ldni, mesh, grid)
    for layers in (0, 6, 64):
        got, _ = _learned(ldni, mesh, grid, layers=layers, slab=max(4, layers) * 3 * 48 * 48)
        for a in range(3):
            assert bit_equal(got[a], ref[a]), (layers, a)


def test_network_capacity_equals_exact(ldni, small_net):
    net, _ = small_net
    for mesh, res in ((M.pr1_pair()[0], 128), (M.icosphere(40, r=0.33, noise=0.05, noise_kind="octave", seed=9), 256)):
        grid = ldni.Grid.cube(O3, 1.0, res)
        ref = _exact(ldni, mesh, grid)
        got, _ = _learned(ldni, mesh, grid, net=net, margin=0.25)
        for a in range(3):
            assert bit_equal(got[a], ref[a])


def test_forward_matches_oracle(ldni, cap):
    net = cap.CapacityNet(seed=3)
    rng = np.random.default_rng(0)
    X = rng.normal(size=(300, 12)).astype(np.float32)
    y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    w, b, w16 = net.params_numpy()
    yo, _ = MLPO.forward(cap.from_bf16_bits(w16).astype(np.float64), b.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(y - yo)) <= 1e-4 * max(1.0, np.max(np.abs(yo)))


def test_gradient_matches_oracle(ldni, cap):
    net = cap.CapacityNet(seed=4)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(500, 12)).astype(np.float32)
    t = rng.normal(loc=1.0, size=500).astype(np.float32)
    w0, b0, w16 = net.params_numpy()
    loss, g = net.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), lr=1e-3, want_grad=True)
    Lo, gw, gb = MLPO.grad(cap.from_bf16_bits(w16).astype(np.float64), b0.astype(np.float64), X.astype(np.float64),
                           t.astype(np.float64), 4.0)
    g = g.cpu().numpy()
    go = np.concatenate([gw, gb])
    assert float(loss.item()) == pytest.approx(Lo, rel=1e-4)
    assert np.linalg.norm(g - go) <= 2e-4 * np.linalg.norm(go)


def test_training_lowers_loss_and_beats_fixed_capacity(ldni, cap, small_net):
    net, losses = small_net
    assert losses[-1] < 0.5 * losses[0]
    held_out = cap.training_meshes(6, seed=99)
    res = 256
    grid = ldni.Grid.cube(O3, 1.0, res)
    over_net = over_k2 = 0
    slab_net = slab_kmax = 0
    for mesh in held_out:
        X, L = cap.tile_rows(*mesh, grid)
        y = net.forward(X)
        k_net = np.clip(np.ceil(np.expm1(np.maximum(y.cpu().numpy(), 0)) * 1.25 - 1e-3), 2, 64)
        k_net = (k_net.astype(int) + 1) & ~1
        k_true = np.rint(np.expm1(L.cpu().numpy())).astype(int)
        over_net += int(np.sum(k_true > k_net))
        over_k2 += int(np.sum(k_true > 2))
        slab_net += int(np.sum(k_net))
        slab_kmax += int(np.max(k_true)) * k_true.size
    assert over_net < over_k2
    assert slab_net < slab_kmax
