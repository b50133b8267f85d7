"""Batched sampling (ldni_sample_batch) and device-resident union chains.

* A batch of meshes of uneven size and resolution gives, image by image, the
  same LDNIs bit for bit as sampling each mesh alone.
* A batch call captured in a CUDA graph and replayed gives the same result.
* A chain of unions of translated copies (the repeated step of Minkowski sums
  and sweeps, Section 4.2) run eagerly, replayed from a CUDA graph, and run
  by the oracle step by step on the same inputs agree bit for bit.
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


def _mixed():
    A, B = M.pr1_pair()
    return [
        (A, 128), (B, 77), (M.flower(96, 96), 160),
        (M.torus_knot(n_ring=128, n_side=16), 100),
        (M.box([-0.45, -0.3, -0.41], [0.37, 0.44, 0.33]), 64),
        (M.icosphere(30, r=0.33, noise=0.05, noise_kind="octave", seed=4), 256),
        (M.tetrahedron([[-0.4, -0.3, -0.2], [0.41, -0.2, -0.3], [0.0, 0.43, -0.1], [0.05, 0.02, 0.45]]), 33),
    ]


def _check(ldni, meshes, grids, outs):
    for (v, t), g, got in zip(meshes, grids, outs):
        ref = ldni.sample(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), g, "all")
        for a in range(3):
            assert got[a].n == ref[a].n
            assert bit_equal(got[a].numpy(), ref[a].numpy()), a


def test_mixed_batch_equals_single(ldni):
    items = _mixed()
    meshes = [m for m, _ in items]
    grids = [ldni.Grid.cube(O3, 1.0, r) for _, r in items]
    plan = ldni.BatchPlan(meshes, grids)
    plan.run()
    _check(ldni, meshes, grids, plan.finish())


def test_deep_rays_batch_equals_single(ldni):
    """Stacked boxes of every ordering tier in one batch, whose warps of 32
    rays straddle images of different meshes (resolutions 5 and 7 have fewer
    rays than a warp)."""
    meshes = [M.slab_stack(k, axis=k % 3, seed=k) for k in (3, 40, 100, 450, 40, 3)]
    res = [48, 5, 40, 48, 7, 33]
    grids = [ldni.Grid.cube(O3, 1.0, r) for r in res]
    plan = ldni.BatchPlan(meshes, grids)
    plan.run()
    _check(ldni, meshes, grids, plan.finish())


def test_many_small_meshes(ldni):
    """96 meshes of 320 to 20,480 triangles, each on its own bounding grid."""
    batch = M.batch_meshes(96, seed=5, tmin=300, tmax=20_000, resolutions=(48, 64, 96, 128))
    meshes = [(v, t) for v, t, _ in batch]
    grids = [ldni.Grid.from_bbox(np.concatenate([v.min(0), v.max(0)]), r) for v, _, r in batch]
    plan = ldni.BatchPlan(meshes, grids)
    plan.run()
    outs = plan.finish()
    pick = [0, 1, 2, 3, 41, 95]
    _check(ldni, [meshes[k] for k in pick], [grids[k] for k in pick], [outs[k] for k in pick])
    for (v, t), g, o in zip(meshes, grids, outs):
        assert all(L.n > 0 for L in o)


def test_batch_graph_replay(ldni):
    items = _mixed()[:4]
    meshes = [m for m, _ in items]
    grids = [ldni.Grid.cube(O3, 1.0, r) for _, r in items]
    plan = ldni.BatchPlan(meshes, grids)
    plan.run()
    first = [[L.numpy() for L in o] for o in plan.finish()]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    for o in plan.outs:
        for L in o:
            L.depth.zero_()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    again = plan.finish()
    for o1, o2 in zip(first, again):
        for a in range(3):
            assert bit_equal(o1[a], o2[a].numpy())


def _torus_chain(steps):
    base = M.torus(R=0.16, r=0.06, nu=48, nv=24)
    offs = M.helix_offsets(steps, seed=11, radius=0.12, pitch=0.4, turns=1.5)
    return [M.translate(base, d) for d in offs]


@pytest.mark.parametrize("res", [64, 96])
def test_union_chain_eager_graph_oracle(ldni, res):
    """64 translated tori (a sweep along a helix): all 192 images sampled by
    one batch call, then each axis' 63 unions run eagerly, as one captured
    graph, and by the oracle."""
    steps = 64
    meshes = _torus_chain(steps)
    grid = ldni.Grid.cube(O3, 1.0, res)
    plan = ldni.BatchPlan(meshes, [grid] * steps)
    plan.run()
    parts = plan.finish()
    for a in range(3):
        P = [parts[k][a] for k in range(steps)]
        run, finish = ldni.union_chain(P)
        run()
        eager = finish().numpy()
        s = torch.cuda.Stream()
        run_g, finish_g = ldni.union_chain(P)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            run_g(stream=s)  # warm-up outside capture
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            run_g(stream=s)
        g.replay()
        torch.cuda.synchronize()
        assert bit_equal(eager, finish_g().numpy())
        acc = P[0].numpy()
        for k in range(1, steps):
            acc = oracle.boolean(acc, P[k].numpy(), "union")
        assert bit_equal(eager, acc)


def test_full_batch_workload(ldni):
    """The batched workload at full size: 256 seeded noisy icospheres and tori
    of 1k-200k triangles at resolutions drawn from {64, 128, 256, 512}, each
    on the cube [-0.5, 0.5]^3, sampled by one batch call; every mesh's three
    images equal a per-mesh sampling bit for bit."""
    batch = M.batch_meshes(256, seed=7)
    meshes = [(v, t) for v, t, _ in batch]
    grids = [ldni.Grid.cube(O3, 1.0, r) for _, _, r in batch]
    plan = ldni.BatchPlan(meshes, grids)
    plan.run()
    outs = plan.finish()
    for (v, t), g, got in zip(meshes, grids, outs):
        ref = ldni.sample(torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda(), g, "all")
        for a in range(3):
            assert ldni.identical(got[a], ref[a])


def test_full_union_chain_workload(ldni):
    """The sweep chain at full size: a 20,000-triangle torus (R 0.1, r 0.04,
    100 x 100 quads) translated along a seeded helix for 64 steps at 512^2;
    the graph-captured chain equals the oracle's step-by-step unions."""
    base = M.torus(R=0.1, r=0.04, nu=100, nv=100)
    offs = M.helix_offsets(64, seed=11)
    meshes = [M.translate(base, d) for d in offs]
    grid = ldni.Grid.cube(O3, 1.0, 512)
    plan = ldni.BatchPlan(meshes, [grid] * 64)
    plan.run()
    parts = plan.finish()
    for a in range(3):
        P = [parts[k][a] for k in range(64)]
        run_g, finish_g = ldni.union_chain(P)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            run_g(stream=s)
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            run_g(stream=s)
        g.replay()
        torch.cuda.synchronize()
        got = finish_g().numpy()
        acc = P[0].numpy()
        for k in range(1, 64):
            acc = oracle.boolean(acc, P[k].numpy(), "union")
        assert bit_equal(got, acc)
