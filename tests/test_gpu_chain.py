"""Chains of unions in one call (ldni_union_chain, Sections 4.1.1 and 4.2)
and the bounded device waits, through the C ABI.

The chain's result must equal the step-by-step chain of ldni_boolean calls
and the oracle's step-by-step unions bit for bit (counts, depths, normals,
ids), with and without small-interval removal at every step, for one or
three images per call and for packed normals.  A ray whose accumulated
result outgrows the per-ray limit is reported, not answered wrongly.  The
timeout path of a bounded wait is made to run out on purpose (a word that
nothing sets) and must report LDNI_ST_TIMEOUT with the device still usable.
"""
import ctypes

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


def _sweep_parts(ldni, steps, res, packed=False):
    base = M.torus(R=0.16, r=0.06, nu=48, nv=24)
    offs = M.helix_offsets(steps, seed=11, radius=0.12, pitch=0.4, turns=1.5)
    grid = ldni.Grid.cube(O3, 1.0, res)
    return [ldni.sample(*M.translate(base, d), grid, "all", packed=packed) for d in offs]


def _stepwise(ldni, P, eps):
    acc = P[0]
    for k in range(1, len(P)):
        acc = ldni.boolean(acc, P[k], "union", eps=eps)
    return acc


@pytest.mark.parametrize("eps", [0.0, 1e-2])
def test_chain_equals_stepwise_and_oracle(ldni, eps):
    steps, res = 24, 80
    parts = _sweep_parts(ldni, steps, res)
    for a in range(3):
        P = [parts[k][a] for k in range(steps)]
        run, finish = ldni.union_chain(P, eps=eps)
        run()
        got = finish()
        want = _stepwise(ldni, P, eps)
        assert ldni.identical(got, want), a
        acc = P[0].numpy()
        for k in range(1, steps):
            acc = oracle.boolean(acc, P[k].numpy(), "union", eps=eps)
        assert bit_equal(got.numpy(), acc), a


def test_three_images_in_one_call_and_graph(ldni):
    steps, res = 16, 96
    parts = _sweep_parts(ldni, steps, res)
    per_image = [[parts[k][a] for k in range(steps)] for a in range(3)]
    run, finish = ldni.union_chain_many(per_image)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run(stream=s)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        run(stream=s)
    g.replay()
    torch.cuda.synchronize()
    outs = finish()
    for a in range(3):
        r1, f1 = ldni.union_chain(per_image[a])
        r1()
        assert ldni.identical(outs[a], f1()), a
        assert ldni.identical(outs[a], _stepwise(ldni, per_image[a], 0.0)), a


def test_packed_normals_chain(ldni):
    steps, res = 12, 64
    parts = _sweep_parts(ldni, steps, res, packed=True)
    for a in range(3):
        P = [parts[k][a] for k in range(steps)]
        run, finish = ldni.union_chain(P)
        run()
        assert ldni.identical(finish(), _stepwise(ldni, P, 0.0)), a


def test_short_chains_and_empty_parts(ldni):
    grid = ldni.Grid.cube(O3, 1.0, 48)
    A, B = M.pr1_pair()
    LA, LB = ldni.sample(*A, grid, 2), ldni.sample(*B, grid, 2)
    E = ldni.sample(np.zeros((3, 3), np.float32), np.zeros((0, 3), np.int32), grid, 2)
    run, finish = ldni.union_chain([LA])  # one part: the part itself
    run()
    assert ldni.identical(finish(), LA)
    for P in ([LA, LB], [LA, E, LB, E], [E, LA, E], [E, E]):
        run, finish = ldni.union_chain(P, eps=1e-5)
        run()
        assert ldni.identical(finish(), _stepwise(ldni, P, 1e-5))


def test_deep_rays_are_reported(ldni):
    """A stack of 40 slabs gives rays of 80 samples, more than a ray's
    accumulated result may hold: the call reports it instead of answering."""
    grid = ldni.Grid.cube(O3, 1.0, 16)
    L = ldni.sample(*M.slab_stack(40, axis=0, seed=1), grid, 0)
    assert int(L.counts().max()) > 64
    run, finish = ldni.union_chain([L, L])
    run()
    with pytest.raises(ldni.LDNIError):
        finish()


def test_bounded_wait_runs_out(ldni):
    """The bounded wait on a word that nothing sets gives up after the set
    number of polls and reports LDNI_ST_TIMEOUT; the device keeps working."""
    lib = ldni._lib.load()
    assert lib.ldni_set_wait_limit(-1) == -1
    assert lib.ldni_set_wait_limit(2000) == 0
    try:
        assert lib.ldni_get_wait_limit() == 2000
        info = ldni.new_info()
        assert lib.ldni_wait_selftest(info.data_ptr(), None) == 0
        torch.cuda.synchronize()
        assert ldni.info_decode(info)["status"] & ldni._lib.ST_TIMEOUT
    finally:
        assert lib.ldni_set_wait_limit(0) == 0
    assert lib.ldni_get_wait_limit() == 1 << 22
    # the device still answers: a Boolean through the one-launch look-back form
    A, B = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, 128)
    LA, LB = ldni.sample(*A, grid, 0), ldni.sample(*B, grid, 0)
    got = ldni.boolean(LA, LB, "union").numpy()
    assert bit_equal(got, oracle.boolean(LA.numpy(), LB.numpy(), "union"))


def test_tiny_wait_limit_terminates(ldni):
    """With one poll per wait the look-back of a one-launch Boolean over many
    tiles may give up; the call still ends, and either its result is right
    or the timeout is reported."""
    from paper_1009_0794_gb300 import tune
    lib = ldni._lib.load()
    grid = ldni.Grid.cube(O3, 1.0, 512)
    (va, ta), (vb, tb) = M.pr1_pair()
    LA, LB = ldni.sample(va, ta, grid, 0), ldni.sample(vb, tb, grid, 0)
    ref = oracle.boolean(LA.numpy(), LB.numpy(), "union")
    prev = tune.set(bool_split=0, bool_tile_rays=256)
    assert lib.ldni_set_wait_limit(1) == 0
    try:
        info = ldni.new_info()
        out = ldni.boolean(LA, LB, "union", info=info, sync=False)
        torch.cuda.synchronize()
        st = ldni.info_decode(info)["status"]
        if not st & ldni._lib.ST_TIMEOUT:
            out.n = ldni.info_decode(info)["n"][0]
            assert bit_equal(out.numpy(), ref)
    finally:
        lib.ldni_set_wait_limit(0)
        tune.set(**prev)
