"""CUDA grid-node classification (ldni_classify_nodes) against the oracle,
bit for bit, on ragged and multi-word resolutions."""
import numpy as np
import pytest

import meshgen as M
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


@pytest.mark.parametrize("res", [32, 45, 70])
def test_matches_oracle(ldni, res):
    A, B = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, res)
    for mesh in (A, B, M.flower(48, 48)):
        L = ldni.sample(*mesh, grid, "all")
        got = ldni.unpack_nodes(ldni.classify_nodes(L), res)
        ref = nodes.classify([x.numpy() for x in L], O3, 1.0, res)
        assert np.array_equal(got, ref)


def test_padding_bits_are_zero(ldni):
    res = 45
    A, _ = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, res)
    words = ldni.classify_nodes(ldni.sample(*A, grid, "all")).cpu().numpy().view(np.uint32)
    assert words.shape == (res, res, 2)
    assert not (words[:, :, 1] >> (res - 32)).any()


def test_union_of_two_solids(ldni):
    """Nodes of A u B are the nodes inside A or inside B wherever all three
    votes agree (away from either surface)."""
    A, B = M.pr1_pair()
    res = 40
    grid = ldni.Grid.cube(O3, 1.0, res)
    LA, LB = ldni.sample(*A, grid, "all"), ldni.sample(*B, grid, "all")
    U = ldni.boolean_many(LA, LB, "union")
    na = ldni.unpack_nodes(ldni.classify_nodes(LA), res)
    nb = ldni.unpack_nodes(ldni.classify_nodes(LB), res)
    nu = ldni.unpack_nodes(ldni.classify_nodes(U), res)
    ref = nodes.classify([x.numpy() for x in U], O3, 1.0, res)
    assert np.array_equal(nu, ref)
    assert (nu | ~(na | nb)).mean() > 0.99 and (~nu | (na | nb)).mean() > 0.99
