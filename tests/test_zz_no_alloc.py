"""ldni_boolean_static, the Boolean entry point that takes no workspace.

It exists for callers that cannot allocate device memory where they need a
Boolean (code handed only input and output buffers because another framework
owns the allocator, or a loop where an allocation would synchronise the
device); its scratch is a static device array inside the library.  Called
through the C ABI, its result must equal ldni_boolean's bit for bit - the
Boolean tolerance of this suite - on two calls in a row, so that the second
call runs on the scratch the first one left behind.  This file is collected
last on purpose."""
import ctypes

import numpy as np
import pytest

import meshgen as M
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


def _static_boolean(ldni, A, B, op, eps):
    lib = ldni._lib.load()
    out = ldni.empty_layers(A.grid, A.axis, A.capacity + B.capacity)
    info = ldni.new_info()
    la, lb, lo = A.c(), B.c(), out.c()
    ga, gb = A.grid.c(), B.grid.c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.ldni_boolean_static(ctypes.byref(la), ctypes.byref(ga), ctypes.byref(lb), ctypes.byref(gb),
                                 ldni.OPS[op], float(eps), ctypes.byref(lo), info.data_ptr(), stream)
    assert rc == 0, ldni._lib.strerror(rc)
    meta = ldni.info_decode(info)
    assert meta["status"] == 0
    out.n = meta["n"][0]
    return out


def test_static_boolean_matches_workspace_boolean(ldni):
    (va, ta), (vb, tb) = M.pr1_pair()
    (fv, ft), (kv, kt) = M.flower(64, 64), M.torus_knot(n_ring=96, n_side=12)
    for res in (128, 1024):
        grid = ldni.Grid.cube(O3, 1.0, res)
        pairs = [(ldni.sample(va, ta, grid, "all"), ldni.sample(vb, tb, grid, "all")),
                 (ldni.sample(fv, ft, grid, "all"), ldni.sample(kv, kt, grid, "all"))]
        for a in range(3):
            for op in ("union", "inter", "diff"):
                for eps in (0.0, 1e-5):
                    for call in range(2):
                        # alternate operand pairs so that a call starts on the
                        # other pair's leftover scratch
                        A, B = pairs[call % 2][0][a], pairs[call % 2][1][a]
                        ref = ldni.boolean(A, B, op, eps=eps).numpy()
                        got = _static_boolean(ldni, A, B, op, eps).numpy()
                        assert bit_equal(got, ref), (res, a, op, eps, call)


def test_static_boolean_limit_and_grid_checks(ldni):
    lib = ldni._lib.load()
    (va, ta), _ = M.pr1_pair()
    g_big = ldni.Grid.cube(O3, 1.0, 1025)
    A = ldni.sample(va, ta, g_big, 0)
    out = ldni.empty_layers(g_big, 0, 2 * A.capacity)
    info = ldni.new_info()
    la, lo, g = A.c(), out.c(), g_big.c()
    rc = lib.ldni_boolean_static(ctypes.byref(la), ctypes.byref(g), ctypes.byref(la), ctypes.byref(g), 0, 0.0,
                                 ctypes.byref(lo), info.data_ptr(), None)
    assert rc == -4  # res beyond the static scratch: LDNI_ETOOLARGE
    g2 = ldni.Grid.cube(O3, 1.0, 512).c()
    g3 = ldni.Grid.cube((-0.5, -0.5, -0.4), 1.0, 512).c()
    rc = lib.ldni_boolean_static(ctypes.byref(la), ctypes.byref(g2), ctypes.byref(la), ctypes.byref(g3), 0, 0.0,
                                 ctypes.byref(lo), info.data_ptr(), None)
    assert rc == -2  # LDNI_EGRID_MISMATCH
