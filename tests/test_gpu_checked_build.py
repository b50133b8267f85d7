"""The checked build (compiled with LDNI_CHECKS; see ldni_build_checked in
include/ldni.h): the sampling, Boolean and volume kernels test every CSR and
slab range before they touch it and report an out-of-range one as
LDNI_ST_BOUNDS instead of accessing it.  Built into a directory of its own by
a child process, on valid inputs it must report nothing, write every output
slot (outputs are poison-filled first: NaN depths and normals, triangle id
-1) and give the oracle's results."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent('''
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, "tests")
    import meshgen as M
    import oracle
    from ldni_compare import bit_equal, compare_ldni
    import paper_1009_0794_gb300 as ldni
    from paper_1009_0794_gb300 import tune

    lib = ldni._lib.load()
    assert lib.ldni_build_checked() == 1, "not a checked build"
    O3, DIAG = (-0.5, -0.5, -0.5), 3 ** 0.5

    def poison(L):
        for t in (L.depth, L.nx, L.ny, L.nz):
            t.fill_(float("nan"))
        L.tri.fill_(-1)

    def clean(L, n):
        return bool(torch.isfinite(L.depth[:n]).all()) and bool((L.tri[:n] != -1).all())

    def status_ok(info):
        st = ldni.info_decode(info)["status"]
        assert not st & ldni._lib.ST_BOUNDS, "out-of-range index reported"
        return st

    A, B = M.pr1_pair()
    for res in (77, 128):
        grid = ldni.Grid.cube(O3, 1.0, res)
        ref = [oracle.sample(*A, O3, 1.0, res, a, "scan") for a in range(3)]
        caps = [int(r["offsets"][-1]) for r in ref]
        vt, tt = torch.from_numpy(A[0]).cuda(), torch.from_numpy(A[1]).cuda()
        for mode in ("exact2", "binned2"):
            plan = ldni.SamplePlan(len(A[0]), len(A[1]), grid, caps, mode=mode)
            for L in plan.outs:
                poison(L)
            plan.run(vt, tt)
            outs = plan.finish()
            for a in range(3):
                assert clean(outs[a], outs[a].n), (mode, a)
                compare_ldni(outs[a].numpy(), ref[a], DIAG)
        for layers in (2, 0):  # 0: every tile with a crossing overflows and is redone exactly
            plan = ldni.LearnedPlan(len(A[0]), len(A[1]), grid, caps, slab_samples=4 * res * res, net=None,
                                    layers=layers)
            for L in plan.outs:
                poison(L)
            plan.run(vt, tt)
            outs = plan.finish()
            for a in range(3):
                assert clean(outs[a], outs[a].n), ("learned", layers, a)
                compare_ldni(outs[a].numpy(), ref[a], DIAG)
        LA = ldni.sample(*A, grid, "all")
        LB = ldni.sample(*B, grid, "all")
        for split in (0, 1):
            prev = tune.set(bool_split=split)
            try:
                for op in ("union", "inter", "diff"):
                    for a in range(3):
                        out = ldni.empty_layers(grid, a, LA[a].capacity + LB[a].capacity)
                        poison(out)
                        info = ldni.new_info()
                        ldni.boolean(LA[a], LB[a], op, eps=1e-5, out=out, info=info, sync=False)
                        torch.cuda.synchronize()
                        status_ok(info)
                        out.n = ldni.info_decode(info)["n"][0]
                        assert clean(out, out.n), (split, op, a)
                        assert bit_equal(out.numpy(), oracle.boolean(LA[a].numpy(), LB[a].numpy(), op, eps=1e-5))
                vols = torch.zeros(3, dtype=torch.float64, device="cuda")
                U = ldni.boolean_many(LA, LB, "union", vols=vols)
                for a in range(3):
                    want = oracle.volume(U[a].numpy(), grid.h)
                    assert abs(float(vols[a]) - want) <= 1e-12 * abs(want) + 1e-15, (split, a)
            finally:
                tune.set(**prev)
        for L in LA:
            info = ldni.new_info()
            v = ldni.volume(L, info=info)
            status_ok(info)
            assert abs(v - oracle.volume(L.numpy(), grid.h)) <= 1e-12 * abs(v) + 1e-15
    # deep rays (ordered from the slab, or in place after a redo) and multi-layer Booleans (general merge)
    mesh = M.slab_stack(40, axis=1, seed=40)
    grid = ldni.Grid.cube(O3, 1.0, 48)
    ref = [oracle.sample(*mesh, O3, 1.0, 48, a, "scan") for a in range(3)]
    caps = [int(r["offsets"][-1]) for r in ref]
    vt, tt = torch.from_numpy(mesh[0]).cuda(), torch.from_numpy(mesh[1]).cuda()
    for layers in (0, 64):
        plan = ldni.LearnedPlan(len(mesh[0]), len(mesh[1]), grid, caps, slab_samples=64 * 3 * 48 * 48, net=None,
                                layers=layers)
        for L in plan.outs:
            poison(L)
        plan.run(vt, tt)
        outs = plan.finish()
        for a in range(3):
            assert clean(outs[a], outs[a].n), ("deep", layers, a)
            compare_ldni(outs[a].numpy(), ref[a], DIAG)
    grid = ldni.Grid.cube(O3, 1.0, 150)
    FL = ldni.sample(*M.flower(64, 64), grid, "all")
    KN = ldni.sample(*M.torus_knot(n_ring=96, n_side=12), grid, "all")
    for op in ("union", "inter", "diff"):
        for a in range(3):
            info = ldni.new_info()
            out = ldni.boolean(FL[a], KN[a], op, eps=1e-5, info=info, sync=False)
            torch.cuda.synchronize()
            status_ok(info)
            out.n = ldni.info_decode(info)["n"][0]
            assert bit_equal(out.numpy(), oracle.boolean(FL[a].numpy(), KN[a].numpy(), op, eps=1e-5)), (op, a)
    print("checked build ok")
''')


def test_checked_build_reports_nothing_and_writes_every_slot(tmp_path):
    env = dict(os.environ, LDNI_BUILD_DIR=str(tmp_path / "checked"), LDNI_EXTRA_NVCC_FLAGS="-DLDNI_CHECKS")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1500)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "checked build ok" in r.stdout


def test_release_build_is_not_checked():
    import paper_1009_0794_gb300 as ldni
    assert ldni._lib.load().ldni_build_checked() == 0
