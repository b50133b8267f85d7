"""Approximate 8-bit normals (Section 3 item 1) through the C ABI.

* The codec kernels agree with the oracle codec bit for bit.
* Sampling with packed normals (exact two-pass, learned one-pass, every
  ordering tier) gives the offsets, depths and ids of FP32 sampling, and
  codes equal to the oracle codec applied to the oracle's normals except
  where the normal lies within rounding of a code boundary.
* The Boolean on packed images equals the packed-Boolean oracle bit for bit.
"""
import numpy as np
import pytest

import meshgen as M
import oracle
from ldni_compare import bit_equal
from oracle import normals8 as N8

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


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_codec_matches_oracle(ldni):
    rng = np.random.default_rng(3)
    n = rng.normal(size=(200000, 3))
    n = (n / np.linalg.norm(n, axis=1, keepdims=True)).astype(np.float32)
    # exact levels, half-way points between levels, the ends, out of range
    lv = (np.arange(256) / 127.5 - 1.0).astype(np.float32)
    half = ((np.arange(255) + 0.5) / 127.5 - 1.0).astype(np.float32)
    extra = np.concatenate([lv, half, np.float32([-1, 1, 0, -0.0, 2, -2, 1e-30])])
    extra = np.stack([extra, extra[::-1], np.roll(extra, 7)], 1).astype(np.float32)
    n = np.concatenate([n, extra])
    w = ldni.encode_normals8(_t(n[:, 0]), _t(n[:, 1]), _t(n[:, 2])).cpu().numpy().view(np.uint32)
    assert np.array_equal(w, N8.encode(n))
    q = np.arange(256, dtype=np.uint32)
    words = (q[:, None, None] | (q[None, :, None] << 8) | (q[None, None, ::5] << 16)).ravel()
    got = ldni.decode_normals8(_t(words.view(np.int32)))
    want = N8.decode(words)
    for c in range(3):
        assert np.array_equal(got[c].cpu().numpy(), want[:, c])


def _near_boundary(nrm64):
    """Components whose scaled value (n + 1) * 127.5 lies within 1e-3 of a
    rounding boundary (a half-integer), where FP32 and FP64 normals may pick
    neighbouring codes."""
    v = (nrm64 + 1.0) * 127.5
    return np.abs(v - np.floor(v) - 0.5) < 1e-3


def _check_against_oracle(ldni, got_packed, got_fp32, ref):
    """got_packed, got_fp32: numpy dicts of the same sampling in the two
    formats; ref: the FP64 oracle's."""
    for k in ("offsets", "depth", "tri"):
        assert np.array_equal(got_packed[k], got_fp32[k]), k
    # the packed codes are the library's own encoding of its FP32 normals
    n = got_fp32["nrm"]
    own = ldni.encode_normals8(_t(n[:, 0]), _t(n[:, 1]), _t(n[:, 2])).cpu().numpy().view(np.uint32)
    assert np.array_equal(got_packed["nrm8"], own)
    # and the oracle's normals up to rounding at code boundaries: match
    # samples by (ray, triangle)
    off = ref["offsets"]
    ray = np.repeat(np.arange(off.size - 1), np.diff(off))
    ig = np.lexsort((got_packed["tri"], ray))
    ir = np.lexsort((ref["tri"], ray))
    qg = N8.codes(got_packed["nrm8"][ig])
    qr = N8.codes(N8.encode(ref["nrm"][ir].astype(np.float32)))
    diff = np.abs(qg - qr)
    assert diff.max(initial=0) <= 1
    assert np.all(_near_boundary(ref["nrm"][ir])[diff == 1])


@pytest.mark.parametrize("mesh_name", ["pr1_sphere", "flower", "slab_stack_100"])
def test_packed_sampling(ldni, mesh_name):
    mesh = {"pr1_sphere": lambda: M.pr1_pair()[0], "flower": lambda: M.flower(96, 96),
            "slab_stack_100": lambda: M.slab_stack(100, axis=1, seed=100)}[mesh_name]()
    res = 96 if mesh_name != "slab_stack_100" else 48
    grid = ldni.Grid.cube(O3, 1.0, res)
    fp = [L.numpy() for L in ldni.sample(*mesh, grid, "all")]
    pk = [L.numpy() for L in ldni.sample(*mesh, grid, "all", packed=True)]
    for a in range(3):
        ref = oracle.sample(*mesh, O3, 1.0, res, a, "scan")
        _check_against_oracle(ldni, pk[a], fp[a], ref)


def test_packed_learned_equals_exact(ldni):
    for mesh, res in ((M.pr1_pair()[0], 128), (M.slab_stack(40, axis=0, seed=4), 48)):
        grid = ldni.Grid.cube(O3, 1.0, res)
        ex = [L.numpy() for L in ldni.sample(*mesh, grid, "all", packed=True)]
        v, t = torch.from_numpy(mesh[0]).cuda(), torch.from_numpy(mesh[1]).cuda()
        for layers in (0, 2, 64):
            got = ldni.sample_learned(v, t, grid, layers=layers, packed=True,
                                      slab_samples=max(4, layers) * 3 * res * res,
                                      capacity_hint=max(int(L["offsets"][-1]) for L in ex))
            for a in range(3):
                g = got[a].numpy()
                for k in ("offsets", "depth", "tri", "nrm8"):
                    assert np.array_equal(g[k], ex[a][k]), (layers, a, k)


def _packed_oracle_image(mesh, res, a):
    L = oracle.as_f32(oracle.sample(*mesh, O3, 1.0, res, a, "scan"))
    return {"offsets": L["offsets"], "depth": L["depth"], "tri": L["tri"], "nrm8": N8.encode(L["nrm"])}


def _upload_packed(ldni, grid, a, L):
    n = int(L["offsets"][-1])
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    return ldni.LDNI(grid, a, _t(L["offsets"].astype(np.int32)), _t(L["depth"]), e, e, e, _t(L["tri"]), n,
                     nrm8=_t(L["nrm8"].view(np.int32)))


@pytest.mark.parametrize("op", ["union", "inter", "diff"])
def test_packed_boolean(ldni, op):
    A, B = M.pr1_pair()
    res = 100
    grid = ldni.Grid.cube(O3, 1.0, res)
    for a in range(3):
        la, lb = _packed_oracle_image(A, res, a), _packed_oracle_image(B, res, a)
        ga, gb = _upload_packed(ldni, grid, a, la), _upload_packed(ldni, grid, a, lb)
        for eps in (0.0, 0.01):
            got = ldni.boolean(ga, gb, op, eps=eps).numpy()
            want = N8.boolean(la, lb, op, eps)
            assert np.array_equal(got["offsets"], want["offsets"])
            for k in ("depth", "tri", "nrm8"):
                assert np.array_equal(got[k], want[k]), (a, eps, k)
        many = ldni.boolean_many([ga], [gb], op)[0].numpy()
        want = N8.boolean(la, lb, op, 0.0)
        assert np.array_equal(many["nrm8"], want["nrm8"]) and np.array_equal(many["depth"], want["depth"])


def test_mixed_formats_rejected(ldni):
    A, B = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, 32)
    pa = ldni.sample(*A, grid, 0, packed=True)
    fb = ldni.sample(*B, grid, 0)
    with pytest.raises(ldni.LDNIError):
        ldni.boolean(pa, fb, "union")
