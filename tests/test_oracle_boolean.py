"""Pins of the Boolean and volume oracles (Section 4.1, 4.1.1; Figure 6)
against set identities, exact interval answers and point membership."""
import numpy as np
import pytest

import meshgen as M
import oracle

O3 = [-0.5, -0.5, -0.5]


def _ldni(mesh, res, axis):
    return oracle.as_f32(oracle.sample(*mesh, O3, 1.0, res, axis, "scan"))


@pytest.fixture(scope="module")
def pr1_64():
    A, B = M.pr1_pair()
    return [(_ldni(A, 64, ax), _ldni(B, 64, ax)) for ax in range(3)]


def _same_depths(X, Y):
    return np.array_equal(X["offsets"], Y["offsets"]) and np.array_equal(X["depth"], Y["depth"])


def _bit_equal(X, Y):
    return (_same_depths(X, Y) and np.array_equal(X["nrm"], Y["nrm"])
            and np.array_equal(X["tri"], Y["tri"]))


def test_idempotence_and_empty_differences(pr1_64):
    """A u A = A and A n A = A bit for bit; A \\ A and (A n B) \\ A are empty
    when everything lives on one grid (Figure 6 (e)-(f))."""
    for A, B in pr1_64:
        assert _bit_equal(oracle.boolean(A, A, "union"), A)
        assert _bit_equal(oracle.boolean(A, A, "inter"), A)
        assert oracle.boolean(A, A, "diff")["depth"].size == 0
        AB = oracle.boolean(A, B, "inter")
        assert oracle.boolean(AB, A, "diff")["depth"].size == 0


def test_commutativity_and_decomposition(pr1_64):
    """A u B = B u A, A n B = B n A as depth sets, and (A \\ B) u (A n B) = A."""
    for A, B in pr1_64:
        assert _same_depths(oracle.boolean(A, B, "union"), oracle.boolean(B, A, "union"))
        assert _same_depths(oracle.boolean(A, B, "inter"), oracle.boolean(B, A, "inter"))
        D = oracle.boolean(A, B, "diff")
        I = oracle.boolean(A, B, "inter")
        assert _same_depths(oracle.boolean(D, I, "union"), A)


def _inside(d, t):
    return (np.searchsorted(d, t, side="left") % 2) == 1


def test_midpoint_membership(pr1_64):
    """Between consecutive output depths (and outside them) the result's
    membership equals op(member of A, member of B) at the midpoint, checked
    against every event depth of A and B; every output sample is a copy of an
    input sample (normal inverted for B in a difference)."""
    ops = {"union": np.logical_or, "inter": np.logical_and, "diff": lambda a, b: a & ~b}
    for A, B in pr1_64:
        for name, f in ops.items():
            R = oracle.boolean(A, B, name)
            nr = R["offsets"].size - 1
            for p in range(nr):
                da = A["depth"][A["offsets"][p]:A["offsets"][p + 1]]
                db = B["depth"][B["offsets"][p]:B["offsets"][p + 1]]
                dr = R["depth"][R["offsets"][p]:R["offsets"][p + 1]]
                ev = np.unique(np.concatenate([da, db, dr]).astype(np.float64))
                if ev.size == 0:
                    continue
                mids = np.concatenate([[ev[0] - 1], (ev[:-1] + ev[1:]) / 2, [ev[-1] + 1]])
                want = f(_inside(da.astype(np.float64), mids), _inside(db.astype(np.float64), mids))
                got = _inside(dr.astype(np.float64), mids)
                assert np.array_equal(want, got), (name, p)
            # provenance
            for k in range(R["depth"].size):
                tid = int(R["tri"][k])
                src = B if tid < 0 else A
                sid = tid & 0x7FFFFFFF
                m = np.nonzero((src["tri"] == sid) & (src["depth"] == R["depth"][k]))[0]
                assert m.size >= 1
                sgn = -1.0 if (tid < 0 and name == "diff") else 1.0
                assert np.any(np.all(src["nrm"][m] * sgn == R["nrm"][k], axis=1))


def test_two_boxes_exact_intervals():
    """Overlapping boxes along z: intervals are the closed-form 1D answers."""
    res = 16
    a = M.box([-0.3, -0.3, -0.4], [0.3, 0.3, 0.1])
    b = M.box([-0.1, -0.1, -0.05], [0.2, 0.2, 0.3])
    A, B = _ldni(a, res, 2), _ldni(b, res, 2)
    f32 = np.float32
    U = oracle.boolean(A, B, "union")
    I = oracle.boolean(A, B, "inter")
    D = oracle.boolean(A, B, "diff")
    c = -0.5 + (np.arange(res) + 0.5) / res
    for j in range(res):
        for i in range(res):
            p = j * res + i
            ina = -0.3 < c[i] < 0.3 and -0.3 < c[j] < 0.3
            inb = -0.1 < c[i] < 0.2 and -0.1 < c[j] < 0.2
            seg = lambda R: R["depth"][R["offsets"][p]:R["offsets"][p + 1]].tolist()
            if ina and inb:
                assert seg(U) == [f32(-0.4), f32(0.3)]
                assert seg(I) == [f32(-0.05), f32(0.1)]
                assert seg(D) == [f32(-0.4), f32(-0.05)]
                k = D["offsets"][p] + 1
                assert D["tri"][k] < 0 and D["nrm"][k].tolist() == [0.0, 0.0, 1.0]  # inverted bottom face of B
            elif ina:
                assert seg(U) == [f32(-0.4), f32(0.1)] and seg(I) == [] and seg(D) == [f32(-0.4), f32(0.1)]
            elif inb:
                assert seg(U) == [f32(-0.05), f32(0.3)] and seg(I) == [] and seg(D) == []
            else:
                assert seg(U) == seg(I) == seg(D) == []


def test_small_interval_removal():
    """Solid intervals thinner than eps are removed (Section 4.1.1); a
    tangential contact union does not leave a gap or sliver."""
    res = 8
    a = M.box([-0.3, -0.3, -0.4], [0.3, 0.3, 0.1])
    b = M.box([-0.3, -0.3, 0.1 - 4e-6], [0.3, 0.3, 0.35])
    A, B = _ldni(a, res, 2), _ldni(b, res, 2)
    I0 = oracle.boolean(A, B, "inter", eps=0.0)
    I1 = oracle.boolean(A, B, "inter", eps=1e-5)
    assert I0["depth"].size > 0 and I1["depth"].size == 0
    D1 = oracle.boolean(A, B, "diff", eps=1e-5)
    assert np.all(np.diff(D1["offsets"]) % 2 == 0)
    # the test is strict: an interval exactly eps thick survives
    c = M.box([-0.3, -0.3, 0.0], [0.3, 0.3, 0.25])
    C = _ldni(c, res, 2)
    assert oracle.boolean(C, C, "inter", eps=0.25)["depth"].size == C["depth"].size > 0
    assert oracle.boolean(C, C, "inter", eps=np.nextafter(np.float32(0.25), np.float32(1)))["depth"].size == 0


def test_volume_inclusion_exclusion(pr1_64):
    """V(A u B) + V(A n B) = V(A) + V(B) and V(A \\ B) = V(A) - V(A n B)."""
    h = 1.0 / 64
    for A, B in pr1_64:
        vA, vB = oracle.volume(A, h), oracle.volume(B, h)
        vU = oracle.volume(oracle.boolean(A, B, "union"), h)
        vI = oracle.volume(oracle.boolean(A, B, "inter"), h)
        vD = oracle.volume(oracle.boolean(A, B, "diff"), h)
        assert vU + vI == pytest.approx(vA + vB, rel=1e-12)
        assert vD == pytest.approx(vA - vI, rel=1e-12)
        assert vI > 0 and vD > 0


def test_odd_input_rejected():
    L = {"offsets": np.array([0, 1]), "depth": np.array([0.1], np.float32),
         "nrm": np.zeros((1, 3), np.float32), "tri": np.zeros(1, np.int32)}
    with pytest.raises(ValueError):
        oracle.boolean(L, L, "union")
    with pytest.raises(ValueError):
        oracle.volume(L, 1.0)
