"""8-bit normal codec oracle (Section 3, approximate normal sampling)
against closed forms: the codes of the axis directions, the exact round
trip of every code, the quantisation error bound of 256 levels on [-1, 1],
unit length after decoding, and inversion in code space."""
import numpy as np

from oracle import normals8 as N8


def test_axis_directions():
    e = np.eye(3, dtype=np.float32)
    w = N8.encode(np.concatenate([e, -e]))
    q = N8.codes(w)
    # +1 -> 255, -1 -> 0, 0 -> 127.5 rounded half to even -> 128
    assert q.tolist() == [[255, 128, 128], [128, 255, 128], [128, 128, 255],
                          [0, 128, 128], [128, 0, 128], [128, 128, 0]]
    assert np.all(w >> 24 == 0)
    d = N8.decode(w)
    assert np.allclose(d, np.concatenate([e, -e]), atol=6e-3)


def test_every_code_round_trips():
    q = np.arange(256, dtype=np.uint32)
    w = q | (q[::-1] << 8) | (((q * 7) % 256) << 16)
    raw = N8.decode_raw(w)
    want = 2.0 * N8.codes(w) / 255.0 - 1.0
    assert np.abs(raw - want).max() <= 2 ** -23
    assert np.array_equal(N8.encode(raw), w)  # a decoded code encodes to itself


def test_quantisation_bound_and_unit_length():
    rng = np.random.default_rng(5)
    n = rng.normal(size=(20000, 3))
    n = (n / np.linalg.norm(n, axis=1, keepdims=True)).astype(np.float32)
    w = N8.encode(n)
    raw = N8.decode_raw(w).astype(np.float64)
    assert np.abs(raw - n).max() <= 1.0 / 255 + 1e-6  # half of a level of width 2/255
    d = N8.decode(w).astype(np.float64)
    assert np.abs(np.linalg.norm(d, axis=1) - 1.0).max() < 1e-6
    # the decoded direction is within the error of the box around n
    assert np.abs(d - n).max() < 2 * np.sqrt(3) / 255


def test_inversion_and_range():
    q = np.arange(256, dtype=np.uint32)
    w = q | (q << 8) | (q << 16)
    assert np.array_equal(N8.codes(N8.invert(w)), 255 - N8.codes(w))
    assert np.abs(N8.decode_raw(N8.invert(w)) + N8.decode_raw(w)).max() <= 2 ** -23
    odd = np.array([[2.0, -3.0, np.nan], [1.0000001, -1.0000001, 0.0]], np.float32)
    assert N8.codes(N8.encode(odd)).tolist() == [[255, 0, 0], [255, 0, 128]]


def test_boolean_on_codes():
    """The packed Boolean copies codes and inverts B's in a difference: two
    nested boxes along one ray, by hand."""
    off = np.array([0, 2], np.int64)
    wa = N8.encode(np.array([[-1, 0, 0], [1, 0, 0]], np.float32))
    wb = N8.encode(np.array([[-0.6, 0.8, 0], [0.6, -0.8, 0]], np.float32))
    A = {"offsets": off, "depth": np.array([0.0, 4.0], np.float32), "nrm8": wa, "tri": np.array([1, 2], np.int32)}
    B = {"offsets": off, "depth": np.array([1.0, 2.0], np.float32), "nrm8": wb, "tri": np.array([3, 4], np.int32)}
    R = N8.boolean(A, B, "diff")
    assert R["depth"].tolist() == [0.0, 1.0, 2.0, 4.0]
    assert R["nrm8"].tolist() == [wa[0], N8.invert(wb[:1])[0], N8.invert(wb[1:])[0], wa[1]]
    U = N8.boolean(A, B, "union")
    assert U["nrm8"].tolist() == wa.tolist()
    # code 0 and 255 components survive the inversion round trip
    assert set(N8.codes(R["nrm8"]).ravel()) <= set(range(256))
