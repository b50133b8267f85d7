"""The seeded generators yield closed, outward-oriented 2-manifolds of the
stated sizes inside the unit cube (the paper's input class, Remark 2)."""
import numpy as np
import pytest

import meshgen as M


@pytest.mark.parametrize("make,nv,nt", [
    (lambda: M.icosphere(8, noise=0.03, seed=1), 642, 1280),
    (lambda: M.icosphere(100, noise=0.03, noise_kind="octave", seed=2), 100002, 200000),
    (lambda: M.torus(0.25, 0.1, 64, 32, center=(0.15, 0, 0)), 2048, 4096),
    (lambda: M.flower(64, 64), 63 * 64 + 2, 2 * 64 + 2 * 62 * 64),
    (lambda: M.torus_knot(), 8192, 16384),
    (lambda: M.box([-0.2] * 3, [0.1] * 3), 8, 12),
    (lambda: M.octahedron([0, 0, 0], 0.2), 6, 8),
])
def test_closed_oriented(make, nv, nt):
    v, t = make()
    assert v.dtype == np.float32 and t.dtype == np.int32
    assert v.shape == (nv, 3) and t.shape == (nt, 3)
    M.check_closed_oriented(t, nv)
    assert M.signed_volume(v, t) > 0
    assert np.all(np.abs(v) <= 0.5)


def test_seeded_and_deterministic():
    a = M.icosphere(8, noise=0.03, seed=5)
    b = M.icosphere(8, noise=0.03, seed=5)
    c = M.icosphere(8, noise=0.03, seed=6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])


def test_geodesic_sphere_volume_and_locality():
    v, t = M.icosphere(32, r=0.35)
    assert M.signed_volume(v, t) == pytest.approx(4 / 3 * np.pi * 0.35**3, rel=2e-3)
    # consecutive triangles share vertices most of the time (memory locality)
    share = [len(set(t[i]) & set(t[i + 1])) > 0 for i in range(len(t) - 1)]
    assert np.mean(share) > 0.9


def test_torus_knot_tube_embedded():
    """Tube radius below the curvature radius and half the strand clearance."""
    p, q, R, rho, tube = 2, 3, 0.25, 0.1, 0.035
    s = np.linspace(0, 2 * np.pi, 1500, endpoint=False)
    c = np.stack([(R + rho * np.cos(q * s)) * np.cos(p * s), (R + rho * np.cos(q * s)) * np.sin(p * s),
                  rho * np.sin(q * s)], -1)
    d = np.linalg.norm(c[:, None] - c[None], axis=-1)
    ds = np.abs(s[:, None] - s[None])
    ds = np.minimum(ds, 2 * np.pi - ds)
    assert d[ds > 0.6].min() > 2 * tube
