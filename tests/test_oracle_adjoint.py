"""Pins of the FP64 adjoint oracle: central finite differences of the
frozen-set depths and volume, translation invariance, and convergence of the
LDNI volume gradient to the exact mesh-volume gradient (divergence theorem)."""
import numpy as np
import pytest

import meshgen as M
import oracle
from oracle import adjoint as AD

O3 = [-0.5, -0.5, -0.5]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_volume_gradient_matches_central_differences(axis):
    v, t = M.icosphere(4, r=0.3, noise=0.04, seed=3)
    res = 48
    L = oracle.sample(v, t, O3, 1.0, res, axis, "scan")
    fs = AD.frozen_set(L, res, axis, O3, 1.0)
    h = 1.0 / res
    g = AD.volume_grad(v, t, fs, axis, h)
    rng = np.random.default_rng(axis)
    V = v.astype(np.float64)
    eps = 1e-6
    for j in rng.choice(len(v), 25, replace=False):
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[j, c] += eps
            Vm[j, c] -= eps
            fd = (AD.volume(Vp, t, fs, axis, h) - AD.volume(Vm, t, fs, axis, h)) / (2 * eps)
            assert abs(fd - g[j, c]) <= 1e-6 * max(1e-3, abs(fd)), (j, c, fd, g[j, c])


def test_depth_vjp_matches_central_differences():
    v, t = M.torus(0.25, 0.1, 12, 8)
    axis, res = 2, 40
    L = oracle.sample(v, t, O3, 1.0, res, axis, "scan")
    fs = AD.frozen_set(L, res, axis, O3, 1.0)
    w = np.random.default_rng(0).normal(size=fs[0].size)
    g = AD.depth_vjp(v, t, fs, axis, w)
    V = v.astype(np.float64)
    f = lambda X: float(np.sum(w * AD.depths(X, t, fs[0], fs[1], fs[2], axis)))
    for j in range(0, len(v), 13):
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[j, c] += 1e-6
            Vm[j, c] -= 1e-6
            fd = (f(Vp) - f(Vm)) / 2e-6
            assert abs(fd - g[j, c]) <= 1e-5 * max(1.0, abs(fd))


def test_frozen_depths_equal_sampled_depths_up_to_snap():
    """The continuous plane depth of a recorded sample differs from the
    sampled (snapped-barycentric) depth only through the subpixel snap: at
    most the face slope |n_uv| / |n_a| times the snap shift (h/512 per
    coordinate, to first order)."""
    v, t = M.icosphere(6, r=0.3, noise=0.02, seed=1)
    res = 64
    for axis in range(3):
        L = oracle.sample(v, t, O3, 1.0, res, axis, "scan")
        fs = AD.frozen_set(L, res, axis, O3, 1.0)
        d = AD.depths(v, t, fs[0], fs[1], fs[2], axis)
        n = L["nrm"]
        iu, iv = (axis + 1) % 3, (axis + 2) % 3
        slope = (np.abs(n[:, iu]) + np.abs(n[:, iv])) / np.abs(n[:, axis])
        bound = 1.5 * slope * (1.0 / res) / 512 + 1e-12
        assert np.all(np.abs(d - L["depth"]) <= bound)


def test_translation_invariance():
    """Moving the whole mesh along the view axis leaves the volume unchanged:
    the a-components of the gradient sum to zero."""
    v, t = M.icosphere(5, r=0.3, noise=0.05, seed=2)
    for axis in range(3):
        L = oracle.sample(v, t, O3, 1.0, 64, axis, "scan")
        fs = AD.frozen_set(L, 64, axis, O3, 1.0)
        g = AD.volume_grad(v, t, fs, axis, 1.0 / 64)
        assert abs(g[:, axis].sum()) < 1e-12


def test_converges_to_mesh_volume_gradient():
    v, t = M.icosphere(6, r=0.33, noise=0.03, noise_kind="octave", seed=4)
    ref = AD.mesh_volume_grad(v, t)
    errs = []
    for res in (64, 128, 256):
        gs = []
        for axis in range(3):
            L = oracle.sample(v, t, O3, 1.0, res, axis, "scan")
            gs.append(AD.volume_grad(v, t, AD.frozen_set(L, res, axis, O3, 1.0), axis, 1.0 / res))
        g = sum(gs) / 3.0
        errs.append(np.linalg.norm(g - ref) / np.linalg.norm(ref))
    assert errs[2] < errs[0]
    assert errs[2] < 0.15
