"""Pins of the FP64 network oracle: its gradient against central finite
differences, and its forward pass on a network whose output has a closed form."""
import numpy as np

from oracle import mlp as M


def _params(seed):
    rng = np.random.default_rng(seed)
    w = np.concatenate([rng.normal(0, np.sqrt(2.0 / i), size=o * i) for o, i in M.SHAPES])
    b = rng.normal(0, 0.1, size=193)
    return w, b


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    w, b = _params(2)
    X = rng.normal(size=(7, 12))
    t = rng.normal(size=7)
    L, gw, gb = M.grad(w, b, X, t, under_weight=4.0)
    h = 1e-6
    idx_w = rng.choice(w.size, 40, replace=False)
    for k in idx_w:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (M.loss(wp, b, X, t) - M.loss(wm, b, X, t)) / (2 * h)
        assert abs(fd - gw[k]) <= 1e-6 * max(1.0, abs(fd))
    for k in range(0, 193, 7):
        bp, bm = b.copy(), b.copy()
        bp[k] += h
        bm[k] -= h
        fd = (M.loss(w, bp, X, t) - M.loss(w, bm, X, t)) / (2 * h)
        assert abs(fd - gb[k]) <= 1e-6 * max(1.0, abs(fd))
    assert L == M.loss(w, b, X, t)


def test_forward_closed_form_and_asymmetric_loss():
    """A network that copies feature 0 through one unit per layer and scales
    it by 3: y = 3 * relu(x0) + 0.5."""
    w = np.zeros(9024)
    b = np.zeros(193)
    w[0 * 12 + 0] = 1.0            # W0[0][0]
    w[768 + 0 * 64 + 0] = 1.0      # W1[0][0]
    w[4864 + 0 * 64 + 0] = 1.0     # W2[0][0]
    w[8960 + 0] = 3.0              # W3[0][0]
    b[192] = 0.5
    X = np.zeros((4, 12))
    X[:, 0] = [-1.0, 0.0, 0.25, 2.0]
    y, _ = M.forward(w, b, X)
    assert np.allclose(y, [0.5, 0.5, 1.25, 6.5])
    t = np.array([1.5, 0.5, 1.25, 5.5])  # errors -1, 0, 0, +1
    assert M.loss(w, b, X, t, under_weight=4.0) == (4.0 * 1.0 + 1.0) / 4
