"""FP64 statement of the per-tile capacity network (TEST INFRASTRUCTURE ONLY).

Architecture 12 -> 64 -> 64 -> 64 -> 1, ReLU on hidden layers; parameters in
the flat layout of the library (weights row-major [out][in], layers
concatenated; biases b0, b1, b2, b3).  Weights enter as the BF16 values the
kernels use, widened exactly to FP64.  Loss: mean_r w_r (y_r - t_r)^2 with
w_r = under_weight when y_r < t_r, else 1.  The gradient is the textbook
backward pass of that composition; test_oracle_mlp pins it with central
finite differences.
"""
import numpy as np

SHAPES = [(64, 12), (64, 64), (64, 64), (1, 64)]


def unpack(w, b):
    Ws, Bs, k, j = [], [], 0, 0
    for (o, i) in SHAPES:
        Ws.append(np.asarray(w[k:k + o * i], dtype=np.float64).reshape(o, i))
        Bs.append(np.asarray(b[j:j + o], dtype=np.float64))
        k += o * i
        j += o
    return Ws, Bs


def forward(w, b, X):
    Ws, Bs = unpack(w, b)
    A = np.asarray(X, dtype=np.float64)
    cache = [A]
    for l, (W, B) in enumerate(zip(Ws, Bs)):
        Z = A @ W.T + B
        A = np.maximum(Z, 0.0) if l < 3 else Z
        cache.append((Z, A))
    return A[:, 0], cache


def loss(w, b, X, t, under_weight=4.0):
    y, _ = forward(w, b, X)
    d = y - np.asarray(t, dtype=np.float64)
    wr = np.where(d < 0, under_weight, 1.0)
    return float(np.mean(wr * d * d))


def grad(w, b, X, t, under_weight=4.0):
    """(loss, dL/dw flat, dL/db flat)."""
    Ws, Bs = unpack(w, b)
    y, cache = forward(w, b, X)
    n = y.shape[0]
    d = y - np.asarray(t, dtype=np.float64)
    wr = np.where(d < 0, under_weight, 1.0)
    L = float(np.mean(wr * d * d))
    dZ = (2.0 * wr * d / n)[:, None]
    gWs, gBs = [None] * 4, [None] * 4
    for l in range(3, -1, -1):
        A_in = cache[l] if l == 0 else cache[l][1]
        gWs[l] = dZ.T @ A_in
        gBs[l] = dZ.sum(0)
        if l > 0:
            dA = dZ @ Ws[l]
            Zp = cache[l][0]
            dZ = dA * (Zp > 0)
    return L, np.concatenate([g.reshape(-1) for g in gWs]), np.concatenate(gBs)
