"""The per-tile capacity network of the one-pass sampler: parameters,
training on exact layer counts, persistence.

Every computation (features, labels, forward, backward, Adam) runs in the
library's CUDA kernels; this module only holds the device buffers.  The
network predicts log1p(largest ray count of a tile) from the tile's features
(ldni_tile_features); the label comes from an exact sampling of the same mesh
(ldni_sample_count + ldni_tile_labels).
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence, Tuple

import numpy as np
import torch

from . import _lib
from .ldni import Grid, _dev, _stream_ptr, auto_stride, empty_layers, new_info, ntiles, sample_workspace_size

H = 64
LAYERS = [(12, H), (H, H), (H, H), (H, 1)]  # (in, out)


def init_params(seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """He-uniform weights, zero biases except the output bias (log1p(2): the
    two-layer answer of a convex patch)."""
    rng = np.random.default_rng(seed)
    ws = []
    for fi, fo in LAYERS:
        lim = np.sqrt(6.0 / fi)
        ws.append(rng.uniform(-lim, lim, size=(fo, fi)).reshape(-1))
    b = np.zeros(_lib.MLP_BIASES, dtype=np.float32)
    b[-1] = np.log1p(2.0)
    return np.concatenate(ws).astype(np.float32), b


def to_bf16_bits(w: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even FP32 -> BF16, as uint16 bit patterns."""
    u = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) >> 16).astype(np.uint16)


def from_bf16_bits(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32)


class CapacityNet:
    def __init__(self, seed: int = 0, w: np.ndarray = None, b: np.ndarray = None):
        if w is None:
            w, b = init_params(seed)
        self.w = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda()
        self.b = torch.from_numpy(np.ascontiguousarray(b, dtype=np.float32)).cuda()
        self.w16 = torch.from_numpy(to_bf16_bits(w).view(np.int16)).cuda()
        n = _lib.MLP_WEIGHTS + _lib.MLP_BIASES
        self.m = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.v = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.step = 0
        self._mlp_keep = []

    def c(self, margin: float = 0.25) -> _lib.MLP:
        m = _lib.MLP()
        m.w = self.w16.data_ptr()
        m.b = self.b.data_ptr()
        m.margin = float(margin)
        return m

    def forward(self, X: torch.Tensor, stream=None) -> torch.Tensor:
        X = X.contiguous()
        y = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        m = self.c()
        _lib.check(_lib.load().ldni_mlp_forward(ctypes.byref(m), X.data_ptr(), X.shape[0], y.data_ptr(),
                                                _stream_ptr(stream)), "ldni_mlp_forward")
        return y

    def train_step(self, X: torch.Tensor, label: torch.Tensor, lr: float = 1e-3, under_weight: float = 4.0,
                   want_grad: bool = False, ws: torch.Tensor = None):
        lib = _lib.load()
        n = X.shape[0]
        if ws is None:
            sz = ctypes.c_size_t(0)
            _lib.check(lib.ldni_mlp_train_workspace_size(n, ctypes.byref(sz)), "ldni_mlp_train_workspace_size")
            ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        grad = torch.empty(_lib.MLP_WEIGHTS + _lib.MLP_BIASES, dtype=torch.float32, device="cuda") if want_grad else None
        self.step += 1
        _lib.check(lib.ldni_mlp_train_step(self.w.data_ptr(), self.b.data_ptr(), self.w16.data_ptr(),
                                           self.m.data_ptr(), self.v.data_ptr(), X.data_ptr(), label.data_ptr(), n,
                                           float(lr), self.step, float(under_weight), loss.data_ptr(),
                                           grad.data_ptr() if grad is not None else None, ws.data_ptr(), ws.numel(),
                                           _stream_ptr(None)), "ldni_mlp_train_step")
        return (loss, grad) if want_grad else loss

    def fit(self, X: torch.Tensor, label: torch.Tensor, steps: int = 1500, batch: int = 4096, lr: float = 2e-3,
            under_weight: float = 4.0, seed: int = 0) -> List[float]:
        """Adam on minibatches of a once-shuffled copy of the rows."""
        perm = torch.from_numpy(np.random.default_rng(seed).permutation(X.shape[0])).cuda()
        Xs, Ls = X[perm].contiguous(), label[perm].contiguous()
        n = X.shape[0]
        batch = min(batch, n)
        sz = ctypes.c_size_t(0)
        _lib.check(_lib.load().ldni_mlp_train_workspace_size(batch, ctypes.byref(sz)), "ldni_mlp_train_workspace_size")
        ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
        losses = []
        nb = max(1, n // batch)
        for k in range(steps):
            s0 = (k % nb) * batch
            lrk = lr * (0.1 ** (k / max(1, steps)))  # decays to lr / 10
            loss = self.train_step(Xs[s0:s0 + batch], Ls[s0:s0 + batch], lrk, under_weight, ws=ws)
            if k % 50 == 0 or k == steps - 1:
                losses.append(float(loss.item()))
        return losses

    def params_numpy(self):
        return (self.w.cpu().numpy(), self.b.cpu().numpy(), self.w16.cpu().numpy().view(np.uint16))

    def save(self, path: str):
        w, b, w16 = self.params_numpy()
        np.savez(path, master_w=w, b=b, w_bf16=w16)

    @staticmethod
    def load(path: str) -> "CapacityNet":
        z = np.load(path)
        net = CapacityNet(w=z["master_w"], b=z["b"])
        net.w16.copy_(torch.from_numpy(z["w_bf16"].view(np.int16)))
        return net


def tile_rows(verts, tris, grid: Grid, feature_stride: int = None, stream=None):
    """(X [3 * ntiles, 12], label [3 * ntiles]) of one mesh: features from the
    subsample, labels from the exact count pass."""
    lib = _lib.load()
    v = _dev(verts, torch.float32).reshape(-1, 3)
    t = _dev(tris, torch.int32).reshape(-1, 3)
    nti = ntiles(grid.res)
    feature_stride = feature_stride or auto_stride(t.shape[0])
    raw = torch.empty(3 * nti * 11, dtype=torch.float32, device="cuda")
    X = torch.empty(3 * nti, 12, dtype=torch.float32, device="cuda")
    g = grid.c()
    sp = _stream_ptr(stream)
    _lib.check(lib.ldni_tile_features(v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], ctypes.byref(g),
                                      _lib.AXIS_ALL, int(feature_stride), raw.data_ptr(), X.data_ptr(), sp),
               "ldni_tile_features")
    ws = torch.empty(sample_workspace_size(v.shape[0], t.shape[0], grid.res, _lib.AXIS_ALL), dtype=torch.uint8,
                     device="cuda")
    info = new_info()
    outs = [empty_layers(grid, a, 0) for a in range(3)]
    arr = (_lib.Layers * 3)(*[o.c() for o in outs])
    _lib.check(lib.ldni_sample_count(v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], ctypes.byref(g),
                                     _lib.AXIS_ALL, arr, info.data_ptr(), ws.data_ptr(), ws.numel(), sp),
               "ldni_sample_count")
    label = torch.empty(3 * nti, dtype=torch.float32, device="cuda")
    for a in range(3):
        _lib.check(lib.ldni_tile_labels(outs[a].offsets.data_ptr(), grid.res, label[a * nti:].data_ptr(), sp),
                   "ldni_tile_labels")
    return X, label


def training_meshes(count: int = 200, seed: int = 21):
    """Seeded noisy geodesic spheres: frequency 16..128 (log-uniform), radius
    0.2..0.42, smooth or per-vertex radial noise of 0..25% of the radius, so
    that tiles range from empty through convex two-layer patches to folded
    multi-layer ones."""
    import meshgen
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        freq = int(round(np.exp(rng.uniform(np.log(16), np.log(128)))))
        r = float(rng.uniform(0.2, 0.42))
        amp = float(rng.uniform(0.0, 0.25)) * r
        kind = "octave" if rng.uniform() < 0.7 else "uniform"
        if kind == "uniform":
            amp = min(amp, 0.15 * r)
        out.append(meshgen.icosphere(freq, r=r, noise=amp, noise_kind=kind, seed=int(rng.integers(1 << 30)),
                                     center=tuple(rng.uniform(-0.04, 0.04, size=3))))
    return out


def build_dataset(meshes: Sequence, res: int = 512, feature_stride: int = None):
    grid = Grid.cube((-0.5, -0.5, -0.5), 1.0, res)
    xs, ls = [], []
    for v, t in meshes:
        X, L = tile_rows(v, t, grid, feature_stride)
        xs.append(X)
        ls.append(L)
    return torch.cat(xs), torch.cat(ls)


def train_default(count: int = 200, res: int = 512, steps: int = 1500, seed: int = 0) -> Tuple["CapacityNet", dict]:
    """The network used by the benchmark: 200 seeded noisy spheres at 512^2."""
    X, L = build_dataset(training_meshes(count), res)
    net = CapacityNet(seed=seed)
    losses = net.fit(X, L, steps=steps)
    return net, {"rows": int(X.shape[0]), "loss_first": losses[0], "loss_last": losses[-1], "steps": steps}
