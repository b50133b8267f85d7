"""Python face of the LDNI library: PyTorch supplies device memory and the
stream, libldni.so does all the work.

    import paper_1009_0794_gb300 as ldni
    g = ldni.Grid.cube((-0.5, -0.5, -0.5), 1.0, 1024)
    X, Y, Z = ldni.sample(verts, tris, g)          # Definition 3: three LDNIs
    U = ldni.boolean(X, X2, "union")               # Section 4.1
    v = ldni.volume(X)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence, Union

import numpy as np
import torch

from . import _lib
from ._lib import Grid as _CGrid, Layers as _CLayers

OPS = {"union": _lib.OP_UNION, "inter": _lib.OP_INTER, "intersection": _lib.OP_INTER,
       "diff": _lib.OP_DIFF, "difference": _lib.OP_DIFF}


@dataclass(frozen=True)
class Grid:
    """The cube shared by the three images (Definition 3)."""
    origin: tuple
    width: float
    res: int

    @staticmethod
    def cube(origin, width, res) -> "Grid":
        return Grid(tuple(float(np.float32(x)) for x in origin), float(np.float32(width)), int(res))

    @staticmethod
    def from_bbox(bbox, res) -> "Grid":
        b = np.ascontiguousarray(bbox, dtype=np.float32).reshape(6)
        g = _CGrid()
        _lib.check(_lib.load().ldni_grid_from_bbox(b.ctypes.data_as(ctypes.c_void_p), int(res), ctypes.byref(g)),
                   "ldni_grid_from_bbox")
        return Grid(tuple(g.origin), float(g.width), int(g.res))

    @property
    def h(self) -> float:
        return self.width / self.res

    def c(self) -> _CGrid:
        g = _CGrid()
        for k in range(3):
            g.origin[k] = self.origin[k]
        g.width = self.width
        g.res = self.res
        return g


class LDNI:
    """One layered depth-normal image in CSR form on the device.  Normals are
    FP32 in nx, ny, nz, or, with ``nrm8`` given, packed 8-bit codes
    (approximate normals, Section 3 item 1; int32 tensor holding the words)
    and nx, ny, nz empty."""

    def __init__(self, grid: Grid, axis: int, offsets, depth, nx, ny, nz, tri, n: int, nrm8=None):
        self.grid, self.axis = grid, axis
        self.offsets, self.depth, self.nx, self.ny, self.nz, self.tri = offsets, depth, nx, ny, nz, tri
        self.nrm8 = nrm8
        self.n = int(n)

    @property
    def packed(self) -> bool:
        return self.nrm8 is not None

    @property
    def capacity(self) -> int:
        return int(self.depth.numel())

    def c(self) -> _CLayers:
        L = _CLayers()
        L.offsets = self.offsets.data_ptr()
        L.depth = self.depth.data_ptr() if self.depth.numel() else None
        L.nx = self.nx.data_ptr() if self.nx.numel() else None
        L.ny = self.ny.data_ptr() if self.ny.numel() else None
        L.nz = self.nz.data_ptr() if self.nz.numel() else None
        L.tri_id = self.tri.data_ptr() if self.tri.numel() else None
        L.capacity = self.capacity
        L.nrm8 = (self.nrm8.data_ptr() if self.nrm8.numel() else None) if self.packed else None
        return L

    def counts(self):
        return self.offsets[1:] - self.offsets[:-1]

    def numpy(self) -> dict:
        n = self.n
        out = {"offsets": self.offsets.cpu().numpy().astype(np.int64), "depth": self.depth[:n].cpu().numpy(),
               "tri": self.tri[:n].cpu().numpy()}
        if self.packed:
            out["nrm8"] = self.nrm8[:n].cpu().numpy().view(np.uint32)
        else:
            out["nrm"] = torch.stack([self.nx[:n], self.ny[:n], self.nz[:n]], 1).cpu().numpy()
        return out


def identical(A: "LDNI", B: "LDNI") -> bool:
    """Bit-for-bit equality of two LDNIs (offsets and every sample array)."""
    if A.n != B.n or A.offsets.numel() != B.offsets.numel():
        return False
    n = A.n
    if A.packed != B.packed:
        return False
    same = torch.equal(A.offsets, B.offsets) and torch.equal(A.tri[:n], B.tri[:n])
    pairs = [(A.depth, B.depth)]
    pairs += [(A.nrm8, B.nrm8)] if A.packed else [(A.nx, B.nx), (A.ny, B.ny), (A.nz, B.nz)]
    for x, y in pairs:
        same = same and torch.equal(x[:n].view(torch.int32), y[:n].view(torch.int32))
    return bool(same)


def _stream_ptr(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(x, dtype) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        t = x.to(device="cuda", dtype=dtype)
    else:
        t = torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)
    return t.contiguous()


def _axes(axis) -> List[int]:
    if axis in ("all", None, _lib.AXIS_ALL):
        return [0, 1, 2]
    return [int(axis)]


def new_info() -> torch.Tensor:
    return torch.zeros(_lib.INFO_BYTES // 8, dtype=torch.int64, device="cuda")


def info_decode(info: torch.Tensor) -> dict:
    h = info.cpu().numpy()
    st = int(h[3]) & 0xFFFFFFFF
    odd = (int(h[3]) >> 32) & 0xFFFFFFFF
    return {"n": [int(x) for x in h[:3]], "status": st, "odd_rays": odd}


def _raise_status(st: int, what: str):
    if st & _lib.ST_BOUNDS:  # checked builds only
        raise _lib.LDNIError(-1, what + " (an index outside its array; checked build)")
    if st & _lib.ST_INDEX:
        raise _lib.LDNIError(-1, what + " (triangle vertex index out of range)")
    if st & _lib.ST_RANGE:
        raise _lib.LDNIError(-8, what)
    if st & _lib.ST_TOOLARGE:
        raise _lib.LDNIError(-4, what)
    if st & _lib.ST_CAPACITY:
        raise _lib.LDNIError(-9, what)
    if st & _lib.ST_TIMEOUT:
        raise _lib.LDNIError(-7, what)


def sample_workspace_size(nv: int, nt: int, res: int, axis=_lib.AXIS_ALL) -> int:
    sz = ctypes.c_size_t(0)
    _lib.check(_lib.load().ldni_sample_workspace_size(int(nv), int(nt), int(res),
                                                      _lib.AXIS_ALL if axis in ("all", None) else int(axis),
                                                      ctypes.byref(sz)), "ldni_sample_workspace_size")
    return int(sz.value)


def empty_layers(grid: Grid, axis: int, capacity: int, packed: bool = False) -> LDNI:
    """Device buffers of one image; packed: 8-bit normals (one int32 word per
    sample) instead of three FP32 arrays."""
    N = grid.res * grid.res
    f = lambda k: torch.empty(k, dtype=torch.float32, device="cuda")
    i = lambda k: torch.empty(k, dtype=torch.int32, device="cuda")
    nc = 0 if packed else capacity
    return LDNI(grid, axis, i(N + 1), f(capacity), f(nc), f(nc), f(nc), i(capacity), 0,
                nrm8=i(capacity) if packed else None)


def empty_layers_flat(grid: Grid, axes: Sequence[int], capacities: Sequence[int], packed: bool = False):
    """Device buffers of several images carved from one allocation (every
    array 256-byte aligned), so that a caller can move all of them with a
    single copy.  Returns (images, the flat uint8 tensor behind them)."""
    N = grid.res * grid.res
    plan = []  # (element count, dtype) per array, in allocation order
    for cap in capacities:
        nc = 0 if packed else int(cap)
        plan.append([(N + 1, torch.int32), (int(cap), torch.float32), (nc, torch.float32), (nc, torch.float32),
                     (nc, torch.float32), (int(cap), torch.int32)] + ([(int(cap), torch.int32)] if packed else []))
    align = lambda b: (b + 255) // 256 * 256
    total = sum(align(4 * k) for arrs in plan for k, _ in arrs)
    flat = torch.empty(max(total, 256), dtype=torch.uint8, device="cuda")
    at = 0
    out = []
    for axis, arrs in zip(axes, plan):
        views = []
        for k, dt in arrs:
            views.append(flat[at:at + 4 * k].view(dt))
            at += align(4 * k)
        nrm8 = views[6] if packed else None
        out.append(LDNI(grid, int(axis), *views[:6], 0, nrm8=nrm8))
    return out, flat


def sample_binned_workspace_size(nv: int, nt: int, res: int, axis=_lib.AXIS_ALL) -> int:
    sz = ctypes.c_size_t(0)
    _lib.check(_lib.load().ldni_sample_binned_workspace_size(int(nv), int(nt), int(res),
                                                             _lib.AXIS_ALL if axis in ("all", None) else int(axis),
                                                             ctypes.byref(sz)), "ldni_sample_binned_workspace_size")
    return int(sz.value)


def sample(verts, tris, grid: Grid, axis="all", mode: str = "exact2", stream=None,
           check_odd: bool = False, packed: bool = False) -> Union[LDNI, List[LDNI]]:
    """Sample a closed mesh into LDNIs (Section 3, Definitions 1-4); packed:
    approximate 8-bit normals (Section 3 item 1).  mode "exact2" traverses
    triangle by triangle, "binned2" tile by tile (identical output).

    Exact sizing: the count pass runs, the sample totals are read back (one
    device->host read, the only synchronisation), the sample arrays are
    allocated to size, then the fill pass and per-ray sort run."""
    lib = _lib.load()
    if mode not in ("exact2", "binned2"):
        raise _lib.LDNIError(-1, f"sample: mode {mode!r}")
    binned = mode == "binned2"
    count_fn = lib.ldni_sample_binned_count if binned else lib.ldni_sample_count
    fill_fn = lib.ldni_sample_binned_fill if binned else lib.ldni_sample_fill
    v = _dev(verts, torch.float32).reshape(-1, 3)
    t = _dev(tris, torch.int32).reshape(-1, 3)
    axes = _axes(axis)
    cax = _lib.AXIS_ALL if len(axes) == 3 else axes[0]
    wsz = (sample_binned_workspace_size if binned else sample_workspace_size)(v.shape[0], t.shape[0], grid.res, cax)
    ws = torch.empty(wsz, dtype=torch.uint8, device="cuda")
    info = new_info()
    outs = [empty_layers(grid, a, 0) for a in axes]
    arr = (_CLayers * len(axes))(*[o.c() for o in outs])
    g = grid.c()
    sp = _stream_ptr(stream)
    _lib.check(count_fn(v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], ctypes.byref(g), cax, arr,
                        info.data_ptr(), ws.data_ptr(), ws.numel(), sp), "ldni_sample_count")
    meta = info_decode(info)
    _raise_status(meta["status"], "ldni_sample_count")
    res_list = []
    for k, a in enumerate(axes):
        n = meta["n"][a]
        L = empty_layers(grid, a, n, packed)
        L.offsets = outs[k].offsets
        L.n = n
        res_list.append(L)
    arr = (_CLayers * len(axes))(*[o.c() for o in res_list])
    _lib.check(fill_fn(v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], ctypes.byref(g), cax, arr,
                       info.data_ptr(), ws.data_ptr(), ws.numel(), sp), "ldni_sample_fill")
    if check_odd:
        meta = info_decode(info)
        _raise_status(meta["status"], "ldni_sample_fill")
        if meta["status"] & _lib.ST_ODD:
            raise _lib.LDNIError(-3, f"ldni_sample: {meta['odd_rays']} odd rays")
    return res_list if len(axes) > 1 else res_list[0]


class SamplePlan:
    """Pre-sized buffers for repeated sampling of one mesh size without any
    host synchronisation (for benchmarks and pipelines).  Capacities come
    from a first exact call; a later call that needs more sets
    LDNI_ST_CAPACITY in ``info``."""

    def __init__(self, nv: int, nt: int, grid: Grid, capacities: Sequence[int], axis="all", slack: float = 1.0,
                 packed: bool = False, mode: str = "exact2"):
        self.grid = grid
        self.axes = _axes(axis)
        self.cax = _lib.AXIS_ALL if len(self.axes) == 3 else self.axes[0]
        self.mode = _lib.MODE_BINNED2 if mode == "binned2" else _lib.MODE_EXACT2
        wsz = (sample_binned_workspace_size if mode == "binned2" else sample_workspace_size)(nv, nt, grid.res,
                                                                                           self.cax)
        self.ws = torch.empty(wsz, dtype=torch.uint8, device="cuda")
        self.info = new_info()
        self.outs = [empty_layers(grid, a, int(np.ceil(c * slack)), packed) for a, c in zip(self.axes, capacities)]
        self._arr = (_CLayers * len(self.axes))(*[o.c() for o in self.outs])
        self._g = grid.c()

    def run(self, verts: torch.Tensor, tris: torch.Tensor, stream=None):
        lib = _lib.load()
        _lib.check(lib.ldni_sample(verts.data_ptr(), verts.shape[0], tris.data_ptr(), tris.shape[0],
                                   ctypes.byref(self._g), self.cax, self.mode, self._arr, self.info.data_ptr(),
                                   self.ws.data_ptr(), self.ws.numel(), _stream_ptr(stream)), "ldni_sample")

    def finish(self) -> List[LDNI]:
        """Synchronise, check status and set the sample counts."""
        meta = info_decode(self.info)
        _raise_status(meta["status"], "ldni_sample")
        for o in self.outs:
            o.n = meta["n"][o.axis]
        return self.outs


def boolean_workspace_size(res: int) -> int:
    sz = ctypes.c_size_t(0)
    _lib.check(_lib.load().ldni_boolean_workspace_size(int(res), ctypes.byref(sz)), "ldni_boolean_workspace_size")
    return int(sz.value)


def boolean(A: LDNI, B: LDNI, op, eps: float = 0.0, stream=None, out: Optional[LDNI] = None,
            ws: Optional[torch.Tensor] = None, info: Optional[torch.Tensor] = None, sync: bool = True) -> LDNI:
    """A op B per ray (Section 4.1) with small-interval removal (Section
    4.1.1).  Output capacity A.capacity + B.capacity always suffices."""
    lib = _lib.load()
    opc = OPS[op] if isinstance(op, str) else int(op)
    if out is None:
        out = empty_layers(A.grid, A.axis, A.capacity + B.capacity, A.packed)
    if ws is None:
        ws = torch.empty(boolean_workspace_size(A.grid.res), dtype=torch.uint8, device="cuda")
    if info is None:
        info = new_info()
    la, lb, lo = A.c(), B.c(), out.c()
    ga, gb = A.grid.c(), B.grid.c()
    _lib.check(lib.ldni_boolean(ctypes.byref(la), ctypes.byref(ga), ctypes.byref(lb), ctypes.byref(gb), opc,
                                float(eps), ctypes.byref(lo), info.data_ptr(), ws.data_ptr(), ws.numel(),
                                _stream_ptr(stream)), "ldni_boolean")
    if sync:
        meta = info_decode(info)
        _raise_status(meta["status"], "ldni_boolean")
        if meta["status"] & _lib.ST_ODD:
            raise _lib.LDNIError(-3, "ldni_boolean")
        out.n = meta["n"][0]
    return out


def volume_workspace_size(res: int) -> int:
    sz = ctypes.c_size_t(0)
    _lib.check(_lib.load().ldni_volume_workspace_size(int(res), ctypes.byref(sz)), "ldni_volume_workspace_size")
    return int(sz.value)


def volume(L: LDNI, stream=None, out: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None,
           info: Optional[torch.Tensor] = None, sync: bool = True):
    """Enclosed volume seen by one LDNI (odd-to-even ranges inside)."""
    lib = _lib.load()
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
    if ws is None:
        ws = torch.empty(volume_workspace_size(L.grid.res), dtype=torch.uint8, device="cuda")
    if info is None:
        info = new_info()
    lc, g = L.c(), L.grid.c()
    _lib.check(lib.ldni_volume(ctypes.byref(lc), ctypes.byref(g), out.data_ptr(), info.data_ptr(), ws.data_ptr(),
                               ws.numel(), _stream_ptr(stream)), "ldni_volume")
    if not sync:
        return out
    meta = info_decode(info)
    if meta["status"] & _lib.ST_ODD:
        raise _lib.LDNIError(-3, "ldni_volume")
    return float(out.item())


def boolean_many_workspace_size(res: int, count: int) -> int:
    sz = ctypes.c_size_t(0)
    _lib.check(_lib.load().ldni_boolean_many_workspace_size(int(res), int(count), ctypes.byref(sz)),
               "ldni_boolean_many_workspace_size")
    return sz.value


def boolean_many(As: Sequence[LDNI], Bs: Sequence[LDNI], op, eps: float = 0.0, stream=None,
                 outs: Optional[Sequence[LDNI]] = None, ws: Optional[torch.Tensor] = None,
                 infos: Optional[torch.Tensor] = None, sync: bool = True,
                 vols: Optional[torch.Tensor] = None) -> List[LDNI]:
    """A[j] op B[j] for every j (all on one grid) in one set of launches;
    with `vols` (device float64[count]) also the volume of every result."""
    lib = _lib.load()
    count = len(As)
    grid = As[0].grid
    for X in list(As) + list(Bs):
        if X.grid != grid:
            raise _lib.LDNIError(-2, "boolean_many")
    opc = OPS[op] if isinstance(op, str) else int(op)
    if outs is None:
        outs = [empty_layers(grid, A.axis, A.capacity + B.capacity, A.packed) for A, B in zip(As, Bs)]
    if ws is None:
        ws = torch.empty(boolean_many_workspace_size(grid.res, count), dtype=torch.uint8, device="cuda")
    if infos is None:
        infos = torch.zeros(count, _lib.INFO_BYTES // 8, dtype=torch.int64, device="cuda")
    arr = lambda xs: (_CLayers * count)(*[x.c() for x in xs])
    la, lb, lo = arr(As), arr(Bs), arr(outs)
    g = grid.c()
    _lib.check(lib.ldni_boolean_many(count, la, lb, ctypes.byref(g), opc, float(eps), lo, infos.data_ptr(),
                                     vols.data_ptr() if vols is not None else None, ws.data_ptr(), ws.numel(),
                                     _stream_ptr(stream)), "ldni_boolean_many")
    if sync:
        h = infos.cpu().numpy()
        for j, o in enumerate(outs):
            st = int(h[j, 3]) & 0xFFFFFFFF
            _raise_status(st, "ldni_boolean_many")
            if st & _lib.ST_ODD:
                raise _lib.LDNIError(-3, "ldni_boolean_many")
            o.n = int(h[j, 0])
    return list(outs)


def volume_many_workspace_size(res: int, count: int) -> int:
    sz = ctypes.c_size_t(0)
    _lib.check(_lib.load().ldni_volume_many_workspace_size(int(res), int(count), ctypes.byref(sz)),
               "ldni_volume_many_workspace_size")
    return sz.value


def volume_many(Ls: Sequence[LDNI], stream=None, out: Optional[torch.Tensor] = None,
                ws: Optional[torch.Tensor] = None, infos: Optional[torch.Tensor] = None, sync: bool = True):
    """Volumes of several images of one grid in one launch."""
    lib = _lib.load()
    count = len(Ls)
    grid = Ls[0].grid
    if out is None:
        out = torch.zeros(count, dtype=torch.float64, device="cuda")
    if ws is None:
        ws = torch.empty(volume_many_workspace_size(grid.res, count), dtype=torch.uint8, device="cuda")
    if infos is None:
        infos = torch.zeros(count, _lib.INFO_BYTES // 8, dtype=torch.int64, device="cuda")
    arr = (_CLayers * count)(*[x.c() for x in Ls])
    g = grid.c()
    _lib.check(lib.ldni_volume_many(count, arr, ctypes.byref(g), out.data_ptr(), infos.data_ptr(), ws.data_ptr(),
                                    ws.numel(), _stream_ptr(stream)), "ldni_volume_many")
    if not sync:
        return out
    h = infos.cpu().numpy()
    if any((int(h[j, 3]) & 0xFFFFFFFF) & _lib.ST_ODD for j in range(count)):
        raise _lib.LDNIError(-3, "ldni_volume_many")
    return [float(v) for v in out.cpu().numpy()]


# ---- one-pass sampling with learned capacity -------------------------------------

def auto_stride(nt: int, budget: int = 65536) -> int:
    """Feature subsample stride: about `budget` triangles feed the features."""
    return max(1, -(-int(nt) // budget))


def ntiles(res: int) -> int:
    return (res * res + _lib.TILE_RAYS - 1) // _lib.TILE_RAYS


def sample_learned_workspace_size(nv: int, nt: int, res: int, axis, slab_samples: int) -> int:
    sz = ctypes.c_size_t(0)
    cax = _lib.AXIS_ALL if axis in ("all", None, _lib.AXIS_ALL) else int(axis)
    _lib.check(_lib.load().ldni_sample_learned_workspace_size(int(nv), int(nt), int(res), cax, int(slab_samples),
                                                              ctypes.byref(sz)), "ldni_sample_learned_workspace_size")
    return int(sz.value)


class LearnedPlan:
    """Buffers for repeated one-pass sampling of one mesh size (no host
    synchronisation per call).  `net` is a capacity.CapacityNet or None for
    fixed `layers` per ray (the baseline without the network)."""

    def __init__(self, nv: int, nt: int, grid: Grid, capacities, slab_samples: int, axis="all", net=None,
                 layers: int = 2, margin: float = 0.25, feature_stride: Optional[int] = None, packed: bool = False):
        self.grid = grid
        self.axes = _axes(axis)
        self.cax = _lib.AXIS_ALL if len(self.axes) == 3 else self.axes[0]
        self.slab = int(slab_samples)
        self.ws = torch.empty(sample_learned_workspace_size(nv, nt, grid.res, self.cax, self.slab), dtype=torch.uint8,
                              device="cuda")
        self.info = new_info()
        self.n_over = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.outs = [empty_layers(grid, a, int(c), packed) for a, c in zip(self.axes, capacities)]
        self._arr = (_CLayers * len(self.axes))(*[o.c() for o in self.outs])
        self._g = grid.c()
        self.net, self.layers = net, int(layers)
        self.stride = int(feature_stride) if feature_stride else auto_stride(nt)
        self._mlp = net.c(margin) if net is not None else None

    def run(self, verts: torch.Tensor, tris: torch.Tensor, stream=None):
        lib = _lib.load()
        mp = ctypes.byref(self._mlp) if self._mlp is not None else None
        _lib.check(lib.ldni_sample_learned(verts.data_ptr(), verts.shape[0], tris.data_ptr(), tris.shape[0],
                                           ctypes.byref(self._g), self.cax, mp, self.layers, self.stride, self.slab,
                                           self._arr, self.info.data_ptr(), self.n_over.data_ptr(),
                                           self.ws.data_ptr(), self.ws.numel(), _stream_ptr(stream)),
                   "ldni_sample_learned")

    def finish(self) -> List[LDNI]:
        meta = info_decode(self.info)
        _raise_status(meta["status"], "ldni_sample_learned")
        for o in self.outs:
            o.n = meta["n"][o.axis]
        return self.outs

    def overflow_tiles(self) -> int:
        return int(self.n_over.item())


def sample_learned(verts, tris, grid: Grid, axis="all", net=None, layers: int = 2, margin: float = 0.25,
                   feature_stride: Optional[int] = None, slab_samples: Optional[int] = None,
                   capacity_hint: Optional[int] = None,
                   stream=None, packed: bool = False):
    """One-traversal sampling (identical output to sample()).  Output arrays
    are sized by capacity_hint per image (default: 3 * res^2 / 2); a call
    that needs more raises LDNIError(LDNI_ECAPACITY)."""
    v = _dev(verts, torch.float32).reshape(-1, 3)
    t = _dev(tris, torch.int32).reshape(-1, 3)
    axes = _axes(axis)
    n_img = len(axes)
    cap = capacity_hint if capacity_hint is not None else max(16, 3 * grid.res * grid.res // 2)
    slab = slab_samples if slab_samples is not None else n_img * grid.res * grid.res * 4
    plan = LearnedPlan(v.shape[0], t.shape[0], grid, [cap] * n_img, slab, axis, net, layers, margin, feature_stride,
                       packed)
    plan.run(v, t, stream)
    outs = plan.finish()
    return outs if n_img > 1 else outs[0]


# ---- approximate normals (Section 3 item 1) -------------------------------------

def encode_normals8(nx: torch.Tensor, ny: torch.Tensor, nz: torch.Tensor, stream=None) -> torch.Tensor:
    """Packed 8-bit codes (int32 tensor of words) of FP32 normals."""
    n = nx.numel()
    w = torch.empty(n, dtype=torch.int32, device="cuda")
    _lib.check(_lib.load().ldni_normals_encode8(nx.data_ptr(), ny.data_ptr(), nz.data_ptr(), n, w.data_ptr(),
                                                _stream_ptr(stream)), "ldni_normals_encode8")
    return w


def decode_normals8(w: torch.Tensor, stream=None):
    """Unit FP32 normals (nx, ny, nz) from packed words."""
    n = w.numel()
    out = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(3)]
    _lib.check(_lib.load().ldni_normals_decode8(w.data_ptr(), n, out[0].data_ptr(), out[1].data_ptr(),
                                                out[2].data_ptr(), _stream_ptr(stream)), "ldni_normals_decode8")
    return tuple(out)


# ---- grid-node classification (Section 5.1, Step 1) -----------------------------

def classify_nodes(Ls: Sequence[LDNI], stream=None, out: Optional[torch.Tensor] = None,
                   ws: Optional[torch.Tensor] = None, info: Optional[torch.Tensor] = None,
                   sync: bool = True) -> torch.Tensor:
    """Inside bits of the res^3 grid nodes from the three images of one
    solid (2-of-3 vote): int32 tensor [res(k), res(j), ceil(res/32)] whose
    bit i % 32 of word [k, j, i // 32] is node (i, j, k)."""
    lib = _lib.load()
    grid = Ls[0].grid
    if len(Ls) != 3 or any(L.grid != grid for L in Ls) or [L.axis for L in Ls] != [0, 1, 2]:
        raise _lib.LDNIError(-1, "classify_nodes needs the x, y and z images of one grid")
    res = grid.res
    W = (res + 31) // 32
    if out is None:
        out = torch.empty(res, res, W, dtype=torch.int32, device="cuda")
    if ws is None:
        sz = ctypes.c_size_t(0)
        _lib.check(lib.ldni_classify_nodes_workspace_size(res, ctypes.byref(sz)), "ldni_classify_nodes_workspace_size")
        ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    if info is None:
        info = new_info()
    arr = (_CLayers * 3)(*[L.c() for L in Ls])
    g = grid.c()
    _lib.check(lib.ldni_classify_nodes(arr, ctypes.byref(g), out.data_ptr(), info.data_ptr(), ws.data_ptr(),
                                       ws.numel(), _stream_ptr(stream)), "ldni_classify_nodes")
    if sync:
        meta = info_decode(info)
        _raise_status(meta["status"], "ldni_classify_nodes")
        if meta["status"] & _lib.ST_ODD:
            raise _lib.LDNIError(-3, "ldni_classify_nodes")
    return out


def offset_workspace_size(n: Sequence[int], res: int, r: float, width: float) -> int:
    sz = ctypes.c_size_t(0)
    nn = (ctypes.c_int64 * 3)(*[int(x) for x in n])
    _lib.check(_lib.load().ldni_offset_workspace_size(nn, int(res), float(r), float(width), ctypes.byref(sz)),
               "ldni_offset_workspace_size")
    return int(sz.value)


def offset(Ls: Sequence[LDNI], r: float, inner: bool = False, eps: float = 0.0, capacity: Optional[int] = None,
           stream=None) -> List[LDNI]:
    """Offset of the solid given by its x, y and z images (Section 4.2): the
    union with (inner: difference with) a sphere of radius r about every
    sample, then small-interval removal with eps.  Sizes the outputs with one
    readback: a first call with `capacity` samples per image (default: twice
    the input's plus 2 per ray), repeated once with the exact sizes if that
    was too small."""
    lib = _lib.load()
    grid = Ls[0].grid
    if len(Ls) != 3 or any(L.grid != grid for L in Ls) or [L.axis for L in Ls] != [0, 1, 2]:
        raise _lib.LDNIError(-1, "offset needs the x, y and z images of one grid")
    n = [int(L.n) for L in Ls]
    nn = (ctypes.c_int64 * 3)(*n)
    ws = torch.empty(offset_workspace_size(n, grid.res, r, grid.width), dtype=torch.uint8, device="cuda")
    info = new_info()
    H = (_CLayers * 3)(*[L.c() for L in Ls])
    g = grid.c()
    caps = [int(capacity)] * 3 if capacity is not None else [2 * x + 2 * grid.res * grid.res for x in n]
    for attempt in range(2):
        outs = [empty_layers(grid, a, caps[a]) for a in range(3)]
        arr = (_CLayers * 3)(*[o.c() for o in outs])
        info.zero_()
        _lib.check(lib.ldni_offset(H, nn, ctypes.byref(g), float(r), 1 if inner else 0, float(eps), arr,
                                   info.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream)), "ldni_offset")
        meta = info_decode(info)
        if meta["status"] & _lib.ST_CAPACITY and attempt == 0:
            caps = [max(int(x), 1) for x in meta["n"]]
            continue
        _raise_status(meta["status"], "ldni_offset")
        if meta["status"] & _lib.ST_ODD:
            raise _lib.LDNIError(-3, "ldni_offset")
        if meta["status"] & _lib.ST_EVENTS:
            raise _lib.LDNIError(-4, "ldni_offset (a ray meets more sphere samples than one warp orders)")
        for a in range(3):
            outs[a].n = meta["n"][a]
        return outs
    raise _lib.LDNIError(-9, "ldni_offset")


def unpack_nodes(words: torch.Tensor, res: int) -> np.ndarray:
    """Bit words of classify_nodes -> bool array [k, j, i]."""
    w = words.cpu().numpy().view(np.uint32)
    bits = (w[..., None] >> np.arange(32, dtype=np.uint32)) & 1
    return bits.reshape(res, res, -1)[:, :, :res].astype(bool)


# ---- contouring, Steps 2-3 (Section 5.1) ----------------------------------------

CELL_DTYPE = np.dtype([("cell", "<i8"), ("labels", "<u4"), ("npts", "<u4"), ("nvert", "<i4"), ("pad_", "<i4"),
                       ("v", "<f4", (4, 3))])


def contour_workspace_size(res: int, max_active: int) -> int:
    sz = ctypes.c_size_t(0)
    _lib.check(_lib.load().ldni_contour_workspace_size(int(res), int(max_active), ctypes.byref(sz)),
               "ldni_contour_workspace_size")
    return int(sz.value)


def contour_cells(Ls: Sequence[LDNI], inside: Optional[torch.Tensor] = None, max_active: Optional[int] = None,
                  stream=None) -> np.ndarray:
    """Cell vertices of Steps 2-3 of the contouring (Section 5.1) from the x,
    y and z images of one solid: a NumPy structured array (CELL_DTYPE) of the
    cells that yield a vertex, in ascending cell order.  inside: the node
    bits of classify_nodes (computed when not given).  One readback at the
    end; a first bound on the active cells that proves too small is raised
    once."""
    lib = _lib.load()
    grid = Ls[0].grid
    if len(Ls) != 3 or any(L.grid != grid for L in Ls) or [L.axis for L in Ls] != [0, 1, 2]:
        raise _lib.LDNIError(-1, "contour_cells needs the x, y and z images of one grid")
    if inside is None:
        inside = classify_nodes(Ls, stream=stream)
    res = grid.res
    n3 = (res - 1) ** 3
    bound = int(max_active) if max_active else min(n3, 4 * sum(L.n for L in Ls) + 6 * (res - 1) ** 2 + 64)
    arr = (_CLayers * 3)(*[L.c() for L in Ls])
    g = grid.c()
    info = new_info()
    for attempt in range(2):
        bound = max(1, min(bound, n3, 2 ** 31 - 1))
        ws = torch.empty(contour_workspace_size(res, bound), dtype=torch.uint8, device="cuda")
        out = torch.empty(bound * CELL_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        info.zero_()
        _lib.check(lib.ldni_contour_cells(arr, ctypes.byref(g), inside.data_ptr(), bound, out.data_ptr(), bound,
                                          info.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream)),
                   "ldni_contour_cells")
        meta = info_decode(info)
        if meta["status"] & _lib.ST_CAPACITY and attempt == 0 and bound < n3:
            bound = min(n3, 4 * bound)
            continue
        _raise_status(meta["status"], "ldni_contour_cells")
        m = int(meta["n"][0])
        return out[:m * CELL_DTYPE.itemsize].cpu().numpy().view(CELL_DTYPE)
    raise _lib.LDNIError(-9, "ldni_contour_cells")


# ---- adjoint -------------------------------------------------------------------

def depth_vjp(verts: torch.Tensor, tris: torch.Tensor, L: LDNI, grad_depth: torch.Tensor,
              grad_verts: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """grad_verts += (d depth / d verts)^T grad_depth for the samples of L
    (fixed crossing set; d(d)/d(V_j) = lambda_j n / n_a)."""
    v = verts.contiguous()
    t = tris.contiguous()
    if grad_verts is None:
        grad_verts = torch.zeros(v.shape[0], 3, dtype=torch.float32, device="cuda")
    gd = grad_depth.contiguous().to(torch.float32)
    if gd.numel() < L.capacity:
        gd = torch.cat([gd, torch.zeros(L.capacity - gd.numel(), dtype=torch.float32, device="cuda")])
    info = new_info()
    lc, g = L.c(), L.grid.c()
    _lib.check(_lib.load().ldni_depth_vjp(v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], ctypes.byref(g), L.axis,
                                          ctypes.byref(lc), gd.data_ptr(), grad_verts.data_ptr(), info.data_ptr(),
                                          _stream_ptr(stream)), "ldni_depth_vjp")
    return grad_verts


def volume_grad(verts: torch.Tensor, tris: torch.Tensor, L: LDNI, grad_volume: float = 1.0,
                grad_verts: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """grad_verts += grad_volume * d(volume of L)/d(verts), fixed crossing set."""
    v = verts.contiguous()
    t = tris.contiguous()
    if grad_verts is None:
        grad_verts = torch.zeros(v.shape[0], 3, dtype=torch.float32, device="cuda")
    info = new_info()
    lc, g = L.c(), L.grid.c()
    _lib.check(_lib.load().ldni_volume_grad(v.data_ptr(), v.shape[0], t.data_ptr(), t.shape[0], ctypes.byref(g),
                                            L.axis, ctypes.byref(lc), float(grad_volume), grad_verts.data_ptr(),
                                            info.data_ptr(), _stream_ptr(stream)), "ldni_volume_grad")
    return grad_verts


# ---- batches ---------------------------------------------------------------------

class BatchPlan:
    """Sampling of many meshes (each on its own grid, three images each) by
    one launch per stage for the whole batch (ldni_sample_batch).  Buffers
    are sized from one exact per-mesh count (or given capacities); run() makes
    no host synchronisation and can be captured in a CUDA graph."""

    def __init__(self, meshes, grids: Sequence[Grid], capacities=None):
        lib = _lib.load()
        self.meshes = [(_dev(v, torch.float32).reshape(-1, 3), _dev(t, torch.int32).reshape(-1, 3)) for v, t in meshes]
        self.grids = list(grids)
        if capacities is None:
            capacities = []
            for (v, t), g in zip(self.meshes, self.grids):
                capacities.append([L.n for L in sample(v, t, g, "all")])
        self.outs = [[empty_layers(g, a, int(c[a])) for a in range(3)] for g, c in zip(self.grids, capacities)]
        count = len(self.meshes)
        items = (_lib.BatchItem * count)()
        for m, ((v, t), g) in enumerate(zip(self.meshes, self.grids)):
            it = items[m]
            it.verts, it.tris, it.nv, it.nt = v.data_ptr(), t.data_ptr(), v.shape[0], t.shape[0]
            it.grid = g.c()
            for a in range(3):
                it.out[a] = self.outs[m][a].c()
        self._items_host = items
        raw = bytes(memoryview(items))
        self._items_dev = torch.frombuffer(bytearray(raw), dtype=torch.uint8).cuda()
        sz = ctypes.c_size_t(0)
        _lib.check(lib.ldni_sample_batch_workspace_size(ctypes.byref(items), count, ctypes.byref(sz)),
                   "ldni_sample_batch_workspace_size")
        self.ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
        self.infos = torch.zeros(count, _lib.INFO_BYTES // 8, dtype=torch.int64, device="cuda")
        self.count = count

    def run(self, stream=None):
        _lib.check(_lib.load().ldni_sample_batch(self._items_dev.data_ptr(), ctypes.byref(self._items_host),
                                                 self.count, self.infos.data_ptr(), self.ws.data_ptr(),
                                                 self.ws.numel(), _stream_ptr(stream)), "ldni_sample_batch")

    def finish(self) -> List[List[LDNI]]:
        h = self.infos.cpu().numpy()
        for m in range(self.count):
            st = int(h[m, 3]) & 0xFFFFFFFF
            _raise_status(st, f"ldni_sample_batch item {m}")
            for a in range(3):
                self.outs[m][a].n = int(h[m, a])
        return self.outs


def union_chain_workspace_size(res: int, nimg: int) -> int:
    sz = ctypes.c_size_t(0)
    _lib.check(_lib.load().ldni_union_chain_workspace_size(int(res), int(nimg), ctypes.byref(sz)),
               "ldni_union_chain_workspace_size")
    return int(sz.value)


def union_chain_many(parts_per_image: Sequence[Sequence[LDNI]], eps: float = 0.0,
                     capacities: Optional[Sequence[int]] = None):
    """For each image j (1 to 3, one grid): parts[j][0] u parts[j][1] u ...
    in order (Section 4.1 unions, the repeated operation of offsetting and
    sweeps, Section 4.2), equal to the step-by-step chain of boolean() calls
    bit for bit, in one call (ldni_union_chain).  Returns (run, finish):
    run() enqueues the chain without host synchronisation (capturable in a
    CUDA graph); finish() checks the status and returns the result images
    once run() has completed."""
    lib = _lib.load()
    nimg = len(parts_per_image)
    count = len(parts_per_image[0])
    if nimg < 1 or nimg > 3 or count < 1 or any(len(ps) != count for ps in parts_per_image):
        raise _lib.LDNIError(-1, "union_chain")
    grid = parts_per_image[0][0].grid
    packed = parts_per_image[0][0].packed
    if any(p.grid != grid for ps in parts_per_image for p in ps):
        raise _lib.LDNIError(-2, "union_chain")
    caps = list(capacities) if capacities else [sum(p.capacity for p in ps) for ps in parts_per_image]
    outs = [empty_layers(grid, ps[0].axis, max(1, int(c)), packed) for ps, c in zip(parts_per_image, caps)]
    host = (_CLayers * (nimg * count))(*[p.c() for ps in parts_per_image for p in ps])
    dev = torch.frombuffer(bytearray(bytes(memoryview(host))), dtype=torch.uint8).cuda()
    oarr = (_CLayers * nimg)(*[o.c() for o in outs])
    ws = torch.empty(union_chain_workspace_size(grid.res, nimg), dtype=torch.uint8, device="cuda")
    info = new_info()
    g = grid.c()

    def run(stream=None):
        _lib.check(lib.ldni_union_chain(dev.data_ptr(), host, count, nimg, ctypes.byref(g), float(eps), oarr,
                                        info.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream)),
                   "ldni_union_chain")

    def finish() -> List[LDNI]:
        meta = info_decode(info)
        _raise_status(meta["status"], "ldni_union_chain")
        if meta["status"] & _lib.ST_EVENTS:
            raise _lib.LDNIError(-4, "ldni_union_chain (a ray needs more than 64 samples)")
        if meta["status"] & _lib.ST_ODD:
            raise _lib.LDNIError(-3, "ldni_union_chain")
        for j, o in enumerate(outs):
            o.n = meta["n"][j]
        return outs

    run._keep = (host, dev, oarr, ws, info, g)  # alive as long as run is
    return run, finish


def union_chain(parts: Sequence[LDNI], eps: float = 0.0, capacity: Optional[int] = None):
    """acc = parts[0] u parts[1] u ... in order for one image (see
    union_chain_many).  Returns (run, finish); finish() gives the result."""
    run, fin = union_chain_many([parts], eps, [capacity] if capacity is not None else None)
    return run, (lambda: fin()[0])
