"""Launch-shape tuner: times the library's launch knobs (ldni_tuning_t) on
the caller's own workload and keeps the fastest.

The knobs only change how work is spread over blocks, never a result, so a
choice is safe on any input; it is cached per device and workload class in a
JSON file so that later processes skip the measurement.

    from paper_1009_0794_gb300 import tune
    tune.tune_boolean(A, B, "union")          # picks and applies
    tune.tune_sampling(verts, tris, grid)
    tune.choose_sampling_mode(verts, tris, grid)  # direct or tile-binned traversal
"""
from __future__ import annotations

import ctypes
import json
import os
from typing import Dict, Iterable, List, Optional, Tuple

import torch

from . import _lib
from . import ldni as L

DEFAULT = {"bool_tile_rays": 512, "bool_stage_samples": 4096, "tri_blocks_per_sm": 16, "bool_split": -1}
BOOL_CANDIDATES = [(r, s, k) for r in (256, 512, 1024, 2048) for s in (0, 2048, 4096, 8192) for k in (0, 1)]
TRI_CANDIDATES = [2, 4, 8, 16, 32, 64]
CACHE_ENV = "LDNI_TUNE_CACHE"


def get() -> Dict[str, int]:
    t = _lib.Tuning()
    _lib.check(_lib.load().ldni_get_tuning(ctypes.byref(t)), "ldni_get_tuning")
    return {k: int(getattr(t, k)) for k, _ in _lib.Tuning._fields_}


def set(**knobs) -> Dict[str, int]:
    """Apply knobs (unnamed ones keep their current value); returns the previous setting."""
    prev = get()
    cur = dict(prev)
    cur.update({k: int(v) for k, v in knobs.items()})
    t = _lib.Tuning(**cur)
    _lib.check(_lib.load().ldni_set_tuning(ctypes.byref(t)), "ldni_set_tuning")
    return prev


def reset() -> None:
    _lib.check(_lib.load().ldni_set_tuning(None), "ldni_set_tuning")


def _cache_path() -> str:
    return os.environ.get(CACHE_ENV, os.path.join(os.path.expanduser("~"), ".cache", "ldni_tune.json"))


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store_cache(key: str, value: dict) -> None:
    path = _cache_path()
    data = _load_cache()
    data[key] = value
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _device_key() -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}/{p.multi_processor_count}"


def _time(fn, reps: int, flush: Optional[torch.Tensor]) -> float:
    """Median milliseconds of one replay of fn() captured in a CUDA graph
    (so host launch overhead is not measured), CUDA events on the replaying
    stream, L2 flushed before each replay when a flush buffer is given."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        fn()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        b = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        b.record()
        graph.replay()
        e.record()
        e.synchronize()
        ts.append(b.elapsed_time(e))
    ts.sort()
    return ts[len(ts) // 2]


def _flush_buffer() -> torch.Tensor:
    return torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # larger than L2


def _bucket(x: int) -> int:
    return max(0, int(x).bit_length() - 1)  # log2 class


def tune_boolean(A: "L.LDNI", B: "L.LDNI", op="union", eps: float = 0.0, reps: int = 10,
                 candidates: Iterable[Tuple[int, int, int]] = BOOL_CANDIDATES, use_cache: bool = True,
                 apply: bool = True) -> dict:
    """Time every (tile rays, staged samples, split) choice on A op B and
    keep the fastest.  Returns {"choice": {...}, "ms": {...}, "cached": bool}."""
    key = f"bool/{_device_key()}/res{A.grid.res}/nA{_bucket(A.n)}/nB{_bucket(B.n)}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            if apply:
                set(**hit["choice"])
            return {"choice": hit["choice"], "ms": hit.get("ms", {}), "cached": True}
    out = L.empty_layers(A.grid, A.axis, A.capacity + B.capacity)
    ws = torch.empty(L.boolean_workspace_size(A.grid.res), dtype=torch.uint8, device="cuda")
    info = L.new_info()
    flush = _flush_buffer()
    prev = get()
    ms = {}
    try:
        for r, s, k in candidates:
            set(bool_tile_rays=r, bool_stage_samples=s, bool_split=k)
            ms[f"{r}/{s}/{k}"] = _time(lambda: L.boolean(A, B, op, eps=eps, out=out, ws=ws, info=info, sync=False),
                                   reps, flush)
    finally:
        set(**prev)
    best = min(ms, key=ms.get)
    r, s, k = (int(x) for x in best.split("/"))
    choice = {"bool_tile_rays": r, "bool_stage_samples": s, "bool_split": k}
    if apply:
        set(**choice)
    _store_cache(key, {"choice": choice, "ms": ms})
    return {"choice": choice, "ms": ms, "cached": False}


def tune_sampling(verts, tris, grid: "L.Grid", reps: int = 10, candidates: Iterable[int] = TRI_CANDIDATES,
                  use_cache: bool = True, apply: bool = True) -> dict:
    """Time the exact two-pass sampling of one mesh for every grid size of
    the per-triangle passes and keep the fastest."""
    v = L._dev(verts, torch.float32).reshape(-1, 3)
    t = L._dev(tris, torch.int32).reshape(-1, 3)
    key = f"sample/{_device_key()}/res{grid.res}/T{_bucket(t.shape[0])}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            if apply:
                set(**hit["choice"])
            return {"choice": hit["choice"], "ms": hit.get("ms", {}), "cached": True}
    sizes = [X.n for X in L.sample(v, t, grid, "all")]
    plan = L.SamplePlan(v.shape[0], t.shape[0], grid, sizes)
    flush = _flush_buffer()
    prev = get()
    ms = {}
    try:
        for b in candidates:
            set(tri_blocks_per_sm=b)
            ms[str(b)] = _time(lambda: plan.run(v, t), reps, flush)
    finally:
        set(**prev)
    best = int(min(ms, key=ms.get))
    choice = {"tri_blocks_per_sm": best}
    if apply:
        set(**choice)
    _store_cache(key, {"choice": choice, "ms": ms})
    return {"choice": choice, "ms": ms, "cached": False}


def choose_sampling_mode(verts, tris, grid: "L.Grid", reps: int = 10, use_cache: bool = True) -> dict:
    """Time the two exact traversals of one mesh - triangle by triangle
    ("exact2") and tile by tile after binning ("binned2"), which give the same
    bits - and return the faster: {"mode": ..., "ms": {...}, "cached": bool}.
    The choice is cached per device, resolution and mesh size class; pass it
    to sample(..., mode=) or SamplePlan(..., mode=)."""
    v = L._dev(verts, torch.float32).reshape(-1, 3)
    t = L._dev(tris, torch.int32).reshape(-1, 3)
    key = f"mode/{_device_key()}/res{grid.res}/T{_bucket(t.shape[0])}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return {"mode": hit["mode"], "ms": hit.get("ms", {}), "cached": True}
    sizes = [X.n for X in L.sample(v, t, grid, "all")]
    flush = _flush_buffer()
    ms = {}
    for mode in ("exact2", "binned2"):
        plan = L.SamplePlan(v.shape[0], t.shape[0], grid, sizes, mode=mode)
        ms[mode] = _time(lambda: plan.run(v, t), reps, flush)
        plan.finish()
    mode = min(ms, key=ms.get)
    _store_cache(key, {"mode": mode, "ms": ms})
    return {"mode": mode, "ms": ms, "cached": False}
