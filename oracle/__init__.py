"""LDNI oracle (TEST INFRASTRUCTURE ONLY).

A plain, slow, obviously correct CPU statement of the LDNI hot path, written
from the paper's definitions, in FP64 C (``ldni_oracle.c``) and NumPy.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and does not import it.

Sampling follows Definitions 1-4 and Remark 1 (Section 2) with the
pixel-centre convention of Section 3; the Boolean follows Section 4.1 and the
small-interval removal of Section 4.1.1; offsetting follows Section 4.2; the
volume follows the odd-to-even-inside statement after Proposition 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libldni_oracle.so")
_SRC = os.path.join(_HERE, "ldni_oracle.c")
_lock = threading.Lock()
_lib = None

OP_UNION, OP_INTER, OP_DIFF = 0, 1, 2
OPS = {"union": OP_UNION, "inter": OP_INTER, "intersection": OP_INTER, "diff": OP_DIFF, "difference": OP_DIFF}


def build(force: bool = False) -> str:
    """Compile the C oracle with IEEE semantics (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _OracleLDNI(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nrays", ctypes.c_int64),
                ("offsets", ctypes.POINTER(ctypes.c_int64)), ("depth", ctypes.POINTER(ctypes.c_double)),
                ("nrm", ctypes.POINTER(ctypes.c_double)), ("tri", ctypes.POINTER(ctypes.c_int32))]


class _OracleBool(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nrays", ctypes.c_int64),
                ("offsets", ctypes.POINTER(ctypes.c_int64)), ("depth", ctypes.POINTER(ctypes.c_float)),
                ("nrm", ctypes.POINTER(ctypes.c_float)), ("tri", ctypes.POINTER(ctypes.c_int32))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.oracle_sample.restype = ctypes.POINTER(_OracleLDNI)
            lib.oracle_sample.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_float,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32)]
            lib.oracle_free.argtypes = [ctypes.POINTER(_OracleLDNI)]
            lib.oracle_boolean.restype = ctypes.POINTER(_OracleBool)
            lib.oracle_boolean.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, P, ctypes.c_int32,
                                           ctypes.c_float, ctypes.POINTER(ctypes.c_int32)]
            lib.oracle_bool_free.argtypes = [ctypes.POINTER(_OracleBool)]
            lib.oracle_offset.restype = ctypes.POINTER(_OracleBool)
            lib.oracle_offset.argtypes = [ctypes.c_int32, P, ctypes.c_float, P, P, P, P, P, ctypes.c_int32,
                                          ctypes.c_float, ctypes.c_int32, ctypes.c_float,
                                          ctypes.POINTER(ctypes.c_int32)]
            lib.oracle_volume.restype = ctypes.c_int32
            lib.oracle_volume.argtypes = [ctypes.c_int64, P, P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _copy(ptr, n, dtype):
    if n <= 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def sample(verts, tris, origin, width, res, axis, mode="scan"):
    """One LDNI of a closed mesh (Definitions 1-2).

    Returns dict: offsets int64[res*res+1], depth f64[n], nrm f64[n,3],
    tri int32[n]; pixel (i, j) is row p = j*res + i; rays sorted by
    (depth, tri).  mode 'brute' tests every ray against every triangle;
    'scan' tests each triangle against the centres in its bounding box."""
    lib = _load()
    v = np.ascontiguousarray(verts, dtype=np.float32)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    o = np.ascontiguousarray(origin, dtype=np.float32)
    err = ctypes.c_int32(0)
    h = lib.oracle_sample(_ptr(v), v.shape[0], _ptr(t), t.shape[0], _ptr(o), float(width), int(res), int(axis),
                          0 if mode == "brute" else 1, ctypes.byref(err))
    if not h:
        raise ValueError(f"oracle_sample failed with code {err.value}")
    try:
        L = h.contents
        n, nr = L.n, L.nrays
        out = {
            "offsets": _copy(L.offsets, nr + 1, np.int64),
            "depth": _copy(L.depth, n, np.float64),
            "nrm": _copy(L.nrm, 3 * n, np.float64).reshape(n, 3),
            "tri": _copy(L.tri, n, np.int32),
        }
    finally:
        lib.oracle_free(h)
    out["res"] = int(res)
    out["axis"] = int(axis)
    return out


def boolean(A, B, op, eps=0.0):
    """Boolean of two same-grid LDNIs (Section 4.1) with small-interval
    removal (Section 4.1.1).  A and B: dicts with offsets, depth (f32),
    nrm (f32 [n,3]) and tri (int32).  Output values are copies of input
    values (normals of B inverted for a difference), ids of B-sourced samples
    carry bit 31."""
    lib = _load()
    opc = OPS[op] if isinstance(op, str) else int(op)
    oA = np.ascontiguousarray(A["offsets"], dtype=np.int64)
    oB = np.ascontiguousarray(B["offsets"], dtype=np.int64)
    if oA.shape != oB.shape:
        raise ValueError("grids differ")
    dA = np.ascontiguousarray(A["depth"], dtype=np.float32)
    dB = np.ascontiguousarray(B["depth"], dtype=np.float32)
    nA = np.ascontiguousarray(np.asarray(A["nrm"], dtype=np.float32).reshape(-1, 3))
    nB = np.ascontiguousarray(np.asarray(B["nrm"], dtype=np.float32).reshape(-1, 3))
    tA = np.ascontiguousarray(A["tri"], dtype=np.int32)
    tB = np.ascontiguousarray(B["tri"], dtype=np.int32)
    err = ctypes.c_int32(0)
    h = lib.oracle_boolean(oA.size - 1, _ptr(oA), _ptr(dA), _ptr(nA), _ptr(tA), _ptr(oB), _ptr(dB), _ptr(nB),
                           _ptr(tB), opc, float(eps), ctypes.byref(err))
    if not h:
        raise ValueError(f"oracle_boolean failed with code {err.value}")
    try:
        R = h.contents
        n, nr = R.n, R.nrays
        out = {
            "offsets": _copy(R.offsets, nr + 1, np.int64),
            "depth": _copy(R.depth, n, np.float32),
            "nrm": _copy(R.nrm, 3 * n, np.float32).reshape(n, 3),
            "tri": _copy(R.tri, n, np.int32),
        }
    finally:
        lib.oracle_bool_free(h)
    return out


def offset(Ls, origin, width, res, r, inner=False, eps=0.0, axes=(0, 1, 2)):
    """Offset of the solid given by its three LDNIs Ls (Section 4.2): the
    union of the solid with one sphere of radius r at every sample (inner:
    the difference), sphere by sphere in sample order (x-, y-, z-image, each
    in CSR order), then small-interval removal with eps.  Ls: three dicts
    with offsets, depth (f32), nrm (f32 [n,3]) and tri (int32).  Returns the
    images listed in axes, as oracle.boolean returns an image; sphere
    samples carry id s | 0x80000000 for sphere s."""
    lib = _load()
    nrays = int(res) * int(res)
    offs, ds, ns, ts, cnt = [], [], [], [], []
    for L in Ls:
        o = np.asarray(L["offsets"], dtype=np.int64)
        if o.size != nrays + 1:
            raise ValueError("an image does not match the resolution")
        offs.append(o - o[0])
        ds.append(np.asarray(L["depth"], dtype=np.float32)[o[0]:o[-1]])
        ns.append(np.asarray(L["nrm"], dtype=np.float32).reshape(-1, 3)[o[0]:o[-1]])
        ts.append(np.asarray(L["tri"], dtype=np.int32)[o[0]:o[-1]])
        cnt.append(int(o[-1] - o[0]))
    off = np.ascontiguousarray(np.concatenate(offs))
    d = np.ascontiguousarray(np.concatenate(ds), dtype=np.float32)
    nr = np.ascontiguousarray(np.concatenate(ns), dtype=np.float32)
    t = np.ascontiguousarray(np.concatenate(ts), dtype=np.int32)
    n = np.asarray(cnt, dtype=np.int64)
    org = np.ascontiguousarray(origin, dtype=np.float32)
    out = []
    for b in axes:
        err = ctypes.c_int32(0)
        h = lib.oracle_offset(int(res), _ptr(org), float(width), _ptr(off), _ptr(d), _ptr(nr), _ptr(t), _ptr(n),
                              int(b), float(r), OP_DIFF if inner else OP_UNION, float(eps), ctypes.byref(err))
        if not h:
            raise ValueError(f"oracle_offset failed with code {err.value}")
        try:
            R = h.contents
            out.append({
                "offsets": _copy(R.offsets, R.nrays + 1, np.int64),
                "depth": _copy(R.depth, R.n, np.float32),
                "nrm": _copy(R.nrm, 3 * R.n, np.float32).reshape(R.n, 3),
                "tri": _copy(R.tri, R.n, np.int32),
            })
        finally:
            lib.oracle_bool_free(h)
    return out


def volume(L, h):
    """Enclosed volume from one LDNI: h^2 * sum over rays of inside lengths."""
    lib = _load()
    off = np.ascontiguousarray(L["offsets"], dtype=np.int64)
    d = np.ascontiguousarray(L["depth"], dtype=np.float32)
    vol = ctypes.c_double(0.0)
    rc = lib.oracle_volume(off.size - 1, _ptr(off), _ptr(d), float(h), ctypes.byref(vol))
    if rc != 0:
        raise ValueError(f"oracle_volume failed with code {rc}")
    return vol.value


def as_f32(L):
    """An oracle LDNI with FP32 depth and normals (the kernel's storage
    precision), for feeding the Boolean and volume oracles."""
    return {"offsets": L["offsets"], "depth": L["depth"].astype(np.float32),
            "nrm": L["nrm"].astype(np.float32), "tri": L["tri"]}
