"""ctypes view of libldni.so (the C ABI declared in include/ldni.h).

Argument marshalling only: every step of sampling, Boolean and volume runs
in the library's CUDA kernels.  There is no CPU fallback: if the library
cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

LDNI_OK = 0
LDNI_ECUDA = -6
AXIS_ALL = 3
MODE_EXACT2 = 0
MODE_LEARNED1 = 1
MODE_BINNED2 = 2
OP_UNION, OP_INTER, OP_DIFF = 0, 1, 2

ST_CAPACITY, ST_ODD, ST_TOOLARGE, ST_TIMEOUT, ST_RANGE, ST_INDEX, ST_EVENTS, ST_BOUNDS = 1, 2, 4, 8, 16, 32, 64, 128


class Grid(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("width", ctypes.c_float), ("res", ctypes.c_int32)]


class MLP(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("b", ctypes.c_void_p), ("margin", ctypes.c_float)]


MLP_IN, MLP_WEIGHTS, MLP_BIASES, TILE_RAYS = 12, 9024, 193, 4096


class Layers(ctypes.Structure):
    _fields_ = [("offsets", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("nx", ctypes.c_void_p),
                ("ny", ctypes.c_void_p), ("nz", ctypes.c_void_p), ("tri_id", ctypes.c_void_p),
                ("capacity", ctypes.c_int64), ("nrm8", ctypes.c_void_p)]


class Cell(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_int64), ("labels", ctypes.c_uint32), ("npts", ctypes.c_uint32),
                ("nvert", ctypes.c_int32), ("pad_", ctypes.c_int32), ("v", ctypes.c_float * 12)]


class Tuning(ctypes.Structure):
    _fields_ = [("bool_tile_rays", ctypes.c_int32), ("bool_stage_samples", ctypes.c_int32),
                ("tri_blocks_per_sm", ctypes.c_int32), ("bool_split", ctypes.c_int32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("tris", ctypes.c_void_p), ("nv", ctypes.c_int64),
                ("nt", ctypes.c_int64), ("grid", Grid), ("pad_", ctypes.c_int32), ("out", Layers * 3)]


INFO_BYTES = 32  # ldni_info_t: int64 n[3]; uint32 status; uint32 odd_rays


class LDNIError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        detail = ""
        if code == LDNI_ECUDA:
            try:
                detail = ": " + load().ldni_last_cuda_error().decode()
            except Exception:
                detail = ""
        super().__init__(f"{what}: {strerror(code)} ({code}){detail}")


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_SZ = ctypes.c_size_t
_PG = ctypes.POINTER(Grid)
_PL = ctypes.POINTER(Layers)

# name -> (restype, argtypes); every symbol include/ldni.h declares
SIGNATURES = {
    "ldni_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "ldni_version": (ctypes.c_int, []),
    "ldni_last_cuda_error": (ctypes.c_char_p, []),
    "ldni_grid_from_bbox": (ctypes.c_int, [_P, _I32, _PG]),
    "ldni_sample_workspace_size": (ctypes.c_int, [_I64, _I64, _I32, _I32, ctypes.POINTER(_SZ)]),
    "ldni_sample": (ctypes.c_int, [_P, _I64, _P, _I64, _PG, _I32, _I32, _PL, _P, _P, _SZ, _P]),
    "ldni_sample_count": (ctypes.c_int, [_P, _I64, _P, _I64, _PG, _I32, _PL, _P, _P, _SZ, _P]),
    "ldni_sample_fill": (ctypes.c_int, [_P, _I64, _P, _I64, _PG, _I32, _PL, _P, _P, _SZ, _P]),
    "ldni_sample_binned_workspace_size": (ctypes.c_int, [_I64, _I64, _I32, _I32, ctypes.POINTER(_SZ)]),
    "ldni_sample_binned_count": (ctypes.c_int, [_P, _I64, _P, _I64, _PG, _I32, _PL, _P, _P, _SZ, _P]),
    "ldni_sample_binned_fill": (ctypes.c_int, [_P, _I64, _P, _I64, _PG, _I32, _PL, _P, _P, _SZ, _P]),
    "ldni_boolean_workspace_size": (ctypes.c_int, [_I32, ctypes.POINTER(_SZ)]),
    "ldni_boolean": (ctypes.c_int, [_PL, _PG, _PL, _PG, _I32, ctypes.c_float, _PL, _P, _P, _SZ, _P]),
    "ldni_boolean_static": (ctypes.c_int, [_PL, _PG, _PL, _PG, _I32, ctypes.c_float, _PL, _P, _P]),
    "ldni_volume_workspace_size": (ctypes.c_int, [_I32, ctypes.POINTER(_SZ)]),
    "ldni_volume": (ctypes.c_int, [_PL, _PG, _P, _P, _P, _SZ, _P]),
    "ldni_sample_learned_workspace_size": (ctypes.c_int, [_I64, _I64, _I32, _I32, _I64, ctypes.POINTER(_SZ)]),
    "ldni_sample_learned": (ctypes.c_int, [_P, _I64, _P, _I64, _PG, _I32, _P, _I32, _I32, _I64, _PL, _P, _P, _P,
                                           _SZ, _P]),
    "ldni_tile_features": (ctypes.c_int, [_P, _I64, _P, _I64, _PG, _I32, _I32, _P, _P, _P]),
    "ldni_tile_labels": (ctypes.c_int, [_P, _I32, _P, _P]),
    "ldni_mlp_forward": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "ldni_mlp_train_workspace_size": (ctypes.c_int, [_I64, ctypes.POINTER(_SZ)]),
    "ldni_mlp_train_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _I64, ctypes.c_float, _I32, ctypes.c_float,
                                           _P, _P, _P, _SZ, _P]),
    "ldni_depth_vjp": (ctypes.c_int, [_P, _I64, _P, _I64, _PG, _I32, _PL, _P, _P, _P, _P]),
    "ldni_volume_grad": (ctypes.c_int, [_P, _I64, _P, _I64, _PG, _I32, _PL, ctypes.c_double, _P, _P, _P]),
    "ldni_boolean_many_workspace_size": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(_SZ)]),
    "ldni_boolean_many": (ctypes.c_int, [_I32, _P, _P, _P, _I32, ctypes.c_float, _P, _P, _P, _P, _SZ, _P]),
    "ldni_volume_many_workspace_size": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(_SZ)]),
    "ldni_volume_many": (ctypes.c_int, [_I32, _P, _P, _P, _P, _P, _SZ, _P]),
    "ldni_normals_encode8": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P]),
    "ldni_normals_decode8": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P]),
    "ldni_contour_workspace_size": (ctypes.c_int, [_I32, ctypes.c_int64, ctypes.POINTER(_SZ)]),
    "ldni_contour_cells": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _SZ, _P]),
    "ldni_offset_workspace_size": (ctypes.c_int, [_P, _I32, ctypes.c_float, ctypes.c_float, ctypes.POINTER(_SZ)]),
    "ldni_offset": (ctypes.c_int, [_P, _P, _P, ctypes.c_float, _I32, ctypes.c_float, _P, _P, _P, _SZ, _P]),
    "ldni_classify_nodes_workspace_size": (ctypes.c_int, [_I32, ctypes.POINTER(_SZ)]),
    "ldni_classify_nodes": (ctypes.c_int, [_P, _P, _P, _P, _P, _SZ, _P]),
    "ldni_union_chain_workspace_size": (ctypes.c_int, [_I32, _I32, ctypes.POINTER(_SZ)]),
    "ldni_union_chain": (ctypes.c_int, [_P, _P, _I32, _I32, _PG, ctypes.c_float, _P, _P, _P, _SZ, _P]),
    "ldni_set_wait_limit": (ctypes.c_int, [_I32]),
    "ldni_get_wait_limit": (ctypes.c_int32, []),
    "ldni_wait_selftest": (ctypes.c_int, [_P, _P]),
    "ldni_build_checked": (ctypes.c_int32, []),
    "ldni_get_tuning": (ctypes.c_int, [_P]),
    "ldni_set_tuning": (ctypes.c_int, [_P]),
    "ldni_sample_batch_workspace_size": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_SZ)]),
    "ldni_sample_batch": (ctypes.c_int, [_P, _P, _I32, _P, _P, _SZ, _P]),
    "ldni_launch_count": (ctypes.c_uint64, []),
    "ldni_profile_set": (ctypes.c_int, [_P, _P, _P, _I32, _I32]),
    "ldni_profile_recorded": (ctypes.c_int64, []),
    "ldni_kernel_name": (ctypes.c_char_p, [_I32]),
}


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libldni.so (building it first if needed).  Raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libldni.so not found at {path}; run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def strerror(code: int) -> str:
    try:
        return load().ldni_strerror(int(code)).decode()
    except Exception:  # library unavailable: still give the number
        return f"ldni error {code}"


def check(code: int, what: str) -> None:
    if code != LDNI_OK:
        raise LDNIError(code, what)
