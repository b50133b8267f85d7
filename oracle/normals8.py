"""Approximate (8-bit) surface normals (TEST INFRASTRUCTURE ONLY): Section 3,
"Approximate Surface Normal Sampling".  Written from the paper's
description in plain NumPy; shares no code with the CUDA library.

The paper renders the three components of the unit normal as the RGB
colour of the face and reads them back from an 8-bit-per-channel colour
buffer: 256 levels for the range [-1, 1].  It then normalises the decoded
vector, since an interpolated or quantised normal is not of unit length.

Readings (the paper gives no arithmetic):
  - a component n maps to the code q = rint(fl32(fl32(n + 1) * 127.5)),
    rounded half to even, clamped to [0, 255]; NaN gives 0;
  - the three codes are packed into one 32-bit word, x in bits 0-7, y in
    8-15, z in 16-23, bits 24-31 zero;
  - decoding gives c = fl32(fl32(q / 127.5) - 1) per component, then the
    vector divided by its length, sqrt(fl32(fl32(cx^2 + cy^2) + cz^2)), all
    in FP32 rounded to nearest;
  - the Boolean's inversion of a normal (Section 4.1) maps every code q to
    255 - q, which decodes to minus the decoded component in exact
    arithmetic.
"""
from __future__ import annotations

import numpy as np


def encode(n: np.ndarray) -> np.ndarray:
    """float [m, 3] -> uint32 [m] packed codes."""
    n = np.asarray(n, dtype=np.float32).reshape(-1, 3)
    with np.errstate(invalid="ignore"):
        v = ((n + np.float32(1.0)).astype(np.float32) * np.float32(127.5)).astype(np.float32)
        q = np.where(v >= 255, 255, np.where(v > 0, np.rint(v), 0))
    q = np.nan_to_num(q, nan=0.0).astype(np.uint32)
    return q[:, 0] | (q[:, 1] << 8) | (q[:, 2] << 16)


def codes(w: np.ndarray) -> np.ndarray:
    """uint32 [m] -> uint8-valued int array [m, 3]."""
    w = np.asarray(w).astype(np.uint32)
    return np.stack([w & 255, (w >> 8) & 255, (w >> 16) & 255], axis=1).astype(np.int64)


def decode_raw(w: np.ndarray) -> np.ndarray:
    """Per-component values before normalisation, FP32 [m, 3]."""
    q = codes(w).astype(np.float32)
    return ((q / np.float32(127.5)).astype(np.float32) - np.float32(1.0)).astype(np.float32)


def decode(w: np.ndarray) -> np.ndarray:
    """Unit normals, FP32 [m, 3]."""
    c = decode_raw(w)
    s = (c[:, 0] * c[:, 0]).astype(np.float32) + (c[:, 1] * c[:, 1]).astype(np.float32)
    s = s.astype(np.float32) + (c[:, 2] * c[:, 2]).astype(np.float32)
    ln = np.sqrt(s.astype(np.float32)).astype(np.float32)
    return (c / ln[:, None]).astype(np.float32)


def invert(w: np.ndarray) -> np.ndarray:
    """The inverted normal (Section 4.1), in code space: q -> 255 - q."""
    return (np.asarray(w).astype(np.uint32) ^ np.uint32(0x00FFFFFF)).astype(np.uint32)


def boolean(A: dict, B: dict, op, eps: float = 0.0) -> dict:
    """The Boolean of Section 4.1 on LDNIs whose normals are packed codes
    (key "nrm8"): a sample's normal is copied, or inverted in code space
    when it comes from B in a difference.  Computed with the FP32 Boolean
    oracle on the codes written as float components (an inversion there
    flips their signs, read back as 255 - q)."""
    from . import boolean as _boolean

    def as_float(L):
        return {"offsets": L["offsets"], "depth": L["depth"], "tri": L["tri"],
                "nrm": codes(L["nrm8"]).astype(np.float32)}

    R = _boolean(as_float(A), as_float(B), op, eps)
    v = R["nrm"]
    q = np.where(np.signbit(v), 255 - np.abs(v), v).astype(np.uint32)
    out = {k: R[k] for k in ("offsets", "depth", "tri")}
    out["nrm8"] = q[:, 0] | (q[:, 1] << 8) | (q[:, 2] << 16)
    return out
