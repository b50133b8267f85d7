"""GB300-native Layered Depth-Normal Images (Wang & Chen).

Sampling of closed triangle meshes into three axis-aligned LDNIs, per-ray
Boolean merges and LDNI volume, computed by hand-written sm_103a CUDA
kernels behind the C ABI in include/ldni.h.  PyTorch provides device memory
and streams only.
"""
import importlib

from . import _lib  # noqa: F401
from ._lib import LDNIError  # noqa: F401


def __getattr__(name):
    # the torch-facing API is imported on first use so that building or
    # inspecting the package does not pay for importing torch
    if name.startswith("__"):
        raise AttributeError(name)
    api = importlib.import_module(__name__ + ".ldni")
    try:
        return getattr(api, name)
    except AttributeError:
        raise AttributeError(name) from None
