"""The C-ABI library builds, loads on a machine without a GPU, and exports
every function include/ldni.h declares; host-side argument checks answer
without touching the device."""
import ctypes
import os
import re

import pytest

import paper_1009_0794_gb300 as pkg
from paper_1009_0794_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ldni_\w+)\s*\(", src, flags=re.M))
    return names


def test_every_declared_symbol_is_exported():
    lib = _lib.load()
    declared = _declared()
    assert "ldni_sample" in declared and "ldni_boolean" in declared and "ldni_volume" in declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared <= set(_lib.SIGNATURES)


def test_host_validation_without_gpu():
    lib = _lib.load()
    sz = ctypes.c_size_t(0)
    assert lib.ldni_sample_workspace_size(10, 10, 0, 3, ctypes.byref(sz)) == -1
    assert lib.ldni_sample_workspace_size(10, 10, 128, 3, ctypes.byref(sz)) == 0 and sz.value > 3 * 128 * 128 * 4
    assert lib.ldni_boolean_workspace_size(64, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.ldni_volume_workspace_size(64, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.ldni_strerror(-2).decode().startswith("Boolean operands")
    assert lib.ldni_version() >= 100
    # null arguments are refused before any CUDA call
    assert lib.ldni_sample(None, 0, None, 0, None, 3, 0, None, None, None, 0, None) == -1
    g = _lib.Grid()
    bbox = (ctypes.c_float * 6)(-1, -2, -3, 1, 0, 2)
    assert lib.ldni_grid_from_bbox(ctypes.cast(bbox, ctypes.c_void_p), 32, ctypes.byref(g)) == 0
    assert list(g.origin) == [-1, -2, -3] and g.width == 5 and g.res == 32


def test_grid_mismatch_refused_on_host():
    lib = _lib.load()
    ga, gb = _lib.Grid(), _lib.Grid()
    ga.width = gb.width = 1.0
    ga.res, gb.res = 64, 128
    L = _lib.Layers()
    L.offsets = 16
    L.capacity = 0
    rc = lib.ldni_boolean(ctypes.byref(L), ctypes.byref(ga), ctypes.byref(L), ctypes.byref(gb), 0, 0.0,
                          ctypes.byref(L), 8, 8, 1 << 20, None)
    assert rc == -2


def test_package_import_is_light():
    assert pkg.LDNIError is _lib.LDNIError


def test_tuning_knobs_validate_on_host():
    """ldni_set_tuning rejects out-of-range knobs without changing the
    current ones, and NULL restores the defaults (no GPU needed)."""
    from paper_1009_0794_gb300 import _lib
    lib = _lib.load()
    t = _lib.Tuning()
    assert lib.ldni_get_tuning(ctypes.byref(t)) == 0
    assert (t.bool_tile_rays, t.bool_stage_samples, t.tri_blocks_per_sm, t.bool_split) == (512, 4096, 16, -1)
    for bad in (_lib.Tuning(300, 4096, 16, 0), _lib.Tuning(1024, 20000, 16, 0), _lib.Tuning(1024, 4096, 0, 0),
                _lib.Tuning(1024, 4096, 16, 2)):
        assert lib.ldni_set_tuning(ctypes.byref(bad)) == -1
    good = _lib.Tuning(1024, 0, 4, 1)
    assert lib.ldni_set_tuning(ctypes.byref(good)) == 0
    assert lib.ldni_get_tuning(ctypes.byref(t)) == 0 and (t.bool_tile_rays, t.tri_blocks_per_sm) == (1024, 4)
    assert lib.ldni_set_tuning(None) == 0
    assert lib.ldni_get_tuning(ctypes.byref(t)) == 0 and t.bool_tile_rays == 512


def test_build_stamp_is_the_same_in_another_checkout(tmp_path):
    """The stamp that names a build's sources (and keys the recorded ncu
    traffic) depends on the sources and flags, not on where the repository
    sits: a copy of the tree elsewhere gives the same stamp."""
    import importlib.util
    import shutil
    from paper_1009_0794_gb300 import build
    root = os.path.dirname(os.path.dirname(os.path.abspath(build.__file__)))
    pkg_copy = tmp_path / "elsewhere" / "paper_1009_0794_gb300"
    shutil.copytree(os.path.join(root, "paper_1009_0794_gb300", "csrc"), pkg_copy / "csrc")
    shutil.copytree(os.path.join(root, "include"), tmp_path / "elsewhere" / "include")
    shutil.copy(build.__file__, pkg_copy / "build.py")
    spec = importlib.util.spec_from_file_location("build_copy", pkg_copy / "build.py")
    copy = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(copy)
    assert copy.ROOT != build.ROOT
    assert copy._stamp() == build._stamp()
    assert copy._stamp(["learned.cu"]) == build._stamp(["learned.cu"]) != build._stamp()
