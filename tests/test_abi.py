"""The C-ABI library: it builds, loads, exports every declared symbol, and rejects bad
arguments on the host before touching a device (no GPU needed)."""

import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"GPP_API\s+[\w\s\*]+?\b(gpp_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2008_11326_gb300 import _native, build
    if not build.up_to_date():
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build libgpp")
        build.build()
    return _native.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert {"gpp_sigma", "gpp_sigma_workspace_size", "gpp_last_error", "gpp_peak_launch"} <= names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    from paper_2008_11326_gb300 import _native
    assert {s[0] for s in _native.SIGNATURES} == names


def test_host_side_validation(lib):
    from paper_2008_11326_gb300 import _native as N
    assert lib.gpp_sigma(None, None, None, 0, None) == -1
    assert b"problem is NULL" in lib.gpp_last_error()
    p = N.GppProblem()
    p.number_bands, p.nvband, p.ncouls, p.ngpown, p.nw = 4, 2, 8, 2, 0
    assert lib.gpp_sigma(ctypes.byref(p), None, None, 0, None) == -2
    p.nw = 9
    assert lib.gpp_sigma(ctypes.byref(p), None, None, 0, None) == -2
    p.nw = 3
    p.ncouls = -1
    assert lib.gpp_sigma(ctypes.byref(p), None, None, 0, None) == -2
    p.ncouls = 8
    o = N.GppOptions()
    lib.gpp_options_default(ctypes.byref(o))
    o.precision = 7
    assert lib.gpp_sigma(ctypes.byref(p), ctypes.byref(o), None, 0, None) == -8
    lib.gpp_options_default(ctypes.byref(o))
    o.block_threads = 100
    assert lib.gpp_sigma(ctypes.byref(p), ctypes.byref(o), None, 0, None) == -8
    lib.gpp_options_default(ctypes.byref(o))
    o.reserved = 3
    assert lib.gpp_sigma(ctypes.byref(p), ctypes.byref(o), None, 0, None) == -8
    lib.gpp_options_default(ctypes.byref(o))
    o.physics = 4
    assert lib.gpp_sigma(ctypes.byref(p), ctypes.byref(o), None, 0, None) == -8
    o.physics = N.GPP_PHYS_SX_CUTOFF      # the cutoff without a positive factor
    assert lib.gpp_sigma(ctypes.byref(p), ctypes.byref(o), None, 0, None) == -8
    assert b"sexcut" in lib.gpp_last_error()
    o.sexcut = float("inf")
    assert lib.gpp_sigma(ctypes.byref(p), ctypes.byref(o), None, 0, None) == -8
    lib.gpp_options_default(ctypes.byref(o))
    assert o.physics == 0 and o.sexcut == 0.0
    # outputs missing
    assert lib.gpp_sigma(ctypes.byref(p), ctypes.byref(o), None, 0, None) == -1
    assert b"achtemp" in lib.gpp_last_error()
    assert lib.gpp_version().startswith(b"libgpp")


def test_noalloc_returns_the_validation_codes(lib):
    """gpp_sigma_noalloc reports the code gpp_sigma gives for the same bad arguments (no
    device is touched before the arguments are validated)."""
    from paper_2008_11326_gb300 import _native as N
    assert lib.gpp_sigma_noalloc(None, None, None) == -1
    assert b"problem is NULL" in lib.gpp_last_error()
    p = N.GppProblem()
    p.number_bands, p.nvband, p.ncouls, p.ngpown, p.nw = 4, 2, 8, 2, 0
    assert lib.gpp_sigma_noalloc(ctypes.byref(p), None, None) == -2
    p.nw = 3
    o = N.GppOptions()
    lib.gpp_options_default(ctypes.byref(o))
    o.precision = 7
    assert lib.gpp_sigma_noalloc(ctypes.byref(p), ctypes.byref(o), None) == -8
    assert b"precision" in lib.gpp_last_error()
    lib.gpp_options_default(ctypes.byref(o))
    o.physics = 4
    assert lib.gpp_sigma_noalloc(ctypes.byref(p), ctypes.byref(o), None) == -8


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2008_11326_gb300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "missing" / "libgpp.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _native.lib()
