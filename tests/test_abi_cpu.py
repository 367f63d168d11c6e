"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol include/wasabi.h declares (no compute call: there is no GPU here), and
argument validation answers before any device work."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wlib():
    from paper_1708_04233_gb300 import build, _abi
    build.build()
    return _abi.load()


def _declared():
    hdr = open(os.path.join(ROOT, "include", "wasabi.h")).read()
    return re.findall(r"^(?:wasabi_status|const char\*)\s+(\w+)\(", hdr, re.M)


def test_header_declares_the_entry_points():
    names = set(_declared())
    for n in ["wasabi_build_lut", "wasabi_superpose", "wasabi_inverse_haar", "cgh_direct",
              "wasabi_sync_status", "wasabi_lut_selection", "wasabi_quantize_points"]:
        assert n in names


def test_library_exports_every_declared_symbol(wlib):
    from paper_1708_04233_gb300 import _abi
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, re.M))
    for n in _declared():
        assert n in exported, n
        assert hasattr(wlib, n)
    assert {s[0] for s in _abi.SIGNATURES} == set(_declared())


def test_library_is_sm103a():
    from paper_1708_04233_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_depth_grid_host_only(wlib, orc):
    import paper_1708_04233_gb300 as w
    assert np.array_equal(w.depth_grid(0.3e-3, 1.0e-3, 64), orc.depth_grid(0.3e-3, 1.0e-3, 64))
    with pytest.raises(w.WasabiError):
        w.depth_grid(1.0, 0.5, 4)


def test_build_lut_rejects_bad_arguments(wlib):
    d = np.array([0.5e-3], np.float64)
    h = C.c_void_p()
    dp = d.ctypes.data_as(C.POINTER(C.c_double))
    # window not a multiple of 2^(L+1), window too small for the PSF, bad levels,
    # lambda >= 2 pitch, keep_ratio <= 0: all rejected before any device work.
    assert wlib.wasabi_build_lut(633e-9, 1e-6, dp, 1, 1000, 4, 0.1, 0, None, C.byref(h)) == -1
    assert wlib.wasabi_build_lut(633e-9, 1e-6, dp, 1, 64, 3, 0.1, 0, None, C.byref(h)) == -1
    assert wlib.wasabi_build_lut(633e-9, 1e-6, dp, 1, 1024, 6, 0.1, 0, None, C.byref(h)) == -1
    assert wlib.wasabi_build_lut(3e-6, 1e-6, dp, 1, 1024, 4, 0.1, 0, None, C.byref(h)) == -1
    assert wlib.wasabi_build_lut(633e-9, 1e-6, dp, 1, 1024, 4, 0.0, 0, None, C.byref(h)) == -1
    assert b"window" in wlib.wasabi_last_error() or len(wlib.wasabi_last_error()) > 0


def test_inverse_rejects_bad_arguments(wlib):
    assert wlib.wasabi_inverse_haar(None, 64, 64, 4, None, None, None) == -1
    assert wlib.wasabi_inverse_haar(C.c_void_p(256), 60, 64, 4, C.c_void_p(256), None, None) == -1
    assert wlib.wasabi_inverse_haar(C.c_void_p(256), 64, 64, 1, C.c_void_p(256), None, None) == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import importlib
    from paper_1708_04233_gb300 import _abi, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _abi.load()
