"""ctypes declarations of libwasabi's C ABI (include/wasabi.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

OK, E_INVALID, E_NOMEM, E_CUDA, E_RANGE, E_TIMEOUT = 0, -1, -2, -3, -4, -5
F32, F16S, BF16S = 0, 1, 2
SHIFT_FLOOR, SHIFT_NEAREST = 0, 1

_NAMES = {E_INVALID: "WASABI_E_INVALID", E_NOMEM: "WASABI_E_NOMEM", E_CUDA: "WASABI_E_CUDA",
          E_RANGE: "WASABI_E_RANGE", E_TIMEOUT: "WASABI_E_TIMEOUT"}

# (name, restype, argtypes) for every exported entry point.
_VP, _I32P, _I64P, _F64P, _F32P, _U8P = (C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                         C.POINTER(C.c_double), C.POINTER(C.c_float),
                                         C.POINTER(C.c_uint8))
_i, _i64, _d, _sz = C.c_int, C.c_int64, C.c_double, C.c_size_t
SIGNATURES = [
    ("wasabi_last_error", C.c_char_p, []),
    ("wasabi_depth_grid", _i, [_d, _d, _i, _F64P]),
    ("wasabi_quantize_points", _i, [_VP, _VP, _VP, _VP, _i64, _d, _d, _i, _VP, _VP]),
    ("wasabi_build_lut", _i, [_d, _d, _F64P, _i, _i, _i, _d, _i, _VP, C.POINTER(_VP)]),
    ("wasabi_build_lut_wavelet", _i, [_d, _d, _F64P, _i, _i, _i, _d, _i, _i, _VP, C.POINTER(_VP)]),
    ("wasabi_lut_destroy", _i, [_VP]),
    ("wasabi_lut_counts", _i, [_VP, _I64P]),
    ("wasabi_lut_selection", _i, [_VP, _i, _I32P, _I64P]),
    ("wasabi_lut_entries", _i, [_VP, _i, _I32P, _F32P, _I64P]),
    ("wasabi_scratch_bytes", _i, [_VP, _i64, _i, _i, C.POINTER(_sz)]),
    ("wasabi_superpose", _i, [_VP, _VP, _i64, _i, _i, _i, _VP, _VP, _sz, _VP]),
    ("wasabi_superpose_static", _i, [_VP, _VP, _i64, _i, _i, _i, _VP, _VP]),
    ("wasabi_hologram", _i, [_VP, _VP, _i64, _i, _i, _i, _VP, _VP, _VP, _VP, _sz, _VP]),
    ("wasabi_inverse_haar", _i, [_VP, _i, _i, _i, _VP, _VP, _VP]),
    ("wasabi_hologram_frame", _i, [_VP, _VP, _i64, _i, _i, _i, _VP, _VP, _VP, _VP, _VP, _sz, _VP]),
    ("wasabi_inverse_haar_frame", _i, [_VP, _i, _i, _i, _VP, _VP, _VP, _VP]),
    ("wasabi_hologram_stream", _i, [_VP, _VP, _i64, _i, _i, _i, _i, _VP, _VP, _VP, _VP]),
    ("wasabi_reconstruct_scratch_bytes", _i, [_i, _i, C.POINTER(_sz)]),
    ("wasabi_inverse_wavelet_scratch_bytes", _i, [_i, _i, C.POINTER(_sz)]),
    ("wasabi_inverse_wavelet", _i, [_VP, _i, _i, _i, _i, _VP, _VP, _VP, _VP, _sz, _VP]),
    ("wasabi_reconstruct", _i, [_VP, _i, _i, _i, _d, _d, _d, _VP, _VP, _VP, _VP, _sz, _VP]),
    ("cgh_direct_scratch_bytes", _i, [_i64, _i, _i, C.POINTER(_sz)]),
    ("cgh_direct", _i, [_d, _d, _F64P, _i, _VP, _i64, _i, _i, _i, _VP, _VP, _sz, _VP]),
    ("wasabi_sync_status", _i, [_VP]),
    ("wasabi_haar_forward", _i, [_VP, _i, _i, _i, _VP, _VP]),
    ("wasabi_wbuf_to_mallat", _i, [_VP, _i, _i, _i, _VP, _VP]),
    ("wasabi_test_inverse_stall", _i, [_VP, _i, _i, _i, _VP, _i64, _i64, _VP]),
    ("wasabi_batch_create", _i, [_VP, _i, _i, _i, C.POINTER(_VP)]),
    ("wasabi_batch_destroy", _i, [_VP]),
    ("wasabi_batch_config", _i, [_VP, C.POINTER(_i), C.POINTER(_i)]),
    ("wasabi_batch_scratch_bytes", _i, [_VP, _VP, _i, C.POINTER(_sz)]),
    ("wasabi_batch_run", _i, [_VP, _VP, _i, _VP, _sz, _VP]),
    ("wasabi_autotune", _i, [_VP, _i, _i64, _VP, C.POINTER(_i), C.POINTER(_i)]),
    ("wasabi_server_create", _i, [_VP, _sz, _i, _i, _i, C.POINTER(_VP)]),
    ("wasabi_server_submit", _i, [_VP, _VP, _I64P]),
    ("wasabi_server_wait", _i, [_VP, _i64, _d, _VP]),
    ("wasabi_server_stats", _i, [_VP, C.POINTER(_sz), _I64P, _I64P]),
    ("wasabi_server_destroy", _i, [_VP]),
]


REF_PLANE, REF_SPHERICAL = 0, 1
RECON_FIELD, RECON_BITS = 0, 1
WAVELETS = {"haar": 0, "coif1": 1}


class Reference(C.Structure):
    """wasabi_reference of include/wasabi.h."""
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("lam", C.c_double), ("pitch", C.c_double),
                ("x", C.c_double), ("y", C.c_double), ("z", C.c_double)]


class Frame(C.Structure):
    """wasabi_frame of include/wasabi.h."""
    _fields_ = [("origin_x", C.c_int32), ("origin_y", C.c_int32), ("ref", Reference)]


class Job(C.Structure):
    """wasabi_job of include/wasabi.h."""
    _fields_ = [("points_dev", C.c_void_p), ("n", C.c_int64), ("holo_w", C.c_int),
                ("holo_h", C.c_int), ("rule", C.c_int), ("wbuf_dev", C.c_void_p),
                ("u_dev", C.c_void_p), ("bits_dev", C.c_void_p), ("frame", Frame)]


class Request(C.Structure):
    """wasabi_request of include/wasabi.h."""
    _fields_ = [("points_host", C.c_void_p), ("n", C.c_int64), ("holo_w", C.c_int), ("holo_h", C.c_int),
                ("rule", C.c_int), ("bits_host", C.c_void_p), ("u_host", C.c_void_p), ("frame", Frame)]


class RequestInfo(C.Structure):
    """wasabi_request_info of include/wasabi.h."""
    _fields_ = [("submit_s", C.c_double), ("launch_s", C.c_double), ("done_s", C.c_double),
                ("batch_jobs", C.c_int), ("status", C.c_int)]


_lib = None


class WasabiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib_path() -> str:
    return _build.LIB


# Variant builds (for example with profiling counters) live in another
# directory, chosen by WASABI_BUILD_DIR at build and load time.


def load(build_if_missing: bool = False):
    """Load libwasabi.so; raise if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"libwasabi.so is not built ({_build.LIB}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        _build.build()
    L = C.CDLL(_build.LIB)
    for name, res, args in SIGNATURES:
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(code: int) -> None:
    if code != OK:
        raise WasabiError(code, load().wasabi_last_error().decode(errors="replace"))
