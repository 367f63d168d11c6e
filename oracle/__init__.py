"""WASABI oracle — TEST INFRASTRUCTURE ONLY.

A plain, slow CPU restatement of the WASABI method (arXiv 1708.04233) in
C++ (``wasabi_oracle.cpp``) with this thin numpy wrapper.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the CUDA library never does, and the two share no code.

Functions and the passages they follow:

* ``support_radius``  — Sec. 1, step 1 (PSF radius; reading R1)
* ``keep_target``     — Sec. 1, step 1 (N_r = pi (W_j/2)^2 gamma; reading R3)
* ``depth_grid`` / ``quantize`` — Sec. 1, step 1 and Sec. 2 (Delta z; R2)
* ``psf_f32`` / ``psf_f64`` — Sec. 1, step 1 (u_z = exp(ikr) circ(...))
* ``haar_fwd`` / ``haar_inv`` — Sec. 1, steps 1 and 3 (FWT; Haar, R4)
* ``wavelet_fwd`` / ``wavelet_inv`` / ``coif1_taps`` — the same steps with the
  paper's coiflets (order 1, periodic filter banks; R14)
* ``select``          — Sec. 1, step 1 ("N_r strong coefficients"; R5)
* ``build_lut``       — Sec. 1, step 1 for all depths
* ``superpose``       — Eq. (2) with the shift rule R6
* ``subhologram`` / ``hologram`` — Sec. 1, large-scale steps 2-4
* ``binarize``        — Sec. 2 (binary amplitude hologram; R7)
* ``reference_wave`` / ``binarize_ref`` — Sec. 2 (spherical reference wave,
  bit = Re(u conj R) > 0; R12)
* ``reconstruct``     — numerical reconstruction (Sec. 2, Fig. 3(b)): the
  angular spectrum method, written with numpy's FFT (reading R13)
* ``cgh_direct``      — Eq. (1)

Parity pins live in ``tests/test_oracle_*.py``.  Functions without an
independent pin: none at present (the unaligned-point WASABI error against
Eq. (1) is reported, not bounded, because the paper prints no error figure).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_u32p = C.POINTER(C.c_uint32)
_f32p = C.POINTER(C.c_float)
_f64p = C.POINTER(C.c_double)
_u8p = C.POINTER(C.c_uint8)


def _p(arr, t):
    return arr.ctypes.data_as(t)


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = C.CDLL(path)
    L.orc_support_radius.restype = C.c_double
    L.orc_support_radius.argtypes = [C.c_double] * 3
    L.orc_keep_target.restype = C.c_int64
    L.orc_keep_target.argtypes = [C.c_double, C.c_double]
    L.orc_depth_grid.argtypes = [C.c_double, C.c_double, C.c_int, _f64p]
    L.orc_quantize.restype = C.c_int64
    L.orc_quantize.argtypes = [_f64p, C.c_int64, C.c_double, C.c_double, C.c_int, _u32p]
    L.orc_sincos2pi_f32.argtypes = [_f32p, C.c_int64, _f32p, _f32p]
    L.orc_psf_f32.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, _f32p]
    L.orc_psf_f64.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, _f64p]
    for nm, t in (("orc_haar_fwd_f32", _f32p), ("orc_haar_inv_f32", _f32p),
                  ("orc_haar_fwd_f64", _f64p), ("orc_haar_inv_f64", _f64p)):
        getattr(L, nm).argtypes = [t, C.c_int64, C.c_int]
    for nm, t in (("orc_wavelet_fwd_f32", _f32p), ("orc_wavelet_inv_f32", _f32p),
                  ("orc_wavelet_fwd_f64", _f64p), ("orc_wavelet_inv_f64", _f64p)):
        getattr(L, nm).argtypes = [t, C.c_int64, C.c_int, C.c_int]
    L.orc_coif1_taps.argtypes = [_f64p, _f64p]
    L.orc_mallat_decode.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_int), _i64p, _i64p]
    L.orc_select_f32.restype = C.c_int64
    L.orc_select_f32.argtypes = [_f32p, C.c_int, C.c_double, C.c_double, _i32p]
    L.orc_select_f64.restype = C.c_int64
    L.orc_select_f64.argtypes = [_f64p, C.c_int, C.c_double, C.c_double, _i32p]
    for nm, t in (("orc_build_lut_f32", _f32p), ("orc_build_lut_f64", _f64p)):
        f = getattr(L, nm)
        f.restype = C.c_int
        f.argtypes = [C.c_double, C.c_double, _f64p, C.c_int, C.c_int, C.c_int,
                      C.c_double, _i64p, C.c_int64, _i32p, t, C.c_int]
    L.orc_build_lut_f32.argtypes = L.orc_build_lut_f32.argtypes + [C.c_int]
    L.orc_build_lut_f64.argtypes = L.orc_build_lut_f64.argtypes + [C.c_int, C.c_int]
    for nm, t in (("orc_superpose_f32", _f32p), ("orc_superpose_f64", _f64p)):
        f = getattr(L, nm)
        f.restype = C.c_int
        f.argtypes = [C.c_int, C.c_int, C.c_int, _i64p, _i32p, t, _i32p, _i32p,
                      _f32p, _u32p, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                      C.c_int, t]
    for nm, t in (("orc_subhologram_f32", _f32p), ("orc_subhologram_f64", _f64p)):
        f = getattr(L, nm)
        f.restype = C.c_int
        f.argtypes = [C.c_int, C.c_int, C.c_int, _i64p, _i32p, t, _i32p, _i32p,
                      _f32p, _u32p, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                      C.c_int, t, C.c_int]
    L.orc_binarize_f32.argtypes = [_f32p, C.c_int64, C.c_int64, _u8p]
    L.orc_reference_wave.argtypes = [C.c_double] * 5 + [C.c_int64] * 4 + [_f64p]
    L.orc_binarize_ref_f64.argtypes = ([_f64p, C.c_int64, C.c_int64] + [C.c_double] * 5 +
                                       [C.c_int64, C.c_int64, _u8p, _f64p])
    L.orc_cgh_direct_f64.argtypes = [C.c_double, C.c_double, _i32p, _i32p, _f32p,
                                     _f64p, C.c_int64, C.c_int64, C.c_int64,
                                     C.c_int64, C.c_int64, C.c_int, _f64p, C.c_int]
    L.orc_have_openmp.restype = C.c_int
    _lib = L
    return L


# ------------------------------------------------------------------ geometry

def support_radius(lam: float, pitch: float, z) -> np.ndarray | float:
    """Reading R1: PSF support radius in pixels at depth z."""
    f = lib().orc_support_radius
    if np.isscalar(z):
        return f(lam, pitch, float(z))
    return np.array([f(lam, pitch, float(v)) for v in np.asarray(z).ravel()])


def keep_target(gamma: float, R: float) -> int:
    """Reading R3: coefficient budget ceil(gamma * pi * R^2 - 1e-9); R11: no
    limit (every nonzero kept) when R <= 1, the single-pixel support."""
    return int(lib().orc_keep_target(gamma, R))


def depth_grid(zmin: float, zmax: float, D: int) -> np.ndarray:
    """Reading R2: the D bin-centre depths."""
    zd = np.empty(D, np.float64)
    lib().orc_depth_grid(zmin, zmax, D, _p(zd, _f64p))
    return zd


def quantize(z: np.ndarray, zmin: float, zmax: float, D: int) -> tuple[np.ndarray, int]:
    """Reading R2: depth index per point and the count of out-of-range points."""
    z = np.ascontiguousarray(z, np.float64)
    d = np.empty(z.size, np.uint32)
    bad = lib().orc_quantize(_p(z, _f64p), z.size, zmin, zmax, D, _p(d, _u32p))
    return d, int(bad)


# --------------------------------------------------------------------- phase

def sincos2pi_f32(g: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    g = np.ascontiguousarray(g, np.float32)
    c = np.empty_like(g)
    s = np.empty_like(g)
    lib().orc_sincos2pi_f32(_p(g, _f32p), g.size, _p(c, _f32p), _p(s, _f32p))
    return c, s


def psf_f32(lam: float, pitch: float, z: float, W: int) -> np.ndarray:
    out = np.empty((W, W), np.complex64)
    lib().orc_psf_f32(lam, pitch, z, W, _p(out, _f32p))
    return out


def psf_f64(lam: float, pitch: float, z: float, W: int) -> np.ndarray:
    out = np.empty((W, W), np.complex128)
    lib().orc_psf_f64(lam, pitch, z, W, _p(out, _f64p))
    return out


# ---------------------------------------------------------------------- Haar

def haar_fwd(a: np.ndarray, L: int) -> np.ndarray:
    """L-level orthonormal 2-D Haar of a square complex array (Mallat layout)."""
    out = np.array(a, copy=True, order="C")
    n = out.shape[0]
    assert out.shape == (n, n)
    if out.dtype == np.complex64:
        lib().orc_haar_fwd_f32(_p(out, _f32p), n, L)
    else:
        out = out.astype(np.complex128)
        lib().orc_haar_fwd_f64(_p(out, _f64p), n, L)
    return out


def haar_inv(a: np.ndarray, L: int) -> np.ndarray:
    out = np.array(a, copy=True, order="C")
    n = out.shape[0]
    assert out.shape == (n, n)
    if out.dtype == np.complex64:
        lib().orc_haar_inv_f32(_p(out, _f32p), n, L)
    else:
        out = out.astype(np.complex128)
        lib().orc_haar_inv_f64(_p(out, _f64p), n, L)
    return out


WAVELETS = {"haar": 0, "coif1": 1}


def coif1_taps() -> tuple[np.ndarray, np.ndarray]:
    """Reading R14: the order-1 coiflet scaling filter h_k and wavelet
    filter g_k = (-1)^k h_{1-k}, k = -2 .. 3 (FP64)."""
    lo, hi = np.empty(6), np.empty(6)
    lib().orc_coif1_taps(_p(lo, _f64p), _p(hi, _f64p))
    return lo, hi


def _wavelet_call(a: np.ndarray, L: int, wavelet: str, fwd: bool) -> np.ndarray:
    out = np.array(a, copy=True, order="C")
    n = out.shape[0]
    assert out.shape == (n, n)
    w = WAVELETS[wavelet]
    if out.dtype == np.complex64:
        fn = lib().orc_wavelet_fwd_f32 if fwd else lib().orc_wavelet_inv_f32
        fn(_p(out, _f32p), n, L, w)
    else:
        out = out.astype(np.complex128)
        fn = lib().orc_wavelet_fwd_f64 if fwd else lib().orc_wavelet_inv_f64
        fn(_p(out, _f64p), n, L, w)
    return out


def wavelet_fwd(a: np.ndarray, L: int, wavelet: str = "haar") -> np.ndarray:
    """L-level forward transform (Mallat layout): Haar (R4) or the periodic
    order-1 coiflet (R14)."""
    return _wavelet_call(a, L, wavelet, True)


def wavelet_inv(a: np.ndarray, L: int, wavelet: str = "haar") -> np.ndarray:
    return _wavelet_call(a, L, wavelet, False)


def mallat_decode(row: int, col: int, n: int, L: int) -> tuple[int, int, int, int]:
    lev, band = C.c_int(), C.c_int()
    p, q = C.c_int64(), C.c_int64()
    lib().orc_mallat_decode(row, col, n, L, C.byref(lev), C.byref(band),
                            C.byref(p), C.byref(q))
    return lev.value, band.value, p.value, q.value


def select(coef: np.ndarray, gamma: float, R: float) -> np.ndarray:
    """Reading R5: kept Mallat linear indices (ascending)."""
    W = coef.shape[0]
    out = np.empty(W * W, np.int32)
    if coef.dtype == np.complex64:
        c = np.ascontiguousarray(coef)
        k = lib().orc_select_f32(_p(c, _f32p), W, gamma, R, _p(out, _i32p))
    else:
        c = np.ascontiguousarray(coef, np.complex128)
        k = lib().orc_select_f64(_p(c, _f64p), W, gamma, R, _p(out, _i32p))
    return out[:k].copy()


# ----------------------------------------------------------------------- LUT

@dataclass
class Lut:
    lam: float
    pitch: float
    depths: np.ndarray      # (D,) float64, metres
    W: int
    L: int
    gamma: float
    nr: np.ndarray          # (D,) int64
    idx: np.ndarray         # (sum nr,) int32, Mallat linear index, ascending per depth
    val: np.ndarray         # (sum nr,) complex64 or complex128
    wavelet: str = "haar"

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.nr)]).astype(np.int64)

    def depth(self, d: int) -> tuple[np.ndarray, np.ndarray]:
        o = self.offsets
        return self.idx[o[d]:o[d + 1]], self.val[o[d]:o[d + 1]]


def build_lut(lam, pitch, depths, W, L, gamma, dtype="f32", threads=1,
              select_fp32=False, wavelet="haar") -> Lut:
    """Sec. 1, step 1 at every depth, with the Haar (R4) or the order-1
    coiflet (R14) transform.  dtype 'f32' uses the FP32 PSF form
    (reading R8) that decides the selection; 'f64' is the FP64 definition.
    With select_fp32 (f64 only) the kept index set is the one the FP32 form
    selects and the values are FP64: the reference for precision errors,
    since which coefficients are kept is an integer decision taken in the
    GPU kernel's precision."""
    depths = np.ascontiguousarray(depths, np.float64)
    D = depths.size
    if gamma >= 1.0:
        cap = D * W * W
    else:
        cap = sum(min(keep_target(gamma, support_radius(lam, pitch, z)), W * W) for z in depths)
    nr = np.zeros(D, np.int64)
    idx = np.empty(max(cap, 1), np.int32)
    if dtype == "f32":
        val = np.empty(max(cap, 1), np.complex64)
        rc = lib().orc_build_lut_f32(lam, pitch, _p(depths, _f64p), D, W, L, gamma,
                                     _p(nr, _i64p), cap, _p(idx, _i32p),
                                     _p(val, _f32p), threads, WAVELETS[wavelet])
    else:
        val = np.empty(max(cap, 1), np.complex128)
        rc = lib().orc_build_lut_f64(lam, pitch, _p(depths, _f64p), D, W, L, gamma,
                                     _p(nr, _i64p), cap, _p(idx, _i32p),
                                     _p(val, _f64p), threads, int(select_fp32), WAVELETS[wavelet])
    if rc != 0:
        raise ValueError("oracle build_lut rejected its arguments (window too "
                         "small for a PSF, or capacity)")
    tot = int(nr.sum())
    return Lut(lam, pitch, depths, W, L, gamma, nr, idx[:tot].copy(), val[:tot].copy(), wavelet)


# ---------------------------------------------------------- superposition

def _pts(points):
    x = np.ascontiguousarray(points["x"], np.int32)
    y = np.ascontiguousarray(points["y"], np.int32)
    a = np.ascontiguousarray(points["a"], np.float32)
    d = np.ascontiguousarray(points["d"], np.uint32)
    return x, y, a, d


def superpose(lut: Lut, points, Nh: int, ox: int = 0, oy: int = 0, rule: int = 0,
              psi: np.ndarray | None = None) -> np.ndarray:
    """Eq. (2): returns the Nh x Nh Mallat-layout wavelet buffer psi."""
    x, y, a, d = _pts(points)
    f64 = lut.val.dtype == np.complex128
    if psi is None:
        psi = np.zeros((Nh, Nh), np.complex128 if f64 else np.complex64)
    fn = lib().orc_superpose_f64 if f64 else lib().orc_superpose_f32
    t = _f64p if f64 else _f32p
    rc = fn(lut.W, lut.L, lut.nr.size, _p(lut.nr, _i64p), _p(lut.idx, _i32p),
            _p(lut.val, t), _p(x, _i32p), _p(y, _i32p), _p(a, _f32p), _p(d, _u32p),
            x.size, Nh, ox, oy, rule, _p(psi, t))
    if rc != 0:
        raise ValueError("oracle superpose: a point's depth index is out of range")
    return psi


def subhologram(lut: Lut, points, Ns: int, s: int, t: int, rule: int = 0) -> np.ndarray:
    """Sec. 1, large-scale steps 2-4 for sub-hologram (s, t) of side Ns."""
    x, y, a, d = _pts(points)
    f64 = lut.val.dtype == np.complex128
    u = np.empty((Ns, Ns), np.complex128 if f64 else np.complex64)
    fn = lib().orc_subhologram_f64 if f64 else lib().orc_subhologram_f32
    tp = _f64p if f64 else _f32p
    rc = fn(lut.W, lut.L, lut.nr.size, _p(lut.nr, _i64p), _p(lut.idx, _i32p),
            _p(lut.val, tp), _p(x, _i32p), _p(y, _i32p), _p(a, _f32p), _p(d, _u32p),
            x.size, Ns, s, t, rule, _p(u, tp), WAVELETS[lut.wavelet])
    if rc != 0:
        raise ValueError("oracle subhologram: a point's depth index is out of range")
    return u


def hologram(lut: Lut, points, Nh: int, rule: int = 0) -> np.ndarray:
    """The whole Nh x Nh hologram (one sub-hologram covering everything)."""
    return subhologram(lut, points, Nh, 0, 0, rule)


def binarize(u: np.ndarray) -> np.ndarray:
    """Reading R7: packed bits, row-major, LSB = lowest x."""
    h, w = u.shape
    uf = np.ascontiguousarray(u, np.complex64)
    bits = np.empty((w * h + 7) // 8, np.uint8)
    lib().orc_binarize_f32(_p(uf, _f32p), w, h, _p(bits, _u8p))
    return bits


def reference_wave(lam: float, pitch: float, xr: float, yr: float, zr: float, w: int, h: int,
                   ox: int = 0, oy: int = 0) -> np.ndarray:
    """Reading R12 (Sec. 2): the spherical reference wave over the region
    [ox, ox+w) x [oy, oy+h) of the plane (h x w complex128)."""
    R = np.empty((h, w), np.complex128)
    lib().orc_reference_wave(lam, pitch, xr, yr, zr, ox, oy, w, h, _p(R, _f64p))
    return R


def binarize_ref(u: np.ndarray, lam: float, pitch: float, xr: float, yr: float, zr: float,
                 ox: int = 0, oy: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Reading R12: packed bits of Re(u conj R) > 0 and the values
    Re(u conj R) (h x w float64) for the field u of the region at (ox, oy)."""
    h, w = u.shape
    uf = np.ascontiguousarray(u, np.complex128)
    bits = np.empty((w * h + 7) // 8, np.uint8)
    val = np.empty((h, w), np.float64)
    lib().orc_binarize_ref_f64(_p(uf, _f64p), w, h, lam, pitch, xr, yr, zr, ox, oy, _p(bits, _u8p),
                               _p(val, _f64p))
    return bits, val


def reconstruct(u0: np.ndarray, lam: float, pitch: float, d: float) -> np.ndarray:
    """Reading R13: the field in the plane at signed distance d from the
    field u0 (h x w) by the angular spectrum method, FP64:
    U_d = IFFT2(FFT2(u0) H), H = exp(i 2 pi d sqrt(1/lam^2 - fx^2 - fy^2))
    where fx^2 + fy^2 < 1/lam^2, 0 elsewhere; fx, fy the FFT frequencies of
    the pitch grid.  A point at depth z (Eq. (1), +i sign) focuses at d = -z."""
    h, w = u0.shape
    fx = np.fft.fftfreq(w, d=pitch)[None, :]
    fy = np.fft.fftfreq(h, d=pitch)[:, None]
    s = 1.0 / lam ** 2 - fx ** 2 - fy ** 2
    prop = s > 0
    H = np.where(prop, np.exp(2j * np.pi * d * np.sqrt(np.where(prop, s, 0.0))), 0.0)
    return np.fft.ifft2(np.fft.fft2(np.asarray(u0, np.complex128)) * H)


def transmittance(bits: np.ndarray, w: int, h: int) -> np.ndarray:
    """A packed binary hologram (R7 bit order) as amplitudes 0 / 1 (h x w)."""
    return np.unpackbits(np.asarray(bits, np.uint8), bitorder="little")[: w * h].reshape(h, w).astype(np.float64)


def cgh_direct(lam: float, pitch: float, x, y, a, z, ox: int, oy: int, w: int, h: int,
               aperture: bool = True, threads: int = 1) -> np.ndarray:
    """Eq. (1) in FP64 over the region [ox, ox+w) x [oy, oy+h); z per point."""
    x = np.ascontiguousarray(x, np.int32)
    y = np.ascontiguousarray(y, np.int32)
    a = np.ascontiguousarray(a, np.float32)
    z = np.ascontiguousarray(z, np.float64)
    u = np.empty((h, w), np.complex128)
    lib().orc_cgh_direct_f64(lam, pitch, _p(x, _i32p), _p(y, _i32p), _p(a, _f32p),
                             _p(z, _f64p), x.size, ox, oy, w, h, int(aperture),
                             _p(u, _f64p), threads)
    return u


def have_openmp() -> bool:
    return bool(lib().orc_have_openmp())
