"""Tensor-level wrappers of the libwasabi entry points (marshalling only)."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import check

_DTYPES = {"f32": _abi.F32, "f16s": _abi.F16S, "bf16s": _abi.BF16S}


def _lib():
    return _abi.load()


def _stream(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _keep(stream, *tensors) -> None:
    """Tensors allocated on the current stream that a call used on another
    stream: the caching allocator is told, so their memory is not handed out
    again before that stream's work on them is done."""
    if stream is None or stream == torch.cuda.current_stream():
        return
    for t in tensors:
        if t is not None and t.is_cuda:
            t.record_stream(stream)


def _ptr(t: torch.Tensor | None) -> C.c_void_p | None:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def depth_grid(zmin: float, zmax: float, n_depths: int) -> np.ndarray:
    out = np.empty(n_depths, np.float64)
    check(_lib().wasabi_depth_grid(zmin, zmax, n_depths,
                                   out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


class Lut:
    """A device-resident WASABI look-up table (library-owned)."""

    def __init__(self, handle: C.c_void_p, lam, pitch, depths, window, levels, keep_ratio,
                 dtype, stream):
        self._h = handle
        self.lam, self.pitch = lam, pitch
        self.depths = np.asarray(depths, np.float64)
        self.window, self.levels, self.keep_ratio, self.dtype = window, levels, keep_ratio, dtype
        self.wavelet = "haar"
        self._stream = stream

    @property
    def handle(self) -> C.c_void_p:
        if self._h is None:
            raise ValueError("LUT already destroyed")
        return self._h

    @property
    def n_depths(self) -> int:
        return int(self.depths.size)

    def counts(self) -> np.ndarray:
        out = np.empty(self.n_depths, np.int64)
        check(_lib().wasabi_lut_counts(self.handle, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out

    def selection(self, depth: int) -> np.ndarray:
        n = C.c_int64(self.window * self.window)
        out = np.empty(n.value, np.int32)
        check(_lib().wasabi_lut_selection(self.handle, depth,
                                          out.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n)))
        return out[:n.value].copy()

    def entries(self, depth: int) -> tuple[np.ndarray, np.ndarray]:
        n = C.c_int64(self.window * self.window)
        idx = np.empty(n.value, np.int32)
        val = np.empty(n.value, np.complex64)
        check(_lib().wasabi_lut_entries(self.handle, depth,
                                        idx.ctypes.data_as(C.POINTER(C.c_int32)),
                                        val.ctypes.data_as(C.POINTER(C.c_float)), C.byref(n)))
        return idx[:n.value].copy(), val[:n.value].copy()

    def close(self) -> None:
        if self._h is not None:
            _lib().wasabi_lut_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_lut(lam: float, pitch: float, depths, window: int, levels: int, keep_ratio: float,
              dtype: str = "f32", stream=None, wavelet: str = "haar") -> Lut:
    """The per-depth LUT (wasabi_build_lut_wavelet); wavelet "haar" or
    "coif1" (the order-1 coiflet)."""
    d = np.ascontiguousarray(depths, np.float64)
    h = C.c_void_p()
    check(_lib().wasabi_build_lut_wavelet(lam, pitch, d.ctypes.data_as(C.POINTER(C.c_double)), d.size,
                                          window, levels, keep_ratio, _DTYPES[dtype], _abi.WAVELETS[wavelet],
                                          _stream(stream), C.byref(h)))
    lut = Lut(h, lam, pitch, d, window, levels, keep_ratio, dtype, stream)
    lut.wavelet = wavelet
    return lut


def pack_points(x, y, a, d, device="cuda") -> torch.Tensor:
    """Lay out (x, y, a, d) as the ABI's 16-byte point records, shape (N, 4) int32."""
    x = np.ascontiguousarray(x, np.int32)
    rec = np.empty((x.size, 4), np.int32)
    rec[:, 0] = x
    rec[:, 1] = np.ascontiguousarray(y, np.int32)
    rec[:, 2] = np.ascontiguousarray(a, np.float32).view(np.int32)
    rec[:, 3] = np.ascontiguousarray(d, np.uint32).view(np.int32)
    return torch.from_numpy(rec).to(device)


def quantize_points(x: torch.Tensor, y: torch.Tensor, z: torch.Tensor, a: torch.Tensor,
                    zmin: float, zmax: float, n_depths: int, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    n = x.numel()
    if out is None:
        out = torch.empty((n, 4), dtype=torch.int32, device=x.device)
    check(_lib().wasabi_quantize_points(_ptr(x), _ptr(y), _ptr(z), _ptr(a), n, zmin, zmax,
                                        n_depths, _ptr(out), _stream(stream)))
    _keep(stream, out)
    return out


def scratch_bytes(lut: Lut, n: int, w: int, h: int) -> int:
    out = C.c_size_t()
    check(_lib().wasabi_scratch_bytes(lut.handle, n, w, h, C.byref(out)))
    return int(out.value)


def superpose(lut: Lut, points: torch.Tensor, w: int, h: int, rule: int = 0,
              wbuf: torch.Tensor | None = None, scratch: torch.Tensor | None = None,
              stream=None, origin=(0, 0)) -> torch.Tensor:
    """Eq. (2): the tile-major wavelet buffer (h*w complex64); origin: plane
    pixel of the buffer's pixel (0, 0) (a sub-hologram, through
    wasabi_hologram_frame with the wavelet buffer as the only output)."""
    n = points.shape[0]
    dev = points.device
    if wbuf is None:
        wbuf = torch.empty(h * w, dtype=torch.complex64, device=dev)
    need = scratch_bytes(lut, n, w, h)
    if scratch is None:
        scratch = torch.empty(need, dtype=torch.uint8, device=dev)
    pts = _ptr(points) if n else C.c_void_p(None)
    if tuple(origin) == (0, 0):
        check(_lib().wasabi_superpose(lut.handle, pts, n, w, h, rule, _ptr(wbuf), _ptr(scratch),
                                      scratch.numel(), _stream(stream)))
    else:
        frame = make_frame(origin, None)
        check(_lib().wasabi_hologram_frame(lut.handle, pts, n, w, h, rule, C.byref(frame), _ptr(wbuf),
                                           None, None, _ptr(scratch), scratch.numel(), _stream(stream)))
    _keep(stream, wbuf, scratch)
    return wbuf


def superpose_static(lut: Lut, points: torch.Tensor, w: int, h: int, rule: int = 0,
                     wbuf: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Eq. (2) through wasabi_superpose_static: no scratch argument; the
    library's fixed device array is used, nothing is allocated by the call
    (the output buffer is allocated here only when not given)."""
    n = points.shape[0]
    if wbuf is None:
        wbuf = torch.empty(h * w, dtype=torch.complex64, device=points.device)
    check(_lib().wasabi_superpose_static(lut.handle, _ptr(points) if n else C.c_void_p(None), n, w,
                                         h, rule, _ptr(wbuf), _stream(stream)))
    _keep(stream, wbuf)
    return wbuf


def inverse_wavelet(wbuf: torch.Tensor, w: int, h: int, levels: int, wavelet: str = "coif1",
                    want: str = "complex", u: torch.Tensor | None = None, bits: torch.Tensor | None = None,
                    origin=(0, 0), reference: dict | None = None, stream=None):
    """Inverse transformation of a tile-major wavelet buffer for either
    wavelet (wasabi_inverse_wavelet): want = "complex" | "bits" | "both"."""
    dev = wbuf.device
    if want in ("complex", "both") and u is None:
        u = torch.empty((h, w), dtype=torch.complex64, device=dev)
    if want in ("bits", "both") and bits is None:
        bits = torch.empty((h * w + 7) // 8, dtype=torch.uint8, device=dev)
    need = C.c_size_t()
    check(_lib().wasabi_inverse_wavelet_scratch_bytes(w, h, C.byref(need)))
    scratch = torch.empty(int(need.value), dtype=torch.uint8, device=dev)
    frame = make_frame(origin, reference)
    check(_lib().wasabi_inverse_wavelet(_ptr(wbuf), w, h, levels, _abi.WAVELETS[wavelet], C.byref(frame), _ptr(u),
                                        _ptr(bits), _ptr(scratch), scratch.numel(), _stream(stream)))
    _keep(stream, u, bits, scratch)
    if want == "complex":
        return u
    if want == "bits":
        return bits
    return u, bits


def spherical_reference(lam: float, pitch: float, x: float, y: float, z: float) -> dict:
    """Reference wave of a unit point source at plane pixel coordinates
    (x, y) and signed distance z (metres) from the plane (Sec. 2)."""
    return {"lam": float(lam), "pitch": float(pitch), "x": float(x), "y": float(y), "z": float(z)}


def make_frame(origin=(0, 0), reference: dict | None = None) -> _abi.Frame:
    """wasabi_frame: sub-hologram origin (plane pixel of output pixel
    (0, 0)) and reference wave (None = unit plane wave)."""
    f = _abi.Frame()
    f.origin_x, f.origin_y = int(origin[0]), int(origin[1])
    if reference is not None:
        f.ref.kind = _abi.REF_SPHERICAL
        f.ref.lam, f.ref.pitch = reference["lam"], reference["pitch"]
        f.ref.x, f.ref.y, f.ref.z = reference["x"], reference["y"], reference["z"]
    return f


def inverse_haar(wbuf: torch.Tensor, w: int, h: int, levels: int, u: torch.Tensor | None = None,
                 bits: torch.Tensor | None = None, want: str = "complex", stream=None,
                 origin=(0, 0), reference: dict | None = None):
    """Inverse transform and binarisation (wasabi_inverse_haar_frame); the
    bits use `reference` (None = unit plane wave) at plane pixels offset by
    `origin`."""
    dev = wbuf.device
    if want in ("complex", "both") and u is None:
        u = torch.empty((h, w), dtype=torch.complex64, device=dev)
    if want in ("bits", "both") and bits is None:
        bits = torch.empty((h * w + 7) // 8, dtype=torch.uint8, device=dev)
    frame = make_frame(origin, reference)
    check(_lib().wasabi_inverse_haar_frame(_ptr(wbuf), w, h, levels, C.byref(frame), _ptr(u), _ptr(bits),
                                           _stream(stream)))
    _keep(stream, u, bits)
    if want == "complex":
        return u
    if want == "bits":
        return bits
    return u, bits


def hologram(lut: Lut, points: torch.Tensor, w: int, h: int, want: str = "complex", rule: int = 0,
             u: torch.Tensor | None = None, bits: torch.Tensor | None = None,
             wbuf: torch.Tensor | None = None, scratch: torch.Tensor | None = None, stream=None,
             origin=(0, 0), reference: dict | None = None):
    """Eq. (2) fused with the inverse transform and binarisation
    (wasabi_hologram / wasabi_hologram_frame): want = "complex" | "bits" |
    "both".  A given wbuf also receives the tile-major wavelet buffer.
    origin: plane pixel of the output's pixel (0, 0) (a sub-hologram);
    reference: spherical_reference(...) for the bits, None = unit plane wave."""
    n = points.shape[0]
    dev = points.device
    if want in ("complex", "both") and u is None:
        u = torch.empty((h, w), dtype=torch.complex64, device=dev)
    if want in ("bits", "both") and bits is None:
        bits = torch.empty((h * w + 7) // 8, dtype=torch.uint8, device=dev)
    if scratch is None:
        scratch = torch.empty(scratch_bytes(lut, n, w, h), dtype=torch.uint8, device=dev)
    if tuple(origin) == (0, 0) and reference is None:
        check(_lib().wasabi_hologram(lut.handle, _ptr(points) if n else C.c_void_p(None), n, w, h, rule,
                                     _ptr(wbuf), _ptr(u), _ptr(bits), _ptr(scratch), scratch.numel(),
                                     _stream(stream)))
    else:
        frame = make_frame(origin, reference)
        check(_lib().wasabi_hologram_frame(lut.handle, _ptr(points) if n else C.c_void_p(None), n, w, h, rule,
                                           C.byref(frame), _ptr(wbuf), _ptr(u), _ptr(bits), _ptr(scratch),
                                           scratch.numel(), _stream(stream)))
    _keep(stream, u, bits, wbuf, scratch)
    if want == "complex":
        return u
    if want == "bits":
        return bits
    return u, bits


def hologram_stream(lut: Lut, points: torch.Tensor, w: int, h: int, band_h: int, want: str = "bits",
                    rule: int = 0, origin=(0, 0), reference: dict | None = None,
                    bits: torch.Tensor | None = None, u: torch.Tensor | None = None, stream=None):
    """Sub-hologram streaming (wasabi_hologram_stream): the w x h hologram
    computed in bands of band_h rows, each copied to host memory while the
    next is computed.  Outputs are host tensors (pinned when allocated here);
    want = "bits" | "complex" | "both"."""
    n = points.shape[0]
    if want in ("bits", "both") and bits is None:
        bits = torch.empty((h * w + 7) // 8, dtype=torch.uint8, pin_memory=True)
    if want in ("complex", "both") and u is None:
        u = torch.empty((h, w), dtype=torch.complex64, pin_memory=True)
    for t in (bits, u):
        if t is not None and (t.is_cuda or not t.is_contiguous()):
            raise ValueError("hologram_stream: outputs are contiguous host tensors")
    frame = make_frame(origin, reference)
    host = [C.c_void_p(t.data_ptr()) if t is not None else None for t in (bits, u)]
    check(_lib().wasabi_hologram_stream(lut.handle, _ptr(points) if n else C.c_void_p(None), n, w, h, band_h,
                                        rule, C.byref(frame), host[0], host[1], _stream(stream)))
    if want == "complex":
        return u
    if want == "bits":
        return bits
    return u, bits


def reconstruct(hologram: torch.Tensor, w: int, h: int, lam: float, pitch: float, d: float,
                want: str = "intensity", origin=(0, 0), reference: dict | None = None,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Numerical reconstruction (wasabi_reconstruct): the field (want =
    "complex") or intensity (want = "intensity") in the plane at signed
    distance d, by the angular spectrum method.  hologram: an (h, w) complex64
    field, or packed bits (uint8) illuminated by `reference` (None: R = 1).
    Asynchronous on `stream`, like the other calls."""
    kind = _abi.RECON_BITS if hologram.dtype == torch.uint8 else _abi.RECON_FIELD
    dev = hologram.device
    if out is None:
        out = torch.empty((h, w), dtype=torch.complex64 if want == "complex" else torch.float32, device=dev)
    need = C.c_size_t()
    check(_lib().wasabi_reconstruct_scratch_bytes(w, h, C.byref(need)))
    scratch = torch.empty(int(need.value), dtype=torch.uint8, device=dev)
    frame = make_frame(origin, reference)
    field, inten = (out, None) if want == "complex" else (None, out)
    check(_lib().wasabi_reconstruct(_ptr(hologram), kind, w, h, lam, pitch, d, C.byref(frame), _ptr(field),
                                    _ptr(inten), _ptr(scratch), scratch.numel(), _stream(stream)))
    _keep(stream, out, scratch)
    return out


def cgh_direct_scratch_bytes(n: int, w: int, h: int) -> int:
    out = C.c_size_t()
    check(_lib().cgh_direct_scratch_bytes(n, w, h, C.byref(out)))
    return int(out.value)


def cgh_direct(lam: float, pitch: float, depths, points: torch.Tensor, w: int, h: int,
               aperture: bool = True, u: torch.Tensor | None = None,
               scratch: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Eq. (1) on the GPU (h x w complex64)."""
    d = np.ascontiguousarray(depths, np.float64)
    n = points.shape[0]
    dev = points.device
    if u is None:
        u = torch.empty((h, w), dtype=torch.complex64, device=dev)
    if scratch is None:
        scratch = torch.empty(cgh_direct_scratch_bytes(n, w, h), dtype=torch.uint8, device=dev)
    check(_lib().cgh_direct(lam, pitch, d.ctypes.data_as(C.POINTER(C.c_double)), d.size,
                            _ptr(points) if n else C.c_void_p(None), n, w, h, int(aperture),
                            _ptr(u), _ptr(scratch), scratch.numel(), _stream(stream)))
    _keep(stream, u, scratch)
    return u


class Batch:
    """Many holograms through one launch sequence (wasabi_batch_*).

    A job is a dict: points (N x 4 int32 CUDA tensor), w, h, and optionally
    rule, want ("none" | "complex" | "bits" | "both"), wbuf (a tensor, or
    keep_wbuf=True to have one allocated; always for want "none"), origin and
    reference (as for hologram()); run() allocates missing buffers, returns
    the jobs with their wbuf / u / bits tensors and keeps the scratch alive
    until the next run."""

    def __init__(self, lut: Lut, max_jobs: int, side_hint: int = 4096, use_graph: bool = True):
        self.lut = lut
        self.max_jobs = max_jobs
        h = C.c_void_p()
        check(_lib().wasabi_batch_create(lut.handle, max_jobs, side_hint, int(use_graph), C.byref(h)))
        self._h = h
        self._held = None  # the last run's scratch and outputs

    def config(self) -> tuple[int, int]:
        c, t = C.c_int(), C.c_int()
        check(_lib().wasabi_batch_config(self._h, C.byref(c), C.byref(t)))
        return c.value, t.value

    def run(self, jobs: list[dict], stream=None) -> list[dict]:
        n = len(jobs)
        arr = (_abi.Job * max(n, 1))()
        out = []
        for i, j in enumerate(jobs):
            pts = j["points"]
            dev = pts.device
            w, h = j["w"], j["h"]
            want = j.get("want", "bits")
            wbuf = j.get("wbuf")
            if wbuf is None and (want == "none" or j.get("keep_wbuf", False)):
                wbuf = torch.empty(h * w, dtype=torch.complex64, device=dev)
            u = j.get("u")
            if u is None and want in ("complex", "both"):
                u = torch.empty((h, w), dtype=torch.complex64, device=dev)
            bits = j.get("bits")
            if bits is None and want in ("bits", "both"):
                bits = torch.empty((h * w + 7) // 8, dtype=torch.uint8, device=dev)
            arr[i] = _abi.Job(pts.data_ptr() if pts.shape[0] else None, pts.shape[0], w, h,
                              j.get("rule", 0), wbuf.data_ptr() if wbuf is not None else None,
                              u.data_ptr() if u is not None else None,
                              bits.data_ptr() if bits is not None else None,
                              make_frame(j.get("origin", (0, 0)), j.get("reference")))
            out.append(dict(j, wbuf=wbuf, u=u, bits=bits))
        need = C.c_size_t()
        check(_lib().wasabi_batch_scratch_bytes(self._h, C.cast(arr, C.c_void_p), n, C.byref(need)))
        dev = jobs[0]["points"].device if jobs else torch.device("cuda")
        scratch = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device=dev)
        check(_lib().wasabi_batch_run(self._h, C.cast(arr, C.c_void_p), n, _ptr(scratch),
                                      scratch.numel(), _stream(stream)))
        _keep(stream, scratch, *[o[k] for o in out for k in ("wbuf", "u", "bits")])
        self._held = (scratch, out)
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            _lib().wasabi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop (wasabi_server_*): requests admitted by a device-memory
    budget and continuously batched over `streams` CUDA streams by a native
    scheduler thread.  submit() takes host tensors (pinned for asynchronous
    copies) and returns at once; wait() returns the request's timings with its
    host outputs filled in."""

    def __init__(self, lut: Lut, budget_bytes: int, streams: int = 2, max_batch: int = 64,
                 side_hint: int = 4096):
        self.lut = lut
        h = C.c_void_p()
        check(_lib().wasabi_server_create(lut.handle, int(budget_bytes), streams, max_batch, side_hint,
                                          C.byref(h)))
        self._h = h
        self._live = {}

    def submit(self, points: torch.Tensor, w: int, h: int, want: str = "bits", rule: int = 0,
               origin=(0, 0), reference: dict | None = None, bits: torch.Tensor | None = None,
               u: torch.Tensor | None = None) -> int:
        """Queue a request; its outputs go to `bits` / `u` (host tensors, pinned
        for asynchronous copies), allocated here when not given."""
        if points.is_cuda or not points.is_contiguous() or points.dtype != torch.int32:
            raise ValueError("points: contiguous (N, 4) int32 host tensor")
        pin = points.is_pinned()
        if bits is None and want in ("bits", "both"):
            bits = torch.empty((h * w + 7) // 8, dtype=torch.uint8, pin_memory=pin)
        if u is None and want in ("complex", "both"):
            u = torch.empty((h, w), dtype=torch.complex64, pin_memory=pin)
        for t in (bits, u):
            if t is not None and (t.is_cuda or not t.is_contiguous()):
                raise ValueError("outputs: contiguous host tensors")
        req = _abi.Request(points.data_ptr() if points.shape[0] else None, points.shape[0], w, h, rule,
                           bits.data_ptr() if bits is not None else None,
                           u.data_ptr() if u is not None else None, make_frame(origin, reference))
        rid = C.c_int64()
        check(_lib().wasabi_server_submit(self._h, C.byref(req), C.byref(rid)))
        self._live[rid.value] = (points, bits, u)
        return rid.value

    def wait(self, rid: int, timeout: float = 0.0) -> dict:
        info = _abi.RequestInfo()
        code = _lib().wasabi_server_wait(self._h, rid, timeout, C.byref(info))
        if code == _abi.E_TIMEOUT:
            check(code)
        _, bits, u = self._live.pop(rid)
        check(code)
        return {"submit_s": info.submit_s, "launch_s": info.launch_s, "done_s": info.done_s,
                "latency_s": info.done_s - info.submit_s, "batch_jobs": info.batch_jobs,
                "bits": bits, "u": u}

    def stats(self) -> dict:
        peak, done, nl = C.c_size_t(), C.c_int64(), C.c_int64()
        check(_lib().wasabi_server_stats(self._h, C.byref(peak), C.byref(done), C.byref(nl)))
        return {"peak_bytes": int(peak.value), "completed": int(done.value), "launches": int(nl.value)}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            _lib().wasabi_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(lut: Lut, side: int, n_points: int, stream=None) -> tuple[int, int]:
    """Pick and store the fastest super-tile / block size for this size class."""
    c, t = C.c_int(), C.c_int()
    check(_lib().wasabi_autotune(lut.handle, side, n_points, _stream(stream), C.byref(c), C.byref(t)))
    return c.value, t.value


def sync_status(stream=None) -> None:
    """Wait for the stream and raise if a kernel recorded an error."""
    check(_lib().wasabi_sync_status(_stream(stream)))


def haar_forward(u: torch.Tensor, levels: int, stream=None) -> torch.Tensor:
    h, w = u.shape
    wbuf = torch.empty(h * w, dtype=torch.complex64, device=u.device)
    check(_lib().wasabi_haar_forward(_ptr(u), w, h, levels, _ptr(wbuf), _stream(stream)))
    _keep(stream, wbuf)
    return wbuf


def wbuf_to_mallat(wbuf: torch.Tensor, w: int, h: int, levels: int, stream=None) -> torch.Tensor:
    out = torch.empty((h, w), dtype=torch.complex64, device=wbuf.device)
    check(_lib().wasabi_wbuf_to_mallat(_ptr(wbuf), w, h, levels, _ptr(out), _stream(stream)))
    _keep(stream, out)
    return out


def inverse_stall_for_test(wbuf: torch.Tensor, w: int, h: int, levels: int, skip_strip: int, wait_cycles: int,
                       bits: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Test export (wasabi_test_inverse_stall): the inverse transform to bits
    with strip `skip_strip`'s copy never issued and stage waits bounded by
    `wait_cycles`; sync_status() then raises WASABI_E_TIMEOUT."""
    if bits is None:
        bits = torch.zeros((h * w + 7) // 8, dtype=torch.uint8, device=wbuf.device)
    check(_lib().wasabi_test_inverse_stall(_ptr(wbuf), w, h, levels, _ptr(bits), skip_strip, wait_cycles,
                                           _stream(stream)))
    _keep(stream, wbuf, bits)
    return bits
