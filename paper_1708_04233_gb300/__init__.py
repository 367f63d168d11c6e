"""WASABI (wavelet shrinkage-based superposition) hologram synthesis on GB300.

Thin Python binding over libwasabi (include/wasabi.h): the functions here only
marshal tensors, pointers and streams; every step of the computation runs in
hand-written sm_103a CUDA kernels.  PyTorch provides device memory and
streams.  After Shimobaba et al., "Fast, large-scale hologram calculation in
wavelet domain" (arXiv 1708.04233): Sec. 1 steps 1-3 and Eqs. (1)-(2).
"""
from .api import (Batch, Lut, Server, autotune, build_lut, cgh_direct, cgh_direct_scratch_bytes, depth_grid,
                  haar_forward, hologram, hologram_stream, inverse_haar, inverse_wavelet, reconstruct, pack_points, quantize_points,
                  make_frame, scratch_bytes, spherical_reference, superpose, superpose_static, sync_status,
                  wbuf_to_mallat)
from ._abi import (BF16S, F16S, F32, SHIFT_FLOOR, SHIFT_NEAREST, WasabiError)

__all__ = ["Batch", "Lut", "Server", "autotune", "build_lut", "cgh_direct", "cgh_direct_scratch_bytes", "depth_grid",
           "haar_forward", "hologram", "hologram_stream", "inverse_haar", "inverse_wavelet", "reconstruct", "make_frame", "pack_points", "quantize_points",
           "scratch_bytes", "spherical_reference", "superpose", "superpose_static", "sync_status", "wbuf_to_mallat", "F32", "F16S",
           "BF16S", "SHIFT_FLOOR", "SHIFT_NEAREST", "WasabiError"]
