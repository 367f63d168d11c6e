"""The measured workloads (sizes, optics and seeds) as plain data.

C1 small parity case; C2 8192^2 WASABI vs direct Eq. (1); C3 the paper-scale
65536^2 binarised hologram; C4 the reduced-precision LUT form of C2; C5 the
serving stream; P the geometry of the paper's own experiment (Sec. 2: an
image-type hologram of ~10^5 points from -15 mm to +15 mm in 29 depth bins,
pitch 1 um, a spherical reference wave at (0, 30 mm, -400 mm), 65,536^2,
binarised; the selectivity is not stated there, 1% is taken).  Lengths are in
metres.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from .clouds import heightfield_cloud, uniform_cloud
from .splitmix import uniform01


@dataclass(frozen=True)
class Workload:
    name: str
    Nh: int            # hologram side (pixels)
    lam: float         # wavelength
    pitch: float       # pixel pitch
    N: int             # object points
    zmin: float
    zmax: float
    D: int             # LUT depths
    W: int             # PSF window side
    L: int             # Haar levels
    gamma: float       # keep ratio (selectivity)
    cloud: str         # "uniform" | "heightfield"
    seed: int
    output: str = "complex"   # "complex" | "bits"
    lut_dtype: str = "f32"
    # Spherical reference wave: source offset (x, y) from the hologram centre
    # and signed distance z, or None for the unit plane wave.
    reference: tuple | None = None

    def points(self, N: int | None = None, Nh: int | None = None) -> dict:
        n = self.N if N is None else N
        side = self.Nh if Nh is None else Nh
        if self.cloud == "uniform":
            return uniform_cloud(self.seed, n, side, self.zmin, self.zmax)
        return heightfield_cloud(self.seed, n, side, self.zmin, self.zmax)

    def scaled(self, **kw) -> "Workload":
        return replace(self, **kw)


CONFIGS = {
    "C1": Workload("C1", 1024, 532e-9, 1e-6, 1000, 0.2e-3, 0.9e-3, 16, 512, 3, 0.05,
                   "uniform", 1),
    "C2": Workload("C2", 8192, 633e-9, 1e-6, 100_000, 0.3e-3, 1.0e-3, 64, 1024, 4, 0.02,
                   "heightfield", 2),
    "C3": Workload("C3", 65536, 633e-9, 1e-6, 2_097_152, 0.1e-3, 1.0e-3, 128, 1024, 4,
                   0.01, "heightfield", 3, output="bits"),
    "C4": Workload("C4", 8192, 633e-9, 1e-6, 100_000, 0.3e-3, 1.0e-3, 64, 1024, 4, 0.02,
                   "heightfield", 2, lut_dtype="f16s"),
    "C5": Workload("C5", 8192, 532e-9, 1e-6, 200_000, 0.3e-3, 1.0e-3, 64, 1024, 4, 0.02,
                   "heightfield", 5),
    # W = 9664: the smallest multiple of 2^(L+1) holding 2 R + 1 at the
    # outermost bin centre (|z| = 14.48 mm, R = 4830.5 px).
    "P": Workload("P", 65536, 632.8e-9, 1e-6, 95_949, -15e-3, 15e-3, 29, 9664, 3, 0.01,
                  "heightfield", 6, output="bits", reference=(0.0, 30e-3, -0.4)),
}


@dataclass(frozen=True)
class Job:
    index: int
    arrival_s: float
    Nh: int
    N: int
    seed: int


def serving_stream(n_jobs: int = 512, seed: int = 5, mean_gap_s: float = 0.005,
                   sizes=(1024, 2048, 4096, 8192), n_lo: float = 1e3,
                   n_hi: float = 2e5) -> list[Job]:
    """C5 arrivals: cumulative Exp(mean_gap_s) gaps, side uniform over
    ``sizes``, N = round(exp(U[ln n_lo, ln n_hi])); job i's points use seed
    5000 + i."""
    u = uniform01(seed, 3 * n_jobs, 0).reshape(3, n_jobs)
    gaps = -mean_gap_s * np.log1p(-u[0])
    t = np.cumsum(gaps)
    side = np.asarray(sizes)[np.minimum((u[1] * len(sizes)).astype(int), len(sizes) - 1)]
    n = np.rint(np.exp(np.log(n_lo) + u[2] * (np.log(n_hi) - np.log(n_lo)))).astype(int)
    return [Job(i, float(t[i]), int(side[i]), int(n[i]), 5000 + i) for i in range(n_jobs)]
