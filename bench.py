#!/usr/bin/env python3
"""WASABI hologram benchmark (paper-scale 65,536^2 binarised hologram).

One step = the whole hot path on one batch of synthetic input: LUT build
(PSF + Haar + shrinkage, 128 depths), point quantisation, binning +
superposition into the 34.4 GB tile-major wavelet buffer, and the fused
inverse Haar + binarisation.  Inputs are resident in HBM when the timed region
starts; the wavelet buffer (34.4 GB) is far larger than L2, so no flush is
needed.  `e2e` repeats the same step through the public API with pinned host
buffers: the host->device copy of the points and the device->host copy of the
bits are inside its timed region.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import CONFIGS, heightfield_cloud, serving_stream  # noqa: E402

METRIC = "WASABI hologram Mpoint*coeff/s at 65536^2 (hologram s, HBM fraction)"
UNIT = "Mpoint*coeff/s"


# DRAM bytes per launch of the dominant kernel (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture, scaled to a full launch), valid
# only while the kernel source is the one that was profiled (sha256 prefix of
# superpose.cu).
# Captured on the 32,768^2 slice of C3 (10.6 MB read + 79.2 MB written) and
# scaled by the point-coefficients processed (x4.015).
TRAFFIC = {("C3", "fused"): ("c5b7dd36496046a9", (10.596e6 + 79.180e6) * 4.015)}
# The same kernel's issue-slot utilisation and warp instructions per
# point·coefficient from its full ncu capture (32,768^2 slice of C3): the
# instruction roofline it is bound by.
ISSUE = {("C3", "fused"): ("c5b7dd36496046a9", 0.598, 1.97)}


def _sha(name):
    import hashlib
    src = os.path.join(ROOT, "paper_1708_04233_gb300", "csrc", name)
    with open(src, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _superpose_sha():
    return _sha("superpose.cu")


def _traffic(c, path):
    ent = TRAFFIC.get((c.name, path))
    return ent[1] if ent is not None and _superpose_sha() == ent[0] else None


def _issue(c, path):
    ent = ISSUE.get((c.name, path))
    if ent is None or _superpose_sha() != ent[0]:
        return None
    return {"ncu_issue_active": ent[1], "warp_instructions_per_point_coeff": ent[2]}


def max_over_ranks(x: float, device) -> float:
    """The largest of one float per rank (all ranks get it); the value alone
    when not running distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Replicas: every rank computes the same workload; the whole job's rate
    is all ranks' units over the slowest rank's time (Mpoint*coeff/s)."""
    return units_per_rank * world / (ms_max * 1e-3) / 1e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload_desc(c):
    form = "binarised hologram" if c.output == "bits" else "complex field"
    out_bytes = c.Nh * c.Nh // 8 if c.output == "bits" else c.Nh * c.Nh * 8
    return {"workload": f"{c.name}: {c.Nh}x{c.Nh} {form}, {c.N} {c.cloud} points, "
                        f"{c.D} depths, W={c.W}, L={c.L}, keep={c.gamma}, LUT {c.lut_dtype}",
            "Nh": c.Nh, "N": c.N, "lambda_m": c.lam, "pitch_m": c.pitch, "z_range_m": [c.zmin, c.zmax],
            "depths": c.D, "window": c.W, "levels": c.L, "keep_ratio": c.gamma, "output": c.output,
            "lut_dtype": c.lut_dtype,
            "reference": (f"spherical, source ({c.reference[0] * 1e3:g} mm, {c.reference[1] * 1e3:g} mm, "
                          f"{c.reference[2] * 1e3:g} mm) from the hologram centre" if c.reference
                          else "unit plane wave"),
            "l2": (f"{'outputs larger than L2' if out_bytes > 129e6 else 'outputs NOT larger than L2'} "
                   f"({out_bytes / 1e9:.3g} GB written per step; "
                   f"{c.Nh * c.Nh * 8e-9:.3g} GB wavelet buffer in the two-pass form)")}


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].strip().replace(".", "").isdigit())}


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(c, pts, threads: int, n_sub: int = 2, sub: int = 1024, depths_sample: int = 4):
    """Time the oracle as it stands on a bounded sample of the workload and
    scale to the whole hologram: `depths_sample` LUT depths (of c.D) and
    `n_sub` sub-holograms of sub x sub (of (Nh/sub)^2), paper procedure."""
    import concurrent.futures as cf

    import oracle
    zd = oracle.depth_grid(c.zmin, c.zmax, c.D)
    d, _ = oracle.quantize(pts["z"], c.zmin, c.zmax, c.D)
    idx = np.linspace(0, c.D - 1, depths_sample).astype(int)
    t0 = time.perf_counter()
    oracle.build_lut(c.lam, c.pitch, zd[idx], c.W, c.L, c.gamma, threads=threads)
    t_lut = (time.perf_counter() - t0) * c.D / depths_sample
    full = oracle.build_lut(c.lam, c.pitch, zd, c.W, c.L, c.gamma, threads=threads)  # untimed
    p = dict(pts, d=d)
    per_side = c.Nh // sub
    rng = np.random.default_rng(0)
    cells = [(int(s), int(t)) for s, t in rng.integers(0, per_side, (max(n_sub, threads), 2))][:max(n_sub, threads)]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda st: oracle.subhologram(full, p, sub, st[0], st[1]), cells))
    t_sub = (time.perf_counter() - t0) / len(cells) * threads  # per sub-hologram, one thread
    t_holo = t_sub * per_side * per_side / threads + t_lut
    work = float(np.sum(full.nr[d]))
    return {"value": work / t_holo / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"LUT for {depths_sample} of {c.D} depths (scaled x{c.D / depths_sample:g}) + "
                      f"{len(cells)} random {sub}x{sub} sub-holograms (paper Sec. 1 procedure, scaled to "
                      f"{per_side * per_side}), threads={threads}",
            "est_hologram_s": t_holo}


def run_reference(args, c):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pts = c.points()
    threads = os.cpu_count() or 1
    # The same bounded sample as the GPU arm's cpu_baseline (four LUT depths
    # spread over the range, one 1,024^2 sub-hologram per host thread).
    for _ in range(args.warmup):
        oracle_sample(c, pts, threads)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_sample(c, pts, threads))
    wall = time.perf_counter() - t0
    v = float(np.median([s["value"] for s in vals]))
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": f"synthetic (seeded height-field point cloud, seed {c.seed})",
            "config": _workload_desc(c), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- GPU arm

def _time(torch, stream, fn, reps=5):
    fn()
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def reference_summary(w, torch, c, depths, pbuf, stream, units):
    """The paper's reference wave (Sec. 2): a spherical wave from
    (0, 30 mm, -400 mm) relative to the hologram centre, against the unit
    plane reference of the headline, on the same points and LUT."""
    lut = w.build_lut(c.lam, c.pitch, depths, c.W, c.L, c.gamma, dtype=c.lut_dtype, stream=stream)
    n = pbuf.shape[0]
    bits = torch.empty(c.Nh * c.Nh // 8, dtype=torch.uint8, device=pbuf.device)
    scratch = torch.empty(w.scratch_bytes(lut, n, c.Nh, c.Nh), dtype=torch.uint8, device=pbuf.device)
    ref = w.spherical_reference(c.lam, c.pitch, c.Nh / 2, c.Nh / 2 + 30e-3 / c.pitch, -0.4)

    def run(r):
        return lambda: w.hologram(lut, pbuf, c.Nh, c.Nh, want="bits", bits=bits, scratch=scratch, stream=stream,
                                  reference=r)
    ms_plane = _time(torch, stream, run(None), reps=3)
    ms_ref = _time(torch, stream, run(ref), reps=3)
    w.sync_status(stream)
    lut.close()
    return {"reference": "spherical, source at (0, 30 mm, -400 mm) from the hologram centre",
            "hologram_ms": ms_ref, "plane_reference_hologram_ms": ms_plane,
            "value": units / (ms_ref * 1e-3) / 1e6, "unit": UNIT,
            "note": "complex accumulation (the imaginary parts enter Re(u conj R)) + per-pixel reference phase"}


def _reference_of(w, c):
    """The workload's spherical reference wave in plane pixels (None: R = 1)."""
    if not c.reference:
        return None
    dx, dy, z = c.reference
    return w.spherical_reference(c.lam, c.pitch, c.Nh / 2 + dx / c.pitch, c.Nh / 2 + dy / c.pitch, z)


def paper_setup_summary(w, torch, dev, reps: int = 3):
    """The geometry of the paper's own experiment (workload P): LUT build
    and the fused hologram with the spherical reference, timed apart."""
    c = CONFIGS["P"]
    pts = c.points()
    cols = [torch.from_numpy(pts[k]).to(dev) for k in ("x", "y", "z", "a")]
    pbuf = torch.empty((c.N, 4), dtype=torch.int32, device=dev)
    w.quantize_points(*cols, c.zmin, c.zmax, c.D, out=pbuf)
    depths = w.depth_grid(c.zmin, c.zmax, c.D)
    stream = torch.cuda.Stream(device=dev)
    ref = _reference_of(w, c)
    bits = torch.empty(c.Nh * c.Nh // 8, dtype=torch.uint8, device=dev)
    holder = {}

    def build():
        if "lut" in holder:
            holder.pop("lut").close()
        holder["lut"] = w.build_lut(c.lam, c.pitch, depths, c.W, c.L, c.gamma, stream=stream)
    lut_ms = _time(torch, stream, build, reps=reps)
    lut = holder["lut"]
    scratch = torch.empty(w.scratch_bytes(lut, c.N, c.Nh, c.Nh), dtype=torch.uint8, device=dev)
    holo_ms = _time(torch, stream, lambda: w.hologram(lut, pbuf, c.Nh, c.Nh, want="bits", bits=bits,
                                                      scratch=scratch, stream=stream, reference=ref), reps=reps)
    w.sync_status(stream)
    nr = lut.counts()
    units = float(np.sum(nr[pbuf[:, 3].cpu().numpy().view(np.uint32)]))
    lut.close()
    return {"workload": _workload_desc(c)["workload"], "reference": _workload_desc(c)["reference"],
            "lut_ms": lut_ms, "hologram_ms": holo_ms, "step_ms": lut_ms + holo_ms,
            "value": units / ((lut_ms + holo_ms) * 1e-3) / 1e6, "unit": UNIT, "point_coeff": units,
            "paper_cpu_s": 354.0}


def streaming_summary(w, torch, dev, c, side: int, band_h: int, reps: int = 2):
    """Sub-hologram streaming (Sec. 1, large-scale steps 2-4): a side^2
    binarised hologram at the headline's point density, computed in bands of
    band_h rows with each band's bits copied to pinned host memory while the
    next band is computed (wasabi_hologram_stream; the call's wall time,
    including its band-buffer allocations)."""
    n = int(round(c.N * (side / c.Nh) ** 2))
    pts = c.points(N=n, Nh=side)
    cols = [torch.from_numpy(pts[k]).to(dev) for k in ("x", "y", "z", "a")]
    pbuf = torch.empty((n, 4), dtype=torch.int32, device=dev)
    depths = w.depth_grid(c.zmin, c.zmax, c.D)
    w.quantize_points(*cols, c.zmin, c.zmax, c.D, out=pbuf)
    lut = w.build_lut(c.lam, c.pitch, depths, c.W, c.L, c.gamma, dtype=c.lut_dtype)
    nr = lut.counts()
    units = float(np.sum(nr[pbuf[:, 3].cpu().numpy().view(np.uint32)]))
    del cols
    bits = torch.empty(side * side // 8, dtype=torch.uint8).pin_memory()
    w.hologram_stream(lut, pbuf, side, side, band_h, want="bits", bits=bits)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(reps):
        w.hologram_stream(lut, pbuf, side, side, band_h, want="bits", bits=bits)
    s = (time.perf_counter() - t0) / reps
    w.sync_status()
    lut.close()
    return {"hologram": f"{side}x{side} binarised, {n} {c.cloud} points, bands of {band_h} rows "
                        f"streamed to pinned host memory",
            "s_per_hologram": s, "value": units / s / 1e6, "unit": UNIT,
            "point_coeff": units, "host_bytes": side * side // 8,
            "device_bytes_held": "two bands of bits + two binning scratches"}


# FP32 lane instructions (FFMA + FADD + FMUL, ncu smsp__sass_thread_inst_executed_op_*_pred_on)
# per term of the apertured Eq. (1) kernel at C2 (9.61e11 for 1.714e10 terms),
# valid while direct.cu is the profiled source (sha256 prefix).
DIRECT_FP32 = ("c38be776c999e9af", 9.6120e11 / 17138704217)


def eq1_terms(x, y, z, lam, pitch, w, h):
    """Point-pixel pairs the apertured Eq. (1) sums: pixels (x + dx, y + dy)
    inside the w x h hologram with dx^2 + dy^2 < R(z)^2, R the support radius
    z tan(asin(lambda / 2p)) / p (the point's own pixel always counts)."""
    s = lam / (2 * pitch)
    R2 = (np.abs(z) * (s / np.sqrt(1 - s * s)) / pitch) ** 2
    x = np.asarray(x, np.int64)
    y = np.asarray(y, np.int64)
    rmax = int(np.ceil(np.sqrt(R2.max()))) + 1 if R2.size else 0
    total = 0
    for dy in range(-rmax, rmax + 1):
        T = R2 - dy * dy
        ok = T > 0
        hw = np.where(ok, np.ceil(np.sqrt(np.maximum(T, 0))) - 1, -1).astype(np.int64)
        hw = np.where(ok & ((hw + 1) ** 2 < T), hw + 1, hw)  # |dx| <= hw  <=>  dx^2 < T
        hw = np.where(ok & (hw ** 2 >= T), hw - 1, hw)
        if dy == 0:
            hw = np.maximum(hw, 0)
        yy = y + dy
        lo, hi = np.maximum(x - hw, 0), np.minimum(x + hw, w - 1)
        total += int(np.sum(np.where((yy >= 0) & (yy < h) & (hw >= 0) & (hi >= lo), hi - lo + 1, 0)))
    return total


def direct_comparison(w, torch, dev, c, depths, pbuf, u_wasabi, stream, wasabi_step_ms):
    """C2: Eq. (1) summed directly on the GPU (aperture form) on the same
    points, its time against the WASABI step, and the WASABI approximation
    error against it (rel-L2 over the whole field, norms in FP64)."""
    u_direct = torch.empty_like(u_wasabi)
    scratch = torch.empty(w.cgh_direct_scratch_bytes(pbuf.shape[0], c.Nh, c.Nh), dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        ms = _time(torch, stream, lambda: w.cgh_direct(c.lam, c.pitch, depths, pbuf, c.Nh, c.Nh, True, u=u_direct,
                                                        scratch=scratch, stream=stream), reps=3)
    w.sync_status(stream)
    diff = (u_wasabi.to(torch.complex128) - u_direct.to(torch.complex128)).abs().pow(2).sum().sqrt()
    ref = u_direct.to(torch.complex128).abs().pow(2).sum().sqrt()
    # Numerical reconstruction of both fields at the middle depth (d = -z):
    # how alike the images are (the paper compares reconstructions, Fig. 3).
    zmid = float(depths[len(depths) // 2])
    rec = {}
    for name, u in (("wasabi", u_wasabi), ("eq1", u_direct)):
        rec[name] = w.reconstruct(u, c.Nh, c.Nh, c.lam, c.pitch, -zmid, stream=stream)
    # The reconstructions run asynchronously on `stream`: wait for them before
    # reading the images on the current stream.
    torch.cuda.current_stream().wait_stream(stream)
    rec = {k: v.double() for k, v in rec.items()}
    rms = _time(torch, stream, lambda: w.reconstruct(u_wasabi, c.Nh, c.Nh, c.lam, c.pitch, -zmid, stream=stream),
                reps=3)
    a_, b_ = rec["wasabi"], rec["eq1"]

    def corr_of(x, y):
        x, y = x - x.mean(), y - y.mean()
        return float((x * y).sum() / (x.norm() * y.norm()))
    corr = corr_of(a_, b_)
    # The shift rule moves each level's coefficients by less than 2^L pixels,
    # so the refocused points of the two images sit up to 2^L - 1 pixels apart:
    # compare them also on 2^L x 2^L blocks.
    pool = lambda x: torch.nn.functional.avg_pool2d(x[None, None], 1 << c.L)[0, 0]
    corr_pooled = corr_of(pool(a_), pool(b_))
    direct_comparison.u_direct = u_direct
    # Roofline: FP32 lane instructions per term (ncu, this source) x terms,
    # against 152 SMs x 128 FP32 lanes x the maximum SM clock.
    p_host = pbuf.cpu().numpy()
    terms = eq1_terms(p_host[:, 0], p_host[:, 1], np.asarray(depths)[p_host[:, 3].view(np.uint32)], c.lam,
                      c.pitch, c.Nh, c.Nh)
    peak = 152 * 128 * 2070e6
    roof = {"bound": "alu", "unit": "FP32 lane-instr/s", "terms": terms, "terms_per_s": terms / (ms * 1e-3),
            "peak": peak, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz"}
    if _sha("direct.cu") == DIRECT_FP32[0]:
        ach = DIRECT_FP32[1] * terms / (ms * 1e-3)
        roof.update({"fp32_instr_per_term": DIRECT_FP32[1], "achieved": ach, "frac": ach / peak})
    return {"kernel": "direct_kernel (Eq. (1), aperture form; double-float phase reduction)", "ms": ms,
            "roofline": roof,
            "wasabi_step_ms": wasabi_step_ms, "speedup": ms / wasabi_step_ms,
            "rel_l2_wasabi_vs_eq1": float(diff / ref),
            "reconstruction": {"d_m": -zmid, "ms": rms, "method": "angular spectrum (cuFFT C2C)",
                               "intensity_correlation_wasabi_vs_eq1": corr,
                               f"intensity_correlation_{1 << c.L}px_blocks": corr_pooled,
                               "intensity_rel_l2_wasabi_vs_eq1": float((a_ - b_).norm() / b_.norm())}}


def coiflet_summary(w, torch, dev, c, depths, pbuf, stream, u_direct, units_haar):
    """The paper's wavelet family (order-1 coiflet, periodic) on the same
    workload: LUT build, superposition into the tile-major buffer, the
    separable periodic inverse, and the WASABI-vs-Eq. (1) error beside
    Haar's.  The inverse's HBM fraction counts its algorithmic bytes (8 B
    read + 8 B written per pixel) against its time."""
    holder = {}

    def build():
        if "lut" in holder:
            holder.pop("lut").close()
        holder["lut"] = w.build_lut(c.lam, c.pitch, depths, c.W, c.L, c.gamma, stream=stream, wavelet="coif1")
    lut_ms = _time(torch, stream, build, reps=3)
    lut = holder["lut"]
    n = pbuf.shape[0]
    wb = torch.empty(c.Nh * c.Nh, dtype=torch.complex64, device=dev)
    u = torch.empty((c.Nh, c.Nh), dtype=torch.complex64, device=dev)
    scratch = torch.empty(w.scratch_bytes(lut, n, c.Nh, c.Nh), dtype=torch.uint8, device=dev)
    sup_ms = _time(torch, stream, lambda: w.superpose(lut, pbuf, c.Nh, c.Nh, wbuf=wb, scratch=scratch, stream=stream),
                   reps=5)
    inv_ms = _time(torch, stream, lambda: w.inverse_wavelet(wb, c.Nh, c.Nh, c.L, "coif1", u=u, stream=stream), reps=5)
    w.sync_status(stream)
    nr = lut.counts()
    units = float(np.sum(nr[pbuf[:, 3].cpu().numpy().view(np.uint32)]))
    lut.close()
    err = float((u.to(torch.complex128) - u_direct.to(torch.complex128)).norm() / u_direct.to(torch.complex128).norm())
    peak, peak_kind = _peaks()
    inv_gbs = 16.0 * c.Nh * c.Nh / (inv_ms * 1e-3) / 1e9
    return {"wavelet": "coif1 (order-1 coiflet, 6 taps, periodic)", "lut_ms": lut_ms, "superpose_ms": sup_ms,
            "inverse_ms": inv_ms, "step_ms": lut_ms + sup_ms + inv_ms, "point_coeff": units,
            "point_coeff_haar": units_haar, "value": units / ((lut_ms + sup_ms + inv_ms) * 1e-3) / 1e6,
            "unit": UNIT, "rel_l2_vs_eq1": err,
            "inverse_hbm": {"algorithmic_bytes": 16 * c.Nh * c.Nh, "gbs": inv_gbs, "frac": inv_gbs / peak,
                            "peak": peak, "peak_source": peak_kind}}


def precision_forms(w, torch, dev, c, depths, pbuf, stream):
    """C4: the fused hologram with the LUT stored as FP32, FP16 and BF16
    (per-32 FP32 scales); time of the hologram call per form.  The error of
    each form against the FP64 oracle is measured by the test suite
    (tests/test_gpu_fullsize.py::test_c4_precision_forms_vs_fp64)."""
    out = {"workload": f"{c.name}: {c.Nh}x{c.Nh} complex field, {c.N} {c.cloud} points, {c.D} depths, "
                       f"W={c.W}, L={c.L}, keep={c.gamma}"}
    u = torch.empty((c.Nh, c.Nh), dtype=torch.complex64, device=dev)
    for dt in ("f32", "f16s", "bf16s"):
        lut = w.build_lut(c.lam, c.pitch, depths, c.W, c.L, c.gamma, dtype=dt, stream=stream)
        scratch = torch.empty(w.scratch_bytes(lut, pbuf.shape[0], c.Nh, c.Nh), dtype=torch.uint8, device=dev)
        with torch.cuda.stream(stream):
            ms = _time(torch, stream, lambda: w.hologram(lut, pbuf, c.Nh, c.Nh, want="complex", u=u,
                                                          scratch=scratch, stream=stream), reps=20)
        out[dt] = {"hologram_ms": ms}
        lut.close()
    w.sync_status(stream)
    for dt in ("f16s", "bf16s"):
        out[dt]["speedup_vs_f32"] = out["f32"]["hologram_ms"] / out[dt]["hologram_ms"]
    return out


def precision_summary(w, torch, dev, stream):
    """The C4 precision forms beside the default run: C4's own seeded points."""
    c = CONFIGS["C4"]
    p = c.points()
    t = {k: torch.from_numpy(p[k]).to(dev) for k in "xyza"}
    pbuf = w.quantize_points(t["x"], t["y"], t["z"], t["a"], c.zmin, c.zmax, c.D)
    return precision_forms(w, torch, dev, c, w.depth_grid(c.zmin, c.zmax, c.D), pbuf, stream)


def serving_summary(w, torch, dev, n_jobs: int = 512, budget_gib: float = 4.0, streams: int = 4,
                    max_batch: int = 32):
    """C5: the seeded request stream (Poisson arrivals at 200/s, sides
    1024..8192, N log-uniform in [1e3, 2e5]) through the serving loop, as
    scheduled (p50/p99 latency) and all at once (saturated throughput), next
    to the same holograms computed one call at a time (plain form)."""
    c = CONFIGS["C5"]
    jobs = serving_stream(n_jobs)
    depths = w.depth_grid(c.zmin, c.zmax, c.D)
    lut = w.build_lut(c.lam, c.pitch, depths, c.W, c.L, c.gamma)
    hosts = []
    for j in jobs:
        p = heightfield_cloud(j.seed, j.N, j.Nh, c.zmin, c.zmax)
        t = {k: torch.from_numpy(p[k]).to(dev) for k in "xyza"}
        q = w.quantize_points(t["x"], t["y"], t["z"], t["a"], c.zmin, c.zmax, c.D)
        hosts.append(q.cpu().pin_memory())
    w.sync_status()
    srv = w.Server(lut, int(budget_gib * (1 << 30)), streams=streams, max_batch=max_batch, side_hint=4096)
    for i in range(min(8, n_jobs)):  # warm-up: graph capture on the streams
        srv.wait(srv.submit(hosts[i], jobs[i].Nh, jobs[i].Nh), timeout=120)

    # Pinned output buffers are allocated once, up front: what is timed is the
    # server, not host-memory allocation.
    outs = [torch.empty((j.Nh * j.Nh) // 8, dtype=torch.uint8).pin_memory() for j in jobs]

    def run(paced: bool):
        ids = []
        t0 = time.perf_counter()
        for j, h, o in zip(jobs, hosts, outs):
            if paced:
                dt = t0 + j.arrival_s - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            ids.append(srv.submit(h, j.Nh, j.Nh, bits=o))
        return [srv.wait(i, timeout=600) for i in ids]

    paced = run(True)
    sat = run(False)
    stats = srv.stats()
    srv.close()
    lat = np.array([r["latency_s"] for r in paced]) * 1e3

    def rate(rs):
        return len(rs) / (max(r["done_s"] for r in rs) - min(r["submit_s"] for r in rs))

    # Plain form: one wasabi_hologram call per request, back to back.
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for j, h, o in zip(jobs, hosts, outs):
            d = h.to(dev, non_blocking=True)
            b = w.hologram(lut, d, j.Nh, j.Nh, want="bits", stream=stream)
            o.copy_(b, non_blocking=True)
    stream.synchronize()
    plain = len(jobs) / (time.perf_counter() - t0)
    w.sync_status()
    lut.close()
    return {"workload": f"C5: {len(jobs)} requests, Poisson arrivals at 200/s, sides 1024-8192, "
                        f"N log-uniform [1e3, 2e5], bits out, {c.D}-depth LUT (lambda 532 nm)",
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "holograms_per_s_paced": rate(paced), "holograms_per_s_saturated": rate(sat),
            "holograms_per_s_plain_one_call_each": plain,
            "mean_jobs_per_launch_saturated": float(np.mean([r["batch_jobs"] for r in sat])),
            "launches": stats["launches"], "peak_arena_bytes": stats["peak_bytes"],
            "budget_bytes": int(budget_gib * (1 << 30)), "streams": streams, "max_batch": max_batch}


def run_gpu(args, c):
    import torch
    import torch.distributed as dist

    import paper_1708_04233_gb300 as w
    from paper_1708_04233_gb300 import build as wbuild
    wbuild.build()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    pts = c.points()
    N = c.N
    depths = w.depth_grid(c.zmin, c.zmax, c.D)
    x = torch.from_numpy(pts["x"]).to(dev)
    y = torch.from_numpy(pts["y"]).to(dev)
    z = torch.from_numpy(pts["z"]).to(dev)
    a = torch.from_numpy(pts["a"]).to(dev)
    pbuf = torch.empty((N, 4), dtype=torch.int32, device=dev)
    want = "bits" if c.output == "bits" else "complex"
    bits = torch.empty(c.Nh * c.Nh // 8, dtype=torch.uint8, device=dev) if want == "bits" else None
    ufield = torch.empty((c.Nh, c.Nh), dtype=torch.complex64, device=dev) if want == "complex" else None
    out_dev = bits if want == "bits" else ufield
    stream = torch.cuda.Stream(device=dev)
    fused = args.path == "fused"
    ref = _reference_of(w, c)
    wbuf = None if fused else torch.empty(c.Nh * c.Nh, dtype=torch.complex64, device=dev)

    ev = {k: [] for k in (("lut", "hologram") if fused else ("lut", "superpose", "inverse"))}

    def step(record=False, xs=x, ys=y, zs=z, as_=a, two_pass=not fused, wb=None, out=None):
        with torch.cuda.stream(stream):
            marks = []

            def mark():
                if record:
                    e = torch.cuda.Event(enable_timing=True)
                    e.record(stream)
                    marks.append(e)
            mark()
            lut = w.build_lut(c.lam, c.pitch, depths, c.W, c.L, c.gamma, dtype=c.lut_dtype, stream=stream)
            w.quantize_points(xs, ys, zs, as_, c.zmin, c.zmax, c.D, out=pbuf, stream=stream)
            mark()
            if step.scratch is None:
                step.scratch = torch.empty(w.scratch_bytes(lut, N, c.Nh, c.Nh), dtype=torch.uint8, device=dev)
            o_u = ufield if out is None or want != "complex" else out
            o_b = bits if out is None or want != "bits" else out
            if two_pass:
                w.superpose(lut, pbuf, c.Nh, c.Nh, rule=0, wbuf=wb if wb is not None else wbuf,
                            scratch=step.scratch, stream=stream)
                mark()
                w.inverse_haar(wb if wb is not None else wbuf, c.Nh, c.Nh, c.L, u=o_u, bits=o_b, want=want,
                               stream=stream, reference=ref)
            else:
                w.hologram(lut, pbuf, c.Nh, c.Nh, want=want, rule=0, u=o_u, bits=o_b, scratch=step.scratch,
                           stream=stream, reference=ref)
            mark()
            if record:
                step.marks.append(marks)
            lut.close()
            return lut
    step.scratch = None
    step.marks = []

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    # Warm-up (also sizes the scratch and validates the device status).
    for _ in range(max(args.warmup, 1)):
        step()
    w.sync_status(stream)
    # Work units: sum over points of N_r(d_j) (kept coefficients per point).
    lut = w.build_lut(c.lam, c.pitch, depths, c.W, c.L, c.gamma, dtype=c.lut_dtype, stream=stream)
    nr = lut.counts()
    lut.close()
    d_host = pbuf[:, 3].cpu().numpy().view(np.uint32)
    units = float(np.sum(nr[d_host]))

    peak, peak_kind = _peaks()
    with ClockSampler(local) as clk:
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(record=True)
        t1.record(stream)
        barrier()
    w.sync_status(stream)
    ms = t0.elapsed_time(t1) / args.steps
    for marks in step.marks:
        for k, (e0, e1) in zip(ev, zip(marks, marks[1:])):
            ev[k].append((e0, e1))
    step.marks = []
    ms = max_over_ranks(ms, dev)
    stage_ms = {k: float(np.mean([s.elapsed_time(e) for s, e in v])) for k, v in ev.items()}

    # End to end through the public API with pinned host buffers: every step
    # uploads its points and downloads its result.  The copies run on their
    # own streams with two buffer sets, so step k's download overlaps step
    # k+1's computation (as a user pipelining the calls would).
    hx = torch.from_numpy(pts["x"]).pin_memory()
    hy = torch.from_numpy(pts["y"]).pin_memory()
    hz = torch.from_numpy(pts["z"]).pin_memory()
    ha = torch.from_numpy(pts["a"]).pin_memory()
    hout = [torch.empty(out_dev.shape, dtype=out_dev.dtype).pin_memory() for _ in range(2)]
    din = [[torch.empty_like(t) for t in (x, y, z, a)] for _ in range(2)]
    dout = [out_dev, torch.empty_like(out_dev)]
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    done_down = [None, None]
    computed_ev = [None, None]

    def e2e_step(k):
        j = k % 2
        uploaded = torch.cuda.Event()
        if computed_ev[j] is not None:
            up.wait_event(computed_ev[j])  # step k-2 has finished reading din[j]
        with torch.cuda.stream(up):
            for d_, h_ in zip(din[j], (hx, hy, hz, ha)):
                d_.copy_(h_, non_blocking=True)
            uploaded.record(up)
        stream.wait_event(uploaded)
        if done_down[j] is not None:
            stream.wait_event(done_down[j])  # the download of step k-2 has read dout[j]
        step(xs=din[j][0], ys=din[j][1], zs=din[j][2], as_=din[j][3], out=dout[j])
        computed = torch.cuda.Event()
        computed.record(stream)
        down.wait_event(computed)
        with torch.cuda.stream(down):
            hout[j].copy_(dout[j], non_blocking=True)
            done_down[j] = torch.cuda.Event()
            done_down[j].record(down)
        computed_ev[j] = computed
    for k in range(2):
        e2e_step(k)
    barrier()
    te = time.perf_counter()
    for k in range(args.steps):
        e2e_step(k)
    barrier()
    e2e_ms = (time.perf_counter() - te) * 1e3 / args.steps
    e2e_ms = max_over_ranks(e2e_ms, dev)
    # The latency of one call with nothing else in flight: upload, step,
    # download, synchronise.
    torch.cuda.synchronize(dev)
    one = []
    for _ in range(max(3, min(args.steps, 10))):
        t1 = time.perf_counter()
        with torch.cuda.stream(up):
            for d_, h_ in zip(din[0], (hx, hy, hz, ha)):
                d_.copy_(h_, non_blocking=True)
        stream.wait_stream(up)
        step(xs=din[0][0], ys=din[0][1], zs=din[0][2], as_=din[0][3], out=dout[0])
        with torch.cuda.stream(stream):
            hout[0].copy_(dout[0], non_blocking=True)
        stream.synchronize()
        one.append((time.perf_counter() - t1) * 1e3)
    one_ms = max_over_ranks(float(np.median(one)), dev)
    h2d = sum(t.numel() * t.element_size() for t in (hx, hy, hz, ha))
    d2h = hout[0].numel() * hout[0].element_size()
    assert torch.equal(hout[(args.steps - 1) % 2].to(dev), out_dev), "end-to-end result differs"

    # The two-pass form (superposition into the 34 GB wavelet buffer, then the
    # separate inverse kernel): the inverse kernel's HBM fraction.
    two = None
    if fused and not args.no_two_pass:
        wb = torch.empty(c.Nh * c.Nh, dtype=torch.complex64, device=dev)
        for _ in range(2):
            step(two_pass=True, wb=wb)
        barrier()
        n2 = max(3, min(args.steps, 10))
        for _ in range(n2):
            step(record=True, two_pass=True, wb=wb)
        barrier()
        w.sync_status(stream)
        st = {k: float(np.mean([m[i].elapsed_time(m[i + 1]) for m in step.marks]))
              for i, k in enumerate(("lut", "superpose", "inverse"))}
        step.marks = []
        del wb
        torch.cuda.empty_cache()
        two = {"ms_per_step": sum(st.values()), "stages_ms": st, "steps": n2}
    elif not fused:
        two = {"ms_per_step": ms, "stages_ms": stage_ms, "steps": args.steps}

    inv_bytes = c.Nh * c.Nh * 8 + (c.Nh * c.Nh // 8 if want == "bits" else c.Nh * c.Nh * 8)
    if two is not None:
        inv_gbs = inv_bytes / (two["stages_ms"]["inverse"] * 1e-3) / 1e9
        two["inverse_hbm"] = {"kernel": f"inverse_kernel<{c.L}> (inverse Haar" + (" + binarisation)" if want == "bits" else ")"),
                              "algorithmic_bytes": inv_bytes, "gbs": inv_gbs, "frac": inv_gbs / peak,
                              "peak": peak, "peak_source": peak_kind}
    hot_ms = stage_ms["hologram" if fused else "superpose"]
    # Dominant kernel: the superposition (with the fused inverse + binarisation
    # epilogue in the fused form).  It is a shared-memory scatter-add: per
    # point-coefficient one 32-bit shared-memory atomic add per accumulated
    # part -- the real part alone when only bits are produced (Re u depends
    # only on the real parts), real and imaginary parts otherwise.
    # Peak: one 32-bit access per bank per clock, 32 banks x 152 SMs x max SM clock.
    parts = 1 if (fused and want == "bits" and not c.reference) else 2
    smem_peak = 32 * 152 * 2070e6 / 1e9  # Gop/s
    ach = parts * units / (hot_ms * 1e-3) / 1e9
    roof = {"kernel": (f"superpose_kernel<{c.L},{c.lut_dtype}> with fused inverse"
                       + (" + binarisation" if want == "bits" else "") if fused
                       else f"superpose_kernel<{c.L},{c.lut_dtype}>") + " (+ binning kernels, one ABI call)",
            "bound": "alu", "achieved": ach, "peak": smem_peak, "unit": "Gop/s", "frac": ach / smem_peak,
            "peak_source": "derived: 32 banks x 152 SMs x 2070 MHz (shared-memory 32-bit ops)",
            "algorithmic_ops": parts * units, "ops_per_point_coeff": parts, "traffic": _traffic(c, args.path),
            "issue": _issue(c, args.path)}
    # psf, select, tile count/scan, scatter, codes, level-mask readback (+ encode for FP16/BF16)
    lut_kernels = 7 + (0 if c.lut_dtype in ("f32", 0) else 1)
    per_step = lut_kernels + 1 + 6 + (0 if fused else 1)

    if rank == 0:
        out = {"metric": METRIC, "value": whole_job_rate(units, world, ms), "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": f"synthetic (seeded height-field point cloud, SplitMix64 seed {c.seed})",
               "config": dict(_workload_desc(c), parallelism=f"replicas x{world}"),
               "hologram_s": ms * 1e-3, "point_coeff_per_step": units,
               "stages_ms": stage_ms,
               "path": args.path,
               "superpose_mpc_s": units / (hot_ms * 1e-3) / 1e6,
               "roofline": roof,
               "two_pass": two,
               "e2e": {"value": whole_job_rate(units, world, e2e_ms), "unit": UNIT,
                       "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "pipelined": "two buffer sets: step k's download overlaps step k+1",
                       "one_call_latency_ms": one_ms},
               "gpu_launches": per_step * args.steps,
               "clocks": clk.summary()}
        if c.name == "C2":
            out["direct_eq1"] = direct_comparison(w, torch, dev, c, depths, pbuf, out_dev, stream, ms)
            out["coiflet"] = coiflet_summary(w, torch, dev, c, depths, pbuf, stream, direct_comparison.u_direct,
                                             units)
        if c.name == "C4":
            out["precision_forms"] = precision_forms(w, torch, dev, c, depths, pbuf, stream)
        if not args.no_serving and c.name == "C3":
            out["serving"] = serving_summary(w, torch, dev)
        if c.name == "C3" and args.nh == 0 and not args.no_extras:
            out["paper_reference_wave"] = reference_summary(w, torch, c, depths, pbuf, stream, units)
            out["streaming"] = streaming_summary(w, torch, dev, c, args.stream_side, args.stream_band)
            out["paper_setup"] = paper_setup_summary(w, torch, dev)
            out["precision_forms"] = precision_summary(w, torch, dev, stream)
        if not args.no_cpu_baseline and c.name != "P":
            out["cpu_baseline"] = oracle_sample(c, pts, os.cpu_count() or 1)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wasabi", choices=["wasabi", "reference"])
    ap.add_argument("--config", default="C3", choices=["C2", "C3", "C4", "P"],
                    help="C3 (default): the 65536^2 binarised hologram; C2: 8192^2 complex field "
                         "with direct Eq. (1) beside it; C4: C2 with the precision forms; P: the paper's own "
                         "geometry (+-15 mm, 29 depths, spherical reference)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--path", default="fused", choices=["fused", "two-pass"],
                    help="fused: wasabi_hologram; two-pass: wasabi_superpose + wasabi_inverse_haar")
    ap.add_argument("--no-serving", action="store_true", help="skip the C5 serving-loop summary")
    ap.add_argument("--nh", type=int, default=0,
                    help="profiling cases: hologram side (points scaled by area, same density)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the spherical-reference and sub-hologram streaming summaries")
    ap.add_argument("--stream-side", type=int, default=131072,
                    help="side of the streamed hologram (points scaled by area)")
    ap.add_argument("--stream-band", type=int, default=16384, help="rows per streamed band")
    ap.add_argument("--no-two-pass", action="store_true",
                    help="skip the secondary two-pass measurement (inverse kernel HBM fraction)")
    args = ap.parse_args()
    c = CONFIGS[args.config]
    if args.nh:
        c = c.scaled(Nh=args.nh, N=max(1, c.N * args.nh * args.nh // (c.Nh * c.Nh)),
                     name=f"{c.name}-scaled")
    if args.impl == "reference":
        run_reference(args, c)
    else:
        run_gpu(args, c)


if __name__ == "__main__":
    main()
