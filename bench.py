#!/usr/bin/env python3
"""Throughput benchmark of the EPIC imaging path on GB300.

One step = one integration imaged by one epic_image call: every channel,
polarisation and time sample of the workload (unpack, calibrate, grid,
transform, products, time sum, autocorrelation subtraction).  The metric is
imaged spectra per second, spectra = channels x time samples x polarisations.
The headline form is the split-FP16 tensor-core form (both 64-point DFT stages
on tcgen05, literal gridding, within 1e-5 of the FP64 oracle); the plain FP32
form and the other forms are timed beside it ("variants"), and the uneven-band
and dense-array workloads have their own lines ("workloads").

Default workload: the LWA-station-like configuration (256 dual-pol antennas,
64 channels of 25 kHz from 60 MHz, 1000 spectra per integration, 5x5 kernel,
128x128 grid), seeded synthetic inputs resident in HBM.  L2 is flushed by a
256 MiB write between timed steps.  Under torchrun each rank images its own
band of the same shape (weak scaling, no collective on the data path); with
--split-band the ranks split one fixed band by channel instead (strong
scaling) and the finished images are gathered to rank 0 after the timed
region.

--impl reference times the FP64 CPU oracle (the correctness reference) on the
host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "imaged spectra/s (chan x time x pol)"
UNIT = "spectra/s"
FP32_LANES_PER_SM = 128
SERIES_SPI = 40                      # spectra per image of the time-resolved variant (1.6 ms at 25 k spectra/s)
L2_FLUSH_BYTES = 256 << 20

# DRAM traffic of one launch of a timed kernel from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by (workload, form),
# with the hash of the kernel source it was taken on; ignored (null) once the
# source changes.  Filled in from the committed profiles/ summaries.
NCU_TRAFFIC = {
    ("lwa", "tc_split_fp16"): (197.21e6, "e16cc173ad5d718a"),     # profiles/tc_pair128_kernel_lwa.md
    ("lwa", "fp32"): (144.11e6, "e8796ed7dfd2eaa3"),              # profiles/fp32_reg64_kernel_lwa.md
}
# What the same capture shows about the kernel's limits (same keys and hashes).
NCU_LIMITER = {
    ("lwa", "tc_split_fp16"): ({"tensor_pipe_active_pct": 60.0, "issue_active_pct": 49.7, "warps_active_pct": 18.7,
                               "smem_conflict_wavefront_share": 0.42,
                               "top_stalls": "short_scoreboard 1.18, wait 1.04, long_scoreboard 0.62"},
                              "e16cc173ad5d718a"),
    ("lwa", "fp32"): ({"fma_pipe_active_pct": 41.9, "issue_active_pct": 45.2, "warps_active_pct": 12.5,
                      "registers_per_thread": 228, "smem_conflict_wavefront_share": 0.20,
                      "top_stalls": "wait 1.10, short_scoreboard 0.75, not_selected 0.44"},
                     "e8796ed7dfd2eaa3"),
}


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["lwa", "tiny", "uneven", "dense"], default="lwa")
    ap.add_argument("--precision", choices=["fp32", "tc_split_fp16", "tc_fp16", "tc_split_bf16"],
                    default="tc_split_fp16",
                    help="arithmetic form of the timed plan (default: the split-FP16 tensor-core form)")
    ap.add_argument("--no-workloads", action="store_true", help="skip the uneven-band and dense-array lines")
    ap.add_argument("--no-peaks", action="store_true", help="skip measuring the pipes' peak rates")
    ap.add_argument("--taper", action="store_true", help="apply the kernel as an image-domain taper")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end loop")
    ap.add_argument("--no-variants", action="store_true", help="skip timing the other forms")
    ap.add_argument("--split-band", action="store_true",
                    help="under torchrun: split one fixed band across the ranks (strong scaling) instead of "
                         "giving every rank its own band (weak scaling)")
    ap.add_argument("--channels", type=int, default=None,
                    help="shrink the workload to this many channels (profiling captures only)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the cost model's launch shapes instead of epic_autotune's measured ones")
    ap.add_argument("--search-only", action="store_true",
                    help="time only the transient search of a synthetic image cube and print its JSON")
    return ap.parse_args()


def make_workload(name, channels=None, rank=0):
    """The named workload; under torchrun the LWA-like band of rank r sits next
    to rank r-1's (weak scaling), the other workloads are per-rank replicas."""
    from paper_2301_09662_gb300 import shard, synth
    kw = {} if channels is None else {"C": channels}
    if name == "lwa":
        kw["first_channel"] = shard.rank_first_channel(channels or 64, rank)
    fn = {"lwa": synth.lwa, "tiny": synth.tiny, "uneven": synth.uneven, "dense": synth.dense}[name]
    return fn(**kw)


def describe(wl, name):
    Ns = sorted(set(int(n) for n in wl.grid_n))
    return {
        "workload": f"{wl.name}: {wl.A} antennas x {wl.n_pol} pol, {wl.C} channels, {wl.T} spectra per "
                    f"integration, {wl.K}x{wl.K} kernel, grid {'/'.join(str(n) for n in Ns)}",
        "antennas": wl.A, "pols": wl.n_pol, "channels": wl.C, "spectra_per_integration": wl.T,
        "kernel": wl.K, "grid": Ns, "gains": wl.gains is not None,
        "l2": "flushed between timed steps (256 MiB write)",
        "parallelism": "one integration per GPU; ranks image independent bands",
    }


def fp32_flops_per_spectrum(A, K, N):
    """Algorithmic FLOPs of one spectrum in the FP32 form: gridding 8 A K^2,
    row-pruned radix-2 FFT 5 N log2 N (N/2 + N), products 8 N^2."""
    return 8.0 * A * K * K + 5.0 * N * math.log2(N) * (N / 2 + N) + 8.0 * N * N


def kernel_source_hash(form):
    """Hash of the device code of the imaging kernel a form runs at grid side
    128: the FP32 register kernel (fp32_reg64.cu up to its large-side part, and
    the transform headers) or the tensor pair kernel (tc_pair128.cu and the
    tensor helpers)."""
    csrc = os.path.join(ROOT, "paper_2301_09662_gb300", "csrc")
    if form == "fp32":
        src = open(os.path.join(csrc, "fp32_reg64.cu")).read()
        start = src.index("// Register transforms of the folded side M")
        end = src.index("// Large grid sides: the folded grids", start)
        h = hashlib.sha256(src[start:end].encode())
        files = ("fft64.cuh", "dft_small.cuh")
    else:
        h = hashlib.sha256()
        files = ("tc_pair128.cu", "tc_common.cuh", "tc_ptx.cuh", "dft_small.cuh")
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_record(table, workload, form):
    rec = table.get((workload, form))
    return rec[0] if rec and rec[1] == kernel_source_hash(form) else None


def measure_pipe_peaks():
    """Peak rates of the pipes the kernels use, measured here by epic_measure_peak
    (best of three ~100 ms launches each; TFLOP/s, 2 per multiply-add)."""
    from paper_2301_09662_gb300 import epic
    out = {}
    for k in ("fp32", "fp32x2", "fp64", "fp16_tc"):
        try:
            out[k] = epic.measure_peak(k, 100)
        except Exception as e:       # a probe that fails is reported, not fatal
            out[k] = f"failed: {e}"
    out["how"] = ("epic_measure_peak: independent FMA chains (8 per thread, 4 blocks of 512 threads per SM) or "
                  "back-to-back 128 x 256 x 16 FP16 tcgen05 MMAs (one CTA per SM), ~100 ms launches, best of 3")
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def cpu_baseline(wl, budget_s):
    """Time the FP64 oracle (O1, OpenMP over channels) on a bounded sample of
    about budget_s seconds: whole channels, one per thread per round, all
    spectra when they fit, more channels (in multiples of the thread count)
    while the budget allows."""
    import oracle
    threads = oracle.threads()
    C_s = max(1, min(wl.C, threads))
    # calibrate the per-spectrum cost on a short run over one round of channels
    T_probe = max(1, min(wl.T, 8))
    sub = _sub_workload(wl, list(range(C_s)), T_probe)
    t0 = time.perf_counter()
    oracle.workload_image(sub)
    per_t = (time.perf_counter() - t0) / T_probe          # one spectrum of every channel in the round
    T_s = int(max(1, min(wl.T, budget_s / max(per_t, 1e-9))))
    if T_s == wl.T:                                       # whole integrations fit: add channel rounds
        rounds = int(max(1, min(wl.C // C_s, budget_s / max(per_t * wl.T, 1e-9))))
        C_s = min(wl.C, C_s * rounds)
    chans = list(range(C_s))
    sub = _sub_workload(wl, chans, T_s)
    t0 = time.perf_counter()
    oracle.workload_image(sub)
    dt = time.perf_counter() - t0
    spectra = T_s * C_s * wl.n_pol
    return {"value": spectra / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"O1 (FP64 EPIC direct, own FFT) on {C_s} of {wl.C} channels x {T_s} of {wl.T} spectra "
                      f"x {wl.n_pol} pol = {spectra} spectra in {dt:.1f} s"}


def _sub_workload(wl, chans, T):
    import copy
    sub = copy.copy(wl)
    sub.v = wl.v[:T, chans]
    sub.gains = None if wl.gains is None else wl.gains[chans]
    sub.freq_hz = wl.freq_hz[chans]
    sub.grid_n = wl.grid_n[chans]
    sub.T = T
    return sub


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    wl = make_workload(args.workload, args.channels)
    threads = oracle.threads()
    C_s = max(1, min(wl.C, threads))
    chans = list(range(C_s))
    probe = _sub_workload(wl, chans, max(1, min(wl.T, 4)))
    t0 = time.perf_counter()
    oracle.workload_image(probe)
    per_t = (time.perf_counter() - t0) / probe.T
    # each step a bounded sample sized so the whole run ends within a few minutes
    T_s = int(max(1, min(wl.T, 150.0 / max(args.steps + args.warmup, 1) / max(per_t, 1e-9))))
    sub = _sub_workload(wl, chans, T_s)
    for _ in range(args.warmup):
        oracle.workload_image(sub)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.workload_image(sub)
        times.append(time.perf_counter() - t0)
    spectra = T_s * C_s * wl.n_pol
    mean = sum(times) / len(times)
    value = spectra / mean
    sample = (f"O1 (FP64 EPIC direct) per step on {C_s} of {wl.C} channels x {T_s} of {wl.T} spectra x "
              f"{wl.n_pol} pol = {spectra} spectra")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(wl, args.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def tensor_roofline(wl, form, img_ms, peaks, pair=True):
    """Executed tensor FLOPs of the tensor-core imaging launch over its time.
    Each 64-point DFT stage of one sample is 8 k-blocks x terms MMAs of
    128 x 128 x 16 (a side-96 48-point stage skips 2 of the 8 k-blocks).
    Grid sides 128 and 96 run two pixel classes per CTA from one row stage
    (pair kernel): 3 stage GEMMs per two classes; other sides (and these with
    EPIC_DIAG_NO_PAIR): 2 per class.  Also the method's algorithmic FLOPs (the
    FP32 FFT form's count) over the same time."""
    terms = 1 if form == "tc_fp16" else 3
    stage = 8 * terms * 2.0 * 128 * 128 * 16          # one 64-point stage: 8 k-blocks x terms MMAs
    stages = 0.0
    for n in wl.grid_n:
        n = int(n)
        fold = 48 if n == 96 else 64                    # side 96: 48-point DFTs, 6 of the 8 k-blocks
        classes = max(1, n // fold) ** 2
        per_class = 1.5 if (pair and n in (128, 96)) else 2.0
        stages += classes * per_class * (6.0 / 8.0 if n == 96 else 1.0)
    flops = stages * wl.T * stage
    ach = flops / (img_ms / 1e3) / 1e12
    peak = float(peaks.get("bf16_tflops", 1892.1))
    alg = sum(fp32_flops_per_spectrum(wl.A, wl.K, int(n)) for n in wl.grid_n) * wl.T * wl.n_pol
    sustained = float(peaks.get("bf16_tflops_sustained", 0.0)) or None
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "frac_of_sustained": (ach / sustained) if sustained else None,
            "traffic": None, "executed_flops_per_launch": flops, "ms_per_launch": img_ms,
            "stage_gemms_per_class_and_sample": stages / max(1, sum((int(n) // 64) ** 2 for n in wl.grid_n)),
            "algorithmic_flops_per_launch": alg, "algorithmic_tflops": alg / (img_ms / 1e3) / 1e12,
            "peak_source": "MEASURED_PEAKS bf16_tflops burst (dense FP16 rate equals BF16)"}


def fp32_roofline(wl, stages, peaks, sm_count):
    """The FP32 form's dominant imaging launch against the FP32 FMA peak derived
    from unit counts (alu bound): the method's algorithmic FLOPs of that grid
    side's channels over the launch's event-timed duration."""
    image_stage = max((n for n in stages if n.startswith("image[")), key=lambda n: stages[n])
    side = int(image_stage[8:-1])
    flops = sum(fp32_flops_per_spectrum(wl.A, wl.K, int(n)) for n in wl.grid_n if int(n) == side) * wl.T * wl.n_pol
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    ms = stages[image_stage]
    return {"bound": "alu", "kernel": f"FP32 imaging kernel {image_stage}", "achieved": flops / (ms / 1e3) / 1e12,
            "peak": peak, "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / peak, "traffic": None,
            "peak_source": f"derived: {sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz "
                           f"(max SM clock of MEASURED_PEAKS)",
            "flops_per_launch": flops, "ms_per_launch": ms}


def _time_steps(call, flush, args, stream):
    """Device time per step (CUDA events on the launching stream, L2 flushed between steps)."""
    import torch
    for _ in range(max(args.warmup, 1)):
        call()
    torch.cuda.synchronize()
    ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return sum(ms) / len(ms)


def time_variants(wl, v, g, out, flush, args, stream):
    """Other forms of the same integration, timed the same way (device events
    per step, L2 flushed between steps): the plain FP32 form, the taper and
    tensor forms (same output up to rounding), delay correction, per-antenna
    kernels, time-resolved Stokes images and the E-field images."""
    import numpy as np
    import torch

    from paper_2301_09662_gb300 import epic
    res = {}
    forms = {"fp32": dict(),
             "kernel_taper": dict(flags=epic.EPIC_KERNEL_TAPER),
             "tc_split_fp16": dict(precision=epic.EPIC_TC_SPLIT_FP16),
             "tc_fp16": dict(precision=epic.EPIC_TC_FP16),
             "tc_split_bf16": dict(precision=epic.EPIC_TC_SPLIT_BF16),
             "tc_split_fp16_taper": dict(precision=epic.EPIC_TC_SPLIT_FP16, flags=epic.EPIC_KERNEL_TAPER),
             "tc_split_fp16_one_class": dict(precision=epic.EPIC_TC_SPLIT_FP16, flags=epic.EPIC_DIAG_NO_PAIR),
             "fp32_delays": dict(),
             "fp32_antenna_kernels": dict(flags=epic.EPIC_ANTENNA_KERNELS),
             "fp32_series_stokes": dict(flags=epic.EPIC_STOKES),
             "fp32_efield": dict()}
    notes = {"fp32": "plain FP32 form: gather gridding, register 64-point FFTs on packed FP32 pairs, products "
                     "summed in registers (literal gridding)",
             "kernel_taper": "FP32; image-domain |W^|^2 taper with point gridding (exact for one shared kernel)",
             "tc_split_fp16": "row and column DFTs on tcgen05, FP16 hi+lo operands (3 MMAs per k-block), "
                              "FP32 accumulate in TMEM; at grid side 128 two pixel classes per CTA share one "
                              "gather gridding and one row stage",
             "tc_fp16": "row and column DFTs on tcgen05, single FP16 operands",
             "tc_split_bf16": "row and column DFTs on tcgen05, BF16 hi+lo operands (3 MMAs per k-block)",
             "tc_split_fp16_taper": "tc_split_fp16 with the image-domain kernel taper",
             "tc_split_fp16_one_class": "tc_split_fp16 with one pixel class per CTA at grid side 128 (each class "
                                        "grids the sample itself; the form before the pair kernel)",
             "fp32_delays": "FP32 literal form with per-(t, antenna) geometric-delay phases (epic_image_ex; "
                            "[T][A] FP64 delays resident in HBM, phases formed in the kernel)",
             "fp32_antenna_kernels": "FP32 literal form with a kernel per antenna (seeded Gaussians of +-20 % "
                                     "width and a small phase gradient); auto term sum_a A_a |W_a^|^2",
             "fp32_series_stokes": f"FP32 literal form, epic_image_series: one Stokes (I, Q, U, V) image per "
                                   f"{SERIES_SPI} spectra ({wl.T // SERIES_SPI if wl.T % SERIES_SPI == 0 else 0} "
                                   f"images per integration)",
             "fp32_efield": "epic_image_efield: the complex E-field image of every sample, channel and "
                            "polarisation (FP32 register kernel, no products), written to HBM"}
    import copy

    from paper_2301_09662_gb300 import synth
    delays = torch.from_numpy(synth.geometric_delays(wl.ant_xy, wl.T)).to(v.device)
    wl_ak = copy.copy(wl)
    wl_ak.kernel = synth.antenna_kernels(wl.A, wl.K, np.random.default_rng(20230120))
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    for name, kw in forms.items():
        series = name == "fp32_series_stokes"
        efield = name == "fp32_efield"
        if series and wl.T % SERIES_SPI:
            res[name] = {"unavailable": f"{wl.T} spectra are not a multiple of {SERIES_SPI}"}
            continue
        try:
            p = epic.Plan.from_workload(wl_ak if name == "fp32_antenna_kernels" else wl, **kw)
            if not args.no_autotune and not series and not efield:
                p.autotune(wl.T)
        except epic.EpicError as e:
            res[name] = {"unavailable": str(e)}
            continue
        p.set_profiling(not (series or efield))
        if series:
            o = torch.empty((wl.T // SERIES_SPI, out.numel()), dtype=out.dtype, device=out.device)
        elif efield:
            o = torch.empty((wl.T, int(epic.load().epic_efield_floats(p.handle)) // 2), dtype=torch.complex64,
                            device=out.device)
        else:
            o = torch.empty_like(out)
        dl = delays if name == "fp32_delays" else None

        def call():
            if series:
                p.image_series(v, SERIES_SPI, g, out=o)
            elif efield:
                p.image_efield(v, g, out=o)
            else:
                p.image(v, g, out=o, delays=dl)

        step = _time_steps(call, flush, args, stream)
        stages = None if (series or efield) else p.stage_times()   # series and E-field run unprofiled
        entry = {"value": wl.spectra / (step / 1e3), "unit": UNIT, "ms_per_step": step, "note": notes[name],
                 "stages_ms_last": stages}
        if name.startswith("tc_") and stages:
            img = max((x for k, x in stages.items() if k.startswith("image[")), default=None)
            if img:
                entry["roofline"] = tensor_roofline(wl, name.replace("_taper", "").replace("_one_class", ""), img,
                                                    peaks, pair=name != "tc_split_fp16_one_class")
        if name == "fp32" and stages:
            entry["roofline"] = fp32_roofline(wl, stages, peaks, sm_count)
            entry["roofline"]["traffic"] = ncu_record(NCU_TRAFFIC, "lwa", "fp32")
            entry["roofline"]["measured_limiter"] = ncu_record(NCU_LIMITER, "lwa", "fp32")
        if efield:
            out_bytes = o.numel() * 8
            in_bytes = v.numel() + (g.numel() * 8 if g is not None else 0)
            hbm = float(peaks.get("hbm_gbs", 6658.0))
            entry["hbm"] = {"bound": "hbm", "algorithmic_bytes": out_bytes + in_bytes,
                            "achieved": (out_bytes + in_bytes) / (step / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                            "frac": (out_bytes + in_bytes) / (step / 1e3) / 1e9 / hbm,
                            "peak_source": "MEASURED_PEAKS hbm_gbs"}
        res[name] = entry
        p.close()
        del o
    return res


def time_workloads(flush, args, stream):
    """The uneven-band (192 channels, grid sides 64/96/128) and dense-array
    (2048 antennas, 256 channels, grid side 512) integrations: FP32 and
    split-FP16 tensor forms (and the FP32 taper on the dense array), each with
    its dominant kernel's roofline."""
    import torch

    from paper_2301_09662_gb300 import epic, synth
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    res = {}
    for wname, fn in (("uneven", synth.uneven), ("dense", synth.dense)):
        wl = fn()
        v = torch.from_numpy(wl.v).cuda()
        g = torch.from_numpy(wl.gains).cuda()
        forms = {"fp32": dict(), "tc_split_fp16": dict(precision=epic.EPIC_TC_SPLIT_FP16)}
        if wname == "dense":
            forms["fp32_taper"] = dict(flags=epic.EPIC_KERNEL_TAPER)
        lines = {}
        for fname, kw in forms.items():
            try:
                p = epic.Plan.from_workload(wl, **kw)
                if not args.no_autotune:
                    p.autotune(wl.T)
            except epic.EpicError as e:
                lines[fname] = {"unavailable": str(e)}
                continue
            p.set_profiling(True)
            o = torch.empty(p.out_floats // 2, dtype=torch.complex64, device="cuda")
            step = _time_steps(lambda: p.image(v, g, out=o), flush, args, stream)
            stages = p.stage_times()
            entry = {"value": wl.spectra / (step / 1e3), "unit": UNIT, "ms_per_step": step, "stages_ms_last": stages}
            if fname.startswith("tc_"):
                # every side runs on the tensor cores in a tensor plan; the longest launch alone
                tc_stages = [k for k in stages if k.startswith("image[")]
                img_stage = max(tc_stages, key=lambda k: stages[k])
                side = int(img_stage[8:-1])
                sub = copy_with_side(wl, side)
                longest = tensor_roofline(sub, fname, stages[img_stage], peaks)
                longest["kernel"] = f"tensor-core imaging launch {img_stage}"
                if len(tc_stages) > 1:
                    # the side groups' launches overlap in one graph, so no launch's own duration
                    # measures it: the executed tensor work of all of them over the whole step
                    agg = tensor_roofline(wl, fname, step, peaks)
                    agg["kernel"] = "all tensor-core imaging launches of one integration (" + ", ".join(tc_stages) + ")"
                    agg["note"] = ("the side groups' launches overlap in one graph: executed tensor FLOPs of every "
                                   "group over the whole step (auto power and epilogues included)")
                    longest["note"] = ("this launch's time includes sharing the GPU with the other groups' "
                                       "launches")
                    agg["longest_launch"] = longest
                    entry["roofline"] = agg
                else:
                    entry["roofline"] = longest
            else:
                entry["roofline"] = fp32_roofline(wl, stages, peaks, sm_count)
            lines[fname] = entry
            p.close()
            del o
        res[wname] = {"config": describe(wl, wname), "forms": lines}
        del v, g
        torch.cuda.empty_cache()
    return res


def copy_with_side(wl, side):
    """The workload restricted to the channels of one grid side (for a per-launch roofline)."""
    import copy
    sub = copy.copy(wl)
    sub.grid_n = wl.grid_n[wl.grid_n == side]
    return sub


def time_calibration(plan, wl, v, flush, args, stream):
    """epic_solve_gains on the same integration (2 iterations, one calibrator
    direction), timed per call on the device like the imaging step."""
    import torch
    for _ in range(max(args.warmup, 1)):
        plan.solve_gains(v, 0.3, -0.2, 2)
    torch.cuda.synchronize()
    ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.solve_gains(v, 0.3, -0.2, 2)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    t = sum(ms) / len(ms)
    return {"what": "epic_solve_gains, 2 iterations, all channels and polarisations of the integration",
            "ms": t, "value": wl.spectra / (t / 1e3), "unit": UNIT}


def time_search(flush, args, stream):
    """De-dispersion + single-pulse search of an image cube shaped like the
    deployed system's output (64 x 64 pixels, 72 channels of 25 kHz at 42 MHz,
    40 ms frames), 512 frames, 128 trial DMs 0 .. 25.4 pc cm^-3, boxcars 1 .. 32;
    synthetic Gaussian intensities with a few broadband pulses.  Timed per step
    on the device (both calls), L2 flushed between steps; the de-dispersion's
    bound is its FP32 adds (C per output sample), the single-pulse search's the
    HBM read of the de-dispersed cube."""
    import numpy as np
    import torch

    from paper_2301_09662_gb300 import epic
    T, C, npix = 512, 72, 64 * 64
    freq = 42.1e6 + 25e3 * np.arange(C)
    dms = np.arange(128) * 0.2
    dt = 0.04
    s = epic.Search(freq, dt, dms, npix, T)
    gen = torch.Generator(device="cuda").manual_seed(20230120)
    cube = torch.randn((T, C, npix), generator=gen, device="cuda") + 10.0
    # sixteen broadband pulses (3 sigma in every channel of one frame) at seeded pixels and frames
    rng = np.random.default_rng(20230120)
    for _ in range(16):
        cube[int(rng.integers(T)), :, int(rng.integers(npix))] += 3.0
    dd = torch.empty((s.n_dm, s.t_out, npix), dtype=torch.float32, device="cuda")

    def step():
        s.dedisperse(cube, out=dd)
        return s.single_pulse(dd, threshold=7.0)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    ms_dd, ms_sp = [], []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        s.dedisperse(cube, out=dd)
        b.record(stream)
        s.single_pulse(dd, threshold=7.0)
        c.record(stream)
        c.synchronize()
        ms_dd.append(a.elapsed_time(b))
        ms_sp.append(b.elapsed_time(c))
    t_dd, t_sp = sum(ms_dd) / len(ms_dd), sum(ms_sp) / len(ms_sp)
    if s.status() != epic.EPIC_OK:
        raise RuntimeError("a bounded device-side wait of the de-dispersion ran out")
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6791.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    add_peak = sm_count * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12       # FP32 adds, T/s
    cube_b = T * C * npix * 4
    dd_b = s.n_dm * s.t_out * npix * 4
    adds = s.n_dm * s.t_out * npix * C
    res = {"metric": "searched cube samples/s (frame x channel x pixel)", "unit": "samples/s",
           "value": T * C * npix / ((t_dd + t_sp) / 1e3), "ms_per_step": t_dd + t_sp,
           "config": {"frames": T, "channels": C, "pixels": npix, "trial_dms": s.n_dm, "t_out": s.t_out,
                      "max_shift": s.max_shift, "widths": [1, 2, 4, 8, 16, 32], "dt_s": dt,
                      "l2": "flushed between timed steps (256 MiB write)"},
           "dedisperse": {"ms": t_dd, "bound": "alu", "adds_per_launch": adds,
                          "achieved": adds / (t_dd / 1e3) / 1e12, "peak": add_peak, "unit": "T FP32 adds/s",
                          "frac": adds / (t_dd / 1e3) / 1e12 / add_peak,
                          "peak_source": f"derived: {sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                         f"{sm_max:.0f} MHz",
                          "hbm": {"algorithmic_bytes": cube_b + dd_b,
                                  "achieved_gbs": (cube_b + dd_b) / (t_dd / 1e3) / 1e9, "peak_gbs": hbm,
                                  "frac": (cube_b + dd_b) / (t_dd / 1e3) / 1e9 / hbm}},
           "single_pulse": {"ms": t_sp, "bound": "hbm", "algorithmic_bytes": dd_b,
                            "achieved_gbs": dd_b / (t_sp / 1e3) / 1e9, "peak_gbs": hbm,
                            "frac": dd_b / (t_sp / 1e3) / 1e9 / hbm, "peak_source": "MEASURED_PEAKS hbm_gbs"}}
    s.close()
    return res


def run_e2e(plan, wl, args, world, barrier, spectra, band_spectra=None):
    """Same metric end to end through the host-buffer entry points, each step
    copying its pinned host voltages and gains in and its image out:
    `value` with the pipelined epic_image_host_async (steps queued back to back,
    the next upload and the previous download overlapping the current imaging;
    one epic_host_wait at the end, inside the timed region), `sync_value` with the
    blocking epic_image_host (copy in, image, copy out, one step at a time)."""
    import torch

    from paper_2301_09662_gb300 import shard
    vh = torch.from_numpy(wl.v).pin_memory()
    gh = None if wl.gains is None else torch.from_numpy(wl.gains).pin_memory()
    oh = [torch.empty(plan.out_floats // 2, dtype=torch.complex64).pin_memory() for _ in range(2)]
    for k in range(3):
        plan.image_host_async(vh, gh, out=oh[k & 1])
    plan.host_wait()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        plan.image_host_async(vh, gh, out=oh[k & 1])
    plan.host_wait()
    async_s = (time.perf_counter() - t0) / args.steps
    barrier()
    for _ in range(2):
        plan.image_host(vh, gh, out=oh[0])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        plan.image_host(vh, gh, out=oh[0])
        times.append(time.perf_counter() - t0)
    barrier()
    step_s = shard.max_over_ranks(async_s, device="cuda")
    sync_s = shard.max_over_ranks(sum(times) / len(times), device="cuda")

    def rate(sec):
        return shard.whole_job_rate(spectra, world, sec) if band_spectra is None else band_spectra / sec
    return {"value": rate(step_s), "unit": UNIT,
            "h2d_bytes_per_step": vh.numel() + (gh.numel() * 8 if gh is not None else 0),
            "d2h_bytes_per_step": oh[0].numel() * 8,
            "api": "epic_image_host_async (pipelined, two slots) + epic_host_wait",
            "sync_value": rate(sync_s), "sync_api": "epic_image_host (blocking)"}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2301_09662_gb300 import epic, shard

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    band = None
    if args.split_band and world > 1:
        # one fixed band: every rank plans and images its cost-balanced block of channels
        from paper_2301_09662_gb300 import synth
        band = make_workload(args.workload, args.channels, 0)
        mine, _, _ = shard.band_slice(band.grid_n, band.n_pol, world, rank)
        if not mine:
            raise SystemExit(f"rank {rank}: no channel of the {band.C}-channel band is left for this rank")
        wl = synth.select_channels(band, mine)
    else:
        wl = make_workload(args.workload, args.channels, rank)
    precision = {"fp32": epic.EPIC_FP32, "tc_split_fp16": epic.EPIC_TC_SPLIT_FP16, "tc_fp16": epic.EPIC_TC_FP16,
                 "tc_split_bf16": epic.EPIC_TC_SPLIT_BF16}[args.precision]
    plan = epic.Plan.from_workload(wl, precision=precision, flags=epic.EPIC_KERNEL_TAPER if args.taper else 0)
    if not args.no_autotune:
        plan.autotune(wl.T)      # plan-time launch-shape measurement, outside the timed region
    v = torch.from_numpy(wl.v).cuda()
    g = None if wl.gains is None else torch.from_numpy(wl.gains).cuda()
    out = torch.empty(plan.out_floats // 2, dtype=torch.complex64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    spectra = wl.spectra

    for _ in range(max(args.warmup, 0)):
        plan.image(v, g, out=out)
    torch.cuda.synchronize()
    if plan.status() != epic.EPIC_OK:
        raise RuntimeError("device status not OK after warm-up")

    names = plan.stage_names()
    stage_sum = {n: 0.0 for n in names}
    plan.set_profiling(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            plan.image(v, g, out=out)
            ends[k].record(stream)
            for n, ms in plan.stage_times().items():
                stage_sum[n] += ms
        torch.cuda.synchronize()
        barrier()
    plan.set_profiling(False)
    clocks = clk.summary()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    max_total_ms = shard.max_over_ranks(sum(step_ms), device="cuda")
    ms_per_step = max_total_ms / args.steps
    if band is None:
        value = shard.whole_job_rate(spectra, world, ms_per_step / 1e3)
    else:
        value = band.spectra / (ms_per_step / 1e3)
        # the finished band collected on rank 0, once, after the timed region
        whole = shard.assemble_band(out, band.grid_n, band.n_pol)
        if rank == 0 and whole.numel() != shard.packed_offsets(band.grid_n, band.n_pol)[-1]:
            raise RuntimeError("assembled band has the wrong size")
    launches = len(names) * args.steps

    # end to end through the host-buffer entry point: pinned inputs copied in,
    # image copied out, every step
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(plan, wl, args, world, barrier, spectra, None if band is None else band.spectra)


    # roofline of the dominant kernel (the fused imaging launch)
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    stages_avg = {n: stage_sum[n] / args.steps for n in names}
    image_stage = max((n for n in names if n.startswith("image[")), key=lambda n: stage_sum[n])
    img_ms = stages_avg[image_stage]
    config = describe(wl if band is None else band, args.workload)
    if band is not None:
        config["parallelism"] = f"one band split across {world} ranks by channel (cost-balanced), images gathered to rank 0"
    config["launch_shapes"] = "cost model" if args.no_autotune else "measured per channel group (epic_autotune)"
    config["form"] = args.precision + (" + image-domain kernel taper" if args.taper else " (literal gridding)")
    if args.precision == "fp32":
        roofline = fp32_roofline(wl, stages_avg, peaks, sm_count)
    else:
        roofline = tensor_roofline(wl, args.precision, img_ms, peaks)
        roofline["kernel"] = f"tensor-core imaging kernel {image_stage}"
    if args.channels is None and not args.taper:
        roofline["traffic"] = ncu_record(NCU_TRAFFIC, args.workload, args.precision)
        roofline["measured_limiter"] = ncu_record(NCU_LIMITER, args.workload, args.precision)
    dtype = "f32" if args.precision == "fp32" else \
        {"tc_split_fp16": "f16 hi+lo operands, f32 accumulate", "tc_fp16": "f16 operands, f32 accumulate",
         "tc_split_bf16": "bf16 hi+lo operands, f32 accumulate"}[args.precision]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak" if band is None else "strong",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic (seeded LWA-like layout, sky, noise, gains)",
        "config": config,
        "roofline": roofline,
        "stages_ms": stages_avg,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if not args.no_variants:
        line["variants"] = time_variants(wl, v, g, out, flush, args, stream)
        line["search"] = time_search(flush, args, stream)
        line["calibration"] = time_calibration(plan, wl, v, flush, args, stream)
    if not args.no_workloads and world == 1 and args.channels is None and args.workload == "lwa":
        line["workloads"] = time_workloads(flush, args, stream)
    if not args.no_peaks and world == 1:
        line["peaks_measured"] = measure_pipe_peaks()
        tc_probe = line["peaks_measured"].get("fp16_tc")
        if roofline.get("bound") == "tensor" and isinstance(tc_probe, float) and tc_probe > 0:
            # the same achieved rate against this run's own back-to-back 128 x 256 x 16 FP16 MMA probe
            roofline["frac_of_fp16_mma_probe"] = roofline["achieved"] / tc_probe
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.search_only:
        import torch
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        print(json.dumps(time_search(flush, args, torch.cuda.current_stream())), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
