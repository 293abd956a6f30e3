#!/usr/bin/env python3
"""Throughput of E-field direct imaging (MOFF / EPIC) on an LWA-station-shaped block.

One step = one epic_image call over the station block: 256 dual-pol antennas,
64 channels spread over 60-76 MHz, 64x64 grid at 0.5-wavelength cells, 5x5
Gaussian kernel, 1250 samples (50 ms at 40 us), autocorrelations removed --
every step of the imaging path (unpack, calibrate, grid, 2-D FFT, XX/YY/XY,
accumulate, autocorrelation removal) in the library's kernels.

Prints one JSON line (rank 0).  Metric: antenna x channel x samples imaged per
second (whole job).  Inputs are 4 rotating device copies of the block (164 MB,
larger than L2).  ``--impl reference`` times the FP64 CPU oracle instead, on a
bounded sample of the same block per step.

Multi-GPU: ``--gpus N`` starts N ranks itself (under torch.distributed.run on
127.0.0.1) unless it already runs under a launcher.  ``--shard replicate``
(default): every rank images its own block (per-GPU work fixed, "weak");
``--shard channels``: the ranks split one block's channels (the paper's per-GPU
bandwidth split, "strong").  Neither has a collective in the data path (channels
are independent); the timing is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "antenna·chan·samples/s imaged, tensor-core vs FP32 path at stated err; %roofline"
UNIT = "antenna·chan·samples/s"
# The paper's per-GPU real-time capacity for 256 dual-pol antennas, 64^2 grid,
# 50 ms gulps: 16 channels x 25 000 samples/s x 256 antennas on a GTX 980.
PAPER_GTX980 = 16 * 25_000 * 256
WORKLOAD = ("station: 256 dual-pol antennas in a 110 m disk (min spacing 5 m), 64 channels of 25 kHz "
            "over 60-76 MHz, 64x64 grid at 0.5 wavelength, 5x5 Gaussian kernel, 1250 samples (50 ms) of "
            "4+4-bit noise + 3 point sources, XX/YY/XY FP32 images, autocorrelations removed")
N_COPIES = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--shard", default="replicate", choices=["replicate", "channels"],
                    help="multi-GPU: one block per rank (weak scaling) or one block's channels split (strong)")
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="epic", choices=["epic", "reference"])
    ap.add_argument("--xform", default="fft_fp32",
                    help="primary transform (the JSON value); see --paths for the others timed")
    ap.add_argument("--paths", default="dft_bf16x3,dft_fp16",
                    help="further transforms timed the same way and reported under 'paths' ('' for none)")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--fma-iterations", type=int, default=100000,
                    help="loop trips of the FMA-chain rate measurement (0: skip)")
    ap.add_argument("--cpu-mode-seconds", type=float, default=3.0,
                    help="seconds per additional oracle mode timed beside cpu_baseline (0: skip)")
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="CPU time budget of the whole --impl reference run")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--soak-seconds", type=float, default=1.5)
    ap.add_argument("--grid128-steps", type=int, default=20,
                    help="calls timed on the station block at 128 x 128 (0 to skip)")
    ap.add_argument("--grid128-paths", default="fft_fp32,dft_bf16x3,dft_fp16",
                    help="transforms timed on the station block at 128 x 128")
    ap.add_argument("--batch-steps", type=int, default=20,
                    help="graph launches timed for the batching workload (0 to skip)")
    ap.add_argument("--grad-steps", type=int, default=20,
                    help="epic_grad calls timed on the gain-calibration config (0: skip)")
    ap.add_argument("--accuracy-paths", default=ALL_XFORMS,
                    help="transforms whose per-image errors against the oracle are reported at 64^2 and 128^2")
    ap.add_argument("--accuracy128-seconds", type=float, default=10.0,
                    help="oracle seconds for the 128^2 error sample (0: skip)")
    return ap.parse_args()


def fp32_flops_per_tc(A, P, N, S):
    """Algorithmic FP32 flops of one (time, channel) image set on the FFT path."""
    import math
    calib = 6 * A * P                            # complex x integer sample
    grid = 4 * A * S * S * P                     # real weight x complex, accumulated
    fft = P * 5 * N * N * int(math.log2(N * N))  # 5 N^2 log2(N^2) per 2-D FFT
    prod = N * N * (4 if P == 1 else 16)         # |X|^2, |Y|^2, X conj(Y), accumulated
    return calib + grid + fft + prod


# Error bound stated for each transform, relative to the channel's image peak
# (checked against the FP64 oracle by the parity tests, which state how each
# was chosen).
ERROR_BOUND = {"fft_fp32": 1e-5, "dft_bf16x3": 5e-5, "dft_fp16x3": 2e-5, "dft_fp16": 5e-3, "dft_bf16": 5e-2}
ALL_XFORMS = "fft_fp32,dft_bf16x3,dft_fp16x3,dft_bf16,dft_fp16"


def tensor_flops_per_tc(xform):
    """Issued tensor-core flops of one (time, channel) image set: two stages of an
    M = N = K = 128 real GEMM, times 3 for the hi+lo transforms."""
    products = 3 if xform.endswith("x3") else 1
    return products * 2 * (2 * 128 * 128 * 128)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def strip_comments(src):
    """C/CUDA source without its comments and with whitespace runs collapsed:
    edits to comments or layout leave it unchanged, any change to the code does
    not."""
    out, i, n = [], 0, len(src)
    while i < n:
        ch = src[i]
        if ch in "\"'":  # a string or character literal, copied whole
            j = i + 1
            while j < n and src[j] != ch:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(ch)
            i += 1
    return " ".join("".join(out).split())


def src_sha(name):
    """Hash of a kernel source's code (comments and layout excluded), which keys
    the ncu traffic figures taken on it."""
    with open(os.path.join(ROOT, "paper_1904_11422_gb300", "csrc", name), encoding="utf-8") as f:
        return hashlib.sha256(strip_comments(f.read()).encode()).hexdigest()[:16]


def dram_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if the code of the
    kernel's source file is unchanged since it was taken; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f).get(kernel)
        if rec and rec.get("source_sha") == src_sha(rec["source"]):
            return rec["bytes_per_launch"]
    except Exception:
        pass
    return None


# --------------------------------------------------------------------------
def _oracle_setup(w):
    import oracle
    oracle.build()
    arr = oracle.OracleArray(w.ant_xy, w.freq_hz, w.n_pol, w.grid_n, w.support, w.cell_lambda, w.sigma_cells)
    return oracle, arr, oracle.max_threads()


def _oracle_sample(oracle, arr, w, cores, target_s, keep=None):
    """Grow a sample of the block (channels first up to the core count, then
    samples, then more channels) until one oracle run takes about target_s.
    Returns (n_chan, n_time, seconds of the last run); keep (a dict), if given,
    receives the last run's images."""
    n_c, n_t = min(cores, w.n_chan), 1
    while True:
        t0 = time.perf_counter()
        img = oracle.image(arr, w.volts[:n_t], subtract=True, c_lo=0, c_hi=n_c, use_fft=True, n_threads=cores)
        dt = time.perf_counter() - t0
        if dt >= 0.8 * target_s or (n_t == w.n_time and n_c == w.n_chan):
            if keep is not None:
                keep["image"] = img
            return n_c, n_t, dt
        grow = max(2.0, min(8.0, target_s / max(dt, 1e-3)))
        if n_t < w.n_time:
            n_t = min(w.n_time, int(n_t * grow) + 1)
        else:
            n_c = min(w.n_chan, int(n_c * grow) + 1)


def cpu_oracle_rate(w, seconds):
    """The FP64 oracle (FFT mode, as it stands) on a bounded sample of the block,
    all host cores.  Returns (units/s, cores, sample description, (n_chan,
    n_time, oracle images of the sample))."""
    oracle, arr, cores = _oracle_setup(w)
    keep = {}
    n_c, n_t, dt = _oracle_sample(oracle, arr, w, cores, seconds, keep)
    units = w.n_ant * n_c * n_t
    sample = (f"{n_c} channels x {n_t} samples x {w.n_ant} antennas of the station block, "
              f"FP64 oracle FFT mode with autocorrelation removal, {cores} OpenMP threads, {dt:.1f} s")
    return units / dt, cores, sample, (n_c, n_t, keep["image"])


def measured_errors(epic, torch, w, dv, xforms, n_c, n_t, ref):
    """Each transform's images of the oracle's sample (the first n_t samples,
    channels 0 .. n_c-1) against the oracle's: per image (channel c, plane XX,
    YY, Re XY, Im XY), max |GPU - oracle| / the channel's image peak
    max(|XX|, |YY|) of the oracle.  Returns {xform: {"max", "per_plane" (max over
    channels), "per_channel" (max over planes), "bound"}}."""
    import numpy as np
    peak = np.maximum(np.abs(ref[:, 0]).max(axis=(1, 2)), np.abs(ref[:, 1]).max(axis=(1, 2)))
    errs = {}
    for xf in xforms:
        plan = epic.plan_for(w, epic.XFORMS[xf], subtract_autos=True)
        out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
        epic.epic_image(plan, dv[:n_t], n_t, out, 0)
        epic.epic_sync(plan)
        got = out[:n_c].double().cpu().numpy()
        plan.close()
        e = np.abs(got - ref).max(axis=(2, 3)) / peak[:, None]  # [C][4]
        errs[xf] = {"max": float(e.max()), "bound": ERROR_BOUND.get(xf),
                    "per_plane": [float(f"{x:.3g}") for x in e.max(axis=0)],
                    "per_channel": [float(f"{x:.3g}") for x in e.max(axis=1)]}
    return errs


def accuracy128(epic, torch, synth, xforms, seconds):
    """The per-image errors of every transform on the station block at 128 x 128
    against the oracle (FFT mode, all host cores) on a bounded sample of it."""
    w = synth.station(grid_n=128)
    oracle, arr, cores = _oracle_setup(w)
    keep = {}
    n_c, n_t, dt = _oracle_sample(oracle, arr, w, cores, seconds, keep)
    dv = torch.from_numpy(w.volts).cuda()
    errs = measured_errors(epic, torch, w, dv, xforms, n_c, n_t, keep["image"])
    return {"errors": errs,
            "sample": f"{n_c} channels x {n_t} samples x {w.n_ant} antennas of the station block on a 128x128 "
                      f"grid, FP64 oracle FFT mode, {cores} OpenMP threads, {dt:.1f} s"}


def _grow(run, n_max, target_s):
    """Smallest n (doubling from 1, at most n_max) whose run(n) takes about
    target_s seconds; returns (n, seconds)."""
    n = 1
    while True:
        t0 = time.perf_counter()
        run(n)
        dt = time.perf_counter() - t0
        if dt >= 0.8 * target_s or n == n_max:
            return n, dt
        n = min(n_max, max(n + 1, int(n * min(8.0, target_s / max(dt, 1e-3)))))


def cpu_oracle_modes(w, seconds):
    """The oracle's other modes, each on a bounded sample of the station block
    (about `seconds` each): the FFT mode on one thread, the direct separable DFT
    on all cores, and the gridded FX image (visibilities of every antenna pair,
    gridded with the kernels' cross-correlations, one transform; one thread).
    Returns {mode: {"value", "unit", "cores", "sample"}}."""
    oracle, arr, cores = _oracle_setup(w)
    out = {}

    def fft1(n_t):
        oracle.image(arr, w.volts[:n_t], subtract=True, c_lo=0, c_hi=1, use_fft=True, n_threads=1)

    def direct(n_t):
        oracle.image(arr, w.volts[:n_t], subtract=True, c_lo=0, c_hi=min(cores, w.n_chan), use_fft=False,
                     n_threads=cores)

    def fx(n_t):
        oracle.fx_gridded(arr, w.volts[:n_t], 0, include_autos=False)

    for mode, fn, n_c, thr, what in [
            ("fft_1thread", fft1, 1, 1, "FFT mode"),
            ("direct_dft", direct, min(cores, w.n_chan), cores, "direct separable DFT"),
            ("fx_gridded", fx, 1, 1, "gridded FX (visibilities, kernel cross-correlations, one DFT)")]:
        n_t, dt = _grow(fn, w.n_time, seconds)
        out[mode] = {"value": w.n_ant * n_c * n_t / dt, "unit": UNIT, "cores": thr,
                     "sample": f"{n_c} channels x {n_t} samples x {w.n_ant} antennas, FP64 oracle {what}, "
                               f"{thr} thread(s), {dt:.1f} s"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1904_11422_gb300 import synth
    w = synth.station()
    budget = args.ref_seconds  # seconds for the whole reference run
    per_step = max(0.2, budget / max(1, args.steps + args.warmup))
    oracle, arr, cores = _oracle_setup(w)
    n_c, n_t, _ = _oracle_sample(oracle, arr, w, cores, per_step)

    def step():
        oracle.image(arr, w.volts[:n_t], subtract=True, c_lo=0, c_hi=n_c, use_fft=True, n_threads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    units = w.n_ant * n_c * n_t
    value = units * args.steps / dt
    sample = (f"per step {n_c} channels x {n_t} samples x {w.n_ant} antennas of the station block, "
              f"FP64 oracle FFT mode with autocorrelation removal, {cores} OpenMP threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_GTX980, "dtype": "f64",
            "data": "synthetic (seeded, LWA-station-shaped)",
            "config": {"workload": WORKLOAD, "xform": "oracle FFT mode (FP64, CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
def time_grid128(args, epic, synth, torch, stream, world, shard, sms, pk, pk_kind):
    """The station block imaged on a 2x padded 128 x 128 grid (the precision
    study's 128^2 variant): the FP32 path (clusters of two CTAs) and the tensor
    paths (four 64 x 64 DFT-GEMMs per image set), each with its kernel's
    fraction of its roofline."""
    w = synth.station(grid_n=128)
    dv = [torch.from_numpy(w.volts).cuda() for _ in range(2)]
    res = {"workload": "station block (256 dual-pol antennas, 64 channels, 1250 samples, 5x5) on a 2x padded "
                       "128x128 grid"}
    for xf in [x for x in args.grid128_paths.split(",") if x]:
        plan = epic.plan_for(w, epic.XFORMS[xf])
        out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
        for i in range(3):
            epic.epic_image(plan, dv[i % 2], w.n_time, out, 0, stream)
        torch.cuda.synchronize()
        epic.epic_timing_enable(plan, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.grid128_steps):
            epic.epic_image(plan, dv[i % 2], w.n_time, out, 0, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = shard.max_over_ranks(e0.elapsed_time(e1) / args.grid128_steps, device="cuda")
        kt = epic.epic_timing_read(plan)
        epic.epic_timing_enable(plan, False)
        epic.epic_sync(plan)
        kname = "fft_image" if xf == "fft_fp32" else "dft_image"
        n, tot = kt[kname]
        avg_s = tot / n / 1e3
        if xf == "fft_fp32":
            flops = w.n_chan * w.n_time * fp32_flops_per_tc(w.n_ant, w.n_pol, w.grid_n, w.support)
            peak = sms * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            clustered = plan.info["cluster_dim"] == 2
            roof = {"bound": "alu",
                    "kernel": ("fft128_image (2-CTA clusters)" if clustered else
                               "fft_image (each image set as four folded 64x64 problems)"),
                    "traffic": (dram_traffic("fft128_image") if clustered else
                                dram_traffic("fft_image_128fold")),
                    "peak_basis": f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x "
                                  f"{pk.get('sm_max_mhz', 2070.0):.0f} MHz ({pk_kind})"}
        else:
            flops = w.n_chan * w.n_time * 4 * tensor_flops_per_tc(xf)
            peak = pk.get("bf16_tflops", 1900.0)
            roof = {"bound": "tensor", "kernel": "dft_image (4 parity sub-problems of 64x64 per image set)",
                    "traffic": dram_traffic("dft_image_128") if xf == "dft_bf16x3" else None,
                    "peak_basis": f"measured dense BF16 cuBLAS burst ({pk_kind})",
                    "useful_tflops": flops / (3 if xf.endswith("x3") else 1) / avg_s / 1e12}
        roof.update({"achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": flops / avg_s / 1e12 / peak, "kernel_ms": 1e3 * avg_s, "flops_per_launch": flops})
        res[xf] = {"ms_per_call": ms, "value": w.units * world / (ms / 1e3), "unit": UNIT,
                   "error_bound": ERROR_BOUND[xf], "roofline": roof,
                   "kernel_times_ms": {k: {"launches": v[0], "total_ms": v[1]} for k, v in kt.items()}}
        plan.close()
    return res


def time_batch(args, epic, synth, torch, stream, world, shard, pk, pk_kind):
    """Arrays A, B and C of the batching recipe (T = 1250 each) in one autotuned
    graph launch, three times: every array on the FP32 path, on the compensated
    BF16 tensor-core path, and on the plain FP16 tensor-core path (error 1.6e-4 of
    the image peak on the station block).  The same plans imaged by separate
    epic_image calls one after another are timed for comparison."""
    ws = [synth.batching_array(k) for k in ("A", "B", "C")]
    vols = [torch.from_numpy(w.volts).cuda() for w in ws]

    def timed(fn, n):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return shard.max_over_ranks(e0.elapsed_time(e1) / n, device="cuda")

    res = {}
    for name, xforms in (("fp32", ["fft_fp32"] * 3), ("tensor", ["dft_bf16x3"] * 3),
                         ("tensor_fp16", ["dft_fp16"] * 3)):
        plans = [epic.plan_for(w, epic.XFORMS[x]) for w, x in zip(ws, xforms)]
        outs = [torch.empty(p.out_shape, dtype=torch.float32, device="cuda") for p in plans]
        b = epic.epic_batch_create(plans, vols, [w.n_time for w in ws], outs, tune=True, stream=stream)
        ms = timed(lambda: epic.epic_batch_launch(b, stream), args.batch_steps)

        def separate():
            for p, v, w, o in zip(plans, vols, ws, outs):
                epic.epic_image(p, v, w.n_time, o, 0, stream)

        ms_sep = timed(separate, args.batch_steps)
        units = sum(w.units for w in ws)
        r = {"ms_per_launch": ms, "value": units * world / (ms / 1e3), "unit": UNIT, "units_per_launch": units,
             "xforms": dict(zip([w.name for w in ws], xforms)), "ctas_chosen": dict(zip([w.name for w in ws], b.ctas)),
             "ms_separate_calls": ms_sep, "graph_launches_per_step": 1,
             # FP32 plans: an imaging kernel each (and a reduction); tensor-core plans of one
             # transform: one persistent kernel that images them all (and, as the tuner
             # chose, reduces them too, or leaves that to one reduction per plan)
             "imaging_kernels_per_step": sum(x == "fft_fp32" for x in xforms)
                                         + len({x for x in xforms if x != "fft_fp32"})}
        if name != "fp32":
            # issued tensor-core flops of the batch over the graph time (a 32^2
            # image set is one 64^2 transform, a 128^2 one four)
            fl = sum(w.n_chan * w.n_time * (4 if w.grid_n == 128 else 1) * tensor_flops_per_tc(x)
                     for w, x in zip(ws, xforms))
            peak = pk.get("bf16_tflops", 1900.0)
            r["roofline"] = {"bound": "tensor", "achieved": fl / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                             "frac": fl / (ms / 1e3) / 1e12 / peak, "flops_per_launch": fl,
                             "basis": f"issued {xforms[0]} tensor flops of arrays A, B and C over the whole "
                                      f"graph time; peak: measured dense BF16 cuBLAS burst ({pk_kind}; "
                                      f"FP16 dense rate taken equal)"}
        else:
            # algorithmic FP32 flops of the batch (each grid's transform counted as
            # one N x N FFT, as in the single-plan rooflines) over the graph time
            fl = sum(w.n_chan * w.n_time * fp32_flops_per_tc(w.n_ant, w.n_pol, w.grid_n, w.support) for w in ws)
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            peak = sms * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            r["roofline"] = {"bound": "alu", "achieved": fl / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                             "frac": fl / (ms / 1e3) / 1e12 / peak, "flops_per_launch": fl,
                             "basis": f"algorithmic FP32 flops of arrays A, B and C over the whole graph time; "
                                      f"peak derived: {sms} SMs x 128 FP32 lanes x 2 flop x "
                                      f"{pk.get('sm_max_mhz', 2070.0):.0f} MHz ({pk_kind})"}
        res[name] = r
        b.close()
        for p in plans:
            p.close()
    res["workload"] = "batching arrays A (64 ants, 32x32, 16 ch) + B (station, 64x64, 64 ch) + C (1024 ants, " \
                      "220 m, 128x128, 32 ch), T = 1250 each, one graph launch"
    return res


def torchrun_command(argv, n_gpus, port):
    """The command that runs this script as n_gpus ranks on one node (one rank
    per GPU, rendezvous on 127.0.0.1)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n_gpus}",
            "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + list(argv)


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # started without a launcher: start the ranks (each sees WORLD_SIZE)
        return subprocess.call(torchrun_command(sys.argv[1:], args.gpus, _free_port()))
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    from paper_1904_11422_gb300 import build_lib, epic, shard, synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build_lib.build()
    if dist is not None:
        dist.barrier()

    block = synth.station()
    # this rank's share of the band: the whole block, or its channel range of it
    c_lo, c_hi = shard.rank_channels(block.n_chan, rank, world, args.shard)
    w = block if (c_lo, c_hi) == (0, block.n_chan) else synth.channel_slice(block, c_lo, c_hi)
    T = w.n_time
    copies = [torch.from_numpy(w.volts).cuda() for _ in range(N_COPIES)]
    stream = torch.cuda.current_stream()
    pk, pk_kind = peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()

    def time_path(xf, soak):
        plan = epic.plan_for(w, epic.XFORMS[xf], subtract_autos=True)
        out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")

        def step(i):
            epic.epic_image(plan, copies[i % N_COPIES], T, out, 0, stream)

        for i in range(max(3, args.warmup)):
            step(i)
        torch.cuda.synchronize()
        epic.epic_sync(plan)
        t_soak = time.perf_counter()
        i = 0
        while time.perf_counter() - t_soak < soak:  # untimed load, for the clock record
            step(i)
            i += 1
            if i % 50 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        epic.epic_timing_enable(plan, True)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(args.steps):
            step(i)
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        kt = epic.epic_timing_read(plan)
        epic.epic_timing_enable(plan, False)
        epic.epic_sync(plan)
        ms = shard.max_over_ranks(ms, device="cuda")
        value = shard.job_units(block.units, world, args.shard) * args.steps / (ms / 1e3)
        launches = sum(v[0] for v in kt.values())
        dom = max(kt.items(), key=lambda kv: kv[1][1])[0]
        n, tot = kt[dom]
        avg_s = tot / n / 1e3
        share = tot / sum(v[1] for v in kt.values())
        if dom == "fft_image":
            flops = w.n_chan * T * fp32_flops_per_tc(w.n_ant, w.n_pol, w.grid_n, w.support)
            peak = sms * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "traffic": dram_traffic("fft_image"), "kernel": dom,
                    "peak_basis": f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x "
                                  f"{pk.get('sm_max_mhz', 2070.0):.0f} MHz (max SM clock, {pk_kind})"}
        else:
            flops = w.n_chan * T * tensor_flops_per_tc(xf)
            peak = pk.get("bf16_tflops", 1900.0)
            roof = {"bound": "tensor", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "traffic": dram_traffic("dft_image"), "kernel": dom,
                    "peak_basis": f"measured dense BF16 cuBLAS burst ({pk_kind}); FP16 dense rate taken equal",
                    "useful_tflops": flops / (3 if xf.endswith("x3") else 1) / avg_s / 1e12}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof.update({"kernel_ms": 1e3 * avg_s, "kernel_share": share, "flops_per_launch": flops})
        res = {"value": value, "ms_per_step": ms / args.steps, "roofline": roof, "gpu_launches": launches,
               "error_bound": ERROR_BOUND.get(xf), "kernel_times_ms": {k: {"launches": v[0], "total_ms": v[1]}
                                                                       for k, v in kt.items()}}
        return plan, res

    plan, primary = time_path(args.xform, args.soak_seconds)
    others = {}
    for xf in [x for x in args.paths.split(",") if x and x != args.xform]:
        p2, r2 = time_path(xf, 0.0)
        p2.close()
        others[xf] = r2
    clocks = sampler.stop()
    units_step = shard.job_units(block.units, world, args.shard)
    value = primary["value"]
    ms = primary["ms_per_step"] * args.steps

    # end to end through the public host-buffer entry point
    e2e = None
    if args.e2e_steps > 0:
        # N_COPIES rotating pinned input blocks (larger than L2 together), as on the
        # device path, and as many pinned result buffers
        h_ins, h_outs = [], []
        for _ in range(N_COPIES):
            h = torch.empty(w.volts.shape, dtype=torch.uint8, pin_memory=True)
            h.numpy()[...] = w.volts
            h_ins.append(h)
            h_outs.append(torch.empty(plan.out_shape, dtype=torch.float32, pin_memory=True))

        def host_steps(call, inputs, n):
            for i in range(n):
                call(plan, inputs[i % len(inputs)], T, h_outs[i % len(h_outs)], 0, stream)
            epic.epic_sync(plan, stream)

        def timed_host(call, inputs):
            host_steps(call, inputs, 3)
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
            host_steps(call, inputs, args.e2e_steps)
            return shard.max_over_ranks(time.perf_counter() - t0, device="cuda")

        def rate(dt):
            return shard.job_units(block.units, world, args.shard) * args.e2e_steps / dt

        dt = timed_host(epic.epic_image_host_async, h_ins)
        dt_sync = timed_host(epic.epic_image_host, h_ins)
        dt_pageable = timed_host(epic.epic_image_host, [np.ascontiguousarray(w.volts) for _ in range(N_COPIES)])
        e2e = {"value": rate(dt), "unit": UNIT,
               "h2d_bytes_per_step": int(w.volts.nbytes), "d2h_bytes_per_step": int(h_outs[0].numel() * 4),
               "steps": args.e2e_steps,
               "api": "epic_image_host_async: pinned host buffers, every step copies its block to the device "
                      "and its images back; the next block's copy overlaps this block's imaging; one "
                      "epic_sync after the last step",
               "synchronous_call": {"value": rate(dt_sync), "api": "epic_image_host (pinned; copy, image, copy "
                                                                    "back, wait, per step)"},
               "pageable_input": {"value": rate(dt_pageable), "api": "epic_image_host from pageable memory"}}

    # gain calibration (differentiation config): loss + gradient per block
    grad = None
    if args.grad_steps > 0:
        wg, sky = synth.differentiation()
        gplan = epic.plan_for(wg)
        dvg = torch.from_numpy(wg.volts).cuda()
        model_full = torch.empty(gplan.out_shape, dtype=torch.float32, device="cuda")
        splan = epic.plan_for(sky)  # model: the noise-free 5-source sky imaged with unit gains
        epic.epic_image(splan, torch.from_numpy(sky.volts).cuda(), sky.n_time, model_full, 0)
        model = model_full[:, :2].contiguous()
        gains = torch.from_numpy(np.stack([wg.gains.real, wg.gains.imag], -1).astype(np.float32)).cuda()
        g_out = torch.empty_like(gains)
        loss = torch.empty((), dtype=torch.float32, device="cuda")
        for _ in range(3):
            epic.epic_grad(gplan, dvg, wg.n_time, gains, model, g_out, loss)
        torch.cuda.synchronize()
        epic.epic_timing_enable(gplan, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.grad_steps):
            epic.epic_grad(gplan, dvg, wg.n_time, gains, model, g_out, loss)
        e1.record(stream)
        torch.cuda.synchronize()
        gms = e0.elapsed_time(e1) / args.grad_steps
        gkt = epic.epic_timing_read(gplan)
        grad = {"workload": "gain calibration: station block with seeded gains (|g| 1 +- 0.1, phase +- 0.3 rad), "
                            "model = 5-source noise-free sky imaged with unit gains",
                "ms_per_call": gms, "value": wg.units / (gms / 1e3), "unit": UNIT,
                "loss": float(loss.item()),
                "kernel_times_ms": {k: {"launches": v[0], "total_ms": v[1]} for k, v in gkt.items()}}
        gplan.close()
        splan.close()

    # the precision study's 128 x 128 variant of the station block
    grid128 = None
    if args.grid128_steps > 0:
        grid128 = time_grid128(args, epic, synth, torch, stream, world, shard, sms, pk, pk_kind)

    # batching: the arrays of the batching recipe imaged by one graph launch
    batch = None
    if args.batch_steps > 0:
        batch = time_batch(args, epic, synth, torch, stream, world, shard, pk, pk_kind)

    # the FP32 roofline's derived peak against a measured FMA-chain rate (after
    # the timed regions, so it does not heat the GPU before them)
    if args.fma_iterations > 0:
        fma = epic.epic_debug_fma_rate(args.fma_iterations, stream)
        roofs = [primary["roofline"]] + [r["roofline"] for r in (grid128 or {}).values()
                                          if isinstance(r, dict) and "roofline" in r]
        for roof in roofs:
            if roof.get("bound") == "alu":
                roof["fma_chain_tflops"] = fma
                roof["fma_chain_of_peak"] = fma / roof["peak"]

    cpu, accuracy = None, None
    if rank == 0 and world == 1 and not args.no_cpu and w is block:
        rate, cores, sample, (n_c, n_t, ref) = cpu_oracle_rate(w, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        # every transform's images of the same sample against the oracle's images,
        # per image (channel, plane), at 64 x 64 and on the 128 x 128 variant
        xfs = [x for x in args.accuracy_paths.split(",") if x]
        errs = measured_errors(epic, torch, w, copies[0], xfs, n_c, n_t, ref)
        accuracy = {"max_error_vs_oracle": {x: e["max"] for x, e in errs.items()},
                    "error_bound": {x: ERROR_BOUND.get(x) for x in xfs},
                    "measure": "per image (channel, plane): max over pixels of |GPU - FP64 oracle| / the "
                               "channel's image peak; per_plane = max over channels, per_channel = max over planes",
                    "grid64": {"errors": errs, "sample": sample}}
        if args.accuracy128_seconds > 0:
            accuracy["grid128"] = accuracy128(epic, torch, synth, xfs, args.accuracy128_seconds)
        if args.cpu_mode_seconds > 0:
            cpu["modes"] = cpu_oracle_modes(w, args.cpu_mode_seconds)

    plan.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": shard.scaling(args.shard), "vs_baseline": value / PAPER_GTX980,
                "dtype": "f32" if args.xform == "fft_fp32" else args.xform,
                "data": "synthetic (seeded, LWA-station-shaped; no LWA-SV captures exist here)",
                "config": {"workload": WORKLOAD, "xform": args.xform, "units_per_step": units_step,
                           "error_bound": ERROR_BOUND.get(args.xform),
                           "parallelism": (f"one block per GPU x {world}" if args.shard == "replicate" else
                                           f"one block's 64 channels split over {world} GPUs"),
                           "shard": args.shard,
                           "l2": f"inputs larger than L2: {N_COPIES} rotating device copies of the block "
                                 f"({N_COPIES * w.volts.nbytes / 1e6:.0f} MB)"},
                "roofline": primary["roofline"], "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": primary["gpu_launches"], "kernel_times_ms": primary["kernel_times_ms"],
                "paths": others, "grad": grad, "grid128": grid128, "batch": batch, "accuracy": accuracy,
                # seconds of data per block (40 us samples of 25 kHz channels) over seconds per block
                "real_time_factor": (T * 40e-6) / (ms / args.steps / 1e3),
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
