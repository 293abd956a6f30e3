"""Shared test helpers: run the CUDA path through the C ABI and compare with the
oracle.  Imported by the test modules only."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1904_11422_gb300 import epic, synth

# FP32 path tolerance: max |GPU - oracle| over a plane, relative to the peak of
# the channel's image (max |XX|, |YY| of the oracle), as the target states.
TOL_FP32 = 1e-5

# Stated bounds of every transform, on the same scale, about three times the
# largest error measured on GB300 over the parity cases (random small arrays and
# a seeded sweep of 24 configurations, the station block at 64 x 64 and
# 128 x 128, saturated plane waves): compensated hi + lo transforms (three
# products, ~16 (BF16) or ~22 (FP16) mantissa bits per operand) 1.6e-5 (BF16)
# and 4.8e-6 (FP16), plain FP16 1.2e-3, plain BF16 1.6e-2, all at their worst
# on a three-antenna array, whose subtracted image peak is small beside the raw
# one (the station block's errors are ten to a hundred times smaller).  FP16
# keeps its bits only with its power-of-two operand scales.
TOL = {"fft_fp32": TOL_FP32, "dft_bf16x3": 5e-5, "dft_fp16x3": 2e-5, "dft_bf16": 5e-2, "dft_fp16": 5e-3}


def oracle_array(w: synth.Workload, gains="workload"):
    g = w.gains if isinstance(gains, str) else gains
    return oracle.OracleArray(w.ant_xy, w.freq_hz, w.n_pol, w.grid_n, w.support, w.cell_lambda,
                              w.sigma_cells, gains=g, delays=w.delays_s)


def oracle_image(w: synth.Workload, subtract=True, channels=None, use_fft=False, volts=None):
    arr = oracle_array(w)
    v = w.volts if volts is None else volts
    if channels is None:
        return oracle.image(arr, v, subtract=subtract, use_fft=use_fft)
    return np.stack([oracle.image(arr, v, subtract=subtract, c_lo=c, c_hi=c + 1, use_fft=use_fft)[0]
                     for c in channels])


def gpu_image(w: synth.Workload, xform=epic.EPIC_XFORM_FFT_FP32, subtract=True, volts=None, plan=None):
    import torch
    own = plan is None
    if own:
        plan = epic.plan_for(w, xform, subtract)
    v = w.volts if volts is None else volts
    dv = torch.from_numpy(np.ascontiguousarray(v)).cuda()
    out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    epic.epic_image(plan, dv, v.shape[0], out, 0)
    epic.epic_sync(plan)
    res = out.cpu().numpy()
    if own:
        plan.close()
    return res


def rel_errors(gpu, ref, n_pol):
    """[C][4] max |gpu - ref| per plane over the channel's image peak."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    C = ref.shape[0]
    out = np.zeros((C, 4))
    for c in range(C):
        peak = np.abs(ref[c, 0]).max() if n_pol == 1 else max(np.abs(ref[c, 0]).max(), np.abs(ref[c, 1]).max())
        peak = max(peak, 1e-30)
        for pl in range(4):
            out[c, pl] = np.abs(gpu[c, pl] - ref[c, pl]).max() / peak
    return out


def assert_close(gpu, ref, n_pol, tol=TOL_FP32):
    err = rel_errors(gpu, ref, n_pol)
    if n_pol == 1:
        assert np.all(np.asarray(gpu)[:, 1:] == 0.0), "single-pol planes 1-3 must be zero"
    assert err.max() <= tol, f"max relative error {err.max():.3e} > {tol:.1e} (per channel/plane: {err})"
    return err
