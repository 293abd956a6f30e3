"""The benchmark itself on a GPU: a short run prints one JSON line carrying the
contract's keys and this library's own evidence (roofline of the dominant
kernel, end-to-end rate through host buffers, kernel launches, clocks, the
per-image error table at both grid sides, the batch and the gradient), and the
channel-split mode reports strong scaling."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=900):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         timeout=timeout, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_short_bench_line_has_the_contract_and_evidence():
    d = _run("--steps", "3", "--warmup", "3", "--e2e-steps", "2", "--grad-steps", "2", "--grid128-steps", "2",
             "--grid128-paths", "fft_fp32", "--batch-steps", "2", "--soak-seconds", "0", "--paths", "dft_bf16x3",
             "--fma-iterations", "1000", "--cpu-seconds", "1", "--cpu-mode-seconds", "0",
             "--accuracy-paths", "fft_fp32,dft_bf16x3", "--accuracy128-seconds", "1")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert key in d, key
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 3 and d["scaling"] == "weak"
    r = d["roofline"]
    assert r["bound"] == "alu" and 0 < r["frac"] < 1.5 and r["kernel"] == "fft_image"
    assert d["e2e"]["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 40_960_000
    assert d["gpu_launches"] == 6  # an imaging kernel and a reduction per step
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    acc = d["accuracy"]
    for grid in ("grid64", "grid128"):
        errs = acc[grid]["errors"]
        for xf in ("fft_fp32", "dft_bf16x3"):
            e = errs[xf]
            assert 0 <= e["max"] <= e["bound"], (grid, xf, e)
            assert len(e["per_plane"]) == 4 and len(e["per_channel"]) >= 1
    assert d["paths"]["dft_bf16x3"]["roofline"]["bound"] == "tensor"
    assert d["batch"]["tensor"]["imaging_kernels_per_step"] == 1
    assert d["grad"]["ms_per_call"] > 0


def test_channel_split_mode_is_strong_scaling():
    d = _run("--steps", "3", "--warmup", "3", "--shard", "channels", "--no-cpu", "--e2e-steps", "0",
             "--grad-steps", "0", "--grid128-steps", "0", "--batch-steps", "0", "--soak-seconds", "0", "--paths=",
             "--fma-iterations", "0")
    assert d["scaling"] == "strong" and d["config"]["shard"] == "channels" and d["value"] > 0
