"""The benchmark's reference arm (the FP64 oracle timed on the host cores) runs
on a CPU-only machine and prints one JSON line with the keys the benchmark
contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-seconds", "4"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_source_hash_ignores_comments_but_not_code():
    b = _bench()
    code = 'int f(int a) { return a + 1; }  // adds one\nconst char* s = "// kept";\n'
    assert b.strip_comments(code) == b.strip_comments("/* doc */ int f(int a)\n{ return a + 1; }\n"
                                                      'const char* s = "// kept";')
    assert b.strip_comments(code) != b.strip_comments(code.replace("a + 1", "a + 2"))
    assert '"// kept"' in b.strip_comments(code)


def test_traffic_records_are_reported_only_for_the_code_they_were_taken_on():
    """Each ncu traffic record names its summary and its kernel source; the
    benchmark reports its bytes while the source's code hash matches the
    recorded one and null once the kernel has changed."""
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        recs = json.load(f)
    assert {"fft_image", "dft_image"} <= set(recs)
    for name, rec in recs.items():
        assert rec["bytes_per_launch"] == rec["read_bytes"] + rec["write_bytes"], name
        assert os.path.exists(os.path.join(ROOT, rec["summary"])), name
        current = rec["source_sha"] == b.src_sha(rec["source"])
        assert b.dram_traffic(name) == (rec["bytes_per_launch"] if current else None), name


def test_flop_model_matches_the_papers_grid_scaling():
    """The FFT term of the benchmark's flop model grows as N^2 log2(N^2): from a
    64^2 to a 128^2 grid by (128^2 x 14) / (64^2 x 12) = 4.67, the theoretical
    factor the paper quotes for its grid-size scaling (Sec. 5)."""
    b = _bench()
    fft = lambda n: b.fp32_flops_per_tc(0, 1, n, 1) - n * n * 4  # one polarisation, no antennas
    assert abs(fft(128) / fft(64) - (128 ** 2 * 14) / (64 ** 2 * 12)) < 1e-12
    assert abs(fft(128) / fft(64) - 4.67) < 0.005
    # and the station figure: 2 388 algorithmic flops per antenna-channel-sample on the 64^2 FP32 path
    assert round(b.fp32_flops_per_tc(256, 2, 64, 5) / 256) == 2388
