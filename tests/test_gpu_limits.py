"""Parity at the largest accepted sizes: the most antennas each transform takes
on each grid side (2048 on the FP32 path, 1024 on the tensor path), and the
widest kernel support (15 x 15 boxes), where the gather tables no longer fit in
shared memory and are read from L2."""
import numpy as np
import pytest

from paper_1904_11422_gb300 import build_lib, epic, synth

from _helpers import TOL, TOL_FP32, gpu_image, oracle_image, rel_errors

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return epic.load_library()


@pytest.mark.parametrize("xf,grid_n,n_ant,support", [
    ("fft_fp32", 32, 2048, 1),
    ("fft_fp32", 64, 2048, 3),
    ("fft_fp32", 128, 2048, 3),
    ("dft_bf16x3", 32, 1024, 3),
    ("dft_bf16x3", 64, 1024, 5),
    ("dft_bf16x3", 128, 1024, 3),
])
def test_most_antennas(xf, grid_n, n_ant, support):
    w = synth.random_small(2201 + grid_n, n_ant=n_ant, n_pol=2, n_chan=2, grid_n=grid_n, support=support,
                           n_time=3)
    d, keep = epic.desc_from_workload(w, epic.XFORMS[xf], True)
    assert epic.epic_plan_validate(d) == epic.EPIC_OK
    err = rel_errors(gpu_image(w, xform=epic.XFORMS[xf]), oracle_image(w), 2)
    assert err.max() <= TOL[xf], err.max()


@pytest.mark.parametrize("xf,grid_n,n_ant", [
    ("fft_fp32", 32, 40),
    ("fft_fp32", 64, 300),
    ("fft_fp32", 128, 200),   # 45 000 entries per channel: the two-CTA cluster kernel
    ("fft_fp32", 128, 1500),  # beyond the clusters' antenna limit: four folded 64 x 64 problems
    ("dft_bf16x3", 64, 300),
    ("dft_bf16x3", 128, 200),
])
def test_widest_support(xf, grid_n, n_ant):
    w = synth.random_small(2301 + n_ant, n_ant=n_ant, n_pol=2, n_chan=2, grid_n=grid_n, support=15, n_time=3)
    plan = epic.plan_for(w, epic.XFORMS[xf])
    if grid_n == 128 and xf == "fft_fp32":
        assert plan.info["cluster_dim"] == (2 if n_ant <= 1024 else 1)
    err = rel_errors(gpu_image(w, xform=epic.XFORMS[xf], plan=plan), oracle_image(w), 2)
    plan.close()
    assert err.max() <= TOL[xf], err.max()
