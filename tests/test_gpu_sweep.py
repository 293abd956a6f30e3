"""A seeded sweep of random array configurations through every transform that
accepts them, against the FP64 oracle: grid sides 32, 64 and 128, one or two
polarisations, supports 1 to 7, a few to a few hundred antennas, one to a few
dozen channels and samples, with and without gains and delays, with and
without autocorrelation removal."""
import numpy as np
import pytest

from paper_1904_11422_gb300 import build_lib, epic, synth

from _helpers import TOL, TOL_FP32, gpu_image, oracle_image, rel_errors

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return epic.load_library()


def _config(i):
    rng = np.random.default_rng(3000 + i)
    grid_n = int(rng.choice([32, 64, 128]))
    n_pol = int(rng.choice([1, 2]))
    support = int(rng.choice([1, 3, 5, 7]))
    n_ant = int(rng.integers(2, 300 if grid_n > 32 else 60))
    n_chan = int(rng.integers(1, 6))
    n_time = int(rng.integers(1, 12))
    gains = bool(rng.integers(0, 2))
    return dict(seed=3100 + i, n_ant=n_ant, n_pol=n_pol, n_chan=n_chan, grid_n=grid_n, support=support,
                n_time=n_time, with_gains=gains, with_delays=gains), bool(rng.integers(0, 2))


@pytest.mark.parametrize("i", range(24))
def test_random_configuration(i):
    kw, subtract = _config(i)
    w = synth.random_small(**kw)
    ref = oracle_image(w, subtract=subtract)
    xforms = ["fft_fp32"]
    if w.n_pol == 2:
        xforms += ["dft_bf16x3", "dft_fp16x3", "dft_bf16", "dft_fp16"]
    for xf in xforms:
        d, keep = epic.desc_from_workload(w, epic.XFORMS[xf], subtract)
        if epic.epic_plan_validate(d) != epic.EPIC_OK:
            continue
        got = gpu_image(w, xform=epic.XFORMS[xf], subtract=subtract)
        err = rel_errors(got, ref, w.n_pol)
        assert err.max() <= TOL[xf], (kw, subtract, xf, err.max())
        if w.n_pol == 1:
            assert np.all(got[:, 1:] == 0.0)
