"""Parity of the tensor-core path (DFT-by-GEMM on tcgen05) with the FP64 oracle.

Every transform must stay within its stated bound (tests/_helpers.TOL, relative
to the channel's image peak): about ten times the largest error measured on
GB300, so that a regression of the hi + lo split fails.  Errors are measured
against the oracle on the same seeded inputs, including saturated plane waves
whose stage-1 magnitudes exceed FP16's range unless the FP16 transforms scale
their operands."""
import numpy as np
import pytest

from paper_1904_11422_gb300 import build_lib, epic, synth

from _helpers import TOL, gpu_image, oracle_image, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return epic.load_library()


@pytest.fixture(scope="module")
def station():
    return synth.station()


def test_small_array_bf16x3():
    w = synth.random_small(901, n_ant=12, n_pol=2, n_chan=2, grid_n=64, support=3, n_time=3)
    got = gpu_image(w, xform=epic.XFORMS["dft_bf16x3"])
    ref = oracle_image(w)
    err = rel_errors(got, ref, 2)
    print("small bf16x3 errors", err.max())
    assert err.max() <= TOL["dft_bf16x3"]


@pytest.mark.parametrize("xf", ["dft_bf16x3", "dft_fp16x3", "dft_bf16", "dft_fp16"])
def test_random_arrays(xf):
    for seed, kw in [(902, dict(n_ant=20, n_chan=3, support=5, n_time=11)),
                     (903, dict(n_ant=40, n_chan=2, support=1, n_time=7))]:
        w = synth.random_small(seed, n_pol=2, grid_n=64, **kw)
        for sub in (True, False):
            err = rel_errors(gpu_image(w, xform=epic.XFORMS[xf], subtract=sub), oracle_image(w, subtract=sub), 2)
            assert err.max() <= TOL[xf], (xf, seed, sub, err.max())


@pytest.mark.parametrize("xf", ["dft_bf16x3", "dft_fp16x3", "dft_bf16", "dft_fp16"])
def test_station_block_sampled_channels(station, xf):
    w = station
    got = gpu_image(w, xform=epic.XFORMS[xf])
    chans = [0, 31, 63]
    ref = oracle_image(w, channels=chans, use_fft=True)
    err = rel_errors(got[chans], ref, 2)
    print(f"{xf}: max error / image peak per plane {err.max(axis=0)}")
    assert err.max() <= TOL[xf], (xf, err.max())


def test_tensor_and_fp32_paths_agree_at_full_size(station):
    w = station
    a = gpu_image(w, xform=epic.XFORMS["dft_bf16x3"])
    b = gpu_image(w, xform=epic.XFORMS["fft_fp32"])
    assert rel_errors(a, b, 2).max() <= TOL["dft_bf16x3"] + TOL["fft_fp32"]


def test_tensor_path_deterministic_and_additive(station):
    import torch
    w = station
    plan = epic.plan_for(w, epic.XFORMS["dft_bf16x3"])
    dv = torch.from_numpy(w.volts).cuda()
    a = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    epic.epic_image(plan, dv, w.n_time, a, 0)
    epic.epic_image(plan, dv, w.n_time, b, 0)
    epic.epic_sync(plan)
    assert torch.equal(a, b)
    T1 = 600
    epic.epic_image(plan, dv[:T1].contiguous(), T1, b, 0)
    epic.epic_image(plan, dv[T1:].contiguous(), w.n_time - T1, b, 1)
    epic.epic_sync(plan)
    assert rel_errors(b.cpu().numpy(), a.cpu().numpy(), 2).max() < 1e-5
    plan.close()


def test_unsupported_shapes_are_rejected():
    w = synth.random_small(904, n_ant=8, n_pol=1, n_chan=1, grid_n=64, support=3, n_time=2)
    d, keep = epic.desc_from_workload(w, epic.XFORMS["dft_bf16x3"])
    assert epic.epic_plan_validate(d) == epic.EPIC_ERR_UNSUPPORTED
    w = synth.random_small(905, n_ant=8, n_pol=2, n_chan=1, grid_n=16, support=3, n_time=2)
    d, keep = epic.desc_from_workload(w, epic.XFORMS["dft_bf16x3"])
    assert epic.epic_plan_validate(d) == epic.EPIC_ERR_UNSUPPORTED
    w = synth.random_small(906, n_ant=1025, n_pol=2, n_chan=1, grid_n=64, support=3, n_time=2)
    d, keep = epic.desc_from_workload(w, epic.XFORMS["dft_bf16x3"])
    assert epic.epic_plan_validate(d) == epic.EPIC_ERR_UNSUPPORTED


# ------------------------------------------------- 128 x 128 grids (parity split)
@pytest.mark.parametrize("xf", ["dft_bf16x3", "dft_fp16x3", "dft_bf16", "dft_fp16"])
def test_grid128_random_arrays(xf):
    """128 x 128 grids: four 64 x 64 transforms of the parity-folded fields, the
    sub-images interleaved by the reduction."""
    for seed, kw in [(1901, dict(n_ant=24, n_chan=3, support=5, n_time=7)),
                     (1902, dict(n_ant=60, n_chan=2, support=3, n_time=4))]:
        w = synth.random_small(seed, n_pol=2, grid_n=128, **kw)
        for sub in (True, False):
            err = rel_errors(gpu_image(w, xform=epic.XFORMS[xf], subtract=sub), oracle_image(w, subtract=sub), 2)
            assert err.max() <= TOL[xf], (xf, seed, sub, err.max())


def test_more_than_512_antennas():
    """Two antennas per thread in the unpack (A up to 1024), gather entries read
    from L2 when they do not fit in shared memory; 64^2 and 128^2."""
    for seed, grid_n in [(1903, 64), (1904, 128)]:
        w = synth.random_small(seed, n_ant=900, n_pol=2, n_chan=2, grid_n=grid_n, support=5, n_time=3)
        err = rel_errors(gpu_image(w, xform=epic.XFORMS["dft_bf16x3"]), oracle_image(w), 2)
        assert err.max() <= TOL["dft_bf16x3"], (grid_n, err.max())


@pytest.mark.parametrize("xf", ["dft_bf16x3", "dft_fp16x3", "dft_bf16", "dft_fp16"])
def test_grid128_station_sampled_channels(xf):
    """The precision study's 128^2 variant: the station block on a 2x padded
    grid, full size, channels 0, 40, 63 against the oracle's FFT mode."""
    w = _station128()
    got = gpu_image(w, xform=epic.XFORMS[xf])
    chans = [0, 40, 63]
    ref = _station128_ref(chans)
    err = rel_errors(got[chans], ref, 2)
    print(f"128^2 {xf}: max error / image peak per plane {err.max(axis=0)}")
    assert err.max() <= TOL[xf], (xf, err.max())


_S128 = {}


def _station128():
    if "w" not in _S128:
        _S128["w"] = synth.station(grid_n=128)
    return _S128["w"]


def _station128_ref(chans):
    key = tuple(chans)
    if key not in _S128:
        _S128[key] = oracle_image(_station128(), channels=chans, use_fft=True)
    return _S128[key]


# ---------------------------------------------- 32 x 32 grids (zero-padded to 64)
@pytest.mark.parametrize("xf", ["dft_bf16x3", "dft_fp16x3", "dft_bf16", "dft_fp16"])
def test_grid32_random_arrays(xf):
    """32 x 32 grids: the 64 x 64 transform of the zero-padded grid, whose even
    output pixels are the 32-point transform."""
    for seed, kw in [(2001, dict(n_ant=16, n_chan=3, support=3, n_time=9)),
                     (2002, dict(n_ant=40, n_chan=2, support=5, n_time=5))]:
        w = synth.random_small(seed, n_pol=2, grid_n=32, **kw)
        for sub in (True, False):
            err = rel_errors(gpu_image(w, xform=epic.XFORMS[xf], subtract=sub), oracle_image(w, subtract=sub), 2)
            assert err.max() <= TOL[xf], (xf, seed, sub, err.max())


# --------------------------------------- the edge of FP16's range (65 504)
@pytest.mark.parametrize("xf", ["dft_bf16x3", "dft_fp16x3", "dft_bf16", "dft_fp16"])
@pytest.mark.parametrize("grid_n,gain", [(64, 16.0), (128, 16.0), (64, 4096.0), (128, 4096.0), (32, 4096.0)])
def test_saturated_plane_wave(xf, grid_n, gain):
    """1 024 antennas all at the 4-bit limit, one coherent source, gains of
    modulus 16 or 4 096: with 4 096 the stage-1 result reaches ~1e6 and the
    gridded field ~2e4, far beyond FP16's 65 504, so the FP16 transforms stay
    finite and within bound only through their power-of-two operand scales.
    On the 128 x 128 grid the folded fields sum four quadrants."""
    w = synth.saturated_plane_wave(3001 + grid_n, n_ant=1024, grid_n=grid_n, gain_amp=gain)
    got = gpu_image(w, xform=epic.XFORMS[xf])
    assert np.isfinite(got).all()
    ref = oracle_image(w)
    err = rel_errors(got, ref, 2)
    print(f"saturated plane wave N={grid_n} |g|={gain} {xf}: {err.max():.3e}")
    assert err.max() <= TOL[xf], (xf, grid_n, gain, err.max())
