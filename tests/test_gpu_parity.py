"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bit-exact on the unpacked integers; within 1e-5 of the channel's image peak for
the FP32 path; full-size station blocks in the launch configuration the
benchmark times, compared on sampled channels and through properties that hold
at any size."""
import numpy as np
import pytest

import oracle
from paper_1904_11422_gb300 import build_lib, epic, synth

from _helpers import TOL_FP32, assert_close, gpu_image, oracle_array, oracle_image, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return epic.load_library()


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def station():
    return synth.station()


# ---------------------------------------------------------------- unpack (A1)
def test_unpack_bit_exact_all_bytes(torch):
    data = np.arange(256, dtype=np.uint8).repeat(3)
    d_in = torch.from_numpy(data).cuda()
    d_out = torch.empty((data.size, 2), dtype=torch.int8, device="cuda")
    epic.epic_debug_unpack(d_in, data.size, d_out)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().astype(np.int32)
    re, im = oracle.unpack(data)
    assert np.array_equal(got[:, 0], re) and np.array_equal(got[:, 1], im)


# ----------------------------------------------------- plan + grid (A0, A2, A3)
GRID_CASES = [
    dict(seed=101, n_ant=7, n_pol=2, n_chan=3, grid_n=32, support=3, n_time=4),
    dict(seed=102, n_ant=12, n_pol=1, n_chan=2, grid_n=64, support=5, n_time=3),
    dict(seed=103, n_ant=5, n_pol=2, n_chan=1, grid_n=32, support=1, n_time=2),
]


@pytest.mark.parametrize("case", GRID_CASES, ids=lambda c: f"s{c['seed']}")
def test_debug_grid_matches_oracle(torch, case):
    w = synth.random_small(**case)
    plan = epic.plan_for(w)
    arr = oracle_array(w)
    dv = torch.from_numpy(w.volts).cuda()
    g = torch.empty((w.grid_n, w.grid_n, 2), dtype=torch.float32, device="cuda")
    for t in range(w.n_time):
        for c in range(w.n_chan):
            for p in range(w.n_pol):
                epic.epic_debug_grid(plan, dv, w.n_time, t, c, p, g)
                torch.cuda.synchronize()
                got = g.cpu().numpy()
                got = got[..., 0] + 1j * got[..., 1]
                ref = oracle.grid(arr, w.volts, t, c, p)
                assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()
    plan.close()


def test_debug_grid_station_sample(torch, station):
    w = station
    plan = epic.plan_for(w)
    arr = oracle_array(w)
    dv = torch.from_numpy(w.volts).cuda()
    g = torch.empty((w.grid_n, w.grid_n, 2), dtype=torch.float32, device="cuda")
    for (t, c, p) in [(0, 0, 0), (777, 31, 1), (1249, 63, 0)]:
        epic.epic_debug_grid(plan, dv, w.n_time, t, c, p, g)
        torch.cuda.synchronize()
        got = g.cpu().numpy()
        got = got[..., 0] + 1j * got[..., 1]
        ref = oracle.grid(arr, w.volts, t, c, p)
        assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()
    plan.close()


def _round_f32(q):
    """The float32 nearest to the rational q (ties to even), exactly."""
    from fractions import Fraction
    if q == 0:
        return np.float32(0.0)
    sign, q = (-1, -q) if q < 0 else (1, q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    scaled = q / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    n, rem = divmod(scaled.numerator, scaled.denominator)
    twice = 2 * rem
    if twice > scaled.denominator or (twice == scaled.denominator and n % 2 == 1):
        n += 1
    return np.float32(sign * n * 2.0 ** (e - 23))


def _fma32(a, b, c):
    """Elementwise a * b + c with a single rounding to float32 (a fused multiply-add)."""
    from fractions import Fraction
    out = np.empty(a.shape, np.float32)
    for idx in np.ndindex(a.shape):
        out[idx] = _round_f32(Fraction(float(a[idx])) * Fraction(float(b[idx])) + Fraction(float(c[idx])))
    return out


@pytest.mark.parametrize("case", GRID_CASES, ids=lambda c: f"s{c['seed']}")
def test_debug_transform_matches_oracle(torch, case):
    """The pre-square image Y of every (t, c, p): the imaging kernel's line
    transforms against the oracle's direct transform of the oracle's grid."""
    w = synth.random_small(**case)
    plan = epic.plan_for(w)
    arr = oracle_array(w)
    dv = torch.from_numpy(w.volts).cuda()
    y = torch.empty((w.grid_n, w.grid_n, 2), dtype=torch.float32, device="cuda")
    for t in range(w.n_time):
        for c in range(w.n_chan):
            for p in range(w.n_pol):
                epic.epic_debug_transform(plan, dv, w.n_time, t, c, p, y)
                torch.cuda.synchronize()
                got = y.cpu().numpy()
                got = got[..., 0] + 1j * got[..., 1]
                ref = oracle.dft2(oracle.grid(arr, w.volts, t, c, p))
                assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max(), (t, c, p)
    plan.close()


def test_debug_transform_squares_to_the_imaged_sample(torch, station):
    """For one sample without autocorrelation removal the imaging kernel's XX,
    YY and XY are the products of the dumped transforms, bit for bit (same
    gather order, same line transforms, same fused multiply-adds)."""
    w = station
    plan = epic.plan_for(w, subtract_autos=False)
    for t in (0, 611):
        dv = torch.from_numpy(np.ascontiguousarray(w.volts[t:t + 1])).cuda()
        img = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
        epic.epic_image(plan, dv, 1, img, 0)
        ys = []
        for p in range(2):
            y = torch.empty((w.grid_n, w.grid_n, 2), dtype=torch.float32, device="cuda")
            epic.epic_debug_transform(plan, dv, 1, 0, 17, p, y)
            ys.append(y)
        torch.cuda.synchronize()
        X, Y = ys[0].cpu().numpy(), ys[1].cpu().numpy()
        im = img.cpu().numpy()[17]
        zero = np.zeros_like(X[..., 0])
        # XX = fma(x.re, x.re, fma(x.im, x.im, 0)): each fused multiply-add rounded once
        assert np.array_equal(im[0], _fma32(X[..., 0], X[..., 0], _fma32(X[..., 1], X[..., 1], zero)))
        assert np.array_equal(im[1], _fma32(Y[..., 0], Y[..., 0], _fma32(Y[..., 1], Y[..., 1], zero)))
        assert np.array_equal(im[2], _fma32(X[..., 0], Y[..., 0], _fma32(X[..., 1], Y[..., 1], zero)))
        assert np.array_equal(im[3], _fma32(X[..., 1], Y[..., 0], _fma32(-X[..., 0], Y[..., 1], zero)))
    plan.close()


def test_debug_transform_unsupported_plans(torch):
    w = synth.random_small(1702, n_ant=6, n_pol=2, n_chan=1, grid_n=128, support=3, n_time=2)
    plan = epic.plan_for(w)
    y = torch.empty((128, 128, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(epic.EpicError) as ei:
        epic.epic_debug_transform(plan, torch.from_numpy(w.volts).cuda(), 2, 0, 0, 0, y)
    assert ei.value.status == epic.EPIC_ERR_UNSUPPORTED
    plan.close()


# ------------------------------------------------------ whole path (A1-A7)
def test_tiny_config(torch):
    w = synth.tiny()
    for sub in (True, False):
        assert_close(gpu_image(w, subtract=sub), oracle_image(w, subtract=sub), w.n_pol)


IMAGE_CASES = [
    dict(seed=201, n_ant=9, n_pol=2, n_chan=3, grid_n=32, support=3, n_time=7),
    dict(seed=202, n_ant=16, n_pol=1, n_chan=2, grid_n=64, support=5, n_time=13),
    dict(seed=203, n_ant=6, n_pol=2, n_chan=5, grid_n=64, support=1, n_time=3),
    dict(seed=204, n_ant=30, n_pol=2, n_chan=2, grid_n=64, support=3, n_time=40),
    dict(seed=205, n_ant=3, n_pol=1, n_chan=1, grid_n=32, support=5, n_time=1),
    # 128 x 128 grids (clusters of two CTAs)
    dict(seed=206, n_ant=24, n_pol=2, n_chan=3, grid_n=128, support=5, n_time=9),
    dict(seed=207, n_ant=10, n_pol=1, n_chan=2, grid_n=128, support=3, n_time=5),
    dict(seed=208, n_ant=70, n_pol=2, n_chan=5, grid_n=128, support=1, n_time=4),
]


@pytest.mark.parametrize("case", IMAGE_CASES, ids=lambda c: f"s{c['seed']}")
def test_random_arrays_match_oracle(torch, case):
    w = synth.random_small(**case)
    for sub in (True, False):
        assert_close(gpu_image(w, subtract=sub), oracle_image(w, subtract=sub), w.n_pol)


def test_single_antenna_subtracts_to_zero(torch):
    w = synth.random_small(301, n_ant=1, n_pol=2, n_chan=2, grid_n=32, support=5, n_time=9)
    raw = gpu_image(w, subtract=False)
    sub = gpu_image(w, subtract=True)
    assert np.abs(sub).max() <= 1e-6 * np.abs(raw).max()


def test_station_block_sampled_channels(torch, station):
    """The full station block (256 ants, 64 ch, 1250 samples, 64^2) in the launch
    the benchmark times; channels 0, 31 and 63 against the oracle's FFT mode
    (pinned to its direct mode)."""
    w = station
    gpu = gpu_image(w)
    ref = oracle_image(w, channels=[0, 31, 63], use_fft=True)
    err = assert_close(gpu[[0, 31, 63]], ref, 2)
    # the three point sources are where the recipe put them (rows m, columns l)
    xx = gpu[:, 0].sum(0)
    for (i, j, _) in w.sources[:1]:
        assert np.unravel_index(np.argmax(xx), xx.shape) == (j, i)
    assert err.max() < TOL_FP32


def test_station_properties(torch, station):
    """Properties at full size: determinism, time additivity (accumulate=1 over
    halves equals one call), and that a plan over a channel subset equals the
    matching slice."""
    w = station
    plan = epic.plan_for(w)
    dv = torch.from_numpy(w.volts).cuda()
    a = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    epic.epic_image(plan, dv, w.n_time, a, 0)
    epic.epic_image(plan, dv, w.n_time, b, 0)
    epic.epic_sync(plan)
    assert torch.equal(a, b)
    h = torch.empty_like(a)
    T1 = 517
    epic.epic_image(plan, dv[:T1].contiguous(), T1, h, 0)
    epic.epic_image(plan, dv[T1:].contiguous(), w.n_time - T1, h, 1)
    epic.epic_sync(plan)
    whole = a.cpu().numpy()
    err = rel_errors(h.cpu().numpy(), whole, 2)
    assert err.max() < 2e-6
    plan.close()
    sub = synth.Workload("sub", w.ant_xy, w.freq_hz[10:13], 2, w.grid_n, w.support, w.cell_lambda,
                         w.sigma_cells, np.ascontiguousarray(w.volts[:, 10:13]))
    part = gpu_image(sub)
    assert rel_errors(part, whole[10:13], 2).max() < 2e-6


def test_empty_and_short_blocks(torch):
    w = synth.random_small(401, n_ant=8, n_pol=2, n_chan=3, grid_n=32, support=3, n_time=2)
    plan = epic.plan_for(w)
    out = torch.full(plan.out_shape, 7.0, dtype=torch.float32, device="cuda")
    epic.epic_image(plan, None, 0, out, 1)
    epic.epic_sync(plan)
    assert torch.all(out == 7.0)
    epic.epic_image(plan, None, 0, out, 0)
    epic.epic_sync(plan)
    assert torch.all(out == 0.0)
    one = np.ascontiguousarray(w.volts[:1])
    assert_close(gpu_image(w, volts=one, plan=plan), oracle_image(w, volts=one), 2)
    plan.close()


def test_image_host_equals_device(torch):
    w = synth.random_small(501, n_ant=20, n_pol=2, n_chan=4, grid_n=64, support=5, n_time=25)
    plan = epic.plan_for(w)
    dev = gpu_image(w, plan=plan)
    h_out = np.empty(plan.out_shape, np.float32)
    epic.epic_image_host(plan, np.ascontiguousarray(w.volts), w.n_time, h_out, 0)
    assert np.array_equal(h_out, dev)
    epic.epic_image_host(plan, np.ascontiguousarray(w.volts), w.n_time, h_out, 1)
    assert np.allclose(h_out, 2 * dev, rtol=1e-6, atol=1e-6 * np.abs(dev).max())
    plan.close()


def test_gains_and_delays_enter_as_the_oracle_says(torch):
    w = synth.random_small(601, n_ant=10, n_pol=2, n_chan=2, grid_n=32, support=3, n_time=6)
    base = gpu_image(w)
    w2 = synth.Workload(w.name, w.ant_xy, w.freq_hz, 2, w.grid_n, w.support, w.cell_lambda, w.sigma_cells,
                        w.volts, gains=w.gains * (0.5 + 1.5j), delays_s=w.delays_s)
    scaled = gpu_image(w2)
    assert rel_errors(scaled, abs(0.5 + 1.5j) ** 2 * base, 2).max() < 1e-5
    assert_close(scaled, oracle_image(w2), 2)


def test_plan_create_errors(torch):
    w = synth.random_small(701, n_ant=4, n_pol=2, n_chan=1, grid_n=32, support=3)
    d, keep = epic.make_desc(w.ant_xy * 100.0, w.freq_hz, 2, 32, 3)
    with pytest.raises(epic.EpicError) as ei:
        epic.epic_plan_create(d, keep)
    assert ei.value.status == epic.EPIC_ERR_OFFGRID
    plan = epic.plan_for(w)
    out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    dv = torch.from_numpy(w.volts).cuda()
    with pytest.raises(epic.EpicError):
        epic.epic_image(plan, dv, -1, out, 0)
    with pytest.raises(epic.EpicError):
        epic.epic_image(plan, dv, 1, out, 2)
    plan.close()


def test_postprocess_matches_oracle(torch):
    w = synth.random_small(1501, n_ant=20, n_pol=2, n_chan=3, grid_n=64, support=5, n_time=6)
    plan = epic.plan_for(w)
    dv = torch.from_numpy(w.volts).cuda()
    img = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    epic.epic_image(plan, dv, w.n_time, img, 0)
    ref = oracle_image(w)
    arr = oracle_array(w)
    floor = 0.05
    for flags in (epic.EPIC_POST_STOKES, epic.EPIC_POST_BEAM, epic.EPIC_POST_STOKES | epic.EPIC_POST_BEAM):
        out = torch.empty_like(img)
        epic.epic_postprocess(plan, img, out, flags, floor)
        epic.epic_sync(plan)
        got = out.cpu().numpy()
        exp = ref.copy()
        for c in range(w.n_chan):
            if flags & epic.EPIC_POST_STOKES:
                exp[c] = oracle.stokes(exp[c])
            if flags & epic.EPIC_POST_BEAM:
                b = oracle.beam(arr, c)
                exp[c] = np.where(b >= floor, exp[c] / np.maximum(b, floor), 0.0)
        scale = np.abs(exp).max()
        assert np.abs(got - exp).max() <= 1e-5 * scale
    plan.close()


def test_plans_coexist_after_a_smaller_plan(torch, station):
    """A kernel's shared-memory limit is a property of the function, not of a
    plan: creating a plan that needs less shared memory must leave an existing,
    larger plan of the same kernel working."""
    big = epic.plan_for(station)
    dv = torch.from_numpy(station.volts[:40]).cuda()
    a = torch.empty(big.out_shape, dtype=torch.float32, device="cuda")
    epic.epic_image(big, dv, 40, a, 0)
    epic.epic_sync(big)
    w = synth.random_small(1701, n_ant=12, n_pol=2, n_chan=2, grid_n=64, support=3, n_time=4)
    small = epic.plan_for(w)
    b = torch.empty_like(a)
    epic.epic_image(big, dv, 40, b, 0)
    epic.epic_sync(big)
    assert torch.equal(a, b)
    assert_close(gpu_image(w, plan=small), oracle_image(w), 2)
    small.close()
    big.close()


def test_grid128_largest_array(torch):
    """1024 antennas on a 128 x 128 grid (the largest array the clusters take;
    gather entries are read from L2 instead of shared memory)."""
    w = synth.random_small(1801, n_ant=1024, n_pol=2, n_chan=2, grid_n=128, support=5, n_time=3)
    plan = epic.plan_for(w)
    assert plan.info["ctas"] >= 1
    got = gpu_image(w, plan=plan)
    assert_close(got, oracle_image(w), 2)
    plan.close()


def test_grid128_station_sampled_channels(torch):
    """The station block on a 2x padded 128 x 128 grid (the precision study's
    128^2 variant), full size in the benchmark's launch, channels 0, 40 and 63
    against the oracle's FFT mode; the brightest source is where the recipe put
    it, and the image is additive over time halves."""
    w = synth.station(grid_n=128)
    plan = epic.plan_for(w)
    dv = torch.from_numpy(w.volts).cuda()
    out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    epic.epic_image(plan, dv, w.n_time, out, 0)
    epic.epic_sync(plan)
    gpu = out.cpu().numpy()
    err = assert_close(gpu[[0, 40, 63]], oracle_image(w, channels=[0, 40, 63], use_fft=True), 2)
    assert err.max() < TOL_FP32
    xx = gpu[:, 0].sum(0)
    i, j, _ = w.sources[0]
    assert np.unravel_index(np.argmax(xx), xx.shape) == (j, i)
    h = torch.empty_like(out)
    epic.epic_image(plan, dv[:600].contiguous(), 600, h, 0)
    epic.epic_image(plan, dv[600:].contiguous(), w.n_time - 600, h, 1)
    epic.epic_sync(plan)
    assert rel_errors(h.cpu().numpy(), gpu, 2).max() < 2e-6
    plan.close()
