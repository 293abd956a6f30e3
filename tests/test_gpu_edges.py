"""Edge cases of the 128 x 128 and 32 x 32 paths (FP32 clusters, tensor-core
parity split and zero-padded transform): single samples, more channels than
clusters or CTAs, time additivity through accumulate = 1, the host-buffer entry
point, the no-allocation entry point's limits, host-side fault injection (a
staging allocation that cannot succeed), and arrays with most antennas stacked on
one position (the most uneven gather tables)."""
import numpy as np
import pytest

from paper_1904_11422_gb300 import build_lib, epic, synth

from _helpers import TOL, TOL_FP32, assert_close, gpu_image, oracle_image, rel_errors

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return epic.load_library()


@pytest.mark.parametrize("xf,grid_n", [("fft_fp32", 128), ("dft_bf16x3", 128), ("dft_bf16x3", 32),
                                       ("dft_fp16", 128)])
def test_single_sample(xf, grid_n):
    w = synth.random_small(2101, n_ant=11, n_pol=2, n_chan=3, grid_n=grid_n, support=3, n_time=1)
    err = rel_errors(gpu_image(w, xform=epic.XFORMS[xf]), oracle_image(w), 2)
    assert err.max() <= TOL[xf], err.max()


@pytest.mark.parametrize("xf,grid_n", [("fft_fp32", 128), ("dft_bf16x3", 128), ("dft_bf16x3", 32)])
def test_more_channels_than_ctas(xf, grid_n):
    """Hundreds of channels of two samples each: a CTA (or cluster) spans many
    channels, and the partial-image slots per CTA are at their largest."""
    C = 400
    w = synth.random_small(2102, n_ant=5, n_pol=2, n_chan=C, grid_n=grid_n, support=1, n_time=2,
                           freq_hz=np.linspace(50e6, 60e6, C))
    got = gpu_image(w, xform=epic.XFORMS[xf])
    chans = [0, 1, 199, 398, 399]
    ref = oracle_image(w, channels=chans)
    assert rel_errors(got[chans], ref, 2).max() <= TOL[xf]
    # every channel has the same array and statistics: no channel is left empty
    assert np.all(np.abs(got[:, 0]).max(axis=(1, 2)) > 0)


@pytest.mark.parametrize("xf,grid_n", [("fft_fp32", 128), ("dft_bf16x3", 128), ("dft_bf16x3", 32)])
def test_time_halves_accumulate(xf, grid_n):
    import torch
    w = synth.random_small(2103, n_ant=30, n_pol=2, n_chan=4, grid_n=grid_n, support=5, n_time=37)
    plan = epic.plan_for(w, epic.XFORMS[xf])
    dv = torch.from_numpy(w.volts).cuda()
    whole = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    halves = torch.empty_like(whole)
    epic.epic_image(plan, dv, w.n_time, whole, 0)
    epic.epic_image(plan, dv[:20].contiguous(), 20, halves, 0)
    epic.epic_image(plan, dv[20:].contiguous(), w.n_time - 20, halves, 1)
    epic.epic_sync(plan)
    assert rel_errors(halves.cpu().numpy(), whole.cpu().numpy(), 2).max() < 1e-5
    plan.close()


@pytest.mark.parametrize("xf", ["fft_fp32", "dft_bf16x3"])
def test_host_entry_point_at_128(xf):
    w = synth.random_small(2104, n_ant=14, n_pol=2, n_chan=2, grid_n=128, support=3, n_time=6)
    plan = epic.plan_for(w, epic.XFORMS[xf])
    dev = gpu_image(w, xform=epic.XFORMS[xf], plan=plan)
    h_out = np.empty(plan.out_shape, np.float32)
    epic.epic_image_host(plan, np.ascontiguousarray(w.volts), w.n_time, h_out, 0)
    assert np.array_equal(h_out, dev)
    plan.close()


def test_noalloc_at_128_is_rejected_when_the_workspace_exceeds_the_scratch():
    import torch
    w = synth.random_small(2105, n_ant=6, n_pol=2, n_chan=2, grid_n=128, support=3, n_time=3)
    plan = epic.plan_for(w)
    out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    dv = torch.from_numpy(w.volts).cuda()
    if plan.info["workspace_bytes"] > epic.EPIC_NOALLOC_SCRATCH_BYTES:
        with pytest.raises(epic.EpicError) as ei:
            epic.epic_image_noalloc(plan, dv, w.n_time, out, 0)
        assert ei.value.status == epic.EPIC_ERR_UNSUPPORTED
    else:
        epic.epic_image_noalloc(plan, dv, w.n_time, out, 0)
        epic.epic_sync(plan)
        assert_close(out.cpu().numpy(), oracle_image(w), 2)
    plan.close()


def test_single_antenna_at_128_subtracts_to_zero():
    for xf in ("fft_fp32", "dft_bf16x3"):
        w = synth.random_small(2106, n_ant=1, n_pol=2, n_chan=2, grid_n=128, support=5, n_time=5)
        raw = gpu_image(w, xform=epic.XFORMS[xf], subtract=False)
        sub = gpu_image(w, xform=epic.XFORMS[xf], subtract=True)
        assert np.abs(sub).max() <= 1e-5 * np.abs(raw).max(), xf


def test_failed_staging_allocation_reports_oom_and_the_plan_keeps_working():
    """Host-side fault injection: a host-buffer call whose staging area (2^24
    samples of the station block, about 550 GB) cannot be allocated returns
    EPIC_ERR_OOM without touching the host buffers, and the failed allocation is
    not reported again by the next call."""
    import torch
    w = synth.station(n_time=4, n_chan=64)
    plan = epic.plan_for(w)
    h_in = np.zeros(16, np.uint8)
    h_out = np.empty(plan.out_shape, np.float32)
    with pytest.raises(epic.EpicError) as ei:  # a bare address: only the library sees the size
        epic.epic_image_host(plan, h_in.ctypes.data, 1 << 24, h_out, 0)
    assert ei.value.status == epic.EPIC_ERR_OOM
    dv = torch.from_numpy(w.volts).cuda()
    out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    epic.epic_image(plan, dv, w.n_time, out, 0)
    epic.epic_sync(plan)
    assert_close(out.cpu().numpy()[[0, 63]], oracle_image(w, channels=[0, 63]), 2)
    plan.close()


def test_grid128_fold_beyond_the_cluster_limit():
    """1500 antennas on a 128 x 128 grid: more than the clusters take, so the
    channel runs as four folded 64 x 64 problems."""
    w = synth.random_small(2107, n_ant=1500, n_pol=2, n_chan=2, grid_n=128, support=1, n_time=3)
    assert_close(gpu_image(w), oracle_image(w), 2)


def test_two_plans_on_two_streams_match_sequential_calls():
    """Different plans share nothing on the device: imaging two arrays
    concurrently on two streams gives exactly the sequential results."""
    import torch
    wa = synth.random_small(2108, n_ant=40, n_pol=2, n_chan=6, grid_n=64, support=5, n_time=30)
    wb = synth.random_small(2109, n_ant=25, n_pol=2, n_chan=4, grid_n=128, support=3, n_time=20)
    pa, pb = epic.plan_for(wa), epic.plan_for(wb, epic.XFORMS["dft_bf16x3"])
    va, vb = torch.from_numpy(wa.volts).cuda(), torch.from_numpy(wb.volts).cuda()
    ra = torch.empty(pa.out_shape, dtype=torch.float32, device="cuda")
    rb = torch.empty(pb.out_shape, dtype=torch.float32, device="cuda")
    epic.epic_image(pa, va, wa.n_time, ra, 0)
    epic.epic_image(pb, vb, wb.n_time, rb, 0)
    torch.cuda.synchronize()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    oa, ob = torch.full_like(ra, float("nan")), torch.full_like(rb, float("nan"))
    torch.cuda.synchronize()
    for _ in range(3):
        epic.epic_image(pa, va, wa.n_time, oa, 0, sa)
        epic.epic_image(pb, vb, wb.n_time, ob, 0, sb)
    torch.cuda.synchronize()
    assert torch.equal(oa, ra) and torch.equal(ob, rb)
    pa.close()
    pb.close()


def test_fma_chain_rate_is_near_the_derived_fp32_peak():
    """The FP32 roofline's denominator (SMs x 128 lanes x 2 flop x the maximum
    SM clock, 2070 MHz on GB300) checked against a measured FMA-chain rate."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * 128 * 2 * 2070e6 / 1e12
    rate = epic.epic_debug_fma_rate(20000)
    assert 0.3 * derived < rate < 1.1 * derived, (rate, derived)
    with pytest.raises(epic.EpicError):
        epic.epic_debug_fma_rate(0)


def test_undersized_buffers_are_refused_before_any_launch():
    """The binding refuses buffers smaller than the plan's shapes (the kernels
    would index past their ends); the plan keeps working."""
    import torch
    w = synth.random_small(2110, n_ant=8, n_pol=2, n_chan=3, grid_n=64, support=3, n_time=4)
    plan = epic.plan_for(w)
    dv = torch.from_numpy(w.volts).cuda()
    out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError, match="d_out"):
        epic.epic_image(plan, dv, w.n_time, out[:2], 0)
    with pytest.raises(ValueError, match="d_volts"):
        epic.epic_image(plan, dv[:2].contiguous(), w.n_time, out, 0)
    with pytest.raises(ValueError, match="h_out"):
        epic.epic_image_host(plan, np.ascontiguousarray(w.volts), w.n_time, np.empty(10, np.float32), 0)
    epic.epic_image(plan, dv, w.n_time, out, 0)
    epic.epic_sync(plan)
    assert_close(out.cpu().numpy(), oracle_image(w), 2)
    plan.close()


@pytest.mark.parametrize("xf,grid_n,n_ant", [("fft_fp32", 64, 40), ("fft_fp32", 32, 20), ("dft_bf16x3", 64, 40),
                                             ("fft_fp32", 128, 450), ("fft_fp32", 128, 30), ("dft_bf16x3", 128, 30)])
def test_pinned_host_buffers_equal_device_call(xf, grid_n, n_ant):
    """Page-locked host buffers through the host entry point give the
    device-buffer call's result bit for bit, also on the 128 x 128 cluster (450
    antennas x 5 x 5) and folded (30 antennas) kernels."""
    import torch
    w = synth.random_small(2111 + n_ant, n_ant=n_ant, n_pol=2, n_chan=3, grid_n=grid_n, support=5, n_time=17)
    plan = epic.plan_for(w, epic.XFORMS[xf])
    dev = gpu_image(w, xform=epic.XFORMS[xf], plan=plan)
    h_in = torch.from_numpy(w.volts).pin_memory()
    h_out = torch.empty(plan.out_shape, dtype=torch.float32).pin_memory()
    epic.epic_image_host(plan, h_in, w.n_time, h_out, 0)
    assert np.array_equal(h_out.numpy(), dev)
    epic.epic_image_host(plan, h_in, w.n_time, h_out, 1)
    assert np.allclose(h_out.numpy(), 2 * dev, rtol=1e-6, atol=1e-6 * np.abs(dev).max())
    plan.close()


def test_async_host_calls_in_flight_equal_device_calls():
    """Five pipelined calls from pinned buffers over three different blocks, then
    one epic_sync: every result equals its device-buffer call bit for bit."""
    import torch
    w = synth.random_small(2120, n_ant=30, n_pol=2, n_chan=4, grid_n=64, support=5, n_time=23)
    plan = epic.plan_for(w)
    rng = np.random.default_rng(5)
    blocks = [w.volts, rng.integers(0, 256, w.volts.shape, dtype=np.uint8), w.volts[::-1].copy()]
    want = [gpu_image(w, plan=plan, volts=b) for b in blocks]
    h_in = [torch.from_numpy(np.ascontiguousarray(b)).pin_memory() for b in blocks]
    outs = [torch.full(plan.out_shape, np.nan, dtype=torch.float32).pin_memory() for _ in range(5)]
    order = [0, 1, 2, 1, 0]
    for i, b in enumerate(order):
        epic.epic_image_host_async(plan, h_in[b], w.n_time, outs[i], 0)
    epic.epic_sync(plan)
    for i, b in enumerate(order):
        assert np.array_equal(outs[i].numpy(), want[b]), i
    plan.close()


def test_async_host_accumulation_chain_and_mixed_calls():
    """Accumulating pipelined calls into one pinned buffer sees each previous
    result; synchronous host calls and device calls interleave on the same plan."""
    import torch
    w = synth.random_small(2121, n_ant=12, n_pol=2, n_chan=3, grid_n=32, support=3, n_time=9)
    plan = epic.plan_for(w)
    dev = gpu_image(w, plan=plan)
    h_in = torch.from_numpy(w.volts).pin_memory()
    acc = torch.zeros(plan.out_shape, dtype=torch.float32).pin_memory()
    for i in range(4):
        epic.epic_image_host_async(plan, h_in, w.n_time, acc, 1)
    epic.epic_sync(plan)
    assert np.allclose(acc.numpy(), 4 * dev, rtol=1e-5, atol=1e-5 * np.abs(dev).max())
    h_out = np.empty(plan.out_shape, np.float32)
    epic.epic_image_host(plan, np.ascontiguousarray(w.volts), w.n_time, h_out, 0)
    assert np.array_equal(h_out, dev)
    one = torch.empty(plan.out_shape, dtype=torch.float32).pin_memory()
    epic.epic_image_host_async(plan, h_in, w.n_time, one, 0)
    epic.epic_sync(plan)
    assert np.array_equal(one.numpy(), dev)
    plan.close()


def test_async_host_call_rejects_pageable_buffers():
    import torch
    w = synth.random_small(2122, n_ant=6, n_pol=2, n_chan=2, grid_n=32, support=3, n_time=3)
    plan = epic.plan_for(w)
    pinned_out = torch.empty(plan.out_shape, dtype=torch.float32).pin_memory()
    with pytest.raises(epic.EpicError) as ei:
        epic.epic_image_host_async(plan, np.ascontiguousarray(w.volts), w.n_time, pinned_out, 0)
    assert ei.value.status == epic.EPIC_ERR_INVALID_ARG
    with pytest.raises(epic.EpicError) as ei:
        epic.epic_image_host_async(plan, torch.from_numpy(w.volts).pin_memory(), w.n_time,
                                   np.empty(plan.out_shape, np.float32), 0)
    assert ei.value.status == epic.EPIC_ERR_INVALID_ARG
    plan.close()


def test_plans_release_their_device_memory():
    """Creating and destroying plans repeatedly (each used through the pipelined
    host entry point, with per-launch timing on, and on the tensor path) returns
    the device's free memory to where it started: no staging slot, stream, event
    or table outlives its plan."""
    import torch
    w = synth.random_small(2130, n_ant=24, n_pol=2, n_chan=4, grid_n=64, support=3, n_time=12)
    h_in = torch.from_numpy(w.volts).pin_memory()

    def cycle():
        for xf in ("fft_fp32", "dft_bf16x3"):
            plan = epic.plan_for(w, epic.XFORMS[xf])
            epic.epic_timing_enable(plan, True)
            out = torch.empty(plan.out_shape, dtype=torch.float32).pin_memory()
            for _ in range(3):
                epic.epic_image_host_async(plan, h_in, w.n_time, out, 0)
            epic.epic_sync(plan)
            epic.epic_timing_read(plan)
            plan.close()

    cycle()  # first use: one-time allocations of the runtime and of the library
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(10):
        cycle()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 8 * 1024 * 1024, (free0, free1)


# ------------------------------------------------ failure detection: bounded waits
@pytest.mark.parametrize("xf,grid_n", [("dft_bf16x3", 64), ("dft_fp16", 128)])
def test_tensor_kernel_wait_times_out_and_the_plan_recovers(xf, grid_n):
    """The tensor kernel's first mbarrier wait in every CTA is made on a barrier
    that nothing arrives at, limited to 2 ms: every CTA must give up, report
    EPIC_ERR_TIMEOUT through epic_sync, drain the products it issued and free its
    tensor memory, leaving the plan and the device usable (the next calls, on the
    same plan and on a fresh one, match the oracle)."""
    import time

    import torch
    w = synth.random_small(2301, n_ant=30, n_pol=2, n_chan=3, grid_n=grid_n, support=3, n_time=6)
    plan = epic.plan_for(w, epic.XFORMS[xf])
    dv = torch.from_numpy(w.volts).cuda()
    t0 = time.time()
    epic.epic_debug_image_timeout(plan, dv, w.n_time, 2_000_000)
    with pytest.raises(epic.EpicError) as ei:
        epic.epic_sync(plan)
    assert ei.value.status == epic.EPIC_ERR_TIMEOUT
    assert time.time() - t0 < 60
    epic.epic_sync(plan)  # the status was cleared
    ref = oracle_image(w)
    assert rel_errors(gpu_image(w, xform=epic.XFORMS[xf], plan=plan), ref, 2).max() <= TOL[xf]
    plan.close()
    assert rel_errors(gpu_image(w, xform=epic.XFORMS[xf]), ref, 2).max() <= TOL[xf]


def test_timeout_hook_rejects_fp32_plans_and_bad_limits():
    import torch
    w = synth.random_small(2302, n_ant=8, n_pol=2, n_chan=1, grid_n=64, support=3, n_time=2)
    plan = epic.plan_for(w)
    dv = torch.from_numpy(w.volts).cuda()
    with pytest.raises(epic.EpicError) as ei:
        epic.epic_debug_image_timeout(plan, dv, w.n_time, 2_000_000)
    assert ei.value.status == epic.EPIC_ERR_UNSUPPORTED
    plan.close()
    plan = epic.plan_for(w, epic.XFORMS["dft_bf16x3"])
    for bad in (0, 999, 2_000_000_000):
        with pytest.raises(epic.EpicError) as ei:
            epic.epic_debug_image_timeout(plan, dv, w.n_time, bad)
        assert ei.value.status == epic.EPIC_ERR_INVALID_ARG
    plan.close()


@pytest.mark.parametrize("grid_n", [64, 128])
@pytest.mark.parametrize("xf", ["fft_fp32", "dft_bf16x3", "dft_fp16x3", "dft_bf16", "dft_fp16"])
def test_stacked_antennas(xf, grid_n):
    """160 of 200 antennas at one position: the 25 cells under the stack hold 160
    entries each while most cells hold none, the most uneven gather tables an
    array can give (the tensor path's cell-pair deal, the FP32 path's padded
    trip counts, the FP16 operand scales of a field 160 kernels deep)."""
    w = synth.random_small(1901, n_ant=200, n_pol=2, n_chan=2, grid_n=grid_n, support=5, n_time=3)
    w.ant_xy = np.array(w.ant_xy)
    w.ant_xy[:160] = w.ant_xy[0]
    for sub in (True, False):
        got = gpu_image(w, xform=epic.XFORMS[xf], subtract=sub)
        err = rel_errors(got, oracle_image(w, subtract=sub), 2)
        assert err.max() <= TOL[xf], (xf, grid_n, sub, err.max())


def test_stacked_antennas_on_clusters():
    """The same stacking on the 128 x 128 two-CTA cluster kernel (450 antennas x
    25 = 11 250 entries per channel, above the folding threshold), 400 of them at
    one position."""
    w = synth.random_small(1902, n_ant=450, n_pol=2, n_chan=1, grid_n=128, support=5, n_time=3)
    w.ant_xy = np.array(w.ant_xy)
    w.ant_xy[:400] = w.ant_xy[0]
    plan = epic.plan_for(w)
    assert plan.info["cluster_dim"] == 2
    got = gpu_image(w, plan=plan)
    plan.close()
    assert_close(got, oracle_image(w), 2)


def test_early_unpack_chosen_where_rows_are_empty():
    """The 64 x 64 FP32 kernel lets the four warps with the lightest gather unpack
    each next sample while the others still grid, when the aperture leaves rows
    empty (a compact array), and keeps the plain unpack when every row holds
    antennas (a square array filling the grid); both images equal the oracle's."""
    # 3 x 201 units over at most 152 CTAs: four consecutive samples per CTA, so the
    # early unpack runs, and some CTAs' spans cross a channel boundary
    compact = synth.random_small(1903, n_ant=60, n_pol=2, n_chan=3, grid_n=64, support=5, n_time=201,
                                 diameter_m=60.0)
    square = synth.random_small(1904, n_ant=300, n_pol=2, n_chan=2, grid_n=64, support=5, n_time=6)
    lam_min = synth.C_LIGHT / square.freq_hz.max()
    half = 0.25 * lam_min * (64 - 5 - 3)  # boxes stay inside the grid at the highest channel
    rng = np.random.default_rng(1905)
    square.ant_xy = rng.uniform(-half, half, size=(300, 2))
    for w, early in ((compact, True), (square, False)):
        plan = epic.plan_for(w)
        mask = plan.info["unpack_warps"]
        assert (bin(mask).count("1") == 4) if early else mask == 0, (w.name, hex(mask))
        got = gpu_image(w, plan=plan)
        plan.close()
        assert_close(got, oracle_image(w, use_fft=True), 2)
