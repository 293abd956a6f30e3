"""Batched imaging: several arrays of different antenna counts, grid sizes and
channel counts in one graph launch, with and without the autotuner."""
import numpy as np
import pytest

from paper_1904_11422_gb300 import build_lib, epic, synth

from _helpers import TOL, assert_close, oracle_image, rel_errors

pytestmark = pytest.mark.gpu

# A tuned batch splits each call into other time tiles than a single call, so
# its partial images are summed in another order: the images agree to FP32
# rounding of the raw (unsubtracted) sums, a few ulps of a raw peak that can be
# several times the subtracted peak these errors are relative to.
REORDER_TOL = 5e-6


@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return epic.load_library()


@pytest.fixture(scope="module")
def arrays():
    return [synth.batching_array("A", n_time=300), synth.batching_array("B", n_time=300),
            synth.random_small(1601, n_ant=40, n_pol=2, n_chan=7, grid_n=64, support=3, n_time=55),
            synth.batching_array("C", n_time=60)]


def _setup(ws, xforms):
    import torch
    plans = [epic.plan_for(w, epic.XFORMS[x]) for w, x in zip(ws, xforms)]
    vols = [torch.from_numpy(w.volts).cuda() for w in ws]
    outs = [torch.empty(p.out_shape, dtype=torch.float32, device="cuda") for p in plans]
    return plans, vols, outs


def _single(plans, vols, ws):
    import torch
    res = []
    for p, v, w in zip(plans, vols, ws):
        o = torch.empty(p.out_shape, dtype=torch.float32, device="cuda")
        epic.epic_image(p, v, w.n_time, o, 0)
        res.append(o)
    torch.cuda.synchronize()
    return [r.cpu().numpy() for r in res]


def test_batch_equals_single_calls_bit_for_bit(arrays):
    import torch
    xforms = ["fft_fp32", "fft_fp32", "dft_bf16x3", "fft_fp32"]
    plans, vols, outs = _setup(arrays, xforms)
    ref = _single(plans, vols, arrays)
    b = epic.epic_batch_create(plans, vols, [w.n_time for w in arrays], outs, tune=False)
    for _ in range(2):
        for o in outs:
            o.fill_(float("nan"))
        epic.epic_batch_launch(b)
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)
    b.close()
    for p in plans:
        p.close()


def test_autotuned_batch_matches_oracle(arrays):
    import torch
    xforms = ["fft_fp32", "fft_fp32", "fft_fp32", "fft_fp32"]
    plans, vols, outs = _setup(arrays, xforms)
    ref = _single(plans, vols, arrays)
    b = epic.epic_batch_create(plans, vols, [w.n_time for w in arrays], outs, tune=True)
    assert all(1 <= c <= p.info["ctas"] for c, p in zip(b.ctas, plans))
    epic.epic_batch_launch(b)
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert rel_errors(o.cpu().numpy(), r, 2).max() <= REORDER_TOL
    # arrays A and C against the oracle on two channels each
    for k, chans in ((0, [0, 15]), (3, [0, 31])):
        got = outs[k].cpu().numpy()
        assert_close(got[chans], oracle_image(arrays[k], channels=chans, use_fft=True), 2)
    b.close()
    for p in plans:
        p.close()


def test_batch_rejects_bad_arguments(arrays):
    import torch
    plans, vols, outs = _setup(arrays[:1], ["fft_fp32"])
    with pytest.raises(epic.EpicError):
        epic.epic_batch_create(plans + plans, vols + vols, [300, 300], outs + outs)  # same plan twice
    for p in plans:
        p.close()


def test_tensor_batch_matches_single_calls(arrays):
    """The batched tensor-core path: arrays A (32^2), B (64^2) and C (128^2) on
    BF16 x3 in one graph."""
    import torch
    ws = [arrays[0], arrays[1], arrays[3]]
    xforms = ["dft_bf16x3", "dft_bf16x3", "dft_bf16x3"]
    plans, vols, outs = _setup(ws, xforms)
    ref = _single(plans, vols, ws)
    b = epic.epic_batch_create(plans, vols, [w.n_time for w in ws], outs, tune=True)
    epic.epic_batch_launch(b)
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert rel_errors(o.cpu().numpy(), r, 2).max() <= REORDER_TOL
    for k, chans in ((0, [0, 15]), (2, [0, 31])):
        got = outs[k].cpu().numpy()
        assert rel_errors(got[chans], oracle_image(ws[k], channels=chans, use_fft=True), 2).max() <= TOL["dft_bf16x3"]
    b.close()
    for p in plans:
        p.close()


def test_tensor_families_in_one_persistent_launch_bit_for_bit(arrays):
    """Tensor-core plans of one transform share one persistent launch that claims
    time tiles of every plan from a work list (32^2, 64^2 and 128^2 grids, 40 to
    1024 antennas); without tuning every tile is the span a CTA of a single call
    images, so the batch equals separate epic_image calls bit for bit.  Two
    transforms make two families; a plan with no samples is zeroed."""
    import torch
    xforms = ["dft_bf16x3", "dft_bf16x3", "dft_fp16", "dft_bf16x3"]
    plans, vols, outs = _setup(arrays, xforms)
    ref = _single(plans, vols, arrays)
    b = epic.epic_batch_create(plans, vols, [w.n_time for w in arrays], outs, tune=False)
    for _ in range(2):
        for o in outs:
            o.fill_(float("nan"))
        epic.epic_batch_launch(b)
        torch.cuda.synchronize()
        for k, (o, r) in enumerate(zip(outs, ref)):
            assert np.array_equal(o.cpu().numpy(), r), k
    for p in plans:
        epic.epic_sync(p)
    b.close()
    # an empty member
    n_time = [w.n_time for w in arrays]
    n_time[1] = 0
    b = epic.epic_batch_create(plans, vols, n_time, outs, tune=False)
    outs[1].fill_(float("nan"))
    epic.epic_batch_launch(b)
    torch.cuda.synchronize()
    assert not outs[1].any()
    assert np.array_equal(outs[3].cpu().numpy(), ref[3])
    b.close()
    for p in plans:
        p.close()


def test_batch_reduction_wait_times_out_and_the_batch_recovers(arrays):
    """A family's reduction items wait (bounded spin) for their channels' imaging
    items to signal; with one signal more expected than can come and a 2 ms
    limit, every reduction item must give up, its plan's epic_sync report
    EPIC_ERR_TIMEOUT, and the next launch of the same batch image as before."""
    import time

    import torch
    ws = [arrays[0], arrays[2]]
    plans, vols, outs = _setup(ws, ["dft_bf16x3", "dft_bf16x3"])
    ref = _single(plans, vols, ws)
    b = epic.epic_batch_create(plans, vols, [w.n_time for w in ws], outs, tune=False)
    t0 = time.time()
    epic.epic_debug_batch_timeout(b, 2_000_000)
    torch.cuda.synchronize()
    for p in plans:
        with pytest.raises(epic.EpicError) as ei:
            epic.epic_sync(p)
        assert ei.value.status == epic.EPIC_ERR_TIMEOUT
    assert time.time() - t0 < 60
    for o in outs:
        o.fill_(float("nan"))
    epic.epic_batch_launch(b)
    torch.cuda.synchronize()
    for p in plans:
        epic.epic_sync(p)
    for o, r in zip(outs, ref):
        assert np.array_equal(o.cpu().numpy(), r)
    b.close()
    for p in plans:
        p.close()
    # a batch without tensor-core families has nothing to time out
    plans, vols, outs = _setup(ws[:1], ["fft_fp32"])
    b = epic.epic_batch_create(plans, vols, [ws[0].n_time], outs, tune=False)
    with pytest.raises(epic.EpicError) as ei:
        epic.epic_debug_batch_timeout(b, 2_000_000)
    assert ei.value.status == epic.EPIC_ERR_UNSUPPORTED
    b.close()
    plans[0].close()
