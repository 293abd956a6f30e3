"""epic_image_noalloc: imaging without any device allocation.

Callers such as real-time streaming loops, or applications that account for
all device memory through their own allocator, cannot allocate while they run;
this entry point takes its scratch from the library's static device array.
Checked through the C ABI against epic_image, bit for bit (the two use the same
kernels, work split and summation order), on two calls in a row (the array
keeps the first call's contents when the second starts), on every FP32 kernel
family: 64 x 64, 32 x 32 single polarisation, a 128 x 128 grid folded into four
64 x 64 problems, and a 128 x 128 grid on two-CTA clusters.  This file is
collected last so that, if it fails, every other test has already run."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_1904_11422_gb300 import build_lib, epic, synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return epic.load_library()


def _align256(x):
    return (x + 255) // 256 * 256


def noalloc_scratch_bytes(plan, n_time):
    """Scratch one call needs, from the split epic_image uses: CTAs (clusters)
    over the channel-major units, each CTA's partial image slots = the channels
    it touches; partial images and self powers each rounded to 256 bytes."""
    info = plan.info
    vq = info["transforms_per_image"]
    units = info["n_chan"] * vq * n_time
    cap = min(info["ctas"], units)
    W = -(-units // cap)
    ctas = -(-units // W)
    spans = max((min(b * W + W, units) - 1) // n_time - (b * W) // n_time + 1 for b in range(ctas))
    ns = info["grid_n"] // 2 if vq == 4 else info["grid_n"]
    slots = ctas * spans
    return _align256(4 * slots * 4 * ns * ns) + _align256(4 * slots * info["n_ant"] * 4)


CASES = {
    "station": lambda: synth.station(),
    "small_single_pol": lambda: synth.random_small(811, n_ant=13, n_pol=1, n_chan=5, grid_n=32, support=3, n_time=9),
    # 40 x 5 x 5 = 1 000 gather entries per channel: four folded 64 x 64 problems
    "folded128": lambda: synth.random_small(814, n_ant=40, n_pol=2, n_chan=3, grid_n=128, support=5, n_time=5),
    # 450 x 5 x 5 = 11 250 entries per channel: two-CTA clusters
    "cluster128": lambda: synth.random_small(813, n_ant=450, n_pol=2, n_chan=1, grid_n=128, support=5, n_time=3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_equals_epic_image_on_two_calls(name):
    import torch
    w = CASES[name]()
    plan = epic.plan_for(w)
    if name == "folded128":
        assert plan.info["transforms_per_image"] == 4
    if name == "cluster128":
        assert plan.info["cluster_dim"] == 2
    assert noalloc_scratch_bytes(plan, w.n_time) <= epic.EPIC_NOALLOC_SCRATCH_BYTES
    dv = torch.from_numpy(w.volts).cuda()
    ref = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    epic.epic_image(plan, dv, w.n_time, ref, 0)
    epic.epic_sync(plan)
    ref_np = ref.cpu().numpy()
    assert np.isfinite(ref_np).all()
    for call in range(2):
        out = torch.full(plan.out_shape, float("nan"), dtype=torch.float32, device="cuda")
        epic.epic_image_noalloc(plan, dv, w.n_time, out, 0)
        epic.epic_sync(plan)
        assert np.array_equal(out.cpu().numpy(), ref_np), f"call {call}"
    plan.close()


def test_noalloc_accumulates_like_epic_image():
    import torch
    w = synth.random_small(815, n_ant=24, n_pol=2, n_chan=4, grid_n=64, support=5, n_time=7)
    plan = epic.plan_for(w)
    dv = torch.from_numpy(w.volts).cuda()
    start = torch.from_numpy(np.random.default_rng(815).standard_normal(plan.out_shape).astype(np.float32)).cuda()
    ref = start.clone()
    epic.epic_image(plan, dv, w.n_time, ref, 1)
    for call in range(2):
        out = start.clone()
        epic.epic_image_noalloc(plan, dv, w.n_time, out, 1)
        epic.epic_sync(plan)
        assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy()), f"call {call}"
    plan.close()


def test_noalloc_first_call_on_a_fresh_plan_and_allocates_nothing():
    import torch
    w = synth.random_small(816, n_ant=30, n_pol=2, n_chan=3, grid_n=64, support=3, n_time=6)
    plan = epic.plan_for(w)
    dv = torch.from_numpy(w.volts).cuda()
    a = torch.full(plan.out_shape, float("nan"), dtype=torch.float32, device="cuda")
    b = torch.full(plan.out_shape, float("nan"), dtype=torch.float32, device="cuda")
    epic.epic_image_noalloc(plan, dv, w.n_time, a, 0)  # the plan's first imaging call
    epic.epic_sync(plan)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    epic.epic_image_noalloc(plan, dv, w.n_time, b, 0)
    epic.epic_sync(plan)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    ref = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    epic.epic_image(plan, dv, w.n_time, ref, 0)
    epic.epic_sync(plan)
    assert np.array_equal(a.cpu().numpy(), ref.cpu().numpy())
    assert np.array_equal(b.cpu().numpy(), ref.cpu().numpy())
    plan.close()


def test_noalloc_first_call_in_a_fresh_process():
    """The address lookup of the process's first call, before any epic_image."""
    code = textwrap.dedent("""
        import numpy as np, torch
        from paper_1904_11422_gb300 import epic, synth
        w = synth.random_small(817, n_ant=20, n_pol=2, n_chan=2, grid_n=64, support=3, n_time=4)
        plan = epic.plan_for(w)
        dv = torch.from_numpy(w.volts).cuda()
        outs = []
        for k in range(2):
            o = torch.full(plan.out_shape, float("nan"), dtype=torch.float32, device="cuda")
            epic.epic_image_noalloc(plan, dv, w.n_time, o, 0)
            epic.epic_sync(plan)
            outs.append(o.cpu().numpy())
        ref = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
        epic.epic_image(plan, dv, w.n_time, ref, 0)
        epic.epic_sync(plan)
        assert all(np.array_equal(o, ref.cpu().numpy()) for o in outs)
        plan.close()
        print("ok")
    """)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


def test_noalloc_rejects_calls_beyond_the_scratch_size():
    import torch
    # 1 200 one-sample channels on 152 CTAs: each CTA's 8 units touch 8 channels,
    # 1 200 partial 64 x 64 images (78.6 MB) in all
    w = synth.random_small(812, n_ant=4, n_pol=2, n_chan=1200, grid_n=64, support=1, n_time=1,
                           freq_hz=np.full(1200, 50e6))
    plan = epic.plan_for(w)
    need = noalloc_scratch_bytes(plan, w.n_time)
    assert need > epic.EPIC_NOALLOC_SCRATCH_BYTES
    out = torch.zeros(plan.out_shape, dtype=torch.float32, device="cuda")
    dv = torch.from_numpy(w.volts).cuda()
    with pytest.raises(epic.EpicError) as ei:
        epic.epic_image_noalloc(plan, dv, w.n_time, out, 0)
    assert ei.value.status == epic.EPIC_ERR_UNSUPPORTED
    assert not out.any()  # nothing was launched
    plan.close()
