"""epic_image_noalloc: imaging without any device allocation.

Callers such as real-time streaming loops, or applications that account for
all device memory through their own allocator, cannot allocate while they run;
this entry point takes its scratch from the library's static device array.
Checked through the C ABI against epic_image on two calls in a row (the array
keeps the first call's contents when the second starts).  This file is
collected last so that, if it fails, every other test has already run."""
import numpy as np
import pytest

from paper_1904_11422_gb300 import build_lib, epic, synth

from _helpers import TOL_FP32, rel_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return epic.load_library()


@pytest.mark.parametrize("make", [lambda: synth.station(),
                                  lambda: synth.random_small(811, n_ant=13, n_pol=1, n_chan=5, grid_n=32,
                                                             support=3, n_time=9)],
                         ids=["station", "small_single_pol"])
def test_noalloc_matches_epic_image_on_two_calls(make):
    import torch
    w = make()
    plan = epic.plan_for(w)
    dv = torch.from_numpy(w.volts).cuda()
    ref = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    epic.epic_image(plan, dv, w.n_time, ref, 0)
    epic.epic_sync(plan)
    ref_np = ref.cpu().numpy()
    for call in range(2):
        out = torch.full(plan.out_shape, float("nan"), dtype=torch.float32, device="cuda")
        epic.epic_image_noalloc(plan, dv, w.n_time, out, 0)
        epic.epic_sync(plan)
        got = out.cpu().numpy()
        assert np.isfinite(got).all(), f"call {call}"
        assert rel_errors(got, ref_np, w.n_pol).max() <= TOL_FP32, f"call {call}"
    plan.close()


def test_noalloc_rejects_plans_beyond_the_scratch_size():
    import torch
    # enough channels that the partial images of one launch exceed the array
    w = synth.random_small(812, n_ant=4, n_pol=2, n_chan=1200, grid_n=64, support=1, n_time=1,
                           freq_hz=np.full(1200, 50e6))
    plan = epic.plan_for(w)
    assert plan.info["workspace_bytes"] > epic.EPIC_NOALLOC_SCRATCH_BYTES
    out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")
    dv = torch.from_numpy(w.volts).cuda()
    with pytest.raises(epic.EpicError) as ei:
        epic.epic_image_noalloc(plan, dv, w.n_time, out, 0)
    assert ei.value.status == epic.EPIC_ERR_UNSUPPORTED
    plan.close()
