"""Host-checked plan invariants (in place of a sanitizer, which this GPU pool
does not offer): for every gather-table layout the library builds, every index
the imaging kernels dereference lies within the plan's sizes and every lane's
entry list equals the one re-derived from the per-cell table."""
import re

import pytest

from paper_1904_11422_gb300 import build_lib, epic, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return epic.load_library()


CASES = [  # (id, transform, grid, antennas, support): one per table layout
    ("fft64", "fft_fp32", 64, 40, 5),
    ("fft32", "fft_fp32", 32, 20, 3),
    ("fft128_folded", "fft_fp32", 128, 30, 5),
    ("fft128_clusters", "fft_fp32", 128, 450, 5),
    ("pairs64", "dft_bf16x3", 64, 40, 5),
    ("pairs128_folded", "dft_bf16x3", 128, 30, 3),
    ("pairs32_padded", "dft_bf16x3", 32, 16, 3),
    ("fft64_largest", "fft_fp32", 64, 2048, 3),
]


@pytest.mark.parametrize("name,xf,grid_n,n_ant,support", CASES, ids=[c[0] for c in CASES])
def test_tables_hold_their_invariants(name, xf, grid_n, n_ant, support):
    w = synth.random_small(2400 + n_ant, n_ant=n_ant, n_pol=2, n_chan=3, grid_n=grid_n, support=support, n_time=2)
    plan = epic.plan_for(w, epic.XFORMS[xf])
    if name == "fft128_clusters":
        assert plan.info["cluster_dim"] == 2
    if name == "fft128_folded":
        assert plan.info["transforms_per_image"] == 4
    report = epic.epic_debug_check_plan(plan)
    assert report.startswith("ok:"), report
    # the check walked every real entry: table sets x A x S^2 (four sets per channel when folded)
    m = re.search(r"(\d+) table sets, (\d+) entries \((\d+) padding\)", report)
    sets, entries, padding = (int(v) for v in m.groups())
    assert sets == w.n_chan * plan.info["transforms_per_image"]
    assert entries - padding == sets * n_ant * support ** 2
    plan.close()


def test_station_tables_hold_their_invariants():
    w = synth.station(n_time=2)
    for xf in ("fft_fp32", "dft_bf16x3"):
        plan = epic.plan_for(w, epic.XFORMS[xf])
        assert epic.epic_debug_check_plan(plan).startswith("ok:")
        plan.close()
