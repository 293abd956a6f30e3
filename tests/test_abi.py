"""The C ABI without a GPU: the library loads, exports what include/epic.h
declares, and its host-only validation agrees with the oracle's geometry."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1904_11422_gb300 import build_lib, epic, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "epic.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(epic_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return epic.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("epic_plan_create", "epic_plan_destroy", "epic_image", "epic_plan_validate",
              "epic_debug_unpack", "epic_debug_grid", "epic_status_string", "epic_sync"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_exactly_the_header():
    assert sorted(epic.SIGNATURES) == _declared()


def test_struct_layouts_match_header():
    # ctypes mirrors of the two structs: field order and count as in include/epic.h
    src = open(HEADER).read()
    body = re.search(r"typedef struct \{([^{}]*)\} epic_plan_desc;", src).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)\s*;", body)
    assert fields == [f for f, _ in epic.epic_plan_desc._fields_]
    body = re.search(r"typedef struct \{([^{}]*)\} epic_plan_info;", src).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            names += [x.strip().split()[-1] for x in decl.split(",")]
    assert names == [f for f, _ in epic.epic_plan_info._fields_]


def test_status_strings(lib):
    for code, name in [(0, "EPIC_OK"), (1, "EPIC_ERR_INVALID_ARG"), (2, "EPIC_ERR_OFFGRID"),
                       (3, "EPIC_ERR_UNSUPPORTED"), (6, "EPIC_ERR_TIMEOUT"), (7, "EPIC_ERR_NO_DEVICE"),
                       (8, "EPIC_ERR_INTERNAL"), (99, "EPIC_ERR_UNKNOWN")]:
        assert epic.epic_status_string(code) == name


def _desc(**kw):
    w = synth.random_small(3, n_ant=5, n_pol=2, n_chan=2, grid_n=32, support=3)
    args = dict(ant_xy=w.ant_xy, chan_freq_hz=w.freq_hz, n_pol=2, grid_n=32, kernel_support=3,
                gains=w.gains, delays_s=w.delays_s)
    args.update(kw)
    return epic.make_desc(**args)


def test_validate_accepts_valid(lib):
    d, keep = _desc()
    assert epic.epic_plan_validate(d) == epic.EPIC_OK
    d, keep = _desc(grid_n=64)
    assert epic.epic_plan_validate(d) == epic.EPIC_OK
    d, keep = _desc(grid_n=128)
    assert epic.epic_plan_validate(d) == epic.EPIC_OK


@pytest.mark.parametrize("kw,code", [
    (dict(kernel_support=4), epic.EPIC_ERR_INVALID_ARG),
    (dict(kernel_support=17), epic.EPIC_ERR_INVALID_ARG),
    (dict(n_pol=3, gains=None, delays_s=None), epic.EPIC_ERR_INVALID_ARG),
    (dict(grid_n=48), epic.EPIC_ERR_INVALID_ARG),
    (dict(grid_n=256), epic.EPIC_ERR_UNSUPPORTED),
    (dict(n_pol=1, xform=1, gains=None, delays_s=None), epic.EPIC_ERR_UNSUPPORTED),
    (dict(cell_lambda=0.0), epic.EPIC_ERR_INVALID_ARG),
    (dict(kernel_sigma_cells=-1.0), epic.EPIC_ERR_INVALID_ARG),
    (dict(chan_freq_hz=[50e6, -1.0]), epic.EPIC_ERR_INVALID_ARG),
    (dict(chan_freq_hz=[50e6, np.nan]), epic.EPIC_ERR_INVALID_ARG),
    (dict(xform=9), epic.EPIC_ERR_INVALID_ARG),
    (dict(chan_freq_hz=[50e6, 5e9]), epic.EPIC_ERR_OFFGRID),
])
def test_validate_rejects(lib, kw, code):
    d, keep = _desc(**kw)
    assert epic.epic_plan_validate(d) == code


def test_validate_rejects_null_and_nan(lib):
    assert lib.epic_plan_validate(None) == epic.EPIC_ERR_INVALID_ARG
    w = synth.random_small(3, n_ant=5, n_pol=2, n_chan=2, grid_n=32, support=3)
    ant = w.ant_xy.copy()
    ant[2, 1] = np.inf
    d, keep = epic.make_desc(ant, w.freq_hz, 2, 32, 3)
    assert epic.epic_plan_validate(d) == epic.EPIC_ERR_INVALID_ARG
    g = w.gains.copy()
    g[1, 1, 1] = np.nan
    d, keep = epic.make_desc(w.ant_xy, w.freq_hz, 2, 32, 3, gains=g)
    assert epic.epic_plan_validate(d) == epic.EPIC_ERR_INVALID_ARG


def test_validate_offgrid_agrees_with_oracle(lib):
    # antennas scattered across and beyond the grid edge at 1 m cells
    rng = np.random.default_rng(17)
    N, S = 32, 5
    freq = [299792458.0 / 2, 299792458.0 / 2.3]
    agree = 0
    for trial in range(300):
        ant = rng.uniform(-17.5, 17.5, size=(1, 2))
        arr = oracle.OracleArray(ant, freq, 1, N, S, 0.5, 1.0)
        ok = all(oracle.antenna_kernel(arr, c, 0)[-1] for c in range(2))
        d, keep = epic.make_desc(ant, freq, 1, N, S, 0.5, 1.0)
        st = epic.epic_plan_validate(d)
        assert st == (epic.EPIC_OK if ok else epic.EPIC_ERR_OFFGRID), (ant, ok, st)
        agree += 1
    assert agree == 300


def test_no_cpu_fallback(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        epic.load_library(str(tmp_path / "missing.so"))


def test_validate_antenna_limits_per_grid(lib):
    """The FP32 path takes up to 2048 antennas on every grid size (128 x 128
    grids of large arrays run on clusters, the others as four folded 64 x 64
    problems)."""
    rng = np.random.default_rng(5)
    for n_ant, grid_n, code in [(1024, 128, epic.EPIC_OK), (1025, 128, epic.EPIC_OK),
                                (2048, 128, epic.EPIC_OK), (2049, 128, epic.EPIC_ERR_UNSUPPORTED),
                                (2048, 64, epic.EPIC_OK), (2049, 64, epic.EPIC_ERR_UNSUPPORTED)]:
        ant = (rng.random((n_ant, 2)) - 0.5) * 20.0  # within a few cells of the centre at 50 MHz
        d, keep = epic.make_desc(ant, [50e6], 2, grid_n, 3)
        assert epic.epic_plan_validate(d) == code, (n_ant, grid_n)


def test_validate_antenna_limits_small_grid_and_tensor_path(lib):
    """2048 antennas on the FP32 path at 32 x 32 as well; 1024 on the tensor path
    at every grid side it takes."""
    rng = np.random.default_rng(6)
    cases = [(2048, 32, epic.EPIC_XFORM_FFT_FP32, epic.EPIC_OK),
             (2049, 32, epic.EPIC_XFORM_FFT_FP32, epic.EPIC_ERR_UNSUPPORTED)]
    for grid_n in (32, 64, 128):
        cases += [(1024, grid_n, epic.EPIC_XFORM_DFT_BF16X3, epic.EPIC_OK),
                  (1025, grid_n, epic.EPIC_XFORM_DFT_BF16X3, epic.EPIC_ERR_UNSUPPORTED)]
    for n_ant, grid_n, xf, code in cases:
        ant = (rng.random((n_ant, 2)) - 0.5) * 20.0
        d, keep = epic.make_desc(ant, [50e6], 2, grid_n, 3, xform=xf)
        assert epic.epic_plan_validate(d) == code, (n_ant, grid_n, xf)


def test_binding_size_and_layout_checks():
    """Host-side argument checks of the binding (no GPU needed)."""
    import torch
    a = np.zeros(100, np.uint8)
    epic._check_size(a, 100, "x")
    epic._check_size(a.ctypes.data, 10**12, "x")  # a bare address is not checked
    with pytest.raises(ValueError, match="holds 100 bytes"):
        epic._check_size(a, 101, "x")
    with pytest.raises(ValueError):
        epic._check_size(torch.zeros(3, dtype=torch.float32), 13, "x")
    h = np.zeros(4, np.float32)
    assert epic._host_array(h, "float32", "h", 16) == h.ctypes.data
    with pytest.raises(ValueError, match="holds 16 bytes"):
        epic._host_array(h, "float32", "h", 17)
    with pytest.raises(ValueError, match="C-contiguous float32"):
        epic._host_array(np.zeros(4, np.float64), "float32", "h")
    with pytest.raises(ValueError, match="C-contiguous uint8"):
        epic._host_array(np.zeros((4, 4), np.uint8)[:, ::2], "uint8", "h")
    with pytest.raises(ValueError, match="contiguous torch.float32"):
        epic._host_array(torch.zeros(4, dtype=torch.float64), "float32", "h")
