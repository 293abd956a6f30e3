"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a textbook/library special case, brute force on tiny inputs or an
invariant.  ``test_planted_mistakes_are_caught`` plants plausible mistakes in
the oracle (on the CPU) and shows that at least one pin fails for each.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1904_11422_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C0 = 299792458.0


def _arr(w: synth.Workload, **kw):
    args = dict(gains=w.gains, delays=w.delays_s)
    args.update(kw)
    return oracle.OracleArray(w.ant_xy, w.freq_hz, w.n_pol, w.grid_n, w.support, w.cell_lambda,
                              w.sigma_cells, **args)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _unpack_np(volts):
    """Independent decoding for closed forms: two's complement of each nibble."""
    v = volts.astype(np.int64)
    hi, lo = v >> 4, v & 15
    return np.where(hi >= 8, hi - 16, hi), np.where(lo >= 8, lo - 16, lo)


# --------------------------------------------------------------------------
# Step 1: unpack (Sec. 3.2, reading R1)
# --------------------------------------------------------------------------
def test_unpack_golden_bytes(oracle_lib):
    rows = []
    with open(os.path.join(GOLDEN, "unpack_bytes.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                b, r, i = line.split()
                rows.append((int(b, 16), int(r), int(i)))
    data = np.array([r[0] for r in rows], np.uint8)
    re, im = oracle.unpack(data)
    assert list(re) == [r[1] for r in rows]
    assert list(im) == [r[2] for r in rows]


def test_unpack_inverts_packing_exhaustively(oracle_lib):
    # every (re, im) pair in [-8, 7]^2, encoded by arithmetic on non-negative residues
    pairs = [(r, i) for r in range(-8, 8) for i in range(-8, 8)]
    data = np.array([((r % 16) << 4) | (i % 16) for r, i in pairs], np.uint8)
    assert sorted(set(data.tolist())) == list(range(256))
    re, im = oracle.unpack(data)
    assert list(zip(re.tolist(), im.tolist())) == pairs


# --------------------------------------------------------------------------
# Step 2: kernel weights (reading R6)
# --------------------------------------------------------------------------
def test_kernel_weights_closed_form(oracle_lib):
    # frequency c0/2 gives lambda = 2 m, so with 0.5-wavelength cells one cell is 1 m
    N, S, sigma = 16, 5, 1.0
    ant = np.array([[0.0, 0.0], [1.3, -2.2], [-3.5, 0.49]])
    arr = oracle.OracleArray(ant, [C0 / 2], 1, N, S, 0.5, sigma)
    for a in range(3):
        u, v, i0, j0, w, ok = oracle.antenna_kernel(arr, 0, a)
        assert ok
        assert u == pytest.approx(ant[a, 0] + N / 2, abs=1e-12)
        assert v == pytest.approx(ant[a, 1] + N / 2, abs=1e-12)
        assert i0 == int(np.floor(u + 0.5)) - 2 and j0 == int(np.floor(v + 0.5)) - 2
        ii = np.arange(S) + i0
        jj = np.arange(S) + j0
        g = np.exp(-((ii[None, :] - u) ** 2 + (jj[:, None] - v) ** 2) / (2 * sigma ** 2))
        assert np.allclose(w, g / g.sum(), rtol=1e-13, atol=0)
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
    # antenna exactly on a cell centre: symmetric, centre/neighbour = exp(1/(2 sigma^2))
    _, _, _, _, w, _ = oracle.antenna_kernel(arr, 0, 0)
    assert np.allclose(w, w.T, atol=1e-16) and np.allclose(w, w[::-1, ::-1], atol=1e-16)
    assert w[2, 2] / w[2, 3] == pytest.approx(np.exp(0.5), rel=1e-13)
    # S = 1: the kernel is the single cell under the antenna with weight 1
    arr1 = oracle.OracleArray(ant, [C0 / 2], 1, N, 1, 0.5, 0.25)
    _, _, i0, j0, w1, ok = oracle.antenna_kernel(arr1, 0, 1)
    assert ok and w1.shape == (1, 1) and w1[0, 0] == 1.0 and (i0, j0) == (9, 6)


def test_offgrid_is_reported(oracle_lib):
    arr = oracle.OracleArray(np.array([[7.0, 0.0]]), [C0 / 2], 1, 16, 3, 0.5, 0.5)
    assert oracle.antenna_kernel(arr, 0, 0)[-1] is False  # box reaches column 16
    arr = oracle.OracleArray(np.array([[6.0, -6.0]]), [C0 / 2], 1, 16, 3, 0.5, 0.5)
    assert oracle.antenna_kernel(arr, 0, 0)[-1] is True
    arr = oracle.OracleArray(np.array([[6.0, -8.0]]), [C0 / 2], 1, 16, 3, 0.5, 0.5)
    assert oracle.antenna_kernel(arr, 0, 0)[-1] is False  # box reaches row -1


# --------------------------------------------------------------------------
# Step 3: calibration coefficient (reading R8)
# --------------------------------------------------------------------------
def test_coefficient_closed_form(oracle_lib):
    w = synth.random_small(11, n_ant=3, n_pol=2, n_chan=2)
    arr = _arr(w)
    for c in range(2):
        for a in range(3):
            for p in range(2):
                expect = w.gains[c, a, p] * np.exp(-2j * np.pi * w.freq_hz[c] * w.delays_s[a, p])
                assert oracle.coef(arr, c, a, p) == pytest.approx(expect, rel=1e-14)


# --------------------------------------------------------------------------
# Step 5: the transform (Eq. (5) sign, reading R3/R4) against numpy
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [4, 8, 16, 32, 64, 128])
def test_dft2_is_shifted_unnormalised_inverse_fft(oracle_lib, N):
    rng = np.random.default_rng(N)
    g = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    ref = np.fft.fftshift(np.fft.ifft2(g)) * N * N
    assert _rel(oracle.dft2(g), ref) < 1e-12
    assert _rel(oracle.fft2(g), ref) < 1e-12


def test_dft2_single_cell_closed_form(oracle_lib):
    # a unit value at cell (y0, x0) transforms to exp(+2 pi i ((i-N/2) x0 + (j-N/2) y0)/N)
    N, x0, y0 = 16, 5, 11
    g = np.zeros((N, N), complex)
    g[y0, x0] = 1.0
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ref = np.exp(2j * np.pi * ((ii - N / 2) * x0 + (jj - N / 2) * y0) / N)
    assert np.abs(oracle.dft2(g) - ref).max() < 1e-13


# --------------------------------------------------------------------------
# Steps 2-7 against step 8: EPIC == FX on tiny inputs (Eq. (2) and Eq. (5))
# --------------------------------------------------------------------------
CASES = [
    dict(seed=1, n_ant=5, n_pol=2, n_chan=2, grid_n=16, support=3),
    dict(seed=2, n_ant=8, n_pol=1, n_chan=1, grid_n=8, support=1),
    dict(seed=3, n_ant=4, n_pol=2, n_chan=1, grid_n=16, support=5),
    dict(seed=4, n_ant=7, n_pol=2, n_chan=2, grid_n=8, support=3, with_gains=False, with_delays=False),
    dict(seed=5, n_ant=3, n_pol=1, n_chan=3, grid_n=16, support=5, n_time=9),
    # the grid size of the 128^2 variants (2x padded station, batching array C)
    dict(seed=6, n_ant=6, n_pol=2, n_chan=1, grid_n=128, support=5, n_time=3),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"s{c['seed']}")
def test_epic_equals_fx_bruteforce_and_gridded(oracle_lib, case):
    w = synth.random_small(**case)
    arr = _arr(w)
    raw = oracle.image(arr, w.volts, subtract=False)
    sub = oracle.image(arr, w.volts, subtract=True)
    for c in range(w.n_chan):
        fx_all = oracle.fx_brute(arr, w.volts, c, include_autos=True)
        fx_cross = oracle.fx_brute(arr, w.volts, c, include_autos=False)
        fg_all = oracle.fx_gridded(arr, w.volts, c, include_autos=True)
        fg_cross = oracle.fx_gridded(arr, w.volts, c, include_autos=False)
        scale = np.abs(fx_all).max()
        assert np.abs(raw[c] - fx_all).max() / scale < 1e-12
        assert np.abs(raw[c] - fg_all).max() / scale < 1e-12
        assert np.abs(sub[c] - fx_cross).max() / scale < 1e-12
        assert np.abs(sub[c] - fg_cross).max() / scale < 1e-12


def test_tiny_config_equals_fx(oracle_lib):
    w = synth.tiny()
    arr = _arr(w)
    sub = oracle.image(arr, w.volts)[0]
    fg = oracle.fx_gridded(arr, w.volts, 0, include_autos=False)
    assert np.abs(sub - fg).max() / np.abs(fg).max() < 1e-12


# --------------------------------------------------------------------------
# Whole pipeline: plane wave (closed form)
# --------------------------------------------------------------------------
def _integer_array(seed, n_ant, N, half):
    """Antennas on integer cells (1 cell = 1 m at c0/2 with 0.5-wavelength cells)."""
    rng = np.random.default_rng(seed)
    cells = set()
    while len(cells) < n_ant:
        cells.add(tuple(int(x) for x in rng.integers(-half, half + 1, size=2)))
    return np.array(sorted(cells), np.float64)


def test_plane_wave_closed_form_every_pixel(oracle_lib):
    # S = 1 and integer cells: the image is T |sum_a q_a exp(+2 pi i f.x_a / N)|^2 exactly
    N, A, T = 16, 9, 3
    ant = _integer_array(7, A, N, 6)
    pi, pj = N // 2 + 3, N // 2 - 2
    l0, m0 = synth.pixel_direction(N, 0.5, pi, pj)
    ph = synth.geometric_phase(ant, np.array([C0 / 2]), l0, m0)[0]  # [A]
    z = np.broadcast_to((7.0 * ph)[None, None, :, None], (T, 1, A, 1))
    volts = synth.quantize4(z)
    arr = oracle.OracleArray(ant, [C0 / 2], 1, N, 1, 0.5, 0.25)
    img = oracle.image(arr, volts, subtract=False)[0, 0]
    re, im = _unpack_np(volts[0, 0, :, 0])
    q = re + 1j * im
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    phase = 2j * np.pi * ((ii[..., None] - N / 2) * ant[:, 0] + (jj[..., None] - N / 2) * ant[:, 1]) / N
    expect = T * np.abs((q * np.exp(phase)).sum(-1)) ** 2
    assert np.abs(img - expect).max() / expect.max() < 1e-12
    assert np.unravel_index(np.argmax(img), img.shape) == (pj, pi)


def test_plane_wave_peak_tiny_noise_free(oracle_lib):
    w = synth.tiny(noise_free=True)
    img = oracle.image(_arr(w), w.volts, subtract=False)[0, 0]
    (pi, pj, _), = w.sources
    assert np.unravel_index(np.argmax(img), img.shape) == (pj, pi)


def test_delay_compensation_moves_zenith_source(oracle_lib):
    # zenith voltages calibrated with tau_a = (x_a l0 + y_a m0)/c image like a source at (l0, m0)
    N, A, T = 16, 9, 2
    ant = _integer_array(8, A, N, 6)
    pi, pj = N // 2 - 4, N // 2 + 1
    l0, m0 = synth.pixel_direction(N, 0.5, pi, pj)
    tau = (ant[:, 0] * l0 + ant[:, 1] * m0) / C0
    volts = synth.quantize4(np.full((T, 1, A, 1), 5.0 + 2.0j))
    arr = oracle.OracleArray(ant, [C0 / 2], 1, N, 1, 0.5, 0.25, delays=tau[:, None])
    img = oracle.image(arr, volts, subtract=False)[0, 0]
    assert np.unravel_index(np.argmax(img), img.shape) == (pj, pi)
    assert img.max() == pytest.approx(T * A * A * 29.0, rel=1e-12)


# --------------------------------------------------------------------------
# Parseval, special cases and invariants
# --------------------------------------------------------------------------
def test_parseval(oracle_lib):
    w = synth.random_small(21, n_ant=6, n_pol=2, n_chan=1, grid_n=16, support=3, n_time=4)
    arr = _arr(w)
    raw = oracle.image(arr, w.volts, subtract=False)[0]
    N = w.grid_n
    for p, plane in ((0, 0), (1, 1)):
        energy = sum(np.sum(np.abs(oracle.grid(arr, w.volts, t, 0, p)) ** 2) for t in range(w.n_time))
        assert raw[plane].sum() == pytest.approx(N * N * energy, rel=1e-12)


def test_single_antenna_subtracts_to_zero(oracle_lib):
    w = synth.random_small(31, n_ant=1, n_pol=2, n_chan=2, grid_n=16, support=5)
    arr = _arr(w)
    raw = oracle.image(arr, w.volts, subtract=False)
    sub = oracle.image(arr, w.volts, subtract=True)
    assert np.abs(sub).max() < 1e-12 * np.abs(raw).max()


def test_two_antenna_fringe_closed_form(oracle_lib):
    N, T = 16, 6
    ant = np.array([[3.0, -2.0], [-1.0, 4.0]])
    rng = np.random.default_rng(5)
    volts = synth.pack4(rng.integers(-8, 8, (T, 1, 2, 1)), rng.integers(-8, 8, (T, 1, 2, 1)))
    arr = oracle.OracleArray(ant, [C0 / 2], 1, N, 1, 0.5, 0.25)
    sub = oracle.image(arr, volts, subtract=True)[0, 0]
    re, im = _unpack_np(volts[:, 0, :, 0])
    e = re + 1j * im
    v12 = np.sum(e[:, 0] * np.conj(e[:, 1]))
    jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    d = ant[0] - ant[1]
    expect = 2 * np.real(v12 * np.exp(2j * np.pi * ((ii - N / 2) * d[0] + (jj - N / 2) * d[1]) / N))
    assert np.abs(sub - expect).max() < 1e-12 * np.abs(expect).max()


def test_invariants(oracle_lib):
    w = synth.random_small(41, n_ant=6, n_pol=2, n_chan=2, grid_n=16, support=3, n_time=6)
    arr = _arr(w)
    raw = oracle.image(arr, w.volts, subtract=False)
    scale = np.abs(raw).max()
    xx, yy, xyr, xyi = raw[:, 0], raw[:, 1], raw[:, 2], raw[:, 3]
    assert xx.min() >= -1e-12 * scale and yy.min() >= -1e-12 * scale
    assert np.all(xyr ** 2 + xyi ** 2 <= xx * yy * (1 + 1e-10) + 1e-12 * scale ** 2)
    # gains x alpha -> images x |alpha|^2
    alpha = 0.7 - 1.9j
    arr2 = _arr(w, gains=w.gains * alpha)
    for sub in (False, True):
        a = oracle.image(arr, w.volts, subtract=sub)
        b = oracle.image(arr2, w.volts, subtract=sub)
        assert np.abs(b - abs(alpha) ** 2 * a).max() < 1e-12 * abs(alpha) ** 2 * scale
    # additive in time, with and without subtraction
    for sub in (False, True):
        whole = oracle.image(arr, w.volts, subtract=sub)
        halves = oracle.image(arr, w.volts[:2], subtract=sub) + oracle.image(arr, w.volts[2:], subtract=sub)
        assert np.abs(whole - halves).max() < 1e-12 * scale
    # channels independent: a channel imaged alone equals its slice of the whole
    one = oracle.OracleArray(w.ant_xy, w.freq_hz[1:2], 2, w.grid_n, w.support, 0.5, w.sigma_cells,
                             gains=w.gains[1:2], delays=w.delays_s)
    alone = oracle.image(one, np.ascontiguousarray(w.volts[:, 1:2]))
    assert np.abs(alone[0] - oracle.image(arr, w.volts)[1]).max() < 1e-13 * scale


def test_integer_translation_leaves_image(oracle_lib):
    # moving every antenna by whole cells changes no kernel and only a common phase
    N, A = 16, 5
    rng = np.random.default_rng(9)
    ant = rng.uniform(-3.0, 3.0, size=(A, 2))
    volts = synth.pack4(rng.integers(-8, 8, (4, 1, A, 2)), rng.integers(-8, 8, (4, 1, A, 2)))
    a1 = oracle.OracleArray(ant, [C0 / 2], 2, N, 3, 0.5, 0.5)
    a2 = oracle.OracleArray(ant + np.array([2.0, -3.0]), [C0 / 2], 2, N, 3, 0.5, 0.5)
    for sub in (False, True):
        x1 = oracle.image(a1, volts, subtract=sub)
        x2 = oracle.image(a2, volts, subtract=sub)
        assert np.abs(x1 - x2).max() < 1e-12 * np.abs(x1).max()


def test_fft_mode_matches_direct_mode(oracle_lib):
    w = synth.random_small(51, n_ant=6, n_pol=2, n_chan=2, grid_n=16, support=3)
    arr = _arr(w)
    a = oracle.image(arr, w.volts, use_fft=False)
    b = oracle.image(arr, w.volts, use_fft=True)
    assert _rel(b, a) < 1e-12


def test_thread_count_does_not_change_result(oracle_lib):
    w = synth.random_small(61, n_ant=5, n_pol=2, n_chan=4, grid_n=8, support=3)
    arr = _arr(w)
    a = oracle.image(arr, w.volts, n_threads=1)
    b = oracle.image(arr, w.volts, n_threads=4)
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# Planted mistakes: every one must break at least one pin
# --------------------------------------------------------------------------
def _pins_pass():
    """Quick versions of the pins above; returns {name: passed}."""
    res = {}

    def run(name, fn):
        try:
            fn()
            res[name] = True
        except AssertionError:
            res[name] = False

    run("unpack", lambda: test_unpack_golden_bytes(None))
    run("weights", lambda: test_kernel_weights_closed_form(None))
    run("numpy", lambda: test_dft2_is_shifted_unnormalised_inverse_fft(None, 8))
    run("fx", lambda: test_epic_equals_fx_bruteforce_and_gridded(None, CASES[0]))
    run("plane_wave", test_plane_wave_closed_form_every_pixel_wrapper)
    run("delay", lambda: test_delay_compensation_moves_zenith_source(None))
    run("parseval", lambda: test_parseval(None))
    run("fringe", lambda: test_two_antenna_fringe_closed_form(None))
    run("single", lambda: test_single_antenna_subtracts_to_zero(None))
    run("invariants", lambda: test_invariants(None))
    return res


def test_plane_wave_closed_form_every_pixel_wrapper():
    test_plane_wave_closed_form_every_pixel(None)


@pytest.mark.parametrize("name", sorted(oracle.MUTATIONS))
def test_planted_mistakes_are_caught(oracle_lib, name):
    with oracle.mutation(oracle.MUTATIONS[name]):
        res = _pins_pass()
    failed = [k for k, ok in res.items() if not ok]
    assert failed, f"planted mistake {name!r} passed every pin"


def test_pins_pass_without_mutation(oracle_lib):
    res = _pins_pass()
    assert all(res.values()), res


# --------------------------------------------------------------------------
# Gain gradient of the image-plane loss: FX closed form against central
# finite differences of the EPIC-form image (two independent computations)
# --------------------------------------------------------------------------
def _grad_case(seed, **kw):
    w = synth.random_small(seed, **kw)
    arr = _arr(w)
    rng = np.random.default_rng(seed + 1000)
    model = rng.standard_normal((w.n_chan, 2, w.grid_n, w.grid_n)) * 50.0
    return w, arr, model


@pytest.mark.parametrize("seed,kw", [
    (1201, dict(n_ant=5, n_pol=2, n_chan=2, grid_n=16, support=3, n_time=4)),
    (1202, dict(n_ant=4, n_pol=1, n_chan=1, grid_n=16, support=5, n_time=6)),
    (1203, dict(n_ant=6, n_pol=2, n_chan=1, grid_n=8, support=1, n_time=3)),
])
def test_gradient_fx_closed_form_matches_finite_differences(oracle_lib, seed, kw):
    w, arr, model = _grad_case(seed, **kw)
    loss, grad = oracle.grad_fx(arr, w.volts, model)
    assert loss == pytest.approx(oracle.loss_epic(arr, w.volts, model), rel=1e-10)
    rng = np.random.default_rng(seed)
    h = 1e-4
    idx = [tuple(int(x) for x in (rng.integers(w.n_chan), rng.integers(w.n_ant), rng.integers(w.n_pol)))
           for _ in range(12)]
    scale = np.abs(grad).max()
    for (c, a, p) in idx:
        fd = 0j
        for unit in (1.0, 1j):
            gp = w.gains.copy()
            gm = w.gains.copy()
            gp[c, a, p] += h * unit
            gm[c, a, p] -= h * unit
            lp = oracle.loss_epic(_arr(w, gains=gp), w.volts, model)
            lm = oracle.loss_epic(_arr(w, gains=gm), w.volts, model)
            fd += unit * (lp - lm) / (2 * h)
        assert abs(fd - grad[c, a, p]) <= 1e-6 * scale, (c, a, p, fd, grad[c, a, p])


# --------------------------------------------------------------------------
# Post-processing: kernel imprint and pseudo-Stokes
# --------------------------------------------------------------------------
def test_beam_is_one_at_zero_frequency_and_bounded(oracle_lib):
    w = synth.random_small(1401, n_ant=6, n_pol=2, n_chan=2, grid_n=16, support=5)
    arr = _arr(w)
    for c in range(2):
        b = oracle.beam(arr, c)
        N = w.grid_n
        assert b[N // 2, N // 2] == pytest.approx(1.0, abs=1e-14)  # every kernel sums to 1
        assert b.max() <= 1.0 + 1e-14 and b.min() >= 0.0
        # S = 1: a single unit weight, flat imprint
    arr1 = oracle.OracleArray(w.ant_xy, w.freq_hz, 2, w.grid_n, 1, 0.5, 0.25)
    assert np.allclose(oracle.beam(arr1, 0), 1.0, atol=1e-14)


def _four_planes(yx, yy):
    return np.stack([np.sum(np.abs(yx) ** 2, 0), np.sum(np.abs(yy) ** 2, 0),
                     np.sum((yx * np.conj(yy)).real, 0), np.sum((yx * np.conj(yy)).imag, 0)])


def test_stokes_of_unpolarised_linear_and_circular_sources(oracle_lib):
    rng = np.random.default_rng(5)
    N = 4
    yx = rng.standard_normal((200, N, N)) + 1j * rng.standard_normal((200, N, N))
    # unpolarised: the incoherent sum of two orthogonal linear states, samples
    # (s, s) and (s, -s): XX = YY and XY = 0 exactly, so Q = U = V = 0, I = 2 XX
    yx_u = np.concatenate([yx, yx])
    yy_u = np.concatenate([yx, -yx])
    img = _four_planes(yx_u, yy_u)
    st = oracle.stokes(img)
    assert np.allclose(st[0], 2 * img[0]) and np.all(st[0] > 0)
    assert np.allclose(st[1], 0) and np.allclose(st[2], 0) and np.allclose(st[3], 0)
    # linear at 45 degrees: Y_Y = Y_X gives I = 2 XX, Q = 0, U = I, V = 0
    img = _four_planes(yx, yx)
    st = oracle.stokes(img)
    assert np.allclose(st[0], 2 * img[0]) and np.allclose(st[1], 0) and np.allclose(st[2], st[0])
    assert np.allclose(st[3], 0)
    # linear along x: Y_Y = 0 gives Q = I, U = V = 0
    st = oracle.stokes(_four_planes(yx, 0 * yx))
    assert np.allclose(st[1], st[0]) and np.allclose(st[2], 0) and np.allclose(st[3], 0)
    # circular: Y_Y = -i Y_X gives XY = Y_X conj(Y_Y) = i |Y_X|^2, so V = 2 |Y_X|^2 = I
    yy = -1j * yx
    img = np.stack([np.sum(np.abs(yx) ** 2, 0), np.sum(np.abs(yy) ** 2, 0),
                    np.sum((yx * np.conj(yy)).real, 0), np.sum((yx * np.conj(yy)).imag, 0)])
    st = oracle.stokes(img)
    assert np.allclose(st[3], st[0]) and np.allclose(st[1], 0) and np.allclose(st[2], 0)
