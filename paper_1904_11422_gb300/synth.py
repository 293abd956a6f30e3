"""Seeded synthetic inputs shaped like an LWA station (no imaging arithmetic).

This module only draws random numbers and encodes them in the instrument's
formats; it holds none of the imaging method's arithmetic.  It is the one
module that both the CUDA path's tests/benchmark and the FP64 oracle's tests
take their inputs from.

Recipes (seeds: positions 1, voltages 2, sources 3, gains 4, each plus
100 x the config index):

* positions: uniform in a disk of the given diameter (r = R sqrt(U),
  theta = 2 pi U), minimum spacing by seeded rejection (at most 10**6 draws,
  otherwise an error).
* voltages: complex noise plus point sources.  A source in direction (l, m)
  reaches antenna a with the geometric phase exp(-2 pi i nu (x_a l + y_a m) / c)
  and a fresh complex-Gaussian amplitude per (time, channel), identical on X
  and Y.  The sum is quantised per component with round-half-to-even and
  saturated to [-8, 7].
* bytes: one byte per (time, channel, antenna, polarisation), cube order
  [T][C][A][P]; the real part is the high nibble and the imaginary part the
  low nibble, both 4-bit two's complement.
"""
from __future__ import annotations

import dataclasses

import numpy as np

C_LIGHT = 299792458.0


def disk_positions(n: int, diameter_m: float, min_spacing_m: float, seed: int,
                   max_draws: int = 10**6) -> np.ndarray:
    """[n][2] positions in metres, uniform in a disk, with a minimum spacing."""
    rng = np.random.default_rng(seed)
    R = 0.5 * diameter_m
    pts = np.zeros((n, 2), np.float64)
    k = 0
    draws = 0
    while k < n:
        draws += 1
        if draws > max_draws:
            raise RuntimeError(f"disk_positions: placed {k} of {n} antennas in {max_draws} draws")
        r = R * np.sqrt(rng.random())
        th = 2.0 * np.pi * rng.random()
        p = np.array([r * np.cos(th), r * np.sin(th)])
        if k and min_spacing_m > 0 and np.min(np.sum((pts[:k] - p) ** 2, axis=1)) < min_spacing_m ** 2:
            continue
        pts[k] = p
        k += 1
    return pts


def pack4(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Encode integer parts in [-8, 7] as 4+4-bit bytes (real high, imaginary low)."""
    re = np.asarray(re, np.int64)
    im = np.asarray(im, np.int64)
    if re.min(initial=0) < -8 or re.max(initial=0) > 7 or im.min(initial=0) < -8 or im.max(initial=0) > 7:
        raise ValueError("pack4: component outside [-8, 7]")
    return (((re & 15) << 4) | (im & 15)).astype(np.uint8)


def quantize4(z: np.ndarray) -> np.ndarray:
    """Round-half-to-even, saturate to [-8, 7], pack to bytes."""
    re = np.clip(np.rint(z.real), -8, 7).astype(np.int64)
    im = np.clip(np.rint(z.imag), -8, 7).astype(np.int64)
    return pack4(re, im)


def geometric_phase(ant_xy: np.ndarray, freq_hz: np.ndarray, l: float, m: float) -> np.ndarray:
    """[C][A] phase exp(-2 pi i nu (x l + y m) / c) of a far-field source at (l, m)."""
    delay = (ant_xy[:, 0] * l + ant_xy[:, 1] * m) / C_LIGHT  # [A] seconds
    return np.exp(-2j * np.pi * np.outer(freq_hz, delay))


@dataclasses.dataclass
class Workload:
    """Everything a plan and an imaging call need, plus the recipe's metadata."""
    name: str
    ant_xy: np.ndarray            # [A][2] metres
    freq_hz: np.ndarray           # [C]
    n_pol: int
    grid_n: int
    support: int
    cell_lambda: float
    sigma_cells: float
    volts: np.ndarray             # [T][C][A][P] uint8
    gains: np.ndarray | None = None    # [C][A][P] complex
    delays_s: np.ndarray | None = None  # [A][P]
    sources: list = dataclasses.field(default_factory=list)  # (pixel_i, pixel_j, amplitude)

    @property
    def n_ant(self):
        return self.ant_xy.shape[0]

    @property
    def n_chan(self):
        return self.freq_hz.shape[0]

    @property
    def n_time(self):
        return self.volts.shape[0]

    @property
    def units(self):
        """antenna x channel x time samples in the block."""
        return self.n_ant * self.n_chan * self.n_time


def pixel_direction(N: int, cell_lambda: float, i: int, j: int) -> tuple[float, float]:
    """Direction of the centre of output pixel (column i, row j): the recipe places
    sources on pixel centres l = (i - N/2)/(N cell), m = (j - N/2)/(N cell)."""
    return (i - N / 2) / (N * cell_lambda), (j - N / 2) / (N * cell_lambda)


def _source_block(rng, ant_xy, freq, n_time, n_pol, sources_lm_amp):
    """[T][C][A][P] complex sum of point sources with fresh complex-Gaussian amplitudes."""
    C = freq.shape[0]
    A = ant_xy.shape[0]
    out = np.zeros((n_time, C, A, n_pol), np.complex128)
    for (l, m, amp) in sources_lm_amp:
        ph = geometric_phase(ant_xy, freq, l, m)  # [C][A]
        s = (rng.standard_normal((n_time, C)) + 1j * rng.standard_normal((n_time, C))) / np.sqrt(2.0)
        out += (amp * s)[:, :, None, None] * ph[None, :, :, None]
    return out


def tiny(config_index: int = 0, noise_free: bool = False) -> Workload:
    """32 single-pol antennas in a 20 m disk, 1 channel at 50 MHz, 32x32 grid,
    3x3 Gaussian (sigma 0.5 cell), 16 samples of integers uniform in [-8, 7]
    plus one plane wave of amplitude 3 centred on pixel (N/2+3, N/2-2)."""
    base = 100 * config_index
    N, S, T, A = 32, 3, 16, 32
    ant = disk_positions(A, 20.0, 0.0, 1 + base)
    freq = np.array([50e6])
    rng_v = np.random.default_rng(2 + base)
    rng_s = np.random.default_rng(3 + base)
    pi, pj = N // 2 + 3, N // 2 - 2
    l, m = pixel_direction(N, 0.5, pi, pj)
    src = _source_block(rng_s, ant, freq, T, 1, [(l, m, 3.0)])
    if noise_free:
        z = src
    else:
        noise = (rng_v.integers(-8, 8, size=(T, 1, A, 1)) + 1j * rng_v.integers(-8, 8, size=(T, 1, A, 1)))
        z = noise + src
    return Workload("tiny", ant, freq, 1, N, S, 0.5, 0.5, quantize4(z), sources=[(pi, pj, 3.0)])


def station(config_index: int = 1, n_time: int = 1250, n_chan: int = 64, grid_n: int = 64,
            noise_sigma: float = 2.5) -> Workload:
    """256 dual-pol antennas in a 110 m disk (min spacing 5 m), 64 channels with
    centres spread evenly over 60-76 MHz, 64x64 grid at 0.5-wavelength cells,
    5x5 Gaussian (sigma 1 cell), 1250 samples (50 ms at 40 us) of complex
    Gaussian noise (sigma 2.5 per component) plus 3 point sources on pixel
    centres within 0.5 of the zenith, amplitudes 1.0 / 0.7 / 0.5 x sigma."""
    base = 100 * config_index
    A, S = 256, 5
    ant = disk_positions(A, 110.0, 5.0, 1 + base)
    freq = np.linspace(60e6, 76e6, n_chan)
    rng_v = np.random.default_rng(2 + base)
    rng_s = np.random.default_rng(3 + base)
    srcs = []
    lm_amp = []
    for amp in (1.0, 0.7, 0.5):
        while True:
            i, j = (int(x) for x in rng_s.integers(0, grid_n, size=2))
            l, m = pixel_direction(grid_n, 0.5, i, j)
            if l * l + m * m < 0.25 and (i, j) not in [(s[0], s[1]) for s in srcs]:
                break
        srcs.append((i, j, amp * noise_sigma))
        lm_amp.append((l, m, amp * noise_sigma))
    volts = np.empty((n_time, n_chan, A, 2), np.uint8)
    # channel by channel keeps the complex temporaries small
    for c in range(n_chan):
        z = noise_sigma * (rng_v.standard_normal((n_time, 1, A, 2)) + 1j * rng_v.standard_normal((n_time, 1, A, 2)))
        z += _source_block(rng_s, ant, freq[c:c + 1], n_time, 2, lm_amp)
        volts[:, c:c + 1] = quantize4(z)
    return Workload("station", ant, freq, 2, grid_n, S, 0.5, 1.0, volts, sources=srcs)


def random_gains(n_chan: int, n_ant: int, n_pol: int, seed: int, amp_spread: float = 0.1,
                 phase_spread: float = 0.3) -> np.ndarray:
    """[C][A][P] complex gains, |g| uniform in 1 +- amp_spread, phase uniform +- phase_spread rad."""
    rng = np.random.default_rng(seed)
    amp = 1.0 + amp_spread * (2.0 * rng.random((n_chan, n_ant, n_pol)) - 1.0)
    ph = phase_spread * (2.0 * rng.random((n_chan, n_ant, n_pol)) - 1.0)
    return amp * np.exp(1j * ph)


def random_small(seed: int, n_ant: int = 6, n_pol: int = 2, n_chan: int = 2, grid_n: int = 16,
                 support: int = 3, n_time: int = 5, diameter_m: float | None = None,
                 freq_hz=None, with_gains: bool = True, with_delays: bool = True) -> Workload:
    """Small random cases for brute-force checks: a few antennas, a small grid,
    uniform integer voltages, random gains and delays."""
    rng = np.random.default_rng(seed)
    if freq_hz is None:
        freq_hz = 40e6 + 30e6 * rng.random(n_chan)
    freq = np.asarray(freq_hz, np.float64)
    lam_min = C_LIGHT / freq.max()
    if diameter_m is None:
        # keep every box inside the grid at the highest channel
        diameter_m = 0.5 * lam_min * (grid_n - support - 3)
    ant = disk_positions(n_ant, diameter_m, 0.0, seed + 1)
    volts = pack4(rng.integers(-8, 8, size=(n_time, n_chan, n_ant, n_pol)),
                  rng.integers(-8, 8, size=(n_time, n_chan, n_ant, n_pol)))
    gains = random_gains(n_chan, n_ant, n_pol, seed + 2) if with_gains else None
    delays = (rng.random((n_ant, n_pol)) - 0.5) * 2e-8 if with_delays else None
    sigma = max(support - 1, 1) / 4.0
    return Workload(f"random{seed}", ant, freq, n_pol, grid_n, support, 0.5, sigma, volts,
                    gains=gains, delays_s=delays)


def channel_slice(w: Workload, lo: int, hi: int) -> Workload:
    """The channels [lo, hi) of a workload (voltages, frequencies, gains), as
    one rank of a channel-split run holds them."""
    import copy
    out = copy.copy(w)
    out.name = f"{w.name}[{lo}:{hi}]"
    out.freq_hz = np.ascontiguousarray(w.freq_hz[lo:hi])
    out.volts = np.ascontiguousarray(w.volts[:, lo:hi])
    out.gains = None if w.gains is None else np.ascontiguousarray(w.gains[lo:hi])
    return out


def saturated_plane_wave(seed: int, n_ant: int = 1024, grid_n: int = 64, n_chan: int = 2, n_time: int = 3,
                         support: int = 5, gain_amp: float = 16.0) -> Workload:
    """The largest fields a block can hold: one noise-free plane wave from a
    pixel centre near the zenith, at the 4-bit limit on every antenna (amplitude
    7 per component before quantisation, so most samples saturate), both
    polarisations, with gains of modulus gain_amp and random phases.  Antennas
    uniform in the largest disk whose boxes stay inside the grid."""
    rng = np.random.default_rng(seed)
    freq = np.linspace(60e6, 76e6, n_chan)
    lam_min = C_LIGHT / freq.max()
    ant = disk_positions(n_ant, 0.5 * lam_min * (grid_n - support - 3), 0.0, seed + 1)
    i, j = grid_n // 2 + 2, grid_n // 2 - 1
    l, m = pixel_direction(grid_n, 0.5, i, j)
    ph = geometric_phase(ant, freq, l, m)  # [C][A]
    s = np.exp(2j * np.pi * rng.random((n_time, n_chan)))
    z = 7.0 * np.sqrt(2.0) * s[:, :, None, None] * ph[None, :, :, None] * np.ones((1, 1, 1, 2))
    gains = gain_amp * np.exp(2j * np.pi * rng.random((n_chan, n_ant, 2)))
    return Workload(f"saturated{seed}", ant, freq, 2, grid_n, support, 0.5, max(support - 1, 1) / 4.0,
                    quantize4(z), gains=gains, sources=[(i, j, 7.0)])


def differentiation(config_index: int = 4, n_chan: int = 64, n_time: int = 1250, n_sources: int = 5,
                    noise_sigma: float = 2.5):
    """Gain calibration on the station block: the station array, complex gains
    with |g| uniform in 1 +- 0.1 and phase uniform in +- 0.3 rad (seed 4 + 100 x
    config index), and voltages of the station recipe.  Also returns the voltages
    of a noise-free sky of n_sources point sources on pixel centres (unit gains),
    from which the model image is formed by whoever calls this.
    Returns (workload with gains, noise-free sky workload)."""
    w = station(config_index=1, n_time=n_time, n_chan=n_chan)
    base = 100 * config_index
    w.gains = random_gains(w.n_chan, w.n_ant, w.n_pol, 4 + base)
    rng_s = np.random.default_rng(3 + base)
    lm_amp, srcs = [], []
    while len(srcs) < n_sources:
        i, j = (int(x) for x in rng_s.integers(0, w.grid_n, size=2))
        l, m = pixel_direction(w.grid_n, 0.5, i, j)
        if l * l + m * m < 0.25 and (i, j) not in [(q[0], q[1]) for q in srcs]:
            amp = noise_sigma * (1.0 - 0.15 * len(srcs))
            srcs.append((i, j, amp))
            lm_amp.append((l, m, amp))
    sky = np.empty_like(w.volts)
    for c in range(w.n_chan):
        z = _source_block(rng_s, w.ant_xy, w.freq_hz[c:c + 1], w.n_time, 2, lm_amp)
        sky[:, c:c + 1] = quantize4(z)
    sky_w = Workload("sky", w.ant_xy, w.freq_hz, 2, w.grid_n, w.support, w.cell_lambda, w.sigma_cells, sky,
                     sources=srcs)
    w.name = "differentiation"
    return w, sky_w


def batching_array(which: str, config_index: int = 3, n_time: int = 1250) -> Workload:
    """The arrays of the batching recipe, all dual-pol over 60-76 MHz with
    station-style noise + 3 point sources:
      'A': 64 antennas in a 50 m disk (min spacing 3 m), 32x32 grid, 16 channels, 3x3 kernel;
      'B': the station array (256 antennas, 110 m, 64x64, 64 channels, 5x5);
      'C': 1024 antennas in a 220 m disk (min spacing 3 m), 128x128 grid, 32 channels, 5x5."""
    spec = {"A": (64, 50.0, 3.0, 32, 16, 3), "B": (256, 110.0, 5.0, 64, 64, 5), "C": (1024, 220.0, 3.0, 128, 32, 5)}
    A, diam, dmin, N, C, S = spec[which]
    base = 100 * config_index + {"A": 0, "B": 10, "C": 20}[which]
    ant = disk_positions(A, diam, dmin, 1 + base)
    freq = np.linspace(60e6, 76e6, C)
    rng_v = np.random.default_rng(2 + base)
    rng_s = np.random.default_rng(3 + base)
    srcs, lm_amp = [], []
    sigma = 2.5
    for amp in (1.0, 0.7, 0.5):
        while True:
            i, j = (int(x) for x in rng_s.integers(0, N, size=2))
            l, m = pixel_direction(N, 0.5, i, j)
            if l * l + m * m < 0.25 and (i, j) not in [(q[0], q[1]) for q in srcs]:
                break
        srcs.append((i, j, amp * sigma))
        lm_amp.append((l, m, amp * sigma))
    volts = np.empty((n_time, C, A, 2), np.uint8)
    for c in range(C):
        z = sigma * (rng_v.standard_normal((n_time, 1, A, 2)) + 1j * rng_v.standard_normal((n_time, 1, A, 2)))
        z += _source_block(rng_s, ant, freq[c:c + 1], n_time, 2, lm_amp)
        volts[:, c:c + 1] = quantize4(z)
    return Workload(f"batch{which}", ant, freq, 2, N, S, 0.5, (S - 1) / 4.0, volts, sources=srcs)
