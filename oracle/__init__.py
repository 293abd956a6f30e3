"""FP64 CPU oracle for E-field direct imaging (MOFF / EPIC).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, loads or calls it and
shares no code with it.

The arithmetic lives in ``epic_oracle.c`` (plain C, FP64, no blocking or
fusion); this module compiles it with gcc and marshals numpy arrays to it.
Each function cites the passage of the paper it implements (Eq. (2), Eq. (5),
Sec. 3.2, Fig. 2).
"""
from __future__ import annotations

import contextlib
import ctypes
import hashlib
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epic_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libepic_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_INT = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_uint8)


_CMD = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-Wall",
        "-Wno-unused-variable"]


def _stamp() -> str:
    """Hash of the source, the compile command and the host architecture."""
    h = hashlib.sha256()
    with open(_SRC, "rb") as f:
        h.update(f.read())
    h.update(" ".join(_CMD).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile ``libepic_oracle.so`` next to its source (gcc, OpenMP), unless the
    library there was built from the same source, command and architecture."""
    stamp = _stamp()
    stamp_path = _LIB_PATH + ".stamp"
    if not force and os.path.exists(_LIB_PATH) and os.path.exists(stamp_path):
        with open(stamp_path) as f:
            if f.read().strip() == stamp:
                return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(_CMD + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    with open(stamp_path + f".{os.getpid()}.tmp", "w") as f:
        f.write(stamp + "\n")
    os.replace(stamp_path + f".{os.getpid()}.tmp", stamp_path)
    return _LIB_PATH


class _Array(ctypes.Structure):
    _fields_ = [
        ("n_ant", ctypes.c_int), ("n_pol", ctypes.c_int), ("n_chan", ctypes.c_int),
        ("grid_n", ctypes.c_int), ("support", ctypes.c_int),
        ("cell_lambda", ctypes.c_double), ("sigma_cells", ctypes.c_double),
        ("ant_xy", _D), ("freq", _D), ("gains", _D), ("delays", _D),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            A = ctypes.POINTER(_Array)
            lib.eo_set_mutation.argtypes = [ctypes.c_int]
            lib.eo_get_mutation.restype = ctypes.c_int
            lib.eo_unpack.argtypes = [_U8, ctypes.c_int64, _I32, _I32]
            lib.eo_antenna_kernel.argtypes = [A, ctypes.c_int, ctypes.c_int, _D, _D, _INT, _INT, _D]
            lib.eo_antenna_kernel.restype = ctypes.c_int
            lib.eo_coef.argtypes = [A, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
            lib.eo_grid.argtypes = [A, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
            lib.eo_grid.restype = ctypes.c_int
            lib.eo_dft2.argtypes = [ctypes.c_int, _D, _D]
            lib.eo_fft2.argtypes = [ctypes.c_int, _D, _D]
            lib.eo_kernel_power.argtypes = [A, ctypes.c_int, ctypes.c_int, _D]
            lib.eo_image.argtypes = [A, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
            lib.eo_image.restype = ctypes.c_int
            lib.eo_visibilities.argtypes = [A, _U8, ctypes.c_int, ctypes.c_int, _D]
            lib.eo_fx_brute.argtypes = [A, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
            lib.eo_fx_brute.restype = ctypes.c_int
            lib.eo_fx_gridded.argtypes = [A, _U8, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
            lib.eo_fx_gridded.restype = ctypes.c_int
            lib.eo_max_threads.restype = ctypes.c_int
            lib.eo_grad_fx.argtypes = [A, _U8, ctypes.c_int, _D, _D, _D]
            lib.eo_grad_fx.restype = ctypes.c_int
            lib.eo_beam.argtypes = [A, ctypes.c_int, _D]
            lib.eo_stokes.argtypes = [ctypes.c_int, _D, _D]
            _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


class OracleArray:
    """Array description in the oracle's own terms (mirrors what a plan holds).

    ant_xy [A][2] metres, freq [C] Hz, gains [C][A][P] complex or None,
    delays [A][P] seconds or None.
    """

    def __init__(self, ant_xy, freq, n_pol, grid_n, support, cell_lambda=0.5,
                 sigma_cells=None, gains=None, delays=None):
        self.ant_xy = np.ascontiguousarray(ant_xy, dtype=np.float64).reshape(-1, 2)
        self.freq = np.ascontiguousarray(np.atleast_1d(freq), dtype=np.float64)
        self.n_ant = self.ant_xy.shape[0]
        self.n_chan = self.freq.shape[0]
        self.n_pol = int(n_pol)
        self.grid_n = int(grid_n)
        self.support = int(support)
        self.cell_lambda = float(cell_lambda)
        self.sigma_cells = float(sigma_cells if sigma_cells is not None
                                 else max(self.support - 1, 1) / 4.0)
        if gains is not None:
            g = np.asarray(gains, dtype=np.complex128).reshape(self.n_chan, self.n_ant, self.n_pol)
            self.gains = np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))
        else:
            self.gains = None
        self.delays = (np.ascontiguousarray(delays, dtype=np.float64).reshape(self.n_ant, self.n_pol)
                       if delays is not None else None)
        self._s = _Array(self.n_ant, self.n_pol, self.n_chan, self.grid_n, self.support,
                         self.cell_lambda, self.sigma_cells, _dptr(self.ant_xy), _dptr(self.freq),
                         _dptr(self.gains), _dptr(self.delays))

    @property
    def ref(self):
        return ctypes.byref(self._s)


def _volts(arr: OracleArray, volts):
    v = np.ascontiguousarray(volts, dtype=np.uint8)
    v = v.reshape(-1, arr.n_chan, arr.n_ant, arr.n_pol)
    return v, v.shape[0]


def set_mutation(m: int) -> None:
    _load().eo_set_mutation(int(m))


@contextlib.contextmanager
def mutation(m: int):
    """Plant mistake number ``m`` in the oracle for the duration (tests only)."""
    lib = _load()
    old = lib.eo_get_mutation()
    lib.eo_set_mutation(int(m))
    try:
        yield
    finally:
        lib.eo_set_mutation(old)


MUTATIONS = {
    "dft_sign": 1, "no_shift": 2, "transpose": 3, "delay_sign": 4, "no_norm": 5,
    "xy_conj": 6, "drop_last_t": 7, "auto_half": 8, "nibble_swap": 9,
}


def max_threads() -> int:
    return int(_load().eo_max_threads())


def unpack(data) -> tuple[np.ndarray, np.ndarray]:
    """Sec. 3.2: 4+4-bit complex bytes -> (real, imag) integer arrays."""
    d = np.ascontiguousarray(data, dtype=np.uint8).ravel()
    re = np.zeros(d.size, np.int32)
    im = np.zeros(d.size, np.int32)
    _load().eo_unpack(d.ctypes.data_as(_U8), d.size, re.ctypes.data_as(_I32), im.ctypes.data_as(_I32))
    return re, im


def antenna_kernel(arr: OracleArray, c: int, a: int):
    """(u, v, i0, j0, w[S][S], ok) of antenna a in channel c."""
    S = arr.support
    u = ctypes.c_double()
    v = ctypes.c_double()
    i0 = ctypes.c_int()
    j0 = ctypes.c_int()
    w = np.zeros((S, S), np.float64)
    rc = _load().eo_antenna_kernel(arr.ref, c, a, ctypes.byref(u), ctypes.byref(v),
                                   ctypes.byref(i0), ctypes.byref(j0), _dptr(w))
    return u.value, v.value, i0.value, j0.value, w, rc == 0


def coef(arr: OracleArray, c: int, a: int, p: int) -> complex:
    kr = ctypes.c_double()
    ki = ctypes.c_double()
    _load().eo_coef(arr.ref, c, a, p, ctypes.byref(kr), ctypes.byref(ki))
    return complex(kr.value, ki.value)


def grid(arr: OracleArray, volts, t: int, c: int, p: int) -> np.ndarray:
    """Eq. (5) inner bracket W * E' for one (t, c, p): complex [N][N]."""
    v, _ = _volts(arr, volts)
    g = np.zeros((arr.grid_n, arr.grid_n, 2), np.float64)
    rc = _load().eo_grid(arr.ref, v.ctypes.data_as(_U8), t, c, p, _dptr(g))
    if rc != 0:
        raise ValueError("antenna box leaves the grid")
    return g[..., 0] + 1j * g[..., 1]


def _xform(fn, g):
    g = np.asarray(g, dtype=np.complex128)
    N = g.shape[0]
    gi = np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))
    y = np.zeros((N, N, 2), np.float64)
    fn(N, _dptr(gi), _dptr(y))
    return y[..., 0] + 1j * y[..., 1]


def dft2(g) -> np.ndarray:
    """Eq. (5) transform, direct separable sum (pixel N/2 = zero frequency)."""
    return _xform(_load().eo_dft2, g)


def fft2(g) -> np.ndarray:
    """The same transform through the oracle's own radix-2 FFT (timing mode)."""
    return _xform(_load().eo_fft2, g)


def kernel_power(arr: OracleArray, c: int, a: int) -> np.ndarray:
    """|W_a(l,m)|^2 of antenna a in channel c on every pixel, [N][N]."""
    out = np.zeros((arr.grid_n, arr.grid_n), np.float64)
    _load().eo_kernel_power(arr.ref, c, a, _dptr(out))
    return out


def image(arr: OracleArray, volts, subtract: bool = True, c_lo: int = 0, c_hi: int | None = None,
          use_fft: bool = False, n_threads: int | None = None, return_autos: bool = False):
    """Accumulated EPIC images [c_hi-c_lo][4][N][N] (XX, YY, Re XY, Im XY)."""
    v, T = _volts(arr, volts)
    if c_hi is None:
        c_hi = arr.n_chan
    n_c = c_hi - c_lo
    N = arr.grid_n
    out = np.zeros((n_c, 4, N, N), np.float64)
    autos = np.zeros((n_c, arr.n_ant, 3, 2), np.float64)
    if n_threads is None:
        n_threads = max_threads()
    rc = _load().eo_image(arr.ref, v.ctypes.data_as(_U8), T, c_lo, c_hi, int(subtract), int(use_fft),
                          int(n_threads), _dptr(out), _dptr(autos))
    if rc != 0:
        raise ValueError("antenna box leaves the grid")
    if return_autos:
        return out, autos[..., 0] + 1j * autos[..., 1]
    return out


def visibilities(arr: OracleArray, volts, c: int) -> np.ndarray:
    """Eq. (2): V[pq][a][b] for pq in (XX, YY, XY), complex [3][A][A]."""
    v, T = _volts(arr, volts)
    out = np.zeros((3, arr.n_ant, arr.n_ant, 2), np.float64)
    _load().eo_visibilities(arr.ref, v.ctypes.data_as(_U8), T, c, _dptr(out))
    return out[..., 0] + 1j * out[..., 1]


def fx_brute(arr: OracleArray, volts, c: int, include_autos: bool) -> np.ndarray:
    """Brute-force FX image of channel c, [4][N][N]."""
    v, T = _volts(arr, volts)
    out = np.zeros((4, arr.grid_n, arr.grid_n), np.float64)
    rc = _load().eo_fx_brute(arr.ref, v.ctypes.data_as(_U8), T, c, int(include_autos), _dptr(out))
    if rc != 0:
        raise ValueError("antenna box leaves the grid")
    return out


def fx_gridded(arr: OracleArray, volts, c: int, include_autos: bool) -> np.ndarray:
    """Gridded FX image of channel c (visibilities gridded with the kernels'
    cross-correlation, then one transform), [4][N][N]."""
    v, T = _volts(arr, volts)
    out = np.zeros((4, arr.grid_n, arr.grid_n), np.float64)
    rc = _load().eo_fx_gridded(arr.ref, v.ctypes.data_as(_U8), T, c, int(include_autos), _dptr(out))
    if rc != 0:
        raise ValueError("antenna box leaves the grid")
    return out


def pixel_lm(N: int, cell_lambda: float, i: int, j: int) -> tuple[float, float]:
    """Reading R4: direction cosines of pixel (i, j) (column i, row j)."""
    return (i - N / 2) / (N * cell_lambda), (j - N / 2) / (N * cell_lambda)


def grad_fx(arr: OracleArray, volts, model):
    """Gradient of L = sum (I - M)^2 over XX, YY and all pixels and channels with
    respect to the complex gains, closed form from the FX image (small cases).
    Returns (loss, grad) with grad [C][A][P] complex = dL/dRe g + i dL/dIm g."""
    v, T = _volts(arr, volts)
    m = np.ascontiguousarray(model, np.float64).reshape(arr.n_chan, 2, arr.grid_n, arr.grid_n)
    g = np.zeros((arr.n_chan, arr.n_ant, arr.n_pol, 2), np.float64)
    loss = ctypes.c_double()
    rc = _load().eo_grad_fx(arr.ref, v.ctypes.data_as(_U8), T, _dptr(m), _dptr(g), ctypes.byref(loss))
    if rc != 0:
        raise ValueError("antenna box leaves the grid")
    return loss.value, g[..., 0] + 1j * g[..., 1]


def loss_epic(arr: OracleArray, volts, model) -> float:
    """L = sum over channels, XX and YY, pixels of (I - M)^2 with I from eo_image."""
    img = image(arr, volts, subtract=True)
    m = np.asarray(model, np.float64).reshape(arr.n_chan, 2, arr.grid_n, arr.grid_n)
    planes = [0] if arr.n_pol == 1 else [0, 1]
    return float(sum(np.sum((img[:, p] - m[:, p]) ** 2) for p in planes))


def beam(arr: OracleArray, c: int) -> np.ndarray:
    """Image of the illumination kernels of channel c: mean_a |W_a|^2, [N][N]."""
    out = np.zeros((arr.grid_n, arr.grid_n), np.float64)
    _load().eo_beam(arr.ref, c, _dptr(out))
    return out


def stokes(img4) -> np.ndarray:
    """Pseudo-Stokes I, Q, U, V planes from XX, YY, Re XY, Im XY ([4][N][N])."""
    x = np.ascontiguousarray(img4, np.float64)
    out = np.zeros_like(x)
    _load().eo_stokes(x.shape[-1] * x.shape[-2], _dptr(x), _dptr(out))
    return out
