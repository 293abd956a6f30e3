"""Python binding of libepic.so: the C ABI of include/epic.h, same names.

Argument marshalling only.  Every step of the imaging path runs in the
library's CUDA kernels; there is no Python or CPU fallback: if libepic.so is
missing or cannot be loaded, every call raises.

Device buffers are passed as torch CUDA tensors (or raw integer addresses),
streams as ``torch.cuda.Stream`` objects, raw handles or ``None`` (the current
torch stream).  PyTorch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libepic.so")

EPIC_OK = 0
EPIC_ERR_INVALID_ARG = 1
EPIC_ERR_OFFGRID = 2
EPIC_ERR_UNSUPPORTED = 3
EPIC_ERR_OOM = 4
EPIC_ERR_CUDA = 5
EPIC_ERR_TIMEOUT = 6
EPIC_ERR_NO_DEVICE = 7
EPIC_ERR_INTERNAL = 8

EPIC_XFORM_FFT_FP32 = 0
EPIC_XFORM_DFT_BF16X3 = 1
EPIC_XFORM_DFT_FP16X3 = 2
EPIC_XFORM_DFT_BF16 = 3
EPIC_XFORM_DFT_FP16 = 4

EPIC_POST_STOKES = 1
EPIC_POST_BEAM = 2

XFORMS = {"fft_fp32": 0, "dft_bf16x3": 1, "dft_fp16x3": 2, "dft_bf16": 3, "dft_fp16": 4}

_D = ctypes.POINTER(ctypes.c_double)


class epic_plan_desc(ctypes.Structure):
    _fields_ = [
        ("n_ant", ctypes.c_int), ("n_pol", ctypes.c_int), ("n_chan", ctypes.c_int),
        ("grid_n", ctypes.c_int), ("kernel_support", ctypes.c_int),
        ("cell_lambda", ctypes.c_double), ("kernel_sigma_cells", ctypes.c_double),
        ("ant_xy_m", _D), ("chan_freq_hz", _D), ("gains", _D), ("delays_s", _D),
        ("xform", ctypes.c_int), ("subtract_autos", ctypes.c_int),
    ]


class epic_plan_info(ctypes.Structure):
    _fields_ = [
        ("n_ant", ctypes.c_int), ("n_pol", ctypes.c_int), ("n_chan", ctypes.c_int),
        ("grid_n", ctypes.c_int), ("kernel_support", ctypes.c_int), ("xform", ctypes.c_int),
        ("subtract_autos", ctypes.c_int), ("device", ctypes.c_int), ("ctas", ctypes.c_int),
        ("threads_per_cta", ctypes.c_int), ("device_bytes", ctypes.c_size_t),
        ("workspace_bytes", ctypes.c_size_t), ("max_time", ctypes.c_longlong),
        ("cluster_dim", ctypes.c_int), ("transform_n", ctypes.c_int), ("transforms_per_image", ctypes.c_int),
        ("unpack_warps", ctypes.c_uint),
    ]


class epic_kernel_time(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char * 32), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


# name -> (restype, argtypes); exactly the declarations of include/epic.h
_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "epic_plan_validate": (_I, [ctypes.POINTER(epic_plan_desc)]),
    "epic_plan_create": (_I, [ctypes.POINTER(epic_plan_desc), ctypes.POINTER(_P)]),
    "epic_plan_destroy": (_I, [_P]),
    "epic_plan_query": (_I, [_P, ctypes.POINTER(epic_plan_info)]),
    "epic_image": (_I, [_P, _P, _I, _P, _I, _P]),
    "epic_image_host": (_I, [_P, _P, _I, _P, _I, _P]),
    "epic_image_noalloc": (_I, [_P, _P, _I, _P, _I, _P]),
    "epic_sync": (_I, [_P, _P]),
    "epic_grad": (_I, [_P, _P, _I, _P, _P, _P, _P, _P]),
    "epic_postprocess": (_I, [_P, _P, _P, _I, ctypes.c_float, _P]),
    "epic_batch_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_P),
                               _I, ctypes.POINTER(_I), _P, ctypes.POINTER(_P)]),
    "epic_batch_launch": (_I, [_P, _P]),
    "epic_batch_destroy": (_I, [_P]),
    "epic_debug_batch_timeout": (_I, [_P, ctypes.c_longlong, _P]),
    "epic_status_string": (ctypes.c_char_p, [_I]),
    "epic_debug_unpack": (_I, [_P, ctypes.c_size_t, _P, _P]),
    "epic_debug_grid": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
    "epic_debug_transform": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
    "epic_debug_check_plan": (_I, [_P, ctypes.c_char_p, ctypes.c_size_t]),
    "epic_debug_fma_rate": (_I, [ctypes.c_longlong, ctypes.POINTER(ctypes.c_double), _P]),
    "epic_debug_image_timeout": (_I, [_P, _P, _I, ctypes.c_longlong, _P]),
    "epic_image_host_async": (_I, [_P, _P, _I, _P, _I, _P]),
    "epic_timing_enable": (_I, [_P, _I]),
    "epic_timing_read": (_I, [_P, ctypes.POINTER(epic_kernel_time), _I, ctypes.POINTER(_I)]),
}

_lib = None
_lock = threading.Lock()


class EpicError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {status_name(status)} ({status})")


def status_name(s: int) -> str:
    names = {0: "EPIC_OK", 1: "EPIC_ERR_INVALID_ARG", 2: "EPIC_ERR_OFFGRID", 3: "EPIC_ERR_UNSUPPORTED",
             4: "EPIC_ERR_OOM", 5: "EPIC_ERR_CUDA", 6: "EPIC_ERR_TIMEOUT", 7: "EPIC_ERR_NO_DEVICE",
             8: "EPIC_ERR_INTERNAL"}
    return names.get(int(s), "EPIC_ERR_UNKNOWN")


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libepic.so (built by ``build_lib.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libepic.so not found at {p}: build it with "
                               "paper_1904_11422_gb300.build_lib.build() (there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def _check(st: int, where: str):
    if st != EPIC_OK:
        raise EpicError(st, where)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _nbytes(x) -> int | None:
    if hasattr(x, "element_size"):
        return x.numel() * x.element_size()
    if isinstance(x, np.ndarray):
        return x.nbytes
    return None  # a bare address: its extent is the caller's to guarantee


def _check_size(x, nbytes: int | None, what: str) -> None:
    """The kernels index a buffer by the plan's sizes; a smaller one would be read
    or written out of bounds, so it is refused here."""
    have = _nbytes(x)
    if nbytes is not None and have is not None and have < nbytes:
        raise ValueError(f"{what} holds {have} bytes; this call needs {nbytes}")


def _dev_tensor(x, dtype_name: str, what: str, nbytes: int | None = None):
    if hasattr(x, "is_cuda"):
        if not x.is_cuda:
            raise ValueError(f"{what} must be a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        if str(x.dtype) != f"torch.{dtype_name}":
            raise ValueError(f"{what} must be torch.{dtype_name}, got {x.dtype}")
    _check_size(x, nbytes, what)
    return _ptr(x)


def _host_array(x, dtype_name: str, what: str, nbytes: int | None = None):
    """A host buffer: a C-contiguous numpy array or CPU tensor of the given dtype."""
    if hasattr(x, "is_cuda"):
        if x.is_cuda:
            raise ValueError(f"{what} must be a host (CPU) buffer")
        if not x.is_contiguous() or str(x.dtype) != f"torch.{dtype_name}":
            raise ValueError(f"{what} must be a contiguous torch.{dtype_name} tensor")
    elif isinstance(x, np.ndarray):
        if not x.flags.c_contiguous or x.dtype != np.dtype(dtype_name):
            raise ValueError(f"{what} must be a C-contiguous {dtype_name} array")
    _check_size(x, nbytes, what)
    return _ptr(x)


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """Owns an ``epic_plan*``; ``close()`` (or garbage collection) destroys it."""

    def __init__(self, handle: int, desc_arrays: dict):
        self.handle = handle
        self._arrays = desc_arrays
        self.info = epic_plan_query(self)

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None
            epic_plan_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def out_shape(self):
        i = self.info
        return (i["n_chan"], 4, i["grid_n"], i["grid_n"])

    def volts_bytes(self, n_time: int) -> int:
        """Bytes of a [n_time][n_chan][n_ant][n_pol] voltage block."""
        i = self.info
        return max(int(n_time), 0) * i["n_chan"] * i["n_ant"] * i["n_pol"]

    @property
    def out_bytes(self) -> int:
        i = self.info
        return 4 * i["n_chan"] * 4 * i["grid_n"] ** 2

    @property
    def gains_bytes(self) -> int:
        """Bytes of [n_chan][n_ant][n_pol][2] float gains (and gradients)."""
        i = self.info
        return 4 * i["n_chan"] * i["n_ant"] * i["n_pol"] * 2


def make_desc(ant_xy, chan_freq_hz, n_pol, grid_n, kernel_support, cell_lambda=0.5, kernel_sigma_cells=None,
              gains=None, delays_s=None, xform=EPIC_XFORM_FFT_FP32, subtract_autos=True):
    """Build an ``epic_plan_desc`` from numpy inputs; returns (desc, arrays kept alive)."""
    ant = np.ascontiguousarray(ant_xy, np.float64).reshape(-1, 2)
    freq = np.ascontiguousarray(np.atleast_1d(chan_freq_hz), np.float64)
    A, C = ant.shape[0], freq.shape[0]
    g = None
    if gains is not None:
        gc = np.asarray(gains, np.complex128).reshape(C, A, n_pol)
        g = np.ascontiguousarray(np.stack([gc.real, gc.imag], -1))
    dl = np.ascontiguousarray(delays_s, np.float64).reshape(A, n_pol) if delays_s is not None else None
    if kernel_sigma_cells is None:
        kernel_sigma_cells = max(kernel_support - 1, 1) / 4.0
    if isinstance(xform, str):
        xform = XFORMS[xform]
    dp = lambda a: a.ctypes.data_as(_D) if a is not None else None  # noqa: E731
    desc = epic_plan_desc(A, int(n_pol), C, int(grid_n), int(kernel_support), float(cell_lambda),
                          float(kernel_sigma_cells), dp(ant), dp(freq), dp(g), dp(dl), int(xform),
                          int(bool(subtract_autos)))
    return desc, {"ant": ant, "freq": freq, "gains": g, "delays": dl}


def desc_from_workload(w, xform=EPIC_XFORM_FFT_FP32, subtract_autos=True):
    return make_desc(w.ant_xy, w.freq_hz, w.n_pol, w.grid_n, w.support, w.cell_lambda, w.sigma_cells,
                     w.gains, w.delays_s, xform, subtract_autos)


# ---- the C ABI, one function per entry point ---------------------------------
def epic_plan_validate(desc: epic_plan_desc) -> int:
    return int(load_library().epic_plan_validate(ctypes.byref(desc)))


def epic_plan_create(desc: epic_plan_desc, keep=None) -> Plan:
    h = ctypes.c_void_p()
    _check(load_library().epic_plan_create(ctypes.byref(desc), ctypes.byref(h)), "epic_plan_create")
    return Plan(h.value, keep or {})


def epic_plan_destroy(plan) -> None:
    h = plan.handle if isinstance(plan, Plan) else plan
    _check(load_library().epic_plan_destroy(h), "epic_plan_destroy")


def epic_plan_query(plan) -> dict:
    info = epic_plan_info()
    h = plan.handle if isinstance(plan, Plan) else plan
    _check(load_library().epic_plan_query(h, ctypes.byref(info)), "epic_plan_query")
    return {k: getattr(info, k) for k, _ in epic_plan_info._fields_}


def epic_image(plan: Plan, d_volts, n_time: int, d_out, accumulate: int = 0, stream=None) -> None:
    v = _dev_tensor(d_volts, "uint8", "d_volts", plan.volts_bytes(n_time)) if d_volts is not None else None
    o = _dev_tensor(d_out, "float32", "d_out", plan.out_bytes)
    _check(load_library().epic_image(plan.handle, v, int(n_time), o, int(accumulate), _stream(stream)),
           "epic_image")


def epic_image_noalloc(plan: Plan, d_volts, n_time: int, d_out, accumulate: int = 0, stream=None) -> None:
    """epic_image without any device allocation: scratch from the library's static
    device array (EPIC_NOALLOC_SCRATCH_BYTES); calls that overlap on the GPU race."""
    v = _dev_tensor(d_volts, "uint8", "d_volts", plan.volts_bytes(n_time)) if d_volts is not None else None
    o = _dev_tensor(d_out, "float32", "d_out", plan.out_bytes)
    _check(load_library().epic_image_noalloc(plan.handle, v, int(n_time), o, int(accumulate), _stream(stream)),
           "epic_image_noalloc")


EPIC_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def epic_image_host(plan: Plan, h_volts, n_time: int, h_out, accumulate: int = 0, stream=None) -> None:
    v = _host_array(h_volts, "uint8", "h_volts", plan.volts_bytes(n_time)) if h_volts is not None else None
    o = _host_array(h_out, "float32", "h_out", plan.out_bytes)
    _check(load_library().epic_image_host(plan.handle, v, int(n_time), o, int(accumulate), _stream(stream)),
           "epic_image_host")


def epic_image_host_async(plan: Plan, h_volts, n_time: int, h_out, accumulate: int = 0, stream=None) -> None:
    """Enqueues imaging from pinned host buffers (see include/epic.h); the result is
    in h_out once epic_sync(plan, stream) returns."""
    v = _host_array(h_volts, "uint8", "h_volts", plan.volts_bytes(n_time)) if h_volts is not None else None
    o = _host_array(h_out, "float32", "h_out", plan.out_bytes)
    _check(load_library().epic_image_host_async(plan.handle, v, int(n_time), o, int(accumulate), _stream(stream)),
           "epic_image_host_async")


def epic_grad(plan: Plan, d_volts, n_time: int, d_gains, d_model, d_grad, d_loss, stream=None) -> None:
    """Loss and gain gradient of the image-plane calibration loss (see include/epic.h)."""
    model_bytes = 4 * plan.info["n_chan"] * 2 * plan.info["grid_n"] ** 2
    _check(load_library().epic_grad(plan.handle, _dev_tensor(d_volts, "uint8", "d_volts", plan.volts_bytes(n_time)),
                                    int(n_time), _dev_tensor(d_gains, "float32", "d_gains", plan.gains_bytes),
                                    _dev_tensor(d_model, "float32", "d_model", model_bytes),
                                    _dev_tensor(d_grad, "float32", "d_grad", plan.gains_bytes),
                                    _dev_tensor(d_loss, "float32", "d_loss", 4), _stream(stream)), "epic_grad")


def epic_postprocess(plan: Plan, d_in, d_out, flags: int, beam_floor: float = 1e-3, stream=None) -> None:
    """Pseudo-Stokes planes and/or kernel-imprint division (see include/epic.h)."""
    _check(load_library().epic_postprocess(plan.handle, _dev_tensor(d_in, "float32", "d_in", plan.out_bytes),
                                           _dev_tensor(d_out, "float32", "d_out", plan.out_bytes), int(flags),
                                           float(beam_floor), _stream(stream)), "epic_postprocess")


class Batch:
    """Owns an ``epic_batch*`` and keeps its plans and buffers alive."""

    def __init__(self, handle, plans, buffers, ctas):
        self.handle = handle
        self.plans = plans
        self._buffers = buffers
        self.ctas = ctas

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None
            epic_batch_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def epic_batch_create(plans, d_volts, n_time, d_out, tune: bool = False, stream=None) -> Batch:
    n = len(plans)
    hp = (_P * n)(*[p.handle for p in plans])
    if not (len(d_volts) == len(n_time) == len(d_out) == n):
        raise ValueError("plans, d_volts, n_time and d_out must have the same length")
    hv = (_P * n)(*[_dev_tensor(v, "uint8", "d_volts", p.volts_bytes(t)) for p, v, t in zip(plans, d_volts, n_time)])
    ht = (_I * n)(*[int(t) for t in n_time])
    ho = (_P * n)(*[_dev_tensor(o, "float32", "d_out", p.out_bytes) for p, o in zip(plans, d_out)])
    chosen = (_I * n)()
    h = _P()
    _check(load_library().epic_batch_create(hp, n, hv, ht, ho, int(bool(tune)), chosen, _stream(stream),
                                            ctypes.byref(h)), "epic_batch_create")
    return Batch(h.value, list(plans), (list(d_volts), list(d_out)), list(chosen))


def epic_batch_launch(batch: Batch, stream=None) -> None:
    _check(load_library().epic_batch_launch(batch.handle, _stream(stream)), "epic_batch_launch")


def epic_debug_batch_timeout(batch: Batch, wait_ns: int, stream=None) -> None:
    """The batch's tensor-core families with reduction waits that cannot succeed
    (see include/epic.h); the members' next epic_sync raises EPIC_ERR_TIMEOUT."""
    _check(load_library().epic_debug_batch_timeout(batch.handle, int(wait_ns), _stream(stream)),
           "epic_debug_batch_timeout")


def epic_batch_destroy(batch) -> None:
    h = batch.handle if isinstance(batch, Batch) else batch
    _check(load_library().epic_batch_destroy(h), "epic_batch_destroy")


def epic_sync(plan: Plan, stream=None) -> None:
    _check(load_library().epic_sync(plan.handle, _stream(stream)), "epic_sync")


def epic_status_string(status: int) -> str:
    return load_library().epic_status_string(int(status)).decode()


def epic_debug_unpack(d_in, n: int, d_out, stream=None) -> None:
    _check_size(d_in, max(int(n), 0), "d_in")
    _check_size(d_out, 2 * max(int(n), 0), "d_out")
    _check(load_library().epic_debug_unpack(_ptr(d_in), int(n), _ptr(d_out), _stream(stream)),
           "epic_debug_unpack")


def epic_debug_grid(plan: Plan, d_volts, n_time: int, t: int, c: int, p: int, d_grid, stream=None) -> None:
    _check_size(d_volts, plan.volts_bytes(n_time), "d_volts")
    _check_size(d_grid, 8 * plan.info["grid_n"] ** 2, "d_grid")
    _check(load_library().epic_debug_grid(plan.handle, _ptr(d_volts), int(n_time), int(t), int(c), int(p),
                                          _ptr(d_grid), _stream(stream)), "epic_debug_grid")


def epic_debug_transform(plan: Plan, d_volts, n_time: int, t: int, c: int, p: int, d_y, stream=None) -> None:
    _check_size(d_volts, plan.volts_bytes(n_time), "d_volts")
    _check_size(d_y, 8 * plan.info["grid_n"] ** 2, "d_y")
    _check(load_library().epic_debug_transform(plan.handle, _ptr(d_volts), int(n_time), int(t), int(c), int(p),
                                               _ptr(d_y), _stream(stream)), "epic_debug_transform")


def epic_debug_image_timeout(plan: Plan, d_volts, n_time: int, wait_ns: int, stream=None) -> None:
    """Tensor-core imaging whose first bounded wait per CTA cannot succeed (see
    include/epic.h); the next epic_sync raises EpicError(EPIC_ERR_TIMEOUT)."""
    _check_size(d_volts, plan.volts_bytes(n_time), "d_volts")
    _check(load_library().epic_debug_image_timeout(plan.handle, _ptr(d_volts), int(n_time), int(wait_ns),
                                                   _stream(stream)), "epic_debug_image_timeout")


def epic_debug_check_plan(plan: Plan) -> str:
    """Host check of the plan's gridding tables (see include/epic.h); returns the
    summary line, raises EpicError (EPIC_ERR_INTERNAL) with the first violated
    invariant."""
    buf = ctypes.create_string_buffer(512)
    st = load_library().epic_debug_check_plan(plan.handle, buf, len(buf))
    if st != EPIC_OK:
        raise EpicError(st, f"epic_debug_check_plan: {buf.value.decode()}")
    return buf.value.decode()


def epic_debug_fma_rate(iterations: int = 100000, stream=None) -> float:
    """Measured FP32 FMA rate of the GPU in TFLOP/s (synchronous)."""
    out = ctypes.c_double(0.0)
    _check(load_library().epic_debug_fma_rate(int(iterations), ctypes.byref(out), _stream(stream)),
           "epic_debug_fma_rate")
    return out.value


def epic_timing_enable(plan: Plan, enable: bool = True) -> None:
    _check(load_library().epic_timing_enable(plan.handle, int(bool(enable))), "epic_timing_enable")


def epic_timing_read(plan: Plan) -> dict:
    """{kernel kind: (launches, total device ms)} since timing was enabled."""
    buf = (epic_kernel_time * 16)()
    n = ctypes.c_int()
    _check(load_library().epic_timing_read(plan.handle, buf, 16, ctypes.byref(n)), "epic_timing_read")
    return {buf[k].kernel.decode(): (int(buf[k].launches), float(buf[k].total_ms)) for k in range(min(n.value, 16))}


def plan_for(w, xform=EPIC_XFORM_FFT_FP32, subtract_autos=True) -> Plan:
    """Plan for a ``synth.Workload``."""
    desc, keep = desc_from_workload(w, xform, subtract_autos)
    return epic_plan_create(desc, keep)
