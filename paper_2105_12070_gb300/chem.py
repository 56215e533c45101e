"""Python binding of the chemgpu C ABI (include/chemgpu.h): argument marshalling only.

Every step of the chemistry solve runs in the CUDA library; this module converts torch
tensors (device memory, the current stream) or numpy arrays (host memory) to pointers and
checks shapes.  The functions carry the ABI's names.  There is no CPU fallback: without the
built library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

CHEM_PREC_FP64 = 0
CHEM_PREC_MIXED = 1
CELL_STATUS = {0: "ok", 1: "max_steps", 2: "h_underflow", 3: "bad_input"}


class ChemOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("refine_sweeps", ctypes.c_int), ("max_steps", ctypes.c_int),
                ("use_queue", ctypes.c_int), ("cells_per_cta", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("warps_per_cell", ctypes.c_int), ("use_graph", ctypes.c_int), ("batch_cells", ctypes.c_int)]


class ChemStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("rejects", ctypes.c_int64), ("failed_cells", ctypes.c_int64),
                ("refine_fallbacks", ctypes.c_int64)]


class ChemError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libchemgpu.so (building it first if it is missing and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or _build._stale():
            if not build_if_missing:
                raise ChemError(f"libchemgpu.so is not built ({path}); run paper_2105_12070_gb300.build.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        vp, dp, ip, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
        lib.chem_last_error.restype = ctypes.c_char_p
        lib.chem_default_opts.argtypes = [ctypes.POINTER(ChemOpts)]
        lib.chem_load_mechanism.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
        lib.chem_free_mechanism.argtypes = [vp]
        lib.chem_mech_dims.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip)]
        lib.chem_rates.argtypes = [vp, dp, vp, vp, i64, vp, vp]
        lib.chem_jacobian.argtypes = [vp, dp, vp, vp, i64, vp, vp]
        lib.chem_integrate.argtypes = [vp, dp, vp, vp, i64, dp, dp, dp, vp, vp, ctypes.POINTER(ChemOpts),
                                       ctypes.POINTER(ChemStats), vp]
        lib.chem_last_cell_counters.argtypes = [vp, vp, vp, i64, vp]
        lib.chem_probe_fp64_peak.argtypes = [ctypes.POINTER(ctypes.c_double)]
        lib.chem_debug_exp.argtypes = [vp, vp, i64, vp]
        lib.chem_integrate_noalloc.argtypes = [vp, dp, vp, vp, i64, dp, dp, dp, vp, vp, vp, vp,
                                               ctypes.POINTER(ChemOpts), ctypes.POINTER(ChemStats), vp]
        for name in ("chem_load_mechanism", "chem_mech_dims", "chem_rates", "chem_jacobian", "chem_integrate",
                     "chem_last_cell_counters", "chem_probe_fp64_peak", "chem_integrate_noalloc",
                     "chem_debug_exp"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        raise ChemError(f"chemgpu error {rc}: {_lib.chem_last_error().decode()}")


def default_opts(**kw) -> ChemOpts:
    lib = load_library()
    o = ChemOpts()
    lib.chem_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, int(v))
    return o


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, is_device) of a contiguous array of the given numpy dtype; None stays None."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {tdt} tensor")
        return ctypes.c_void_p(x.data_ptr()), x.is_cuda
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    return ctypes.c_void_p(x.ctypes.data), False


def _stream(stream, any_device: bool):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if any_device:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


class Mechanism:
    """A mechanism loaded on the current CUDA device (chem_load_mechanism)."""

    def __init__(self, path: str):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.chem_load_mechanism(path.encode(), ctypes.byref(h)))
        self._h = h
        K, R = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.chem_mech_dims(self._h, ctypes.byref(K), ctypes.byref(R)))
        self.K, self.R, self.N = K.value, R.value, K.value
        self.path = path

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.chem_free_mechanism(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def chem_load_mechanism(path: str) -> Mechanism:
    return Mechanism(path)


def _cells(mech, T, Y):
    n = int(T.shape[0])
    if tuple(Y.shape) != (mech.K, n):
        raise ValueError(f"Y must have shape (K={mech.K}, ncells={n}), got {tuple(Y.shape)}")
    return n


def chem_rates(mech: Mechanism, p_Pa: float, T, Y, out, stream=None):
    """out[N, ncells] = f(phi) (Eq. 1) for every cell."""
    n = _cells(mech, T, Y)
    pT, dT = _ptr(T, np.float64)
    pY, _ = _ptr(Y, np.float64)
    po, _ = _ptr(out, np.float64)
    _check(mech._lib.chem_rates(mech.handle, float(p_Pa), pT, pY, n, po, _stream(stream, dT)))
    return out


def chem_jacobian(mech: Mechanism, p_Pa: float, T, Y, out, stream=None):
    """out[ncells, N, N] = d f / d phi (analytical) for every cell."""
    n = _cells(mech, T, Y)
    pT, dT = _ptr(T, np.float64)
    pY, _ = _ptr(Y, np.float64)
    po, _ = _ptr(out, np.float64)
    _check(mech._lib.chem_jacobian(mech.handle, float(p_Pa), pT, pY, n, po, _stream(stream, dT)))
    return out


def chem_integrate(mech: Mechanism, p_Pa: float, T, Y, dt: float, rtol: float = 1e-6, atol: float = 1e-10,
                   h_inout=None, status=None, opts: ChemOpts | None = None, want_stats: bool = False, stream=None):
    """Integrates every cell over dt in place (T[ncells], Y[K, ncells]).  Returns ChemStats if
    want_stats (this synchronises the stream), else None."""
    n = _cells(mech, T, Y)
    pT, dT = _ptr(T, np.float64)
    pY, _ = _ptr(Y, np.float64)
    ph, _ = _ptr(h_inout, np.float64)
    ps, _ = _ptr(status, np.int32)
    st = ChemStats() if want_stats else None
    _check(mech._lib.chem_integrate(mech.handle, float(p_Pa), pT, pY, n, float(dt), float(rtol), float(atol), ph, ps,
                                    ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(st) if st is not None else None, _stream(stream, dT)))
    return st


def chem_integrate_noalloc(mech: Mechanism, p_Pa: float, T, Y, dt: float, rtol: float = 1e-6, atol: float = 1e-10,
                           h_inout=None, status=None, steps=None, rejects=None, opts: ChemOpts | None = None,
                           want_stats: bool = False, stream=None):
    """chem_integrate for callers that cannot allocate device memory: device tensors only, at most
    262144 cells, scratch in a fixed array inside the library shared by all calls (calls that
    overlap on the GPU race).  Optional steps/rejects receive the per-cell counters."""
    n = _cells(mech, T, Y)
    pT, dT = _ptr(T, np.float64)
    pY, _ = _ptr(Y, np.float64)
    ph, _ = _ptr(h_inout, np.float64)
    ps, _ = _ptr(status, np.int32)
    pst, _ = _ptr(steps, np.int32)
    prj, _ = _ptr(rejects, np.int32)
    st = ChemStats() if want_stats else None
    _check(mech._lib.chem_integrate_noalloc(mech.handle, float(p_Pa), pT, pY, n, float(dt), float(rtol), float(atol),
                                            ph, ps, pst, prj, ctypes.byref(opts) if opts is not None else None,
                                            ctypes.byref(st) if st is not None else None, _stream(stream, dT)))
    return st


def chem_last_cell_counters(mech: Mechanism, steps, rejects, stream=None):
    n = int(steps.shape[0])
    ps, dev = _ptr(steps, np.int32)
    pr, _ = _ptr(rejects, np.int32)
    _check(mech._lib.chem_last_cell_counters(mech.handle, ps, pr, n, _stream(stream, dev)))


def chem_probe_fp64_peak() -> float:
    """Measured FP64 FMA throughput of the current device in TFLOP/s (roofline denominator)."""
    lib = load_library()
    v = ctypes.c_double()
    if lib.chem_probe_fp64_peak(ctypes.byref(v)) != 0:
        raise ChemError(lib.chem_last_error().decode())
    return v.value


def chem_debug_exp(x, out, stream=None):
    """out = the rate kernels' exponential of x (device float64 tensors), for the tests."""
    lib = load_library()
    px, dev = _ptr(x, np.float64)
    po, _ = _ptr(out, np.float64)
    rc = lib.chem_debug_exp(px, po, int(x.numel()), _stream(stream, dev))
    if rc != 0:
        raise ChemError(lib.chem_last_error().decode())
    return out
