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

CHEM_SOLVER_ROSENBROCK = 0
CHEM_SOLVER_SEULEX = 1
CHEM_JAC_ANALYTIC = 0
CHEM_JAC_FD = 1
CHEM_PREC_FP64 = 0
CHEM_PREC_MIXED = 1
CHEM_PREC_MIXED_FF = 2
CELL_STATUS = {0: "ok", 1: "max_steps", 2: "h_underflow", 3: "bad_input", 4: "record_full"}
CHEM_CELL_RECORD_FULL = 4


class ChemOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("refine_sweeps", ctypes.c_int), ("max_steps", ctypes.c_int),
                ("use_queue", ctypes.c_int), ("cells_per_cta", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("warps_per_cell", ctypes.c_int), ("use_graph", ctypes.c_int), ("batch_cells", ctypes.c_int),
                ("solver", ctypes.c_int), ("jacobian", ctypes.c_int)]


class ChemStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("rejects", ctypes.c_int64), ("failed_cells", ctypes.c_int64),
                ("refine_fallbacks", ctypes.c_int64), ("kernel_ms", ctypes.c_double)]


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
        lib.chem_describe_mechanism.argtypes = [ctypes.c_char_p, ctypes.c_char_p, i64, ctypes.POINTER(i64)]
        lib.chem_mech_dims.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip)]
        lib.chem_mech_counts.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip)]
        lib.chem_rates.argtypes = [vp, dp, vp, vp, i64, vp, vp]
        lib.chem_jacobian.argtypes = [vp, dp, vp, vp, i64, vp, vp]
        lib.chem_integrate.argtypes = [vp, dp, vp, vp, i64, dp, dp, dp, vp, vp, ctypes.POINTER(ChemOpts),
                                       ctypes.POINTER(ChemStats), vp]
        lib.chem_last_cell_counters.argtypes = [vp, vp, vp, i64, vp]
        lib.chem_probe_fp64_peak.argtypes = [ctypes.POINTER(ctypes.c_double)]
        lib.chem_debug_exp.argtypes = [vp, vp, i64, vp]
        lib.chem_integrate_noalloc.argtypes = [vp, dp, vp, vp, i64, dp, dp, dp, vp, vp, vp, vp,
                                               ctypes.POINTER(ChemOpts), ctypes.POINTER(ChemStats), vp]
        lib.chem_integrate_record.argtypes = [vp, dp, vp, vp, i64, dp, dp, dp, vp, vp, vp, ctypes.c_int32, vp,
                                              ctypes.POINTER(ChemOpts), ctypes.POINTER(ChemStats), vp]
        lib.chem_adjoint.argtypes = [vp, dp, i64, vp, ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.chem_integrate_mapped.argtypes = [vp, dp, vp, vp, i64, dp, dp, dp, vp, vp, vp, ctypes.c_int32, dp, dp,
                                              vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ChemOpts),
                                              ctypes.POINTER(ChemStats), vp]
        lib.chem_integrate_varp.argtypes = [vp, vp, vp, vp, i64, dp, dp, dp, vp, vp, ctypes.POINTER(ChemOpts),
                                            ctypes.POINTER(ChemStats), vp]
        lib.chem_debug_lu.argtypes = [vp, ctypes.c_int, i64, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp]
        lib.chem_get_lnA.argtypes = [vp, vp]
        lib.chem_set_lnA.argtypes = [vp, vp]
        for name in ("chem_load_mechanism", "chem_mech_dims", "chem_mech_counts", "chem_rates", "chem_jacobian", "chem_integrate",
                     "chem_last_cell_counters", "chem_probe_fp64_peak", "chem_integrate_noalloc",
                     "chem_debug_exp", "chem_integrate_record", "chem_adjoint", "chem_get_lnA", "chem_set_lnA",
                     "chem_integrate_mapped", "chem_integrate_varp", "chem_debug_lu"):
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
        ntb, nfo = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.chem_mech_counts(self._h, ctypes.byref(ntb), ctypes.byref(nfo)))
        self.n_third_body, self.n_falloff = ntb.value, nfo.value
        self.n_pd = ntb.value + nfo.value
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


def chem_describe_mechanism(path: str) -> str:
    """The library's reading of a mechanism file (host only, no GPU): its tables in file order as
    text, the format of include/chemgpu.h's chem_describe_mechanism."""
    lib = load_library()
    need = ctypes.c_int64()
    _check(lib.chem_describe_mechanism(path.encode(), None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(lib.chem_describe_mechanism(path.encode(), buf, need.value, ctypes.byref(need)))
    return buf.value.decode()


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


def chem_integrate_record(mech: Mechanism, p_Pa: float, T, Y, dt: float, rec, nsteps, status, rtol: float = 1e-6,
                          atol: float = 1e-10, h_inout=None, opts: ChemOpts | None = None, want_stats: bool = False,
                          stream=None):
    """chem_integrate (FP64) that also checkpoints every accepted step for chem_adjoint: device
    tensors only; rec is (ncells, max_steps_rec, N + 1) float64, nsteps and status (ncells,) int32."""
    n = _cells(mech, T, Y)
    if rec.dim() != 3 or rec.shape[0] != n or rec.shape[2] != mech.N + 1:
        raise ValueError(f"rec must have shape (ncells={n}, max_steps_rec, N+1={mech.N + 1})")
    pT, dT = _ptr(T, np.float64)
    pY, _ = _ptr(Y, np.float64)
    ph, _ = _ptr(h_inout, np.float64)
    ps, _ = _ptr(status, np.int32)
    pr, _ = _ptr(rec, np.float64)
    pn, _ = _ptr(nsteps, np.int32)
    st = ChemStats() if want_stats else None
    _check(mech._lib.chem_integrate_record(mech.handle, float(p_Pa), pT, pY, n, float(dt), float(rtol), float(atol),
                                           ph, ps, pr, int(rec.shape[1]), pn,
                                           ctypes.byref(opts) if opts is not None else None,
                                           ctypes.byref(st) if st is not None else None, _stream(stream, dT)))
    return st


def chem_adjoint(mech: Mechanism, p_Pa: float, rec, nsteps, status, gT, gY, gT0, gY0, g_lnA=None, g_lnA_cells=None,
                 stream=None):
    """Reverse sweep over the checkpoints of chem_integrate_record: from dL/dT(dt) = gT (ncells,) and
    dL/dY(dt) = gY (K, ncells) writes dL/dT(0) to gT0, dL/dY(0) to gY0, and (if given) the sum over
    cells of dL/d ln A to g_lnA (R,) and its per-cell terms to g_lnA_cells (ncells, R), reactions
    in file order.  Device tensors only."""
    n = int(gT.shape[0])
    if tuple(gY.shape) != (mech.K, n) or tuple(gY0.shape) != (mech.K, n) or tuple(gT0.shape) != (n,):
        raise ValueError("gradient arrays must be (ncells,) and (K, ncells)")
    if rec.dim() != 3 or rec.shape[0] != n or rec.shape[2] != mech.N + 1:
        raise ValueError(f"rec must have shape (ncells={n}, max_steps_rec, N+1={mech.N + 1})")
    if g_lnA is not None and tuple(g_lnA.shape) != (mech.R,):
        raise ValueError(f"g_lnA must have shape (R={mech.R},)")
    if g_lnA_cells is not None and tuple(g_lnA_cells.shape) != (n, mech.R):
        raise ValueError(f"g_lnA_cells must have shape (ncells={n}, R={mech.R})")
    prec, _ = _ptr(rec, np.float64)
    pn, dev = _ptr(nsteps, np.int32)
    ps, _ = _ptr(status, np.int32)
    pgT, _ = _ptr(gT, np.float64)
    pgY, _ = _ptr(gY, np.float64)
    pgT0, _ = _ptr(gT0, np.float64)
    pgY0, _ = _ptr(gY0, np.float64)
    pgA, _ = _ptr(g_lnA, np.float64)
    pgC, _ = _ptr(g_lnA_cells, np.float64)
    _check(mech._lib.chem_adjoint(mech.handle, float(p_Pa), n, prec, int(rec.shape[1]), pn, ps, pgT, pgY, pgT0,
                                  pgY0, pgA, pgC, _stream(stream, dev)))


def chem_integrate_varp(mech: Mechanism, p_Pa, T, Y, dt: float, rtol: float = 1e-6, atol: float = 1e-10,
                        h_inout=None, status=None, opts: ChemOpts | None = None, want_stats: bool = False,
                        stream=None):
    """chem_integrate with a pressure per cell (p_Pa: (ncells,) float64, Pa); device tensors only."""
    n = _cells(mech, T, Y)
    if tuple(p_Pa.shape) != (n,):
        raise ValueError(f"p_Pa must have shape (ncells={n},)")
    pp, _ = _ptr(p_Pa, np.float64)
    pT, dT = _ptr(T, np.float64)
    pY, _ = _ptr(Y, np.float64)
    ph, _ = _ptr(h_inout, np.float64)
    ps, _ = _ptr(status, np.int32)
    st = ChemStats() if want_stats else None
    _check(mech._lib.chem_integrate_varp(mech.handle, pp, pT, pY, n, float(dt), float(rtol), float(atol), ph, ps,
                                         ctypes.byref(opts) if opts is not None else None,
                                         ctypes.byref(st) if st is not None else None, _stream(stream, dT)))
    return st


def chem_integrate_mapped(mech: Mechanism, p_Pa: float, T, Y, dt: float, refs, tol_T: float, tol_Y: float,
                          rtol: float = 1e-6, atol: float = 1e-10, h_inout=None, status=None, zone=None,
                          opts: ChemOpts | None = None, want_stats: bool = False, stream=None):
    """chem_integrate with zonal reference-cell mapping: refs is a host array (n_ref, 1 + K) of
    reference states [T, Y_0..Y_{K-1}]; cells within (tol_T, tol_Y) of a reference take its change
    over dt instead of being solved.  Device tensors otherwise.  Returns (n_mapped, ChemStats or None)."""
    n = _cells(mech, T, Y)
    r = np.ascontiguousarray(np.asarray(refs, dtype=np.float64))
    if r.ndim != 2 or r.shape[1] != mech.K + 1:
        raise ValueError(f"refs must have shape (n_ref, K+1={mech.K + 1})")
    pT, dT = _ptr(T, np.float64)
    pY, _ = _ptr(Y, np.float64)
    ph, _ = _ptr(h_inout, np.float64)
    ps, _ = _ptr(status, np.int32)
    pz, _ = _ptr(zone, np.int32)
    nm = ctypes.c_int64()
    st = ChemStats() if want_stats else None
    _check(mech._lib.chem_integrate_mapped(mech.handle, float(p_Pa), pT, pY, n, float(dt), float(rtol), float(atol),
                                           ph, ps, ctypes.c_void_p(r.ctypes.data), int(r.shape[0]), float(tol_T),
                                           float(tol_Y), pz, ctypes.byref(nm),
                                           ctypes.byref(opts) if opts is not None else None,
                                           ctypes.byref(st) if st is not None else None, _stream(stream, dT)))
    return nm.value, st


def chem_get_lnA(mech: Mechanism) -> np.ndarray:
    """ln A_r of every reaction (file order)."""
    out = np.zeros(mech.R)
    _check(mech._lib.chem_get_lnA(mech.handle, ctypes.c_void_p(out.ctypes.data)))
    return out


def chem_set_lnA(mech: Mechanism, lnA):
    """Replace ln A_r of every reaction (file order, R values); synchronises the device."""
    a = np.ascontiguousarray(np.asarray(lnA, dtype=np.float64))
    if a.shape != (mech.R,):
        raise ValueError(f"lnA must have shape (R={mech.R},)")
    _check(mech._lib.chem_set_lnA(mech.handle, ctypes.c_void_p(a.ctypes.data)))


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


def chem_debug_lu(A, precision: int = CHEM_PREC_FP64, variant: int = 0, stream=None):
    """The kernels' LU with partial pivoting of each matrix of A (n, N, N) float64 (device tensor),
    in the factor precision of `precision`, in schedule `variant` (0 column by column, 1 with the
    next pivot search fused into the update, 2 in panels of 8 columns), for the tests.  Returns
    (factors, invdiag, perm, singular): factors of P A = L D U' (L's multipliers below the
    diagonal, the pivots D on it, U' = D^-1 U above it) (n, N*N) and invdiag (n, N) in the
    precision's storage (float64; float32; FP32 pairs as (n, N*N, 2) / (n, N, 2) float32), perm
    (n, N) int32, singular (n,) int32."""
    import torch
    lib = load_library()
    if A.dim() != 3 or A.shape[1] != A.shape[2] or A.dtype != torch.float64 or not A.is_cuda:
        raise ValueError("A must be a (n, N, N) float64 CUDA tensor")
    A = A.contiguous()
    n, N = int(A.shape[0]), int(A.shape[1])
    dev = A.device
    if precision == CHEM_PREC_MIXED:
        F = torch.empty((n, N * N), dtype=torch.float32, device=dev)
        D = torch.empty((n, N), dtype=torch.float32, device=dev)
    elif precision == CHEM_PREC_MIXED_FF:
        F = torch.empty((n, N * N, 2), dtype=torch.float32, device=dev)
        D = torch.empty((n, N, 2), dtype=torch.float32, device=dev)
    else:
        F = torch.empty((n, N * N), dtype=torch.float64, device=dev)
        D = torch.empty((n, N), dtype=torch.float64, device=dev)
    P = torch.empty((n, N), dtype=torch.int32, device=dev)
    S = torch.empty((n,), dtype=torch.int32, device=dev)
    rc = lib.chem_debug_lu(ctypes.c_void_p(A.data_ptr()), N, n, int(precision), int(variant),
                           ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(P.data_ptr()),
                           ctypes.c_void_p(S.data_ptr()), _stream(stream, True))
    if rc != 0:
        raise ChemError(lib.chem_last_error().decode())
    return F, D, P, S
