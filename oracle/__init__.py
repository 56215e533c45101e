"""Python access to the CPU oracle (oracle/chem_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg use this module to compute reference results.  Nothing on the product path
imports it.  The oracle shares no code with the CUDA library; both read the same mechanism
file, each with its own parser.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  thermo       -- d(h/R)/dT = cp/R and d(s/R)/dT = cp/(R T) by complex step; continuity at Tmid
  rates        -- closed-form kinetics (A=B, A->B->C), element conservation, enthalpy
                  conservation, Gibbs-minimum equilibrium (independent element-potential solve),
                  detailed balance at equilibrium, fall-off limits (Pr->0, Pr->inf, F(center)),
                  the width of the Troe broadening curve (its half- and fifth-depth points)
  jacobian     -- complex-step derivative of rates to 1e-12 row-normwise, central differences
  integrate    -- Rosenbrock order conditions and L-stability from the coefficient table,
                  closed-form A=B and A->B->C solutions, observed convergence order
  replay / TLM -- replay of the recorded steps equals the adaptive run bit for bit; the dual-number
                  tangent-linear result equals central differences of the replay (state and ln A
                  directions) and the ln k / initial-state derivatives of the Bateman solution
  readers      -- CHEMMECH and CHEMKIN-II readings equal each other and the library's own reader
                  (describe), on the synthetic mechanisms and CHEMKIN syntax variants

`planted(n)` switches to a build with planted mistake n (tests/test_oracle_planted.py shows that
each one fails the pin that guards it).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chem_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libchem_oracle.so")
_lock = threading.Lock()
_libs = {}  # compiled oracle per planted-mistake id (0 = the oracle itself)
_plant = 0

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)


def _lib_path(plant: int) -> str:
    return _LIB_PATH if plant == 0 else os.path.join(_BUILD, f"libchem_oracle_plant{plant}.so")


def build(force: bool = False, plant: int = 0) -> str:
    """Compile the oracle with the host C++ compiler (portable flags only).  plant > 0 builds the
    variant with that planted mistake (chem_oracle.cpp, ORACLE_PLANT; pin tests only)."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _lib_path(plant)
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC]
        if plant:
            cmd.insert(1, f"-DORACLE_PLANT={int(plant)}")
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


def _load():
    plant = _plant
    with _lock:
        if plant not in _libs:
            lib = ctypes.CDLL(build(plant=plant))
            lib.oracle_load.restype = ctypes.c_void_p
            lib.oracle_load.argtypes = [ctypes.c_char_p]
            lib.oracle_free.argtypes = [ctypes.c_void_p]
            lib.oracle_last_error.restype = ctypes.c_char_p
            lib.oracle_dims.argtypes = [ctypes.c_void_p, _ip, _ip]
            lib.oracle_thermo.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp, _dp]
            lib.oracle_thermo_cs.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _dp, _dp]
            lib.oracle_rates.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, _dp, _dp, _dp, _dp]
            lib.oracle_reaction_rates.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp,
                                                  _dp, _dp]
            lib.oracle_jacobian.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, _dp, _dp, _dp]
            lib.oracle_jacobian_cs.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _dp, ctypes.c_double,
                                               _dp]
            lib.oracle_integrate.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, _dp, _dp,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _ip, _ip, _ip,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_ros_coefficients.argtypes = [_dp]
            lib.oracle_opcount.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _dp, _lp]
            lib.oracle_integrate_record.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, ctypes.c_double,
                                                    ctypes.c_double, ctypes.c_double, _dp, ctypes.c_int, _ip]
            lib.oracle_replay.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp, ctypes.c_int, _dp, _dp, _dp,
                                          _dp, _dp]
            lib.oracle_jacobian_fd.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp]
            lib.oracle_describe.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int64, _lp]
            lib.oracle_jacobian_dir.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            _libs[plant] = lib
    return _libs[plant]


@contextlib.contextmanager
def planted(plant: int):
    """Pin tests only: OracleMechanism objects and ros_coefficients() made inside the block use
    the oracle compiled with planted mistake `plant` (chem_oracle.cpp, ORACLE_PLANT)."""
    global _plant
    old = _plant
    _plant = int(plant)
    try:
        yield
    finally:
        _plant = old


def _p(a, ptype=_dp):
    return a.ctypes.data_as(ptype) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleMechanism:
    """A mechanism file loaded into the oracle."""

    def __init__(self, path: str):
        self._lib = _load()
        self._h = self._lib.oracle_load(path.encode())
        if not self._h:
            raise RuntimeError("oracle could not load mechanism: " + self._lib.oracle_last_error().decode())
        K = ctypes.c_int32()
        R = ctypes.c_int32()
        self._lib.oracle_dims(self._h, ctypes.byref(K), ctypes.byref(R))
        self.K, self.R = K.value, R.value
        self.N = self.K

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_free(h)
            self._h = None

    def describe(self) -> str:
        """The oracle's reading of the mechanism file, in the text form of the library's
        chem_describe_mechanism (for comparing the two readers)."""
        need = ctypes.c_int64()
        self._lib.oracle_describe(self._h, None, 0, ctypes.byref(need))
        buf = ctypes.create_string_buffer(need.value)
        self._lib.oracle_describe(self._h, buf, need.value, ctypes.byref(need))
        return buf.value.decode()

    def thermo(self, T: float):
        out = [np.zeros(self.K) for _ in range(3)]
        self._lib.oracle_thermo(self._h, float(T), *[_p(o) for o in out])
        return tuple(out)  # cp/R, h/RT, s/R

    def thermo_cs(self, T: float, step: float = 1e-30):
        dh = np.zeros(self.K)
        ds = np.zeros(self.K)
        self._lib.oracle_thermo_cs(self._h, float(T), step, _p(dh), _p(ds))
        return dh, ds

    def rates(self, p_Pa: float, T, Y, gross: bool = False):
        T = _f64(T)
        Y = _f64(Y)
        n = T.shape[0]
        f = np.zeros((self.N, n))
        g = np.zeros((self.N, n)) if gross else None
        self._lib.oracle_rates(self._h, float(p_Pa), n, _p(T), _p(Y), _p(f), _p(g))
        return (f, g) if gross else f

    def reaction_rates(self, p_Pa: float, T: float, Y):
        Y = _f64(Y)
        out = [np.zeros(self.R) for _ in range(4)]
        self._lib.oracle_reaction_rates(self._h, float(p_Pa), float(T), _p(Y), *[_p(o) for o in out])
        return tuple(out)  # kf, kr, qf, qr

    def jacobian(self, p_Pa: float, T, Y):
        T = _f64(T)
        Y = _f64(Y)
        n = T.shape[0]
        J = np.zeros((n, self.N, self.N))
        self._lib.oracle_jacobian(self._h, float(p_Pa), n, _p(T), _p(Y), _p(J))
        return J

    def jacobian_cs(self, p_Pa: float, T: float, Y, step: float = 1e-30):
        Y = _f64(Y)
        J = np.zeros((self.N, self.N))
        self._lib.oracle_jacobian_cs(self._h, float(p_Pa), float(T), _p(Y), step, _p(J))
        return J

    def integrate(self, p_Pa: float, T, Y, dt: float, rtol: float = 1e-6, atol: float = 1e-10, h_inout=None,
                  max_steps: int = 100000, nthreads: int = 1, solver: str = "rosenbrock"):
        """Returns (T, Y, status, steps, rejects); inputs are not modified; h_inout is updated in place.
        solver: "rosenbrock" (the 4-stage method), "seulex" (extrapolated linearly implicit Euler) or
        "rosenbrock_fdjac" (the 4-stage method with the forward-difference Jacobian)."""
        solver_id = {"rosenbrock": 0, "seulex": 1, "rosenbrock_fdjac": 2}[solver]
        T = _f64(T).copy()
        Y = _f64(Y).copy()
        n = T.shape[0]
        status = np.zeros(n, np.int32)
        steps = np.zeros(n, np.int32)
        rej = np.zeros(n, np.int32)
        if h_inout is not None:
            assert h_inout.dtype == np.float64 and h_inout.flags.c_contiguous and h_inout.shape == (n,)
        self._lib.oracle_integrate(self._h, float(p_Pa), n, _p(T), _p(Y), float(dt), float(rtol), float(atol),
                                   _p(h_inout), _p(status, _ip), _p(steps, _ip), _p(rej, _ip), int(max_steps),
                                   int(nthreads), solver_id)
        return T, Y, status, steps, rej

    def integrate_mapped(self, p_Pa: float, T, Y, dt: float, refs, tol_T: float, tol_Y: float, rtol: float = 1e-6,
                         atol: float = 1e-10, nthreads: int = 1):
        """Zonal reference-cell mapping (DLBFoam's, Sec. 2.2) on top of integrate: a cell within
        |T - T_r| <= tol_T and max_k |Y_k - Y_r,k| <= tol_Y of reference r (the first such) is not
        solved; it takes the reference's change over dt (T and Y_0..Y_{K-2}; Y_{K-1} = 1 - sum).
        refs: (n_ref, 1 + K).  Returns (T, Y, status, zone)."""
        T = _f64(T)
        Y = _f64(Y)
        refs = np.atleast_2d(_f64(refs))
        n = T.shape[0]
        zone = np.full(n, -1, np.int32)
        for c in range(n):
            for r in range(refs.shape[0]):
                if abs(T[c] - refs[r, 0]) <= tol_T and np.all(np.abs(Y[:, c] - refs[r, 1:]) <= tol_Y):
                    zone[c] = r
                    break
        solve = np.nonzero(zone < 0)[0]
        Ts = np.concatenate([T[solve], refs[:, 0]])
        Ys = np.concatenate([Y[:, solve], refs[:, 1:].T], axis=1)
        To, Yo, st, _, _ = self.integrate(p_Pa, Ts, Ys, dt, rtol, atol, nthreads=nthreads)
        Tn, Yn, status = T.copy(), Y.copy(), np.zeros(n, np.int32)
        Tn[solve], Yn[:, solve], status[solve] = To[:solve.size], Yo[:, :solve.size], st[:solve.size]
        for c in np.nonzero(zone >= 0)[0]:
            r = zone[c]
            i = solve.size + r
            Tn[c] = T[c] + (To[i] - refs[r, 0])
            Yn[:-1, c] = Y[:-1, c] + (Yo[:-1, i] - refs[r, 1:-1])
            Yn[-1, c] = 1.0 - Yn[:-1, c].sum()
            status[c] = st[i]
        return Tn, Yn, status, zone

    def integrate_record(self, p_Pa: float, phi, dt: float, rtol: float = 1e-6, atol: float = 1e-10,
                         max_hs: int = 100000):
        """One cell, phi = [T, Y_1..Y_{K-1}]: returns (phi_final, accepted step sizes, status)."""
        phi = _f64(phi).copy()
        hs = np.zeros(max_hs)
        n = ctypes.c_int32()
        st = self._lib.oracle_integrate_record(self._h, float(p_Pa), _p(phi), float(dt), float(rtol), float(atol),
                                               _p(hs), max_hs, ctypes.byref(n))
        return phi, hs[:n.value].copy(), st

    def replay(self, p_Pa: float, phi, hs, dphi=None, dlnA=None, lnA_shift=None):
        """Replays accepted steps hs from phi (with ln A_r + lnA_shift[r]); with dphi / dlnA also
        returns the tangent-linear derivative of the final state along that direction (reaction
        arrays in file order)."""
        phi = _f64(phi)
        hs = _f64(hs)
        out = np.zeros(self.N)
        dout = np.zeros(self.N) if (dphi is not None or dlnA is not None) else None
        rc = self._lib.oracle_replay(self._h, float(p_Pa), _p(phi), _p(hs), int(hs.shape[0]),
                                     _p(_f64(lnA_shift)) if lnA_shift is not None else None,
                                     _p(_f64(dphi)) if dphi is not None else None,
                                     _p(_f64(dlnA)) if dlnA is not None else None, _p(out), _p(dout))
        if rc != 0:
            raise RuntimeError("oracle replay hit a singular iteration matrix")
        return (out, dout) if dout is not None else out

    def jacobian_fd(self, p_Pa: float, phi):
        """Forward-difference Jacobian at one state phi = [T, Y_1..Y_{K-1}]."""
        phi = _f64(phi)
        J = np.zeros((self.N, self.N))
        self._lib.oracle_jacobian_fd(self._h, float(p_Pa), _p(phi), _p(J))
        return J

    def jacobian_dir(self, p_Pa: float, phi, dphi=None, dlnA=None):
        """At one state phi: (f, J, df, dJ), df and dJ the derivatives of f and J along
        (dphi, dlnA) (dual numbers; reaction arrays in file order)."""
        phi = _f64(phi)
        f, df = np.zeros(self.N), np.zeros(self.N)
        J, dJ = np.zeros((self.N, self.N)), np.zeros((self.N, self.N))
        self._lib.oracle_jacobian_dir(self._h, float(p_Pa), _p(phi), _p(_f64(dphi)) if dphi is not None else None,
                                      _p(_f64(dlnA)) if dlnA is not None else None, _p(f), _p(J), _p(df), _p(dJ))
        return f, J, df, dJ

    def opcount(self, p_Pa: float, T: float, Y):
        Y = _f64(Y)
        c = np.zeros(20, np.int64)
        self._lib.oracle_opcount(self._h, float(p_Pa), float(T), _p(Y), _p(c, _lp))
        keys = ("add", "mul", "div", "exp", "log")
        parts = ("rates", "jacobian", "lu", "solve")
        return {p: dict(zip(keys, c[5 * i:5 * i + 5].tolist())) for i, p in enumerate(parts)}


def ros_coefficients():
    """Classical-form Rosenbrock table used by the oracle: (gamma, alpha[4,4], gamma_ij[4,4], b[4], bhat[4])."""
    out = np.zeros(41)
    _load().oracle_ros_coefficients(_p(out))
    return out[0], out[1:17].reshape(4, 4), out[17:33].reshape(4, 4), out[33:37], out[37:41]
