"""Oracle for the axisymmetric Shan-Chen LBM step (arXiv:1310.1871): test infrastructure.

A plain FP64 CPU restatement of the paper's update (``amlbm_oracle.cpp``), built
with g++ (no FMA contraction, no fast-math) and loaded with ctypes.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package; the CUDA library never does, and it never imports the CUDA
library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amlbm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

NFIELDS = 23
FIELD_NAMES = ("rho jz jr psi Fsc_z Fsc_r Dr Drr Dzr Fg_z Fg_r Fz Fr uz ur ueqz ueqr "
               "druz dzur drur S Hz Hr").split()
DIAG_NAMES = ("mass2d mass3d momz3d Eke umax a2 A neck p_in p_out dp bad sumS").split()

WALL_FREESLIP, WALL_NOSLIP, WALL_OUTLET = 0, 1, 2
SRC_LOCAL, SRC_LINK = 0, 1
Z_PERIODIC, Z_NOSLIP = 0, 1
RLO_AXIS, RLO_INLET = 0, 1
FORCE_SHIFT, FORCE_GUO = 0, 1


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain -O2, FP contraction off),
    or with ``omp`` into ``oracle/liboracle_omp.so``: the same source with its site
    loops run over OpenMP threads (the same arithmetic; bit-identical results)."""
    lib = _LIB_OMP if omp else _LIB
    with _lock:
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
            cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17", "-fPIC",
                   "-shared"] + (["-fopenmp"] if omp else []) + ["-o", lib + ".tmp", _SRC]
            subprocess.run(cmd, check=True)
            os.replace(lib + ".tmp", lib)
    return lib


class _Params(ctypes.Structure):
    _fields_ = [("Nz", ctypes.c_int), ("Nr", ctypes.c_int), ("tau", ctypes.c_double),
                ("G", ctypes.c_double), ("rho0", ctypes.c_double), ("gz", ctypes.c_double),
                ("wall", ctypes.c_int), ("axisym", ctypes.c_int), ("src_mode", ctypes.c_int),
                ("zbc", ctypes.c_int), ("rlo", ctypes.c_int), ("r_off", ctypes.c_double),
                ("rho_out", ctypes.c_double), ("inlet_uz", ctypes.POINTER(ctypes.c_double)),
                ("inlet_ur", ctypes.POINTER(ctypes.c_double)), ("forcing", ctypes.c_int)]


def _load(omp: bool = False):
    if omp not in _libs:
        lib = ctypes.CDLL(build(omp=omp))
        dp = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(_Params)
        lib.orc_init.argtypes = [P, dp, dp, dp, dp]
        lib.orc_run.argtypes = [P, dp, ctypes.c_int]
        lib.orc_fields.argtypes = [P, dp, dp]
        lib.orc_sources.argtypes = [P, dp, dp]
        lib.orc_stencil.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
        lib.orc_drop_rho.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 5 + \
            [ctypes.c_int, ctypes.c_int, dp, dp]
        lib.orc_objective.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp] + \
            [ctypes.c_double] * 4 + [ctypes.c_int]
        lib.orc_objective.restype = ctypes.c_double
        lib.orc_grad.argtypes = [P, ctypes.c_int] + [ctypes.c_double] * 5 + \
            [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp]
        lib.orc_diag.argtypes = [P, dp] + [ctypes.c_double] * 4 + [dp]
        lib.orc_threads.argtypes = [ctypes.c_int]
        _libs[omp] = lib
    return _libs[omp]


def threads(n: int = 0) -> int:
    """Set (n > 0) and return the thread count of the OpenMP build's site loops."""
    return int(_load(True).orc_threads(int(n)))


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One lattice (Nz x Nr) with fixed parameters; state f is float64 [9, Nr, Nz]."""

    def __init__(self, Nz, Nr, tau=1.0, G=-5.0, rho0=1.0, gz=0.0, wall=WALL_FREESLIP,
                 axisym=1, src_mode=SRC_LOCAL, zbc=Z_PERIODIC, rlo=RLO_AXIS, r_off=0.0,
                 rho_out=1.0, inlet=None, forcing=FORCE_SHIFT, omp=False):
        """inlet: (u_z, u_r) arrays of Nz values imposed on the inlet row (rlo=RLO_INLET).
        omp: run on the OpenMP build (see ``threads``)."""
        self.Nz, self.Nr = int(Nz), int(Nr)
        if inlet is None:
            inlet = (np.zeros(self.Nz), np.zeros(self.Nz))
        # kept alive for as long as the parameter block points at them
        self._inlet = tuple(np.ascontiguousarray(a, dtype=np.float64).reshape(self.Nz) for a in inlet)
        self.p = _Params(self.Nz, self.Nr, float(tau), float(G), float(rho0), float(gz),
                         int(wall), int(axisym), int(src_mode), int(zbc), int(rlo), float(r_off),
                         float(rho_out), _ptr(self._inlet[0]), _ptr(self._inlet[1]), int(forcing))
        self.lib = _load(bool(omp))

    def _c(self, rc):
        if rc != 0:
            raise ValueError("oracle rejected the arguments")

    def init(self, rho, uz=None, ur=None) -> np.ndarray:
        shp = (self.Nr, self.Nz)
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(shp)
        uz = np.zeros(shp) if uz is None else np.ascontiguousarray(uz, dtype=np.float64).reshape(shp)
        ur = np.zeros(shp) if ur is None else np.ascontiguousarray(ur, dtype=np.float64).reshape(shp)
        f = np.empty((9,) + shp)
        self._c(self.lib.orc_init(ctypes.byref(self.p), _ptr(rho), _ptr(uz), _ptr(ur), _ptr(f)))
        return f

    def run(self, f: np.ndarray, nsteps: int) -> np.ndarray:
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        self._c(self.lib.orc_run(ctypes.byref(self.p), _ptr(f), int(nsteps)))
        return f

    def fields(self, f: np.ndarray) -> dict:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty((NFIELDS, self.Nr, self.Nz))
        self._c(self.lib.orc_fields(ctypes.byref(self.p), _ptr(f), _ptr(out)))
        return {n: out[q] for q, n in enumerate(FIELD_NAMES)}

    def sources(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        h = np.empty((9, self.Nr, self.Nz))
        self._c(self.lib.orc_sources(ctypes.byref(self.p), _ptr(f), _ptr(h)))
        return h

    def diag(self, f: np.ndarray, zc=0.0, objR=1.0, rho_l=2.0, rho_v=0.1) -> dict:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(16)
        self._c(self.lib.orc_diag(ctypes.byref(self.p), _ptr(f), float(zc), float(objR),
                                  float(rho_l), float(rho_v), _ptr(out)))
        return {n: out[q] for q, n in enumerate(DIAG_NAMES)}

    def grad(self, T, zc, R, w, rho_l, rho_v, amps, l0=2, kind=0, objR=None, kstar=0,
             with_grad=True):
        """J and dJ/d(G, tau, amplitudes) of drop_rho -> f^eq -> T steps -> J (complex step)."""
        amps = np.ascontiguousarray(amps, dtype=np.float64)
        J = ctypes.c_double(0.0)
        g = np.zeros(2 + amps.size)
        self._c(self.lib.orc_grad(ctypes.byref(self.p), int(T), float(zc), float(R), float(w),
                                  float(rho_l), float(rho_v), int(l0), int(amps.size), _ptr(amps),
                                  int(kind), float(R if objR is None else objR), int(kstar),
                                  ctypes.byref(J), _ptr(g) if with_grad else None))
        return J.value, (g if with_grad else None)


def stencil(padded: np.ndarray, pad: int, op: int) -> np.ndarray:
    """Apply stencil ``op`` (0 iso d_z, 1 iso d_r, 2 1D d_r, 3 1D d_z, 4 d_rr, 5 d_zr)."""
    padded = np.ascontiguousarray(padded, dtype=np.float64)
    Nr, Nz = padded.shape[0] - 2 * pad, padded.shape[1] - 2 * pad
    out = np.empty((Nr, Nz))
    rc = _load().orc_stencil(Nz, Nr, pad, _ptr(padded), op, _ptr(out))
    if rc:
        raise ValueError("bad stencil arguments")
    return out


def drop_rho(Nz, Nr, zc, R, w, rho_l, rho_v, amps, l0=2) -> np.ndarray:
    amps = np.ascontiguousarray(amps, dtype=np.float64)
    rho = np.empty((Nr, Nz))
    _load().orc_drop_rho(Nz, Nr, zc, R, w, rho_l, rho_v, l0, amps.size, _ptr(amps), _ptr(rho))
    return rho


def objective(kind, rho, zc, R, rho_l, rho_v, kstar=0) -> float:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    Nr, Nz = rho.shape
    return _load().orc_objective(kind, Nz, Nr, _ptr(rho), zc, R, rho_l, rho_v, kstar)
