"""Thin ctypes binding of libamlbm.so (the C ABI declared in include/amlbm.h).

Argument marshalling only: every step of the lattice Boltzmann update runs in
the library's CUDA kernels.  PyTorch provides the device workspace and the
stream.  There is no CPU fallback: if the library cannot be built or loaded,
or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamlbm.so")
_lib = None
_lock = threading.Lock()

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE = 0, -1, -2, -3, -5
WALL = {"freeslip": 0, "noslip": 1, "outlet": 2}
Z_BC = {"periodic": 0, "noslip": 1}
R_LO = {"axis": 0, "inlet": 1}
FORCING = {"shift": 0, "guo": 1}
SRC = {"local": 0, "link": 1}
STORAGE = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
SHIFT = {"default": 0, "none": 1, "global": 2, "local": 3, "equilibrium": 4}
ROUNDING = {"default": 0, "nearest": 1, "stochastic": 2}
DIAG_FIELDS = ["mass2d", "mass3d", "momz3d", "Eke", "umax", "a2", "A", "neck", "p_in", "p_out",
               "dp", "bad", "sumS", "steps"]


class AmlbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"amlbm error {code}: {msg}")
        self.code = code


class BC(ctypes.Structure):
    _fields_ = [("wall_r", ctypes.c_int), ("axisym", ctypes.c_int), ("src_mode", ctypes.c_int),
                ("storage", ctypes.c_int), ("shift", ctypes.c_int), ("rounding", ctypes.c_int),
                ("g_z", ctypes.c_double), ("rho_ref", ctypes.c_double),
                ("z_bc", ctypes.c_int), ("r_lo", ctypes.c_int), ("r_off", ctypes.c_double),
                ("rho_out", ctypes.c_double), ("forcing", ctypes.c_int)]


class DiagParams(ctypes.Structure):
    _fields_ = [("zc", ctypes.c_double), ("R", ctypes.c_double), ("rho_l", ctypes.c_double),
                ("rho_v", ctypes.c_double)]


class Diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in DIAG_FIELDS] + [("reserved", ctypes.c_double * 2)]


class InstanceC(ctypes.Structure):
    _fields_ = [("Nz", ctypes.c_int), ("Nr", ctypes.c_int), ("tau", ctypes.c_double),
                ("G", ctypes.c_double), ("rho0", ctypes.c_double), ("bc", BC)]


class AdjointProblem(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("ckpt_every", ctypes.c_int), ("objective", ctypes.c_int),
                ("l0", ctypes.c_int), ("n_amps", ctypes.c_int), ("kstar", ctypes.c_int),
                ("zc", ctypes.c_double), ("R", ctypes.c_double), ("w", ctypes.c_double),
                ("rho_l", ctypes.c_double), ("rho_v", ctypes.c_double), ("obj_R", ctypes.c_double),
                ("amps", ctypes.POINTER(ctypes.c_double))]


OBJECTIVE = {"a2sq": 0, "neck": 1}


class Tune(ctypes.Structure):
    _fields_ = [("tile_z", ctypes.c_int), ("tile_r", ctypes.c_int), ("graph_chunk", ctypes.c_int),
                ("schedule", ctypes.c_int)]


class Interface(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("gamma", "gamma_tilde", "rho_l", "rho_v", "position", "umax")]


class TuneResult(ctypes.Structure):
    _fields_ = [("tune", Tune), ("ms_per_step", ctypes.c_double), ("mlups", ctypes.c_double)]


SCHEDULE = {"auto": 0, "fused": 1, "split": 2, "pair": 3}
SCHEDULE_NAME = {1: "fused", 2: "split", 3: "pair"}


EXPORTS = [
    "amlbm_workspace_bytes", "amlbm_create", "amlbm_init_fields", "amlbm_init_fields_device",
    "amlbm_step", "amlbm_read_fields", "amlbm_diagnostics", "amlbm_save_state", "amlbm_load_state",
    "amlbm_device_state", "amlbm_destroy", "amlbm_tiles", "amlbm_batch_workspace_bytes",
    "amlbm_batch_create", "amlbm_batch_init_fields", "amlbm_batch_step", "amlbm_batch_read",
    "amlbm_batch_diagnostics", "amlbm_batch_sites", "amlbm_batch_destroy", "amlbm_last_error",
    "amlbm_version", "amlbm_diagnostics_noalloc", "amlbm_adjoint_workspace_bytes", "amlbm_adjoint",
    "amlbm_objective", "amlbm_batch_config", "amlbm_batch_init_all", "amlbm_batch_init_all_f32",
    "amlbm_batch_diagnostics_all",
    "amlbm_autotune", "amlbm_set_inlet", "amlbm_batch_set_inlet", "amlbm_flat_interface",
]


def load(build_if_missing: bool = True):
    """Load libamlbm.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1310_1871_gb300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        sz = ctypes.c_size_t
        lib.amlbm_workspace_bytes.argtypes = [ip, ip, ip]
        lib.amlbm_workspace_bytes.restype = sz
        lib.amlbm_create.argtypes = [ip, ip, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(BC), vp, vp, sz, ctypes.POINTER(vp)]
        lib.amlbm_init_fields.argtypes = [vp, dp, dp, dp]
        lib.amlbm_set_inlet.argtypes = [vp, dp, dp]
        lib.amlbm_flat_interface.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int] * 5 + \
            [ctypes.c_double] * 2 + [vp, ctypes.POINTER(Interface)]
        lib.amlbm_init_fields_device.argtypes = [vp, vp, vp, vp]
        lib.amlbm_step.argtypes = [vp, ip]
        lib.amlbm_read_fields.argtypes = [vp, dp, dp, dp, dp]
        lib.amlbm_diagnostics.argtypes = [vp, ctypes.POINTER(DiagParams), ctypes.POINTER(Diag)]
        lib.amlbm_save_state.argtypes = [vp, vp, ctypes.POINTER(sz)]
        lib.amlbm_load_state.argtypes = [vp, vp, sz]
        lib.amlbm_device_state.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(ip)]
        lib.amlbm_destroy.argtypes = [vp]
        lib.amlbm_destroy.restype = None
        lib.amlbm_tiles.argtypes = [ip, ip, ctypes.POINTER(ip), ctypes.POINTER(ip), ip]
        lib.amlbm_batch_workspace_bytes.argtypes = [ip, ctypes.POINTER(InstanceC)]
        lib.amlbm_batch_workspace_bytes.restype = sz
        lib.amlbm_batch_create.argtypes = [ip, ctypes.POINTER(InstanceC), ctypes.POINTER(Tune), vp, vp,
                                           sz, ctypes.POINTER(vp)]
        lib.amlbm_batch_init_fields.argtypes = [vp, ip, dp, dp, dp]
        lib.amlbm_batch_set_inlet.argtypes = [vp, ip, dp, dp]
        lib.amlbm_batch_step.argtypes = [vp, ip]
        lib.amlbm_batch_read.argtypes = [vp, ip, dp, dp, dp, dp]
        lib.amlbm_batch_diagnostics.argtypes = [vp, ip, ctypes.POINTER(DiagParams), ctypes.POINTER(Diag)]
        lib.amlbm_autotune.argtypes = [ip, ctypes.POINTER(InstanceC), ip, vp, ctypes.POINTER(Tune),
                                       ctypes.POINTER(TuneResult), ip]
        lib.amlbm_batch_init_all.argtypes = [vp, dp, dp, dp]
        fp = ctypes.POINTER(ctypes.c_float)
        lib.amlbm_batch_init_all_f32.argtypes = [vp, fp, fp, fp]
        lib.amlbm_batch_diagnostics_all.argtypes = [vp, ctypes.POINTER(DiagParams), ctypes.POINTER(Diag)]
        lib.amlbm_batch_sites.argtypes = [vp]
        lib.amlbm_batch_sites.restype = ctypes.c_longlong
        lib.amlbm_batch_config.argtypes = [vp] + [ctypes.POINTER(ip)] * 4
        lib.amlbm_batch_destroy.argtypes = [vp]
        lib.amlbm_batch_destroy.restype = None
        lib.amlbm_last_error.restype = ctypes.c_char_p
        lib.amlbm_version.restype = ctypes.c_char_p
        lib.amlbm_diagnostics_noalloc.argtypes = [vp, ctypes.POINTER(DiagParams), ctypes.POINTER(Diag)]
        AP = ctypes.POINTER(AdjointProblem)
        lib.amlbm_adjoint_workspace_bytes.argtypes = [vp, AP]
        lib.amlbm_adjoint_workspace_bytes.restype = sz
        lib.amlbm_adjoint.argtypes = [vp, AP, vp, sz, dp, dp, dp, dp]
        lib.amlbm_objective.argtypes = [vp, AP, dp]
        _lib = lib
        return lib


def _check(lib, rc):
    if rc != OK:
        raise AmlbmError(rc, lib.amlbm_last_error().decode())
    return rc


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _is_f32(a):
    if isinstance(a, (list, tuple)):
        return all(np.asarray(x).dtype == np.float32 for x in a)
    return np.asarray(a).dtype == np.float32


def _host(a, shape):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        a = a.reshape(shape)
    return a


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream), s


def _code(table, v):
    return table[v] if isinstance(v, str) else int(v)


def make_bc(wall="freeslip", axisym=True, src="local", storage="f64", gz=0.0, rho_ref=1.0,
            shift="default", rounding="default", z_bc="periodic", r_lo="axis", r_off=0.0,
            rho_out=1.0, forcing="shift") -> BC:
    return BC(_code(WALL, wall), int(bool(axisym)), _code(SRC, src), _code(STORAGE, storage),
              _code(SHIFT, shift), _code(ROUNDING, rounding), float(gz), float(rho_ref),
              _code(Z_BC, z_bc), _code(R_LO, r_lo), float(r_off), float(rho_out), _code(FORCING, forcing))


def _diag_dict(d: Diag) -> dict:
    return {n: getattr(d, n) for n in DIAG_FIELDS}


@dataclass
class InstanceSpec:
    """One lattice of a batch (plain parameters; fields are set with init_fields)."""
    Nz: int
    Nr: int
    tau: float = 1.0
    G: float = -5.0
    rho0: float = 1.0
    wall: str = "freeslip"
    axisym: bool = True
    src: str = "local"
    gz: float = 0.0
    rho_ref: float = 1.0
    shift: str = "default"
    rounding: str = "default"
    z_bc: str = "periodic"
    r_lo: str = "axis"
    r_off: float = 0.0
    rho_out: float = 1.0
    forcing: str = "shift"


def instances_c(specs, storage):
    """The amlbm_instance array of a list of InstanceSpec."""
    specs = list(specs)
    arr = (InstanceC * len(specs))()
    for i, s in enumerate(specs):
        arr[i] = InstanceC(int(s.Nz), int(s.Nr), float(s.tau), float(s.G), float(s.rho0),
                           make_bc(s.wall, s.axisym, s.src, storage, s.gz, s.rho_ref, s.shift,
                                   s.rounding, s.z_bc, s.r_lo, s.r_off, s.rho_out, s.forcing))
    return arr


def flat_interface(G, tau=1.0, rho0=1.0, axisym=True, storage="f64", n=64, steps=20000, rho_l0=2.0,
                   rho_v0=0.15, forcing="shift", stream=None) -> dict:
    """amlbm_flat_interface: coexistence densities and surface tension (Table I) of a
    1 x n flat interface after `steps` timesteps on the GPU."""
    lib = load()
    sh, _ = _stream_handle(stream)
    out = Interface()
    _check(lib, lib.amlbm_flat_interface(float(G), float(tau), float(rho0), int(bool(axisym)),
                                         _code(FORCING, forcing), _code(STORAGE, storage), int(n),
                                         int(steps), float(rho_l0),
                                         float(rho_v0), sh, ctypes.byref(out)))
    return {k: getattr(out, k) for k, _ in Interface._fields_}


def autotune_raw(specs, storage, steps=20, stream=None):
    """Run amlbm_autotune: returns (schedule, (tile_z, tile_r), [candidate dicts])."""
    lib = load()
    arr = instances_c(specs, storage)
    sh, _ = _stream_handle(stream)
    best = Tune()
    cap = 128
    res = (TuneResult * cap)()
    n = lib.amlbm_autotune(len(arr), arr, int(steps), sh, ctypes.byref(best), res, cap)
    if n < 0:
        _check(lib, n)
    names = SCHEDULE_NAME
    cands = [{"schedule": names[r.tune.schedule], "tile": [r.tune.tile_z, r.tune.tile_r],
              "ms_per_step": r.ms_per_step, "mlups": r.mlups} for r in res[:min(n, cap)]]
    return names[best.schedule], (best.tile_z, best.tile_r), cands


class Batch:
    """Independent lattices stepped together, one kernel launch per timestep.

    tile=None lets the library pick the launch shape by a size heuristic;
    tile="auto" takes the autotuner's choice for these lattice shapes (cached,
    see autotune.py); a (tile_z, tile_r) pair with schedule="fused" or "split"
    forces one."""

    def __init__(self, specs, storage="f32", tile=None, graph_chunk=0, stream=None, schedule="auto"):
        import torch
        self.lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("amlbm needs a CUDA device")
        self.specs = list(specs)
        n = len(self.specs)
        self.tuned = None
        if isinstance(tile, str):
            if tile != "auto":
                raise ValueError("tile must be None, 'auto' or a (tile_z, tile_r) pair")
            from . import autotune
            self.tuned = autotune.tune(self.specs, storage, stream=stream)
            schedule, tile = self.tuned["schedule"], tuple(self.tuned["tile"])
        arr = instances_c(self.specs, storage)
        self._arr = arr
        nbytes = self.lib.amlbm_batch_workspace_bytes(n, arr)
        if nbytes == 0:
            raise AmlbmError(EINVAL, self.lib.amlbm_last_error().decode())
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        sh, self.stream = _stream_handle(stream)
        sched = SCHEDULE[schedule] if isinstance(schedule, str) else int(schedule)
        if tile and not sched:
            sched = SCHEDULE["fused"]
        tune = Tune(*(tile if tile else (0, 0)), int(graph_chunk), sched)
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.amlbm_batch_create(n, arr, ctypes.byref(tune), sh,
                                                     ctypes.c_void_p(aligned), nbytes, ctypes.byref(h)))
        self.h = h
        self.storage = storage
        self.sites = int(self.lib.amlbm_batch_sites(h))
        sc, tz, tr, nl = (ctypes.c_int() for _ in range(4))
        _check(self.lib, self.lib.amlbm_batch_config(h, ctypes.byref(sc), ctypes.byref(tz), ctypes.byref(tr),
                                                     ctypes.byref(nl)))
        self.schedule = SCHEDULE_NAME[sc.value]
        self.tile = (tz.value, tr.value)
        self.launches_per_step = nl.value

    def init_fields(self, k, rho, uz=None, ur=None):
        s = self.specs[k]
        shp = (s.Nr, s.Nz)
        rho, uz, ur = _host(rho, shp), _host(uz, shp), _host(ur, shp)
        _check(self.lib, self.lib.amlbm_batch_init_fields(self.h, k, _dptr(rho), _dptr(uz), _dptr(ur)))

    def set_inlet(self, k, uz, ur):
        """Velocity of instance k's inlet row, arrays of Nz values (r_lo="inlet")."""
        n = self.specs[k].Nz
        uz, ur = _host(uz, (n,)), _host(ur, (n,))
        _check(self.lib, self.lib.amlbm_batch_set_inlet(self.h, k, _dptr(uz), _dptr(ur)))

    def step(self, n=1):
        _check(self.lib, self.lib.amlbm_batch_step(self.h, int(n)))

    def read(self, k, with_f=False):
        s = self.specs[k]
        rho, uz, ur = (np.empty((s.Nr, s.Nz)) for _ in range(3))
        f = np.empty((9, s.Nr, s.Nz)) if with_f else None
        _check(self.lib, self.lib.amlbm_batch_read(self.h, k, _dptr(rho), _dptr(uz), _dptr(ur), _dptr(f)))
        return (rho, uz, ur, f) if with_f else (rho, uz, ur)

    def read_f(self, k):
        s = self.specs[k]
        f = np.empty((9, s.Nr, s.Nz))
        _check(self.lib, self.lib.amlbm_batch_read(self.h, k, None, None, None, _dptr(f)))
        return f

    def diagnostics(self, k, zc=None, R=1.0, rho_l=2.0, rho_v=0.1, check=True):
        s = self.specs[k]
        dp = DiagParams(s.Nz / 2 if zc is None else float(zc), float(R), float(rho_l), float(rho_v))
        d = Diag()
        rc = self.lib.amlbm_batch_diagnostics(self.h, k, ctypes.byref(dp), ctypes.byref(d))
        if rc not in (OK, EUNSTABLE) or (check and rc != OK):
            _check(self.lib, rc)
        return _diag_dict(d)

    def _flat(self, a, dtype=np.float64):
        if a is None:
            return None
        if isinstance(a, (list, tuple)):
            a = np.concatenate([np.ravel(x) for x in a])
        a = np.ascontiguousarray(a, dtype=dtype).reshape(-1)
        if a.size != self.sites:
            raise ValueError(f"expected {self.sites} values (all instances back to back), got {a.size}")
        return a

    def init_all(self, rho, uz=None, ur=None):
        """Every instance at once (amlbm_batch_init_all): rho, uz, ur hold all
        instances back to back in instance order, each [Nr][Nz], or are lists of
        per-instance arrays.  When every given array is float32 the call is
        amlbm_batch_init_all_f32 (half the bytes; the same state for the
        FP32-arithmetic forms)."""
        given = [x for x in (rho, uz, ur) if x is not None]
        if all(_is_f32(x) for x in given):
            rho, uz, ur = (self._flat(x, np.float32) for x in (rho, uz, ur))
            _check(self.lib, self.lib.amlbm_batch_init_all_f32(self.h, _fptr(rho), _fptr(uz), _fptr(ur)))
            return
        rho, uz, ur = self._flat(rho), self._flat(uz), self._flat(ur)
        _check(self.lib, self.lib.amlbm_batch_init_all(self.h, _dptr(rho), _dptr(uz), _dptr(ur)))

    def diagnostics_all(self, params=None, check=True, as_array=False):
        """Diagnostics of every instance in one pass (amlbm_batch_diagnostics_all).

        params: None (defaults), one dict per instance with zc, R, rho_l, rho_v, or a
        float64 array of shape (n, 4) in that column order.  Returns one dict per
        instance, or with as_array=True an (n, 16) float64 array whose first columns
        follow DIAG_FIELDS (no per-instance Python objects, for tight loops)."""
        n = len(self.specs)
        dp = None
        if params is not None:
            if isinstance(params, np.ndarray):
                a = np.ascontiguousarray(params, dtype=np.float64)
                if a.shape != (n, 4):
                    raise ValueError(f"params array must have shape ({n}, 4)")
                self._dp_keep = a
                dp = (DiagParams * n).from_buffer(a)
            else:
                dp = (DiagParams * n)()
                for k, (s, q) in enumerate(zip(self.specs, params)):
                    zc = q.get("zc")
                    dp[k] = DiagParams(s.Nz / 2 if zc is None else float(zc), float(q.get("R", 1.0)),
                                       float(q.get("rho_l", 2.0)), float(q.get("rho_v", 0.1)))
        out = (Diag * n)()
        rc = self.lib.amlbm_batch_diagnostics_all(self.h, dp, out)
        if rc not in (OK, EUNSTABLE) or (check and rc != OK):
            _check(self.lib, rc)
        if as_array:
            return np.frombuffer(out, dtype=np.float64).reshape(n, -1).copy()
        return [_diag_dict(d) for d in out]

    def close(self):
        if getattr(self, "h", None):
            self.lib.amlbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice:
    """One Nz x Nr lattice (amlbm_ctx)."""

    def __init__(self, Nz, Nr, tau=1.0, G=-5.0, rho0=1.0, wall="freeslip", axisym=True, src="local",
                 storage="f64", gz=0.0, rho_ref=1.0, shift="default", rounding="default", stream=None,
                 z_bc="periodic", r_lo="axis", r_off=0.0, rho_out=1.0, forcing="shift"):
        import torch
        self.lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("amlbm needs a CUDA device")
        self.Nz, self.Nr = int(Nz), int(Nr)
        bc = make_bc(wall, axisym, src, storage, gz, rho_ref, shift, rounding, z_bc, r_lo, r_off, rho_out,
                     forcing)
        nbytes = self.lib.amlbm_workspace_bytes(self.Nz, self.Nr, bc.storage)
        if nbytes == 0:
            raise AmlbmError(EINVAL, "bad lattice size or storage")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        sh, self.stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.amlbm_create(self.Nz, self.Nr, float(tau), float(G), float(rho0),
                                               ctypes.byref(bc), sh, ctypes.c_void_p(aligned), nbytes,
                                               ctypes.byref(h)))
        self.h = h
        self.storage = storage

    def init_fields(self, rho, uz=None, ur=None):
        shp = (self.Nr, self.Nz)
        rho, uz, ur = _host(rho, shp), _host(uz, shp), _host(ur, shp)
        _check(self.lib, self.lib.amlbm_init_fields(self.h, _dptr(rho), _dptr(uz), _dptr(ur)))

    def set_inlet(self, uz, ur):
        """Velocity of the inlet row (r_lo="inlet"), arrays of Nz values."""
        uz, ur = _host(uz, (self.Nz,)), _host(ur, (self.Nz,))
        _check(self.lib, self.lib.amlbm_set_inlet(self.h, _dptr(uz), _dptr(ur)))

    def init_fields_device(self, rho, uz=None, ur=None):
        """rho, uz, ur: contiguous float64 CUDA tensors [Nr, Nz] (uz, ur optional)."""
        def p(t):
            if t is None:
                return None
            assert t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()
            return ctypes.c_void_p(t.data_ptr())
        _check(self.lib, self.lib.amlbm_init_fields_device(self.h, p(rho), p(uz), p(ur)))

    def step(self, n=1):
        _check(self.lib, self.lib.amlbm_step(self.h, int(n)))

    def read(self):
        rho, uz, ur = (np.empty((self.Nr, self.Nz)) for _ in range(3))
        _check(self.lib, self.lib.amlbm_read_fields(self.h, _dptr(rho), _dptr(uz), _dptr(ur), None))
        return rho, uz, ur

    def read_f(self):
        f = np.empty((9, self.Nr, self.Nz))
        _check(self.lib, self.lib.amlbm_read_fields(self.h, None, None, None, _dptr(f)))
        return f

    def diagnostics(self, zc=None, R=1.0, rho_l=2.0, rho_v=0.1, check=True):
        dp = DiagParams(self.Nz / 2 if zc is None else float(zc), float(R), float(rho_l), float(rho_v))
        d = Diag()
        rc = self.lib.amlbm_diagnostics(self.h, ctypes.byref(dp), ctypes.byref(d))
        if rc not in (OK, EUNSTABLE) or (check and rc != OK):
            _check(self.lib, rc)
        return _diag_dict(d)

    @staticmethod
    def _problem(T, ckpt_every, amps, zc, R, w, rho_l, rho_v, objective, obj_R, kstar, l0):
        amps = np.ascontiguousarray(np.asarray(amps, dtype=np.float64).reshape(-1))
        prob = AdjointProblem(int(T), int(ckpt_every), OBJECTIVE[objective] if isinstance(objective, str)
                              else int(objective), int(l0), int(amps.size), int(kstar), float(zc), float(R),
                              float(w), float(rho_l), float(rho_v), float(R if obj_R is None else obj_R),
                              _dptr(amps) if amps.size else None)
        return prob, amps

    def adjoint(self, T, amps, zc, R, w=2.0, rho_l=1.93, rho_v=0.16, objective="a2sq", obj_R=None,
                kstar=0, l0=2, ckpt_every=None):
        """J and dJ/d(G, tau, amps) of: shape-perturbed drop -> f^eq -> T steps -> J, by the
        hand-written discrete adjoint (state checkpoints every ckpt_every steps, default
        ~sqrt(T)).  Overwrites the lattice state."""
        import torch
        ck = int(ckpt_every) if ckpt_every else max(1, int(round(np.sqrt(T))))
        prob, keep = self._problem(T, ck, amps, zc, R, w, rho_l, rho_v, objective, obj_R, kstar, l0)
        nbytes = self.lib.amlbm_adjoint_workspace_bytes(self.h, ctypes.byref(prob))
        if nbytes == 0:
            raise AmlbmError(EINVAL, self.lib.amlbm_last_error().decode())
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        aligned = (ws.data_ptr() + 255) // 256 * 256
        J, dG, dT = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        dA = np.zeros(max(1, keep.size))
        _check(self.lib, self.lib.amlbm_adjoint(self.h, ctypes.byref(prob), ctypes.c_void_p(aligned), nbytes,
                                                ctypes.byref(J), ctypes.byref(dG), ctypes.byref(dT), _dptr(dA)))
        del ws
        return J.value, dG.value, dT.value, dA[:keep.size].copy()

    def objective(self, T, amps, zc, R, w=2.0, rho_l=1.93, rho_v=0.16, objective="a2sq", obj_R=None,
                  kstar=0, l0=2):
        """J of the same run (no adjoint).  Overwrites the lattice state."""
        prob, keep = self._problem(T, 1, amps, zc, R, w, rho_l, rho_v, objective, obj_R, kstar, l0)
        J = ctypes.c_double()
        _check(self.lib, self.lib.amlbm_objective(self.h, ctypes.byref(prob), ctypes.byref(J)))
        return J.value

    def save_state(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(self.lib, self.lib.amlbm_save_state(self.h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self.lib, self.lib.amlbm_save_state(self.h, buf, ctypes.byref(n)))
        return buf.raw

    def load_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(self.lib, self.lib.amlbm_load_state(self.h, buf, len(data)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.amlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tiles(storage="f32", schedule="fused"):
    lib = load()
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    sc = SCHEDULE[schedule] if isinstance(schedule, str) else int(schedule)
    n = lib.amlbm_tiles(st, sc, None, None, 0)
    tz, tr = (ctypes.c_int * n)(), (ctypes.c_int * n)()
    lib.amlbm_tiles(st, sc, tz, tr, n)
    return list(zip(tz, tr))


@dataclass
class DropRun:
    """A differentiable run for DropObjective: lattice, drop, objective."""
    Nz: int
    Nr: int
    T: int
    zc: float
    R: float
    w: float = 2.0
    rho_l: float = 1.93
    rho_v: float = 0.16
    objective: str = "a2sq"
    obj_R: float = None
    kstar: int = 0
    l0: int = 2
    storage: str = "f64"
    ckpt_every: int = None
    wall: str = "freeslip"


def _drop_objective_class():
    import torch

    class DropObjective(torch.autograd.Function):
        """J(amps, G, tau) of a DropRun; backward returns the discrete-adjoint gradients."""

        @staticmethod
        def forward(ctx, amps, G, tau, run):
            lat = Lattice(run.Nz, run.Nr, tau=float(tau), G=float(G), storage=run.storage, wall=run.wall)
            a = amps.detach().cpu().double().numpy()
            kw = dict(zc=run.zc, R=run.R, w=run.w, rho_l=run.rho_l, rho_v=run.rho_v,
                      objective=run.objective, obj_R=run.obj_R, kstar=run.kstar, l0=run.l0)
            if any(ctx.needs_input_grad[:3]):
                J, dG, dT, dA = lat.adjoint(run.T, a, ckpt_every=run.ckpt_every, **kw)
                ctx.save_for_backward(torch.as_tensor(dA, dtype=amps.dtype, device=amps.device),
                                      torch.tensor(dG, dtype=torch.float64), torch.tensor(dT, dtype=torch.float64))
            else:
                J = lat.objective(run.T, a, **kw)
            lat.close()
            return torch.tensor(J, dtype=torch.float64, device=amps.device)

        @staticmethod
        def backward(ctx, gJ):
            dA, dG, dT = ctx.saved_tensors
            gJ = gJ.to(torch.float64)
            return (gJ.to(dA.dtype) * dA, (gJ.cpu() * dG).to(gJ.device), (gJ.cpu() * dT).to(gJ.device), None)

    return DropObjective


_DO = None


def drop_objective(amps, G, tau, run: DropRun):
    """torch-differentiable J(amps, G, tau) (see DropRun)."""
    global _DO
    if _DO is None:
        _DO = _drop_objective_class()
    return _DO.apply(amps, G, tau, run)
