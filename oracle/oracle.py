"""ctypes wrapper of the FP64 CPU oracle (``lbm_oracle.cpp``).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module. It never imports the CUDA
package, and the CUDA package never imports it.

``build()`` compiles the oracle with g++ (OpenMP, no fast-math, no FMA
contraction, so x86-64 and aarch64 hosts round identically).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NF, NQ = 14, 7
FIELD_NAMES = ("rho", "mx", "my", "mz", "E", "txx", "tyy", "tzz", "txy", "txz", "tyz",
               "qx", "qy", "qz")


# LBM_ORACLE_SANITIZED=1 selects a second build with AddressSanitizer and
# UndefinedBehaviorSanitizer (single-threaded, aborting on the first finding); a process
# that loads it must preload the ASan runtime (the sanitizer test does).
_SANITIZED = os.environ.get("LBM_ORACLE_SANITIZED") == "1"
if _SANITIZED:
    _LIB = os.path.join(_BUILD, "liboracle_sanitized.so")


def build(force: bool = False) -> str:
    """Compile liboracle.so (or the sanitized variant) in place; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    if _SANITIZED:
        cmd = ["g++", "-O1", "-g", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas", "-fsanitize=address,undefined",
               "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-o", tmp, _SRC]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
               "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc_x", ctypes.c_int),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("cfl", ctypes.c_double), ("lambda_ref", ctypes.c_double),
        ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("kappa", ctypes.c_double),
        ("tau_R", ctypes.c_double), ("tau_q", ctypes.c_double), ("T_ref", ctypes.c_double),
        ("relax_in_dt", ctypes.c_int),
        ("sutherland", ctypes.c_int), ("source_mode", ctypes.c_int),
        ("f_mu", ctypes.c_double), ("C_sigma", ctypes.c_double),
        ("J_min", ctypes.c_double), ("omega_min", ctypes.c_double),
        ("sensor_mode", ctypes.c_int), ("collide", ctypes.c_int),
    ]


class OrcDiag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "step", "time", "sum_rho", "sum_mx", "sum_my", "sum_mz", "sum_E", "ek_mean",
        "eps_s_raw", "eps_d_raw", "max_mach", "max_cfl", "min_rho", "min_T", "nonfinite")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
            L.orc_create.restype = vp
            L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
            L.orc_destroy.argtypes = [vp]
            L.orc_dt.restype = ctypes.c_double
            L.orc_dt.argtypes = [vp]
            L.orc_step_count.restype = ctypes.c_longlong
            L.orc_step_count.argtypes = [vp]
            L.orc_set_threads.argtypes = [ip]
            L.orc_get_threads.restype = ip
            L.orc_init_tgv.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ip, ip, ip, ip]
            L.orc_init_riemann.argtypes = [vp, ip, ip, dp, dp]
            L.orc_init_fields.argtypes = [vp, dp, dp, dp, dp, dp]
            L.orc_init_state.argtypes = [vp, dp]
            L.orc_get_populations.argtypes = [vp, dp]
            L.orc_set_populations.argtypes = [vp, dp]
            L.orc_step.argtypes = [vp, ip]
            L.orc_moments.argtypes = [vp, dp]
            L.orc_primitives.argtypes = [vp, dp]
            L.orc_sensor.argtypes = [vp, dp, dp, dp]
            L.orc_equilibrium_of.argtypes = [vp, dp, dp]
            L.orc_flux_of.argtypes = [vp, dp, dp]
            L.orc_closure_of.argtypes = [vp, dp, dp]
            L.orc_chi_of.restype = ctypes.c_double
            L.orc_chi_of.argtypes = [vp, ctypes.c_double]
            L.orc_collide_of.argtypes = [vp, dp, dp, dp]
            L.orc_lattice.argtypes = [dp, ctypes.POINTER(ctypes.c_int)]
            L.orc_diag_get.argtypes = [vp, ctypes.POINTER(OrcDiag)]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


DEFAULTS = dict(bc_x=0, dt=0.0, cfl=0.1, lambda_ref=1.0, gamma=1.4, mu=0.0, kappa=0.0,
                tau_R=1.0, tau_q=1.0, T_ref=1.0, relax_in_dt=0, sutherland=0, source_mode=0, f_mu=0.0,
                C_sigma=0.0, J_min=0.0, omega_min=1.0, sensor_mode=0, collide=1)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def lattice():
    w = np.zeros(7)
    e = (ctypes.c_int * 21)()
    lib().orc_lattice(_dp(w), e)
    return w, np.array(list(e), dtype=np.int64).reshape(7, 3)


class Oracle:
    """One periodic (or x-held) FP64 domain of the scheme."""

    def __init__(self, nx: int, ny: int, nz: int, dx: float, **kw):
        p = dict(DEFAULTS)
        unknown = set(kw) - set(p)
        if unknown:
            raise TypeError(f"unknown oracle parameters {sorted(unknown)}")
        p.update(kw)
        self.params = dict(p, nx=nx, ny=ny, nz=nz, dx=dx)
        s = OrcParams(**{k: v for k, v in self.params.items()})
        self._h = lib().orc_create(ctypes.byref(s))
        if not self._h:
            raise ValueError(f"oracle rejected parameters {self.params}")
        self.shape = (nz, ny, nx)
        self.ncell = nx * ny * nz

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dt(self) -> float:
        return float(lib().orc_dt(self._h))

    @property
    def step_count(self) -> int:
        return int(lib().orc_step_count(self._h))

    def init_tgv(self, U0: float, M0: float, rho0: float, gn: int = 0,
                 origin=(0, 0, 0)):
        lib().orc_init_tgv(self._h, U0, M0, rho0, int(gn), *[int(o) for o in origin])

    def init_riemann(self, axis: int, i_split: int, left, right):
        L = np.ascontiguousarray(left, dtype=np.float64)
        R = np.ascontiguousarray(right, dtype=np.float64)
        if lib().orc_init_riemann(self._h, axis, i_split, _dp(L), _dp(R)) != 0:
            raise ValueError("bad Riemann axis")

    def init_fields(self, rho, ux, uy, uz, p):
        arrs = [np.ascontiguousarray(np.broadcast_to(a, self.shape), dtype=np.float64)
                for a in (rho, ux, uy, uz, p)]
        lib().orc_init_fields(self._h, *[_dp(a) for a in arrs])

    def init_state(self, Q):
        """Equilibrium of given zeroth moments Q (14, nz, ny, nx)."""
        Q = np.ascontiguousarray(np.broadcast_to(Q, (NF,) + self.shape), dtype=np.float64)
        lib().orc_init_state(self._h, _dp(Q))

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def populations(self) -> np.ndarray:
        out = np.empty((NF, NQ) + self.shape)
        lib().orc_get_populations(self._h, _dp(out))
        return out

    def set_populations(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((NF, NQ) + self.shape)
        lib().orc_set_populations(self._h, _dp(f))

    def moments(self) -> np.ndarray:
        out = np.empty((NF,) + self.shape)
        lib().orc_moments(self._h, _dp(out))
        return out

    def primitives(self) -> np.ndarray:
        """rho, u_x, u_y, u_z, T, p as one (6, nz, ny, nx) array."""
        out = np.empty((6,) + self.shape)
        lib().orc_primitives(self._h, _dp(out))
        return out

    def sensor(self):
        th, chi, om = (np.empty(self.shape) for _ in range(3))
        lib().orc_sensor(self._h, _dp(th), _dp(chi), _dp(om))
        return th, chi, om

    def diag(self) -> dict:
        d = OrcDiag()
        lib().orc_diag_get(self._h, ctypes.byref(d))
        return {n: getattr(d, n) for n, _ in OrcDiag._fields_}

    # single-state helpers
    def equilibrium_of(self, Q) -> np.ndarray:
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.empty(NF * NQ)
        lib().orc_equilibrium_of(self._h, _dp(Q), _dp(out))
        return out.reshape(NF, NQ)

    def flux_of(self, Q) -> np.ndarray:
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.empty(NF * 3)
        lib().orc_flux_of(self._h, _dp(Q), _dp(out))
        return out.reshape(NF, 3)

    def closure_of(self, Q) -> dict:
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.empty(9)
        lib().orc_closure_of(self._h, _dp(Q), _dp(out))
        return dict(zip(("rho", "ux", "uy", "uz", "E", "p", "T", "mu_T", "kappa_T"), out))

    def chi_of(self, s: float) -> float:
        return float(lib().orc_chi_of(self._h, float(s)))

    def collide_of(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        out = np.empty(NF * NQ)
        tco = np.empty(3)
        lib().orc_collide_of(self._h, _dp(f), _dp(out), _dp(tco))
        return out.reshape(NF, NQ), tco
