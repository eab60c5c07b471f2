"""Thin Python binding of liblbm.so (the C ABI in include/lbm.h).

Argument marshalling only: every step of the path runs in the CUDA library.
The functions keep the C names; ``Domain`` and ``Batch`` wrap a handle and use
PyTorch for device buffers and the CUDA stream. If the library has not been
built this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY=checked selects the build with address checks (liblbm_checked.so; see
# lbm_check_count in include/lbm.h); the default is the production build.
LIB_VARIANT = os.environ.get("LBM_LIBRARY", "")
LIB_PATH = os.path.join(_PKG, "_lib", "liblbm_checked.so" if LIB_VARIANT == "checked" else "liblbm.so")

LBM_OK, LBM_E_INVAL, LBM_E_NOMEM, LBM_E_CUDA, LBM_E_NONFINITE, LBM_E_STATE, LBM_E_IO, LBM_E_TIMEOUT = range(8)
STORE_F32, STORE_F16, STORE_BF16 = 0, 1, 2
DT_F32, DT_F64, DT_NATIVE = 0, 1, 2
MOM_Q, MOM_PRIM = 0, 1
STORES = {"f32": STORE_F32, "f16": STORE_F16, "bf16": STORE_BF16}


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("bc_x", ctypes.c_int),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
        ("lambda_ref", ctypes.c_double), ("gamma", ctypes.c_double), ("mu", ctypes.c_double),
        ("kappa", ctypes.c_double), ("tau_R", ctypes.c_double), ("tau_q", ctypes.c_double),
        ("T_ref", ctypes.c_double), ("relax_in_dt", ctypes.c_int), ("sutherland", ctypes.c_int),
        ("source_mode", ctypes.c_int), ("f_mu", ctypes.c_double), ("C_sigma", ctypes.c_double),
        ("J_min", ctypes.c_double), ("omega_min", ctypes.c_double), ("sensor_mode", ctypes.c_int),
        ("collide", ctypes.c_int), ("store", ctypes.c_int), ("stochastic_round", ctypes.c_int),
        ("use_graphs", ctypes.c_int), ("streaming", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p), ("pop_buffer", ctypes.c_void_p),
    ]


class LbmInfo(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("c", ctypes.c_double), ("tau_R", ctypes.c_double),
        ("tau_q", ctypes.c_double), ("rho_ref", ctypes.c_double), ("E_ref", ctypes.c_double),
        ("scale", ctypes.c_double * 14), ("step", ctypes.c_longlong), ("ncell", ctypes.c_longlong),
        ("population_bytes", ctypes.c_size_t), ("store", ctypes.c_int), ("block_x", ctypes.c_int),
        ("variant", ctypes.c_int), ("prefetch_tiles", ctypes.c_int), ("device", ctypes.c_int),
    ]


DIAG_FIELDS = ("step", "time", "sum_rho", "sum_mx", "sum_my", "sum_mz", "sum_E", "ek_mean",
               "eps_s_raw", "eps_d_raw", "max_mach", "max_cfl", "min_rho", "min_T", "nonfinite")


class LbmDiag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in DIAG_FIELDS]


class LbmTune(ctypes.Structure):
    _fields_ = [("block_x", ctypes.c_int), ("variant", ctypes.c_int), ("ms_per_step", ctypes.c_float),
                ("candidates", ctypes.c_int), ("prefetch_tiles", ctypes.c_int)]


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_STATUS_NAMES = {0: "LBM_OK", 1: "LBM_E_INVAL", 2: "LBM_E_NOMEM", 3: "LBM_E_CUDA",
                 4: "LBM_E_NONFINITE", 5: "LBM_E_STATE", 6: "LBM_E_IO", 7: "LBM_E_TIMEOUT"}

_lib = None

# name -> (restype, argtypes)
_VP, _IP, _DP = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
_SIGNATURES = {
    "lbm_population_bytes": (ctypes.c_size_t, [ctypes.POINTER(LbmParams)]),
    "lbm_create": (_IP, [ctypes.POINTER(LbmParams), ctypes.POINTER(_VP)]),
    "lbm_destroy": (_IP, [_VP]),
    "lbm_last_error": (ctypes.c_char_p, []),
    "lbm_status_string": (ctypes.c_char_p, [_IP]),
    "lbm_get_info": (_IP, [_VP, ctypes.POINTER(LbmInfo)]),
    "lbm_init_tgv": (_IP, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "lbm_init_riemann": (_IP, [_VP, _IP, _IP, _DP, _DP]),
    "lbm_init_fields": (_IP, [_VP, _VP, _IP, _IP]),
    "lbm_init_state": (_IP, [_VP, _VP, _IP, _IP]),
    "lbm_step": (_IP, [_VP, _IP]),
    "lbm_synchronize": (_IP, [_VP]),
    "lbm_moments": (_IP, [_VP, _IP, _VP, _IP, _IP]),
    "lbm_sensor": (_IP, [_VP, _VP, _IP, _IP]),
    "lbm_diag": (_IP, [_VP, ctypes.POINTER(LbmDiag)]),
    "lbm_diag_static": (_IP, [_VP, ctypes.POINTER(LbmDiag)]),
    "lbm_step_diag": (_IP, [_VP, _IP, ctypes.POINTER(LbmDiag)]),
    "lbm_test_skip_copy": (_IP, [_VP]),
    "lbm_test_encode": (_IP, [_IP, _IP, _VP, _VP, _VP, ctypes.c_longlong, _VP]),
    "lbm_plane_get": (_IP, [_VP, _IP, _IP, _VP, _IP]),
    "lbm_plane_set": (_IP, [_VP, _IP, _IP, _VP, _IP]),
    "lbm_populations_get": (_IP, [_VP, _VP, _IP, _IP]),
    "lbm_populations_set": (_IP, [_VP, _VP, _IP, _IP]),
    "lbm_save": (_IP, [_VP, ctypes.c_char_p]),
    "lbm_load": (_IP, [_VP, ctypes.c_char_p]),
    "lbm_autotune": (_IP, [_VP, _IP, ctypes.POINTER(LbmTune)]),
    "lbm_set_kernel_config": (_IP, [_VP, _IP, _IP]),
    "lbm_set_prefetch": (_IP, [_VP, _IP]),
    "lbm_batch_create": (_IP, [_IP, ctypes.POINTER(LbmParams), ctypes.POINTER(_VP)]),
    "lbm_batch_destroy": (_IP, [_VP]),
    "lbm_batch_init_tgv": (_IP, [_VP, _DP, _DP, _DP]),
    "lbm_batch_step": (_IP, [_VP, _IP]),
    "lbm_batch_step_sequential": (_IP, [_VP, _IP]),
    "lbm_batch_synchronize": (_IP, [_VP]),
    "lbm_batch_moments": (_IP, [_VP, _IP, _IP, _VP, _IP, _IP]),
    "lbm_batch_info": (_IP, [_VP, ctypes.POINTER(ctypes.c_longlong), _IP, _DP]),
    "lbm_batch_diag": (_IP, [_VP, _IP, ctypes.POINTER(LbmDiag)]),
    "lbm_batch_autotune": (_IP, [_VP, _IP, ctypes.POINTER(_IP), ctypes.POINTER(_IP),
                                 ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_IP)]),
    "lbm_batch_set_prefetch": (_IP, [_VP, _IP]),
    "lbm_check_count": (_IP, [_VP, ctypes.POINTER(ctypes.c_ulonglong)]),
    "lbm_batch_check_count": (_IP, [_VP, ctypes.POINTER(ctypes.c_ulonglong)]),
}


def lib():
    """The loaded library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"liblbm.so is not built ({LIB_PATH}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != LBM_OK:
        raise LbmError(status, lib().lbm_last_error().decode())


def make_params(p: dict, store="f32", stream=None, pop_buffer=None, use_graphs=True) -> LbmParams:
    fields = {n for n, _ in LbmParams._fields_}
    kw = {k: v for k, v in p.items() if k in fields}
    unknown = set(p) - fields
    if unknown:
        raise TypeError(f"unknown parameters {sorted(unknown)}")
    kw["store"] = STORES[store] if isinstance(store, str) else int(store)
    kw["use_graphs"] = int(use_graphs)
    kw["cuda_stream"] = stream
    kw["pop_buffer"] = pop_buffer
    return LbmParams(**kw)


def _np_ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


class Domain:
    """One domain. Device buffers and the stream come from PyTorch."""

    def __init__(self, params: dict, store="f32", use_graphs=True, torch_buffer=True,
                 device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        torch.cuda.set_device(self.device)
        self.stream = torch.cuda.current_stream(self.device)
        self.params = dict(params)
        pr = make_params(params, store, stream=self.stream.cuda_stream, use_graphs=use_graphs)
        nbytes = lib().lbm_population_bytes(ctypes.byref(pr))
        if nbytes == 0:
            raise LbmError(LBM_E_INVAL, "invalid grid sizes")
        self._buf = None
        if torch_buffer:
            self._buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            pr.pop_buffer = self._buf.data_ptr()
        h = ctypes.c_void_p()
        check(lib().lbm_create(ctypes.byref(pr), ctypes.byref(h)))
        self._h = h
        self.nx, self.ny, self.nz = params["nx"], params["ny"], params["nz"]
        self.shape = (self.nz, self.ny, self.nx)
        self.ncell = self.nx * self.ny * self.nz
        self.store = pr.store

    # lifecycle ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None
            self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def buffer(self):
        """The population buffer in its stored layout (torch uint8 tensor on the device),
        or None when the library allocated it (torch_buffer=False)."""
        return self._buf

    def info(self) -> dict:
        inf = LbmInfo()
        check(lib().lbm_get_info(self._h, ctypes.byref(inf)))
        d = {n: getattr(inf, n) for n, _ in LbmInfo._fields_}
        d["scale"] = list(inf.scale)
        return d

    @property
    def dt(self) -> float:
        return self.info()["dt"]

    # initial states -------------------------------------------------------
    def init_tgv(self, U0=1.0, M0=1.25, rho0=1.0):
        check(lib().lbm_init_tgv(self._h, U0, M0, rho0))

    def init_riemann(self, axis, i_split, left, right):
        L = (ctypes.c_double * 3)(*left)
        R = (ctypes.c_double * 3)(*right)
        check(lib().lbm_init_riemann(self._h, axis, i_split, L, R))

    def init_fields(self, rho, ux, uy, uz, p, dtype=np.float64):
        arr = np.ascontiguousarray(np.stack([np.broadcast_to(a, self.shape) for a in
                                             (rho, ux, uy, uz, p)]), dtype=dtype)
        check(lib().lbm_init_fields(self._h, _np_ptr(arr), 0,
                                    DT_F64 if arr.dtype == np.float64 else DT_F32))

    def init_state(self, Q, dtype=np.float64):
        """Equilibrium of given zeroth moments Q (14, nz, ny, nx)."""
        arr = np.ascontiguousarray(np.broadcast_to(Q, (14,) + self.shape), dtype=dtype)
        check(lib().lbm_init_state(self._h, _np_ptr(arr), 0,
                                   DT_F64 if arr.dtype == np.float64 else DT_F32))

    def init_fields_device(self, fields, src_on_device=True):
        """fields: torch tensor (5, nz, ny, nx) float32/float64 on the device (or pinned host)."""
        t = fields.contiguous()
        dt = DT_F64 if t.dtype == self.torch.float64 else DT_F32
        check(lib().lbm_init_fields(self._h, ctypes.c_void_p(t.data_ptr()), int(src_on_device), dt))

    # stepping ---------------------------------------------------------------
    def step(self, n=1):
        check(lib().lbm_step(self._h, int(n)))

    def step_diag(self, n=1) -> dict:
        """n steps; the first also returns the diagnostics of the state it starts from
        (computed inside the step kernel). Same keys as diag()."""
        d = LbmDiag()
        st = lib().lbm_step_diag(self._h, int(n), ctypes.byref(d))
        res = {k: getattr(d, k) for k in DIAG_FIELDS}
        if st not in (LBM_OK, LBM_E_NONFINITE):
            check(st)
        res["status"] = st
        return res

    def synchronize(self):
        check(lib().lbm_synchronize(self._h))

    # outputs ----------------------------------------------------------------
    def moments(self, which=MOM_Q, dtype=np.float64) -> np.ndarray:
        nf = 14 if which == MOM_Q else 6
        out = np.empty((nf,) + self.shape, dtype=dtype)
        check(lib().lbm_moments(self._h, which, _np_ptr(out), 0,
                                DT_F64 if out.dtype == np.float64 else DT_F32))
        return out

    def primitives(self, dtype=np.float64) -> np.ndarray:
        return self.moments(MOM_PRIM, dtype)

    def moments_device(self, which=MOM_Q, dtype=None):
        torch = self.torch
        dtype = dtype or torch.float32
        nf = 14 if which == MOM_Q else 6
        out = torch.empty((nf,) + self.shape, dtype=dtype, device=self.device)
        check(lib().lbm_moments(self._h, which, ctypes.c_void_p(out.data_ptr()), 1,
                                DT_F64 if dtype == torch.float64 else DT_F32))
        return out

    def moments_into(self, out, which=MOM_PRIM, on_device=False):
        """Write moments into an existing torch tensor (pinned host or device)."""
        dt = DT_F64 if out.dtype == self.torch.float64 else DT_F32
        check(lib().lbm_moments(self._h, which, ctypes.c_void_p(out.data_ptr()), int(on_device), dt))

    def sensor(self, dtype=np.float64):
        out = np.empty((3,) + self.shape, dtype=dtype)
        check(lib().lbm_sensor(self._h, _np_ptr(out), 0,
                               DT_F64 if out.dtype == np.float64 else DT_F32))
        return out[0], out[1], out[2]

    def diag(self) -> dict:
        d = LbmDiag()
        st = lib().lbm_diag(self._h, ctypes.byref(d))
        res = {n: getattr(d, n) for n in DIAG_FIELDS}
        if st not in (LBM_OK, LBM_E_NONFINITE):
            check(st)
        res["status"] = st
        return res

    def populations(self, dtype=np.float64) -> np.ndarray:
        if dtype == "native":
            nd = np.float32 if self.store == STORE_F32 else np.uint16
            out = np.empty((14, 7) + self.shape, dtype=nd)
            check(lib().lbm_populations_get(self._h, _np_ptr(out), 0, DT_NATIVE))
            return out
        out = np.empty((14, 7) + self.shape, dtype=dtype)
        check(lib().lbm_populations_get(self._h, _np_ptr(out), 0,
                                        DT_F64 if out.dtype == np.float64 else DT_F32))
        return out

    def set_populations(self, f: np.ndarray, native=False):
        f = np.ascontiguousarray(f)
        if native:
            check(lib().lbm_populations_set(self._h, _np_ptr(f), 0, DT_NATIVE))
        else:
            f = np.ascontiguousarray(f, dtype=np.float64)
            check(lib().lbm_populations_set(self._h, _np_ptr(f), 0, DT_F64))

    def plane_get(self, z: int, slot: int, out=None):
        """Raw stored values of storage slot `slot` on plane z, (14, ny, nx): a device
        tensor (int32 for F32 storage, int16 otherwise) unless `out` is a numpy array."""
        if isinstance(out, np.ndarray):
            check(lib().lbm_plane_get(self._h, int(z), int(slot), _np_ptr(out), 0))
            return out
        if out is None:
            out = self.torch.empty((14, self.ny, self.nx), dtype=self.plane_dtype(), device=self.device)
        check(lib().lbm_plane_get(self._h, int(z), int(slot), ctypes.c_void_p(out.data_ptr()), 1))
        return out

    def plane_set(self, z: int, slot: int, buf):
        if isinstance(buf, np.ndarray):
            buf = np.ascontiguousarray(buf)
            check(lib().lbm_plane_set(self._h, int(z), int(slot), _np_ptr(buf), 0))
        else:
            buf = buf.contiguous()
            check(lib().lbm_plane_set(self._h, int(z), int(slot), ctypes.c_void_p(buf.data_ptr()), 1))

    def plane_dtype(self, numpy=False):
        if numpy:
            return np.int32 if self.store == STORE_F32 else np.int16
        return self.torch.int32 if self.store == STORE_F32 else self.torch.int16

    @property
    def step_count(self) -> int:
        return int(self.info()["step"])

    def save(self, path: str):
        check(lib().lbm_save(self._h, path.encode()))

    def load(self, path: str):
        check(lib().lbm_load(self._h, path.encode()))

    def set_kernel_config(self, block_x: int, variant: int):
        check(lib().lbm_set_kernel_config(self._h, int(block_x), int(variant)))

    def set_prefetch(self, tiles: int):
        check(lib().lbm_set_prefetch(self._h, int(tiles)))

    def autotune(self, pairs_per_trial=4) -> dict:
        t = LbmTune()
        check(lib().lbm_autotune(self._h, int(pairs_per_trial), ctypes.byref(t)))
        return {"block_x": t.block_x, "variant": t.variant, "ms_per_step": t.ms_per_step,
                "candidates": t.candidates, "prefetch_tiles": t.prefetch_tiles}


class Batch:
    """Many independent periodic domains (one storage type) advanced together."""

    def __init__(self, param_list: list[dict], store="f32", device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        torch.cuda.set_device(self.device)
        self.stream = torch.cuda.current_stream(self.device)
        arr = (LbmParams * len(param_list))(*[make_params(p, store, stream=self.stream.cuda_stream)
                                              for p in param_list])
        h = ctypes.c_void_p()
        check(lib().lbm_batch_create(len(param_list), arr, ctypes.byref(h)))
        self._h = h
        self.n = len(param_list)
        self.shapes = [(p["nz"], p["ny"], p["nx"]) for p in param_list]

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_tgv(self, U0, M0, rho0):
        a = [np.ascontiguousarray(v, dtype=np.float64) for v in (U0, M0, rho0)]
        check(lib().lbm_batch_init_tgv(self._h, *[x.ctypes.data_as(_DP) for x in a]))

    def step(self, n=1):
        check(lib().lbm_batch_step(self._h, int(n)))

    def step_sequential(self, n=1):
        check(lib().lbm_batch_step_sequential(self._h, int(n)))

    def synchronize(self):
        check(lib().lbm_batch_synchronize(self._h))

    def moments(self, d, which=MOM_Q, dtype=np.float64):
        nf = 14 if which == MOM_Q else 6
        out = np.empty((nf,) + self.shapes[d], dtype=dtype)
        check(lib().lbm_batch_moments(self._h, d, which, _np_ptr(out), 0,
                                      DT_F64 if out.dtype == np.float64 else DT_F32))
        return out

    def diag(self, d) -> dict:
        """lbm_diag of domain d (same keys as Domain.diag)."""
        r = LbmDiag()
        st = lib().lbm_batch_diag(self._h, int(d), ctypes.byref(r))
        res = {n: getattr(r, n) for n in DIAG_FIELDS}
        if st not in (LBM_OK, LBM_E_NONFINITE):
            check(st)
        res["status"] = st
        return res

    def total_cells(self) -> int:
        t = ctypes.c_longlong()
        check(lib().lbm_batch_info(self._h, ctypes.byref(t), 0, None))
        return int(t.value)

    def dt(self, d) -> float:
        v = ctypes.c_double()
        check(lib().lbm_batch_info(self._h, None, int(d), ctypes.byref(v)))
        return float(v.value)

    def set_prefetch(self, tiles: int):
        check(lib().lbm_batch_set_prefetch(self._h, int(tiles)))

    def autotune(self, steps_per_trial=4) -> dict:
        tc, bt, ms, pf = ctypes.c_int(), ctypes.c_int(), ctypes.c_float(), ctypes.c_int()
        check(lib().lbm_batch_autotune(self._h, int(steps_per_trial), ctypes.byref(tc),
                                       ctypes.byref(bt), ctypes.byref(ms), ctypes.byref(pf)))
        return {"tile_cells": tc.value, "block": bt.value, "ms_per_step": ms.value,
                "prefetch_tiles": pf.value}


def encode_pairs(store, values, rbits=None):
    """lbm_test_encode on device tensors: values (float32, 2 n elements), rbits (n
    32-bit words as int32, or None to round to nearest) -> n packed words (int32)."""
    import torch
    v = values.contiguous()
    if v.dtype != torch.float32 or not v.is_cuda or v.numel() % 2:
        raise ValueError("values must be a CUDA float32 tensor of even length")
    n = v.numel() // 2
    out = torch.empty(n, dtype=torch.int32, device=v.device)
    r = None
    if rbits is not None:
        r = rbits.contiguous()
        if r.dtype != torch.int32 or r.numel() != n or r.device != v.device:
            raise ValueError("rbits must be an int32 tensor of one word per pair on the same device")
    stream = torch.cuda.current_stream(v.device)
    check(lib().lbm_test_encode(STORES[store] if isinstance(store, str) else int(store),
                                int(r is not None), v.data_ptr(),
                                r.data_ptr() if r is not None else None, out.data_ptr(), n,
                                stream.cuda_stream))
    stream.synchronize()
    return out
