"""Python binding of libugks.so (include/ugks.h): argument marshalling only.

Every step of the UGKS path runs in the CUDA library; this module converts arguments,
checks statuses and raises.  There is no CPU fallback: without the compiled library
(or without a GPU) the calls fail loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_STATUS = {0: "UGKS_OK", 1: "UGKS_EINVAL", 2: "UGKS_ENOMEM", 3: "UGKS_ECUDA",
           4: "UGKS_ETIMEOUT", 5: "UGKS_ENUMERIC"}
FP64, FP32F, DF64 = 0, 1, 2

# Every symbol include/ugks.h declares.
EXPORTS = ("ugks_create", "ugks_destroy", "ugks_last_error", "ugks_get_grid",
           "ugks_device_bytes", "ugks_set_state", "ugks_set_state_device",
           "ugks_init_maxwellian", "ugks_step", "ugks_sync", "ugks_moments", "ugks_get_state",
           "ugks_get_state_device", "ugks_residual", "ugks_profile", "ugks_kernel_times",
           "ugks_kernel_name", "ugks_step_noalloc", "ugks_state_bytes", "ugks_batch_create",
           "ugks_batch_destroy", "ugks_batch_last_error", "ugks_batch_bytes_used",
           "ugks_batch_admit", "ugks_batch_retire", "ugks_batch_instance", "ugks_batch_step",
           "ugks_batch_sync", "ugks_batch_set_walk_rows", "ugks_batch_get_walk_rows",
           "ugks_batch_set_walk_vtile", "ugks_batch_get_walk_vtile", "ugks_batch_set_persistent",
           "ugks_batch_get_persistent", "ugks_batch_set_wait_limit", "ugks_batch_tune",
           "ugks_fp64_rate", "ugks_set_wait_limit", "ugks_set_sums_split", "ugks_get_sums_split")
NKERNELS = 6


class UGKSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _BC(C.Structure):
    _fields_ = [("kind", C.c_int), ("rho", C.c_double), ("T", C.c_double), ("U", C.c_double)]


class _Config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("nu", C.c_int), ("nv", C.c_int), ("umin", C.c_double), ("umax", C.c_double),
                ("vmin", C.c_double), ("vmax", C.c_double), ("K", C.c_int), ("kn", C.c_double),
                ("omega", C.c_double), ("alpha", C.c_double), ("cfl", C.c_double),
                ("dt", C.c_double), ("bc", _BC * 4), ("precision", C.c_int),
                ("ref_rho", C.c_double), ("ref_U", C.c_double), ("ref_V", C.c_double),
                ("ref_T", C.c_double), ("pr", C.c_double)]


_lib = None
_P = C.POINTER(C.c_double)


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libugks.so (building it first if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise OSError(f"{_build.LIB} is missing; run paper_1810_08137_gb300.build.build()")
            _build.build()
        L = C.CDLL(_build.LIB)
        L.ugks_create.argtypes = [C.POINTER(_Config), C.c_void_p, C.POINTER(C.c_void_p)]
        L.ugks_destroy.argtypes = [C.c_void_p]
        L.ugks_destroy.restype = None
        L.ugks_last_error.argtypes = [C.c_void_p]
        L.ugks_last_error.restype = C.c_char_p
        L.ugks_device_bytes.argtypes = [C.c_void_p]
        L.ugks_device_bytes.restype = C.c_size_t
        L.ugks_get_grid.argtypes = [C.c_void_p, _P, _P, _P, _P]
        for name in ("ugks_set_state", "ugks_get_state", "ugks_moments"):
            getattr(L, name).argtypes = [C.c_void_p, _P, _P]
        for name in ("ugks_set_state_device", "ugks_get_state_device"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.ugks_init_maxwellian.argtypes = [C.c_void_p, _P, _P, _P, _P]
        L.ugks_step.argtypes = [C.c_void_p, C.c_int]
        L.ugks_sync.argtypes = [C.c_void_p]
        L.ugks_residual.argtypes = [C.c_void_p, _P]
        L.ugks_profile.argtypes = [C.c_void_p, C.c_int]
        L.ugks_kernel_times.argtypes = [C.c_void_p, _P, C.POINTER(C.c_long)]
        L.ugks_kernel_name.argtypes = [C.c_int]
        L.ugks_kernel_name.restype = C.c_char_p
        L.ugks_step_noalloc.argtypes = [C.POINTER(_Config), C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
        L.ugks_state_bytes.argtypes = [C.POINTER(_Config)]
        L.ugks_state_bytes.restype = C.c_size_t
        L.ugks_batch_create.argtypes = [C.c_int, C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]
        L.ugks_batch_destroy.argtypes = [C.c_void_p]
        L.ugks_batch_destroy.restype = None
        L.ugks_batch_last_error.argtypes = [C.c_void_p]
        L.ugks_batch_last_error.restype = C.c_char_p
        L.ugks_batch_bytes_used.argtypes = [C.c_void_p]
        L.ugks_batch_bytes_used.restype = C.c_size_t
        L.ugks_batch_admit.argtypes = [C.c_void_p, C.POINTER(_Config), C.POINTER(C.c_int)]
        L.ugks_batch_retire.argtypes = [C.c_void_p, C.c_int]
        L.ugks_batch_instance.argtypes = [C.c_void_p, C.c_int]
        L.ugks_batch_instance.restype = C.c_void_p
        L.ugks_batch_step.argtypes = [C.c_void_p, C.c_int]
        L.ugks_batch_sync.argtypes = [C.c_void_p]
        L.ugks_batch_set_walk_rows.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.ugks_batch_get_walk_rows.argtypes = [C.c_void_p, C.c_int]
        L.ugks_batch_set_walk_vtile.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.ugks_batch_get_walk_vtile.argtypes = [C.c_void_p, C.c_int]
        L.ugks_batch_set_persistent.argtypes = [C.c_void_p, C.c_int]
        L.ugks_batch_get_persistent.argtypes = [C.c_void_p]
        L.ugks_batch_set_wait_limit.argtypes = [C.c_void_p, C.c_ulonglong]
        L.ugks_batch_tune.argtypes = [C.c_void_p, C.c_int, _P]
        L.ugks_fp64_rate.argtypes = [C.c_void_p, _P]
        L.ugks_set_wait_limit.argtypes = [C.c_void_p, C.c_longlong]
        L.ugks_set_sums_split.argtypes = [C.c_void_p, C.c_int]
        L.ugks_get_sums_split.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def to_c_config(cfg, precision: int = FP64) -> _Config:
    c = _Config()
    for k in ("nx", "ny", "nu", "nv", "K"):
        setattr(c, k, int(getattr(cfg, k)))
    for k in ("lx", "ly", "umin", "umax", "vmin", "vmax", "kn", "omega", "alpha", "cfl", "dt"):
        setattr(c, k, float(getattr(cfg, k)))
    for s in range(4):
        b = cfg.bc[s]
        c.bc[s].kind, c.bc[s].rho, c.bc[s].T, c.bc[s].U = int(b.kind), float(b.rho), float(b.T), float(b.U)
    c.precision = int(precision)
    ref = getattr(cfg, "ref", None) or (0.0, 0.0, 0.0, 0.0)
    c.ref_rho, c.ref_U, c.ref_V, c.ref_T = (float(x) for x in ref)
    c.pr = float(getattr(cfg, "pr", 1.0))
    return c


def _arr(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.size != int(np.prod(shape)):
        raise ValueError(f"expected {int(np.prod(shape))} values, got {a.size}")
    return a


def _dptr(x) -> int:
    """Device pointer of a torch CUDA tensor (float64, contiguous) or an int address."""
    if isinstance(x, int):
        return x
    if not (x.is_cuda and x.is_contiguous()) or str(x.dtype) != "torch.float64":
        raise ValueError("device buffers must be contiguous float64 CUDA tensors")
    return x.data_ptr()


def state_bytes(cfg, precision: int = FP64) -> int:
    """Device bytes ugks_create allocates for cfg."""
    return int(lib().ugks_state_bytes(C.byref(to_c_config(cfg, precision))))


class Solver:
    """One UGKS instance on the GPU (ugks_create ... ugks_destroy)."""

    def __init__(self, cfg, precision: int = FP64, stream=None, _handle=None):
        self.cfg = cfg
        self.precision = precision
        self._L = lib()
        self.nc, self.nq = cfg.nx * cfg.ny, cfg.nu * cfg.nv
        self._owned = _handle is None
        if _handle is not None:
            self._h = C.c_void_p(_handle)
            return
        self._h = C.c_void_p()
        c = to_c_config(cfg, precision)
        st = self._L.ugks_create(C.byref(c), C.c_void_p(stream or 0), C.byref(self._h))
        if st:
            raise UGKSError(st, "ugks_create failed (see stderr)")

    def _check(self, st: int):
        if st:
            raise UGKSError(st, self._L.ugks_last_error(self._h).decode())

    def close(self):
        if self._h and self._owned:
            self._L.ugks_destroy(self._h)
        self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def device_bytes(self) -> int:
        return int(self._L.ugks_device_bytes(self._h))

    def grid(self):
        dt = C.c_double()
        u, v, w = np.empty(self.cfg.nu), np.empty(self.cfg.nv), np.empty(self.nq)
        self._check(self._L.ugks_get_grid(self._h, C.byref(dt), u.ctypes.data_as(_P),
                                          v.ctypes.data_as(_P), w.ctypes.data_as(_P)))
        return dt.value, u, v, w

    def set_state(self, f, W):
        f = _arr(f, (self.nc, self.nq, 2))
        W = _arr(W, (4, self.nc))
        self._check(self._L.ugks_set_state(self._h, f.ctypes.data_as(_P), W.ctypes.data_as(_P)))

    def set_state_device(self, f_dev, W_dev):
        self._check(self._L.ugks_set_state_device(self._h, C.c_void_p(_dptr(f_dev)),
                                                  C.c_void_p(_dptr(W_dev))))

    def init_maxwellian(self, rho, U, V, T):
        a = [_arr(x, (self.nc,)) for x in (rho, U, V, T)]
        self._check(self._L.ugks_init_maxwellian(self._h, *[x.ctypes.data_as(_P) for x in a]))

    def step(self, n: int = 1):
        self._check(self._L.ugks_step(self._h, int(n)))

    def sync(self):
        self._check(self._L.ugks_sync(self._h))

    def moments(self, prim: bool = False):
        W = np.empty((4, self.nc))
        p = np.empty((4, self.nc)) if prim else None
        self._check(self._L.ugks_moments(self._h, W.ctypes.data_as(_P),
                                         p.ctypes.data_as(_P) if prim else None))
        return (W, p) if prim else W

    def get_state(self):
        f = np.empty((self.nc, self.nq, 2))
        W = np.empty((4, self.nc))
        self._check(self._L.ugks_get_state(self._h, f.ctypes.data_as(_P), W.ctypes.data_as(_P)))
        return f, W

    def get_state_device(self, f_dev, W_dev):
        self._check(self._L.ugks_get_state_device(self._h, C.c_void_p(_dptr(f_dev)),
                                                  C.c_void_p(_dptr(W_dev))))

    def profile(self, enable: bool = True):
        self._check(self._L.ugks_profile(self._h, int(bool(enable))))

    def kernel_times(self) -> dict:
        """{kernel name: (launches, total ms)} of the steps recorded since profile(True)."""
        ms = np.zeros(NKERNELS)
        n = (C.c_long * NKERNELS)()
        self._check(self._L.ugks_kernel_times(self._h, ms.ctypes.data_as(_P), n))
        return {self._L.ugks_kernel_name(k).decode(): (int(n[k]), float(ms[k]))
                for k in range(NKERNELS)}

    def set_wait_limit(self, polls: int):
        self._check(self._L.ugks_set_wait_limit(self._h, C.c_longlong(int(polls))))

    def set_sums_split(self, warps: int):
        """FP32-f form: warps per cell of the velocity sums (1, 2, 4; 0 = automatic)."""
        self._check(self._L.ugks_set_sums_split(self._h, int(warps)))

    @property
    def sums_split(self) -> int:
        return int(self._L.ugks_get_sums_split(self._h))

    def residual(self) -> np.ndarray:
        r = np.empty(4)
        self._check(self._L.ugks_residual(self._h, r.ctypes.data_as(_P)))
        return r


def fp64_rate(stream=None) -> float:
    """ugks_fp64_rate: measured FP64 FMA throughput of the current device, GFLOP/s."""
    g = C.c_double()
    st = lib().ugks_fp64_rate(C.c_void_p(stream or 0), C.byref(g))
    if st:
        raise UGKSError(st, "ugks_fp64_rate failed")
    return g.value


def step_noalloc(cfg, f_in, W_in, f_out, W_out, stream=None) -> None:
    """ugks_step_noalloc: one FP64 step on caller-owned device buffers (torch CUDA float64
    tensors or integer addresses), with no device allocation by the library."""
    c = to_c_config(cfg, FP64)
    st = lib().ugks_step_noalloc(C.byref(c), C.c_void_p(_dptr(f_in)), C.c_void_p(_dptr(W_in)),
                                 C.c_void_p(_dptr(f_out)), C.c_void_p(_dptr(W_out)),
                                 C.c_void_p(stream or 0))
    if st:
        raise UGKSError(st, "ugks_step_noalloc failed (see stderr)")


class Batch:
    """Independent FP32-f instances stepped together (ugks_batch_*)."""

    def __init__(self, max_slots: int, hbm_budget: int = 0, stream=None):
        self._L = lib()
        self._b = C.c_void_p()
        st = self._L.ugks_batch_create(int(max_slots), C.c_size_t(int(hbm_budget)),
                                       C.c_void_p(stream or 0), C.byref(self._b))
        if st:
            raise UGKSError(st, "ugks_batch_create failed (see stderr)")
        self.cfgs = {}

    def _check(self, st: int):
        if st:
            raise UGKSError(st, self._L.ugks_batch_last_error(self._b).decode())

    def close(self):
        if self._b:
            self._L.ugks_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def bytes_used(self) -> int:
        return int(self._L.ugks_batch_bytes_used(self._b))

    def admit(self, cfg) -> int:
        slot = C.c_int(-1)
        self._check(self._L.ugks_batch_admit(self._b, C.byref(to_c_config(cfg, FP32F)),
                                             C.byref(slot)))
        self.cfgs[slot.value] = cfg
        return slot.value

    def retire(self, slot: int):
        self._check(self._L.ugks_batch_retire(self._b, int(slot)))
        self.cfgs.pop(slot, None)

    def instance(self, slot: int) -> Solver:
        """View of a slot's instance (state I/O and results; not owned, do not step)."""
        h = self._L.ugks_batch_instance(self._b, int(slot))
        if not h:
            raise UGKSError(1, f"slot {slot} is free")
        return Solver(self.cfgs[slot], FP32F, _handle=h)

    def step(self, n: int = 1):
        self._check(self._L.ugks_batch_step(self._b, int(n)))

    def sync(self):
        self._check(self._L.ugks_batch_sync(self._b))

    def set_walk_rows(self, slot: int, rows: int):
        self._check(self._L.ugks_batch_set_walk_rows(self._b, int(slot), int(rows)))

    def walk_rows(self, slot: int) -> int:
        return int(self._L.ugks_batch_get_walk_rows(self._b, int(slot)))

    def set_walk_vtile(self, slot: int, chunks: int):
        self._check(self._L.ugks_batch_set_walk_vtile(self._b, int(slot), int(chunks)))

    def walk_vtile(self, slot: int) -> int:
        return int(self._L.ugks_batch_get_walk_vtile(self._b, int(slot)))

    @property
    def persistent(self) -> bool:
        return bool(self._L.ugks_batch_get_persistent(self._b))

    def set_persistent(self, enable: bool):
        self._check(self._L.ugks_batch_set_persistent(self._b, int(bool(enable))))

    def set_wait_limit(self, polls: int):
        self._check(self._L.ugks_batch_set_wait_limit(self._b, C.c_ulonglong(int(polls))))

    def tune(self, trial_steps: int = 3) -> float:
        ms = C.c_double()
        self._check(self._L.ugks_batch_tune(self._b, int(trial_steps), C.byref(ms)))
        return ms.value
