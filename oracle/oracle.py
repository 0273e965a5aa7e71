"""ctypes binding of the FP64 CPU UGKS oracle (ugks_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU-baseline leg
use it; the product path never imports it.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ugks_oracle.c")
LIB = os.path.join(HERE, "libugks_oracle.so")


def compile_source(src: str, out: str) -> str:
    """Compile one C source file of the oracle into the shared library `out` (gcc, OpenMP
    over faces and cells).  The source must include ugks_oracle.h from this directory."""
    tmp = out + f".tmp{os.getpid()}"
    # no floating-point contraction: the same rounding on x86 and aarch64
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-D_GNU_SOURCE", "-fPIC", "-shared",
                           "-fopenmp", "-I", HERE, "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (if its source is newer than the library)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "ugks_oracle.h"))):
        compile_source(SRC, LIB)
    return LIB


class _Cfg(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("nu", C.c_int), ("nv", C.c_int), ("umin", C.c_double), ("umax", C.c_double),
                ("vmin", C.c_double), ("vmax", C.c_double), ("K", C.c_int),
                ("kn", C.c_double), ("omega", C.c_double), ("alpha", C.c_double),
                ("cfl", C.c_double), ("dt", C.c_double), ("bc_kind", C.c_int * 4),
                ("bc_rho", C.c_double * 4), ("bc_T", C.c_double * 4), ("bc_U", C.c_double * 4),
                ("pr", C.c_double)]


_lib = None
_P = C.POINTER(C.c_double)


def _load(path: str):
    L = C.CDLL(path)
    L.orc_dt.restype = C.c_double
    L.orc_tau.restype = C.c_double
    L.orc_get_threads.restype = C.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _load(LIB)
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Route every call of this module to another build of the oracle (a copy with a
    deliberately planted mistake, in the tests that show the pins catch it)."""
    global _lib
    old = lib()
    threads = old.orc_get_threads()
    _lib = _load(path)
    _lib.orc_set_threads(threads)
    try:
        yield
    finally:
        _lib = old


def _cfg(cfg) -> _Cfg:
    c = _Cfg()
    for k in ("nx", "ny", "nu", "nv", "K"):
        setattr(c, k, int(getattr(cfg, k)))
    for k in ("lx", "ly", "umin", "umax", "vmin", "vmax", "kn", "omega", "alpha", "cfl", "dt"):
        setattr(c, k, float(getattr(cfg, k)))
    for s in range(4):
        c.bc_kind[s] = int(cfg.bc[s].kind)
        c.bc_rho[s] = float(cfg.bc[s].rho)
        c.bc_T[s] = float(cfg.bc[s].T)
        c.bc_U[s] = float(cfg.bc[s].U)
    c.pr = float(getattr(cfg, "pr", 1.0))
    return c


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def vgrid(cfg):
    u = np.empty(cfg.nu)
    v = np.empty(cfg.nv)
    w = np.empty(cfg.nu * cfg.nv)
    lib().orc_vgrid(C.byref(_cfg(cfg)), _p(u), _p(v), _p(w))
    return u, v, w


def dt(cfg) -> float:
    return lib().orc_dt(C.byref(_cfg(cfg)))


def tau(cfg, rho: float, lam: float) -> float:
    return lib().orc_tau(C.byref(_cfg(cfg)), C.c_double(rho), C.c_double(lam))


def mt(dt_: float, tau_: float) -> np.ndarray:
    out = np.empty(5)
    lib().orc_mt(C.c_double(dt_), C.c_double(tau_), _p(out))
    return out


def gauss_moments(U: float, lam: float, nmax: int):
    full, pos, neg = (np.empty(nmax + 1) for _ in range(3))
    lib().orc_gauss_moments(C.c_double(U), C.c_double(lam), C.c_int(nmax), _p(full), _p(pos),
                            _p(neg))
    return full, pos, neg


def slope_solve(prim, K: int, s) -> np.ndarray:
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    a = np.empty(4)
    lib().orc_slope_solve(_p(prim), C.c_int(K), _p(s), _p(a))
    return a


def shakhov_eq(prim, K: int, pr: float, q, u, v) -> np.ndarray:
    """Shakhov equilibrium (h, b) at the velocities (u[i], v[i]): shape (n, 2)."""
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    out = np.empty((u.size, 2))
    lib().orc_shakhov_eq(_p(np.ascontiguousarray(prim, dtype=np.float64)), C.c_int(K),
                         C.c_double(pr), _p(np.ascontiguousarray(q, dtype=np.float64)),
                         C.c_int(u.size), _p(u), _p(v), _p(out))
    return out


def heat_flux(cfg, f_cell, W_cell) -> np.ndarray:
    """Heat flux (qx, qy) of one cell's f[nq][2] about the velocity of W_cell[4]."""
    q = np.empty(2)
    lib().orc_heat_flux(C.byref(_cfg(cfg)), _p(np.ascontiguousarray(f_cell, dtype=np.float64)),
                        _p(np.ascontiguousarray(W_cell, dtype=np.float64)), _p(q))
    return q


def init_maxwellian(cfg, rho, U, V, T):
    """Pointwise Maxwellian f[nc][nq][2] and analytic W[4][nc] from primitive fields."""
    f = np.empty((cfg.nc, cfg.nq, 2))
    W = np.empty((4, cfg.nc))
    arr = [np.ascontiguousarray(x, dtype=np.float64) for x in (rho, U, V, T)]
    lib().orc_init_maxwellian(C.byref(_cfg(cfg)), *[_p(x) for x in arr], _p(f), _p(W))
    return f, W


def fluxes(cfg, f, W):
    nfx = (cfg.nx + 1) * cfg.ny
    nfy = cfg.nx * (cfg.ny + 1)
    Fx = np.empty((nfx, 4))
    Fy = np.empty((nfy, 4))
    fx = np.empty((nfx, cfg.nq, 2))
    fy = np.empty((nfy, cfg.nq, 2))
    lib().orc_fluxes(C.byref(_cfg(cfg)), _p(np.ascontiguousarray(f)),
                     _p(np.ascontiguousarray(W)), _p(Fx), _p(Fy), _p(fx), _p(fy))
    return Fx, Fy, fx, fy


def step(cfg, f, W, nsteps: int = 1):
    """nsteps UGKS steps; returns new (f, W) (inputs untouched)."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    W = np.array(W, dtype=np.float64, order="C", copy=True)
    lib().orc_step(C.byref(_cfg(cfg)), _p(f), _p(W), C.c_int(nsteps))
    return f, W


def step_cells(cfg, f, W, ids):
    """One step for the listed cells only: (f_out[n][nq][2], W_out[n][4])."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    n = len(ids)
    fo = np.empty((n, cfg.nq, 2))
    Wo = np.empty((n, 4))
    lib().orc_step_cells(C.byref(_cfg(cfg)), _p(np.ascontiguousarray(f)),
                         _p(np.ascontiguousarray(W)), C.c_int(n),
                         ids.ctypes.data_as(C.POINTER(C.c_int)), _p(fo), _p(Wo))
    return fo, Wo
