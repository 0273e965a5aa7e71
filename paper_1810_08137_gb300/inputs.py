"""Seeded synthetic inputs for the 2D UGKS channel workloads.

This module holds configurations and random numbers only -- none of the scheme's
arithmetic -- so that both the CUDA library and the CPU oracle can be fed the same
inputs.  The workloads are shaped like the paper's 2D pressure-driven channel
(Sec. 3.A) and its mesh-size and velocity-grid sweeps (Sec. 3.B, Tables 1 and 3).

Random numbers: SplitMix64 (Vigna's published definition) drives a Box-Muller
transform; the i-th draw of a stream depends only on (seed, i), so any subset of a
field can be regenerated independently of the rest.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

BC_PERIODIC, BC_WALL, BC_PRESSURE = 0, 1, 2
SIDE_W, SIDE_E, SIDE_S, SIDE_N = 0, 1, 2, 3
SEED_BASE = 1810_08137

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


@dataclass
class BC:
    kind: int
    rho: float = 1.0
    T: float = 1.0
    U: float = 0.0


@dataclass
class Config:
    """One channel-flow instance: mesh, velocity grid, gas, time step, boundaries."""

    nx: int
    ny: int
    lx: float = 5.0
    ly: float = 1.0
    nu: int = 20
    nv: int = 20
    umin: float = -4.0
    umax: float = 4.0
    vmin: float = -4.0
    vmax: float = 4.0
    K: int = 1
    kn: float = 0.1
    omega: float = 0.5
    alpha: float = 1.0
    cfl: float = 0.8
    dt: float = 0.0
    bc: list = field(default_factory=lambda: [BC(BC_PRESSURE, 1.2), BC(BC_PRESSURE, 1.0),
                                              BC(BC_WALL), BC(BC_WALL)])
    steps: int = 200
    name: str = ""
    # (rho, U, V, T) of the FP32-f form's reference Maxwellian g_ref (f is stored as f - g_ref);
    # None: the library's default (1, 0, 0, 1).  Not used by the FP64 form.
    ref: tuple = None
    # Prandtl number: 1 = the BGK model of Eq. 1; otherwise the Shakhov model
    pr: float = 1.0

    @property
    def nc(self) -> int:
        return self.nx * self.ny

    @property
    def nq(self) -> int:
        return self.nu * self.nv

    @property
    def vc(self) -> int:
        """velocity-cells per step"""
        return self.nc * self.nq

    def replace(self, **kw) -> "Config":
        return dataclasses.replace(self, **kw)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Draws start..start+n-1 of the SplitMix64 stream seeded with `seed`."""
    idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in (0, 1]: top 53 bits of SplitMix64, plus one ulp step."""
    z = splitmix64(seed, n, start)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller: pair p uses draws 2p and 2p+1."""
    npair = (n + 1) // 2
    u = uniform01(seed, 2 * npair)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * math.pi * u[1::2]
    out = np.empty(2 * npair)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:n]


def seed_for(config_id: int, instance: int = 0) -> int:
    return SEED_BASE + 1000 * config_id + instance


def initial_prim(cfg: Config, seed: int, amp: float = 1e-3, mirror_y: bool = False):
    """Initial primitive fields (rho, U, V, T) per cell, row-major (x fastest):
    rho = 1 + amp*N(0,1), U = V = 0, T = 1.  mirror_y makes rho symmetric about the
    channel centre line (row j and row ny-1-j share draws)."""
    n = normal(seed, cfg.nc).reshape(cfg.ny, cfg.nx)
    if mirror_y:
        for j in range(cfg.ny // 2, cfg.ny):
            n[j] = n[cfg.ny - 1 - j]
    rho = (1.0 + amp * n).reshape(-1)
    U = np.zeros(cfg.nc)
    V = np.zeros(cfg.nc)
    T = np.ones(cfg.nc)
    return rho, U, V, T


def perturbation(seed: int, shape, amp: float) -> np.ndarray:
    """Multiplicative factors 1 + amp*(2r-1), r uniform, for non-equilibrium test states."""
    n = int(np.prod(shape))
    r = uniform01(seed, n)
    return (1.0 + amp * (2.0 * r - 1.0)).reshape(shape)


# --------------------------------------------------------------------------------------
# Named workloads (2D pressure-driven channel, Sec. 3.A; sweeps of Sec. 3.B)
# --------------------------------------------------------------------------------------
def channel_config(nx=40, ny=20, n_vel=20, vrange=4.0, kn=0.1, rho_in=1.2, rho_out=1.0,
                   steps=200, name="") -> Config:
    """Pressure-driven channel; the FP32-f reference Maxwellian sits at the mean of the inlet
    and outlet densities (U = V = 0, T = 1), which halves the FP32 deviation f - g_ref at the
    channel ends against the default density 1."""
    return Config(nx=nx, ny=ny, lx=5.0, ly=1.0, nu=n_vel, nv=n_vel,
                  umin=-vrange, umax=vrange, vmin=-vrange, vmax=vrange, K=1, kn=kn,
                  cfl=0.8, bc=[BC(BC_PRESSURE, rho_in), BC(BC_PRESSURE, rho_out),
                               BC(BC_WALL), BC(BC_WALL)], steps=steps, name=name,
                  ref=(0.5 * (rho_in + rho_out), 0.0, 0.0, 1.0))


def workload_channel_small() -> Config:
    """40x20 cells on 5H x H, 20^2 velocities on [-4,4]^2, Kn 0.1, 200 steps."""
    return channel_config(name="channel_40x20_v20")


def workload_mesh_sweep(nx: int) -> Config:
    """Mesh-size sweep: Kn 0.05, 28^2 velocities on [-4,4]^2, nx x nx/2 cells, 500 steps."""
    return channel_config(nx=nx, ny=nx // 2, n_vel=28, kn=0.05, steps=500,
                          name=f"channel_{nx}x{nx // 2}_v28")


MESH_SWEEP = (100, 200, 400, 800)


def workload_large_velocity(n_vel: int) -> Config:
    """Large velocity space: 200x100 cells, [-20,20]^2, Kn 0.01, rho_in 1.05, 200 steps."""
    return channel_config(nx=200, ny=100, n_vel=n_vel, vrange=20.0, kn=0.01, rho_in=1.05,
                          steps=200, name=f"channel_200x100_v{n_vel}_r20")


LARGE_VELOCITY = (51, 101, 151, 201)


def workload_batch(n_inst: int = 64, seed: int = None, steps: int = 1000):
    """Uneven batch: nx log-uniform in [50, 400] (ny = nx/2), N log-uniform integer in
    [16, 64] (N^2 velocities on [-4,4]^2), Kn log-uniform in [1e-3, 1], inlet rho uniform
    in [1.05, 1.5]."""
    seed = seed_for(4) if seed is None else seed
    r = uniform01(seed, 4 * n_inst).reshape(n_inst, 4)
    out = []
    for i in range(n_inst):
        nx = int(round(math.exp(math.log(50) + r[i, 0] * (math.log(400) - math.log(50)))))
        nx = max(50, min(400, nx))
        nvel = int(round(math.exp(math.log(16) + r[i, 1] * (math.log(64) - math.log(16)))))
        nvel = max(16, min(64, nvel))
        kn = math.exp(math.log(1e-3) + r[i, 2] * (math.log(1.0) - math.log(1e-3)))
        rin = 1.05 + r[i, 3] * 0.45
        out.append(channel_config(nx=nx, ny=max(1, nx // 2), n_vel=nvel, kn=kn, rho_in=rin,
                                  steps=steps, name=f"batch{i}"))
    return out


def poisson_arrivals(rate: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    u = uniform01(seed, n)
    return np.cumsum(-np.log(u) / rate)


def workload_serving(n_req: int = 24, seed: int = None, scale: str = "small", rate: float = 20.0):
    """Channel-solve requests drawn as in the uneven batch (log-uniform mesh, velocity grid
    and Kn, uniform inlet density) with Poisson arrival times.  scale="full" uses the batch
    ranges (meshes 50x25..400x200, 16^2..64^2 velocities); scale="small" shrinks meshes to
    nx in [20, 50] and velocity grids to [16, 32] per axis so that requests reach steady
    state in seconds.  Returns (configs, arrival times, initial primitive fields)."""
    seed = seed_for(5) if seed is None else seed
    r = uniform01(seed, 4 * n_req).reshape(n_req, 4)
    lo_x, hi_x, lo_v, hi_v = (50, 400, 16, 64) if scale == "full" else (20, 50, 16, 32)
    cfgs, prims = [], []
    for i in range(n_req):
        nx = int(round(math.exp(math.log(lo_x) + r[i, 0] * (math.log(hi_x) - math.log(lo_x)))))
        nvel = int(round(math.exp(math.log(lo_v) + r[i, 1] * (math.log(hi_v) - math.log(lo_v)))))
        kn = math.exp(math.log(1e-3) + r[i, 2] * (math.log(1.0) - math.log(1e-3)))
        rin = 1.05 + r[i, 3] * 0.45
        c = channel_config(nx=nx, ny=max(1, nx // 2), n_vel=nvel, kn=kn, rho_in=rin,
                           steps=20000, name=f"req{i}")
        cfgs.append(c)
        prims.append(initial_prim(c, seed + 1 + i))
    return cfgs, poisson_arrivals(rate, n_req, seed + 10_000), prims
