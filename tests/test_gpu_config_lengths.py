"""GPU parity at each workload's own length and at its extremes (Sec. 3.A channel; the
mesh-size and velocity-grid sweeps of Sec. 3.B, Tables 1 and 3; the uneven batch).

* Mesh sweep (Kn 0.05, 28^2 velocities, 500 steps): the 100x50 mesh against the oracle
  itself at full length, both forms; 200x100, 400x200 and 800x400 FP32-f against the plain
  FP64 form, which matches the oracle to 1e-12 per step (one-step and sampled full-size
  tests) -- parity of long runs is transitive.
* Large velocity space (200x100 cells, [-20,20]^2, Kn 0.01, 200 steps): all four grids
  51^2 .. 201^2, FP32-f against FP64.
* Uneven batch extremes: instances at Kn 1e-3 and Kn 1 with 64^2 velocities, 1000 steps in
  one batch, FP32-f against the FP64 form, and the FP64 form's last step against the oracle
  on sampled cells.
Tolerances: FP64 per-field relative error 1e-12 per step (3e-11 after 500 steps, where
the per-step rounding differences compound); FP32-f 1e-5 per field after the full run.
The measured errors are printed (pytest -s) and recorded in the design notes.
"""
import os

import numpy as np
import pytest

from paper_1810_08137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("rho", "rho U", "rho V", "rho E")


@pytest.fixture(scope="module")
def U():
    from paper_1810_08137_gb300 import build, ugks
    build.build()
    return ugks


def rel_fields(W, Wr):
    return np.max(np.abs(W - Wr), axis=1) / np.maximum(np.max(np.abs(Wr), axis=1), 1e-300)


def _report(tag, err):
    print(f"{tag}: " + ", ".join(f"{n} {e:.2e}" for n, e in zip(FIELDS, err)))


def _run(U, cfg, prec, prim, steps):
    with U.Solver(cfg, prec) as s:
        s.init_maxwellian(*prim)
        s.step(steps)
        return s.moments()


def test_mesh_sweep_100x50_500_steps_against_oracle(U, oracle):
    cfg = I.workload_mesh_sweep(100)
    prim = I.initial_prim(cfg, I.seed_for(2, 100))
    threads = oracle.lib().orc_get_threads()
    oracle.set_threads(os.cpu_count() or 1)
    try:
        f0, W0 = oracle.init_maxwellian(cfg, *prim)
        _, Wr = oracle.step(cfg, f0, W0, cfg.steps)
    finally:
        oracle.set_threads(threads)
    e64 = rel_fields(_run(U, cfg, U.FP64, prim, cfg.steps), Wr)
    e32 = rel_fields(_run(U, cfg, U.FP32F, prim, cfg.steps), Wr)
    _report("100x50x28^2 500 steps FP64 vs oracle", e64)
    _report("100x50x28^2 500 steps FP32-f vs oracle", e32)
    assert np.all(e64 <= 3e-11), e64
    assert np.all(e32 <= 1e-5), e32


@pytest.mark.parametrize("nx", [200, 400, 800])
def test_mesh_sweep_500_steps_fp32f_vs_fp64(U, nx):
    cfg = I.workload_mesh_sweep(nx)
    prim = I.initial_prim(cfg, I.seed_for(2, nx))
    W64 = _run(U, cfg, U.FP64, prim, cfg.steps)
    W32 = _run(U, cfg, U.FP32F, prim, cfg.steps)
    err = rel_fields(W32, W64)
    _report(f"{nx}x{nx // 2}x28^2 500 steps FP32-f vs FP64", err)
    assert np.all(err <= 1e-5), err


@pytest.mark.parametrize("nvel", [51, 101, 151, 201])
def test_large_velocity_200_steps_fp32f_vs_fp64(U, nvel):
    cfg = I.workload_large_velocity(nvel)
    prim = I.initial_prim(cfg, I.seed_for(3, nvel))
    W64 = _run(U, cfg, U.FP64, prim, cfg.steps)
    W32 = _run(U, cfg, U.FP32F, prim, cfg.steps)
    err = rel_fields(W32, W64)
    _report(f"200x100x{nvel}^2 200 steps FP32-f vs FP64", err)
    assert np.all(err <= 1e-5), err


def _sample_ids(cfg, n_random, seed):
    nx, ny = cfg.nx, cfg.ny
    edge = [0, nx - 1, (ny - 1) * nx, ny * nx - 1, nx // 2, (ny // 2) * nx, (ny // 2) * nx + nx - 1]
    r = I.uniform01(seed, n_random)
    return sorted(set(edge + [int(x * (nx * ny)) for x in r]))


def test_batch_extremes_1000_steps(U, oracle):
    """The stiff and the rarefied end of the uneven batch (Kn 1e-3 and Kn 1, 64^2
    velocities on [-4,4]^2, 100x50 cells, inlet rho 1.5 and 1.05) stepped 1000 times in one
    batch: FP32-f W against the FP64 form after 1000 steps (<= 1e-5 per field), and the FP64
    form's step 1000 against the oracle from its step-999 state on sampled cells (1e-12)."""
    cfgs = [I.channel_config(nx=100, ny=50, n_vel=64, kn=1e-3, rho_in=1.5, steps=1000, name="stiff"),
            I.channel_config(nx=100, ny=50, n_vel=64, kn=1.0, rho_in=1.05, steps=1000, name="rarefied")]
    prims = [I.initial_prim(c, I.seed_for(4, 900 + k)) for k, c in enumerate(cfgs)]
    steps = 1000
    with U.Batch(4) as B:
        slots = [B.admit(c) for c in cfgs]
        for s, p in zip(slots, prims):
            B.instance(s).init_maxwellian(*p)
        B.step(steps)
        B.sync()
        W32 = [B.instance(s).moments() for s in slots]
    for cfg, prim, w32 in zip(cfgs, prims, W32):
        with U.Solver(cfg, U.FP64) as s:
            s.init_maxwellian(*prim)
            s.step(steps - 1)
            f, W = s.get_state()
            s.step(1)
            f1, W1 = s.get_state()
        err = rel_fields(w32, W1)
        _report(f"batch {cfg.name} (Kn {cfg.kn}) 1000 steps FP32-f vs FP64", err)
        assert np.all(err <= 1e-5), (cfg.name, err)
        ids = _sample_ids(cfg, 16, 91)
        fo, Wo = oracle.step_cells(cfg, f, W, ids)
        scale = np.max(np.abs(W1), axis=1)
        eo = np.max(np.abs(W1[:, ids].T - Wo), axis=0) / scale
        _report(f"batch {cfg.name} FP64 step 1000 vs oracle (sampled)", eo)
        assert np.all(eo <= 1e-12), (cfg.name, eo)
        assert np.max(np.abs(f1[ids] - fo)) <= 1e-12 * np.max(np.abs(fo))
