"""Velocity-space split of the FP32-f sums kernel (S1 + S7 of the Sec. 2.B flux table over
1, 2 or 4 warps per cell; the large-velocity-space regime of Sec. 3.B): every split matches
the FP64 oracle to the FP32-f form's one-step bounds, the splits agree with each other to
the FP32 rounding of the chunk sums, and the automatic choice splits small meshes with large
velocity grids only.
"""
import numpy as np
import pytest

from paper_1810_08137_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    from paper_1810_08137_gb300 import build, ugks
    build.build()
    return ugks


def rel_fields(W, Wr):
    return np.max(np.abs(W - Wr), axis=1) / np.maximum(np.max(np.abs(Wr), axis=1), 1e-300)


def rel_f(f, fr):
    return np.max(np.abs(f - fr)) / np.max(np.abs(fr))


def random_state(oracle, cfg, seed, amp=0.2, flow=0.3):
    r = I.uniform01(seed, 4 * cfg.nc).reshape(4, cfg.nc)
    f, W = oracle.init_maxwellian(cfg, 0.8 + 0.4 * r[0], flow * (2 * r[1] - 1),
                                  flow * (2 * r[2] - 1), 0.8 + 0.4 * r[3])
    return f * I.perturbation(seed + 1, f.shape, amp), W


def _periodic(**kw):
    base = dict(nx=6, ny=5, lx=1.0, ly=1.0, nu=37, nv=41, umin=-6.0, umax=6.0, vmin=-6.0,
                vmax=6.0, K=1, kn=0.05, bc=[I.BC(I.BC_PERIODIC)] * 4)
    base.update(kw)
    return I.Config(**base)


def _walls_pressure():
    cfg = I.channel_config(nx=7, ny=9, n_vel=33, kn=0.1)
    cfg.bc = [I.BC(I.BC_WALL, T=1.1), I.BC(I.BC_WALL, T=1.0, U=0.1),
              I.BC(I.BC_PRESSURE, 1.15, 1.05), I.BC(I.BC_PRESSURE, 0.95, 1.0)]
    return cfg


CASES = {
    # channel (pressure ends, diffuse walls) with a large velocity grid on a small mesh
    "channel_12x6_v41": lambda: I.channel_config(nx=12, ny=6, n_vel=41, vrange=8.0, kn=0.01),
    # odd grid (v = 0 row, H(0) = 1/2) and row counts that the split ranges divide unevenly
    "periodic_6x5_v37x41": lambda: _periodic(),
    # halves of different sizes, one of them shorter than a warp range at split 4
    "periodic_5x4_v35x45_asym": lambda: _periodic(nx=5, ny=4, nu=35, nv=45, vmin=-6.0, vmax=2.0),
    "walls_x_pressure_y_7x9_v33": _walls_pressure,
}


def _one_step(U, cfg, f, W, split):
    with U.Solver(cfg, U.FP32F) as s:
        s.set_sums_split(split)
        assert s.sums_split == split
        s.set_state(f, W)
        s.step(1)
        return s.get_state()


@pytest.mark.parametrize("name", list(CASES))
def test_split_one_step_against_oracle(U, oracle, name):
    cfg = CASES[name]()
    f, W = random_state(oracle, cfg, 211)
    fr, Wr = oracle.step(cfg, f, W, 1)
    res = {}
    for split in (1, 2, 4):
        fg, Wg = _one_step(U, cfg, f, W, split)
        ew, ef = rel_fields(Wg, Wr), rel_f(fg, fr)
        print(f"{name} split {split}: W {ew} f {ef:.2e}")
        assert np.all(ew <= 1e-6), (split, ew)
        assert ef <= 1e-5, (split, ef)
        res[split] = (fg, Wg)
    for split in (2, 4):
        d = rel_fields(res[split][1], res[1][1])
        assert np.all(d <= 1e-7), (split, d)


def test_split_multi_step_channel(U, oracle):
    """20 steps of a channel at Kn 0.01 with 41^2 velocities: split 4 against the oracle."""
    cfg = CASES["channel_12x6_v41"]()
    prim = I.initial_prim(cfg, I.seed_for(3, 41))
    f0, W0 = oracle.init_maxwellian(cfg, *prim)
    _, Wr = oracle.step(cfg, f0, W0, 20)
    with U.Solver(cfg, U.FP32F) as s:
        s.set_sums_split(4)
        s.init_maxwellian(*prim)
        s.step(20)
        W = s.moments()
    err = rel_fields(W, Wr)
    print(f"channel_12x6_v41 split 4, 20 steps: {err}")
    assert np.all(err <= 1e-5), err


def test_auto_split_choice(U):
    # small mesh, large velocity grid (64^2: 16 row pairs per half): split 4
    with U.Solver(I.channel_config(nx=12, ny=6, n_vel=64, vrange=8.0), U.FP32F) as s:
        assert s.sums_split == 4
        s.set_sums_split(1)
        assert s.sums_split == 1
        s.set_sums_split(0)
        assert s.sums_split == 4
    # 41^2 (10 row pairs below v = 0): two warps keep at least two chunks each
    with U.Solver(I.channel_config(nx=12, ny=6, n_vel=41, vrange=8.0), U.FP32F) as s:
        assert s.sums_split == 2
    # a mesh that fills the GPU alone: no split
    with U.Solver(I.workload_mesh_sweep(200), U.FP32F) as s:
        assert s.sums_split == 1
    # too few velocity rows per half to split (28^2: 7 row pairs per half)
    with U.Solver(I.channel_config(nx=12, ny=6, n_vel=28), U.FP32F) as s:
        assert s.sums_split == 1


def test_split_rejects_bad_values(U):
    cfg = I.channel_config(nx=6, ny=4, n_vel=8)
    with U.Solver(cfg, U.FP32F) as s:
        for bad in (3, 8, -1):
            with pytest.raises(U.UGKSError):
                s.set_sums_split(bad)
    with U.Solver(cfg, U.FP64) as s:
        with pytest.raises(U.UGKSError):
            s.set_sums_split(2)
        assert s.sums_split == 0
