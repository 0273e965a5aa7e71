"""GPU parity of the Shakhov model (Prandtl number != 1) against the oracle, through the C ABI.

The oracle's Shakhov step is pinned in tests/test_oracle_shakhov.py.  The FP64 form meets
the FP64 tolerance (1e-12 per field and on f after one step; 1e-11 after 50 steps of the
40x20 channel); the FP32-f form its one-step bounds (1e-6 per field, 1e-5 on f) and 1e-5
after 50 steps; a Shakhov instance steps bitwise the same alone and in a batch.
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


def periodic_cfg(**kw):
    base = dict(nx=4, ny=4, lx=1.0, ly=1.0, nu=5, nv=5, umin=-3.0, umax=3.0, vmin=-3.0,
                vmax=3.0, K=1, kn=0.05, bc=[I.BC(I.BC_PERIODIC)] * 4, pr=2.0 / 3.0)
    base.update(kw)
    return I.Config(**base)


def _channel(**kw):
    cfg = I.channel_config(**kw)
    cfg.pr = 2.0 / 3.0
    return cfg


def _walls_pressure():
    cfg = _channel(nx=7, ny=9, n_vel=9, kn=0.1)
    cfg.bc = [I.BC(I.BC_WALL, T=1.1), I.BC(I.BC_WALL, T=1.0, U=0.1),
              I.BC(I.BC_PRESSURE, 1.15, 1.05), I.BC(I.BC_PRESSURE, 0.95, 1.0)]
    return cfg


def _hotwall():
    cfg = _channel(nx=11, ny=6, n_vel=7, vrange=3.5, kn=0.05)
    cfg.bc[2] = I.BC(I.BC_WALL, T=1.3, U=0.2)
    cfg.bc[3] = I.BC(I.BC_WALL, T=0.9, U=-0.1)
    return cfg


CASES = {
    "periodic_4x4_v5x4": lambda: periodic_cfg(nu=5, nv=4),
    "periodic_13x7_v37": lambda: periodic_cfg(nx=13, ny=7, lx=1.3, ly=0.7, nu=37, nv=37, umin=-4,
                                              umax=4, vmin=-4, vmax=4, kn=0.02),
    "periodic_9x5_v33x6_K0_pr05": lambda: periodic_cfg(nx=9, ny=5, nu=33, nv=6, K=0, kn=0.5, pr=0.5),
    "periodic_6x6_v8_K2_pr072": lambda: periodic_cfg(nx=6, ny=6, nu=8, nv=8, K=2, kn=2.0, pr=0.72),
    "channel_11x6_v7_hotwall": _hotwall,
    "walls_x_pressure_y_7x9_v9": _walls_pressure,
    "channel_40x20_v20": lambda: _channel(),
}


def _one_step(U, cfg, f, W, prec):
    with U.Solver(cfg, prec) as s:
        s.set_state(f, W)
        s.step(1)
        return s.get_state()


@pytest.mark.parametrize("name", list(CASES))
def test_shakhov_one_step_fp64(U, oracle, name):
    cfg = CASES[name]()
    f, W = random_state(oracle, cfg, 401)
    fr, Wr = oracle.step(cfg, f, W, 1)
    f0, W0 = oracle.step(cfg.replace(pr=1.0), f, W, 1)
    assert rel_f(fr, f0) > 1e-6  # the Shakhov terms matter in this state
    fg, Wg = _one_step(U, cfg, f, W, U.FP64)
    ew, ef = rel_fields(Wg, Wr), rel_f(fg, fr)
    print(f"shakhov fp64 {name}: W {ew} f {ef:.2e}")
    assert np.all(ew <= 1e-12), ew
    assert ef <= 1e-12, ef


def test_shakhov_channel_50_steps_fp64(U, oracle):
    cfg = _channel(steps=50)
    prim = I.initial_prim(cfg, I.seed_for(1))
    f0, W0 = oracle.init_maxwellian(cfg, *prim)
    fr, Wr = oracle.step(cfg, f0, W0, 50)
    with U.Solver(cfg, U.FP64) as s:
        s.init_maxwellian(*prim)
        s.step(50)
        fg, Wg = s.get_state()
    ew = rel_fields(Wg, Wr)
    print(f"shakhov fp64 channel 50 steps: {ew}")
    assert np.all(ew <= 1e-11), ew
    assert rel_f(fg, fr) <= 1e-11


@pytest.mark.parametrize("name", list(CASES))
def test_shakhov_one_step_fp32f(U, oracle, name):
    cfg = CASES[name]()
    f, W = random_state(oracle, cfg, 403)
    fr, Wr = oracle.step(cfg, f, W, 1)
    fg, Wg = _one_step(U, cfg, f, W, U.FP32F)
    ew, ef = rel_fields(Wg, Wr), rel_f(fg, fr)
    print(f"shakhov fp32f {name}: W {ew} f {ef:.2e}")
    assert np.all(ew <= 1e-6), ew
    assert ef <= 1e-5, ef


def test_shakhov_channel_50_steps_fp32f(U, oracle):
    cfg = _channel(steps=50)
    prim = I.initial_prim(cfg, I.seed_for(1))
    f0, W0 = oracle.init_maxwellian(cfg, *prim)
    _, Wr = oracle.step(cfg, f0, W0, 50)
    with U.Solver(cfg, U.FP32F) as s:
        s.init_maxwellian(*prim)
        s.step(50)
        W = s.moments()
    ew = rel_fields(W, Wr)
    print(f"shakhov fp32f channel 50 steps: {ew}")
    assert np.all(ew <= 1e-5), ew


@pytest.mark.parametrize("persistent", [True, False], ids=["persistent", "phases"])
def test_shakhov_batch_alone_equals_mix(U, persistent):
    """A Shakhov instance steps bitwise the same alone and in a batch with BGK instances, in
    both step modes (one persistent launch; the phase launches)."""
    shk = _channel(nx=20, ny=10, n_vel=16, kn=0.05, name="shk")
    bgk = I.channel_config(nx=30, ny=15, n_vel=20, kn=0.1, name="bgk")
    prim_s = I.initial_prim(shk, I.seed_for(5, 1))
    prim_b = I.initial_prim(bgk, I.seed_for(5, 2))
    with U.Solver(shk, U.FP32F) as s:
        s.init_maxwellian(*prim_s)
        s.step(7)
        f_alone, W_alone = s.get_state()
    with U.Batch(4) as B:
        B.set_persistent(persistent)
        a = B.admit(bgk)
        b = B.admit(shk)
        B.instance(a).init_maxwellian(*prim_b)
        B.instance(b).init_maxwellian(*prim_s)
        B.step(7)
        B.sync()
        f_mix, W_mix = B.instance(b).get_state()
    np.testing.assert_array_equal(W_mix, W_alone)
    np.testing.assert_array_equal(f_mix, f_alone)


def test_shakhov_unsupported_paths_rejected(U):
    cfg = periodic_cfg()
    with pytest.raises(U.UGKSError):
        U.Solver(cfg, U.DF64)
    with U.Solver(cfg, U.FP32F) as s:
        assert s.sums_split == 1
        with pytest.raises(U.UGKSError):
            s.set_sums_split(2)
