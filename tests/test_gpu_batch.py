"""Batched execution of independent instances (ugks_batch_*), FP32-f form.

Each instance's result must be bitwise the same alone (ugks_step on its own handle) and in
a mix of uneven instances stepped together, including instances admitted while others are
running; admission respects the HBM budget; the tile shape and the autotuner do not change
results.
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


def mix_configs():
    """Uneven instances: meshes, velocity grids (odd, even, > 32), Kn, inlet density."""
    a = I.channel_config(nx=20, ny=10, n_vel=16, kn=0.5, rho_in=1.3, name="a")
    b = I.channel_config(nx=37, ny=18, n_vel=33, kn=0.003, rho_in=1.1, name="b")
    c = I.channel_config(nx=9, ny=5, n_vel=21, kn=0.05, rho_in=1.45, name="c")
    c.bc[2] = I.BC(I.BC_WALL, T=1.2, U=0.1)
    d = I.Config(nx=12, ny=8, lx=1.0, ly=1.0, nu=24, nv=19, kn=0.02,
                 bc=[I.BC(I.BC_PERIODIC)] * 4, name="d")
    return [a, b, c, d]


def prim_of(cfg, k):
    return I.initial_prim(cfg, I.seed_for(4, k), amp=0.02)


def alone(U, cfg, prim, steps, rows=None):
    with U.Solver(cfg, U.FP32F) as s:
        s.init_maxwellian(*prim)
        s.step(steps)
        return s.get_state()


def test_batch_alone_vs_mix_bitwise(U):
    cfgs = mix_configs()
    prims = [prim_of(c, k) for k, c in enumerate(cfgs)]
    ref = [alone(U, c, p, 7) for c, p in zip(cfgs, prims)]
    with U.Batch(8) as B:
        slots = [B.admit(c) for c in cfgs]
        for s, p in zip(slots, prims):
            B.instance(s).init_maxwellian(*p)
        B.step(7)
        B.sync()
        for k, s in enumerate(slots):
            f, W = B.instance(s).get_state()
            assert np.array_equal(f, ref[k][0]), cfgs[k].name
            assert np.array_equal(W, ref[k][1]), cfgs[k].name


def test_batch_continuous_admission_and_retire(U):
    """Admission while others run: A runs 9 steps, B joins after 4 and runs 5, C takes the
    slot A leaves; each equals its own alone run with the same number of steps."""
    a, b, c, _ = mix_configs()
    pa, pb, pc = prim_of(a, 10), prim_of(b, 11), prim_of(c, 12)
    ra, rb, rc = alone(U, a, pa, 9), alone(U, b, pb, 5), alone(U, c, pc, 3)
    with U.Batch(2) as B:
        sa = B.admit(a)
        B.instance(sa).init_maxwellian(*pa)
        B.step(4)
        sb = B.admit(b)
        B.instance(sb).init_maxwellian(*pb)
        B.step(5)
        fa, Wa = B.instance(sa).get_state()
        B.retire(sa)
        sc = B.admit(c)
        B.instance(sc).init_maxwellian(*pc)
        B.step(3)
        fc, Wc = B.instance(sc).get_state()
        fb, Wb = B.instance(sb).get_state()
    rb8 = alone(U, b, pb, 8)
    assert np.array_equal(fa, ra[0]) and np.array_equal(Wa, ra[1])
    assert np.array_equal(fb, rb8[0]) and np.array_equal(Wb, rb8[1])
    assert np.array_equal(fc, rc[0]) and np.array_equal(Wc, rc[1])
    del rb


def test_batch_hbm_budget_admission(U):
    a, b, c, _ = mix_configs()
    need = [U.state_bytes(x, U.FP32F) for x in (a, b, c)]
    with U.Batch(8, hbm_budget=need[0] + need[1] + need[2] - 1) as B:
        s0 = B.admit(a)
        B.admit(b)
        with pytest.raises(U.UGKSError) as e:
            B.admit(c)
        assert e.value.status == 2
        assert B.bytes_used == need[0] + need[1]
        B.retire(s0)
        B.admit(c)
        assert B.bytes_used == need[1] + need[2]


def test_batch_tile_shape_and_tuner_do_not_change_results(U):
    cfgs = mix_configs()[:3]
    prims = [prim_of(c, 20 + k) for k, c in enumerate(cfgs)]
    with U.Batch(4) as B1, U.Batch(4) as B2:
        s1 = [B1.admit(c) for c in cfgs]
        s2 = [B2.admit(c) for c in cfgs]
        for x, y, p in zip(s1, s2, prims):
            B1.instance(x).init_maxwellian(*p)
            B2.instance(y).init_maxwellian(*p)
        for k, x in enumerate(s2):
            B2.set_walk_rows(x, 3)  # tiles of 3 rows: many tile seams
            B2.set_walk_vtile(x, 1 + k % 2)  # velocity tiles of 1 and 2 chunks
        B1.step(4)
        B2.step(4)
        ms = B1.tune(1)  # advances B1 by 12*(1+1) per velocity class present, plus 2*(1+1)
        assert ms > 0
        for x in s1:
            assert B1.walk_rows(x) in (16, 32, 64, 128)
            assert B1.walk_vtile(x) in (0, 1, 2)
        for x, y in zip(s1, s2):
            fa, Wa = B2.instance(y).get_state()
            fb, Wb = alone(U, cfgs[s2.index(y)], prims[s2.index(y)], 4)
            assert np.array_equal(fa, fb) and np.array_equal(Wa, Wb)


def test_batch_persistent_and_phase_launches_bitwise(U):
    """The persistent step (one cooperative launch, grid barriers between the phases) and
    the seven phase launches run the same phase code in the same order of work: bitwise
    equal results, and equal to each instance stepped alone."""
    cfgs = mix_configs()
    prims = [prim_of(c, 40 + k) for k, c in enumerate(cfgs)]
    out = []
    for persistent in (True, False):
        with U.Batch(8) as B:
            assert B.persistent  # the default where cooperative launch is available
            B.set_persistent(persistent)
            slots = [B.admit(c) for c in cfgs]
            for s, p in zip(slots, prims):
                B.instance(s).init_maxwellian(*p)
            B.step(5)
            B.sync()
            out.append([B.instance(s).get_state() for s in slots])
    for k in range(len(cfgs)):
        ref = alone(U, cfgs[k], prims[k], 5)
        for mode in (0, 1):
            assert np.array_equal(out[mode][k][0], ref[0]), (cfgs[k].name, mode)
            assert np.array_equal(out[mode][k][1], ref[1]), (cfgs[k].name, mode)


def test_batch_persistent_barrier_timeout_is_reported(U):
    """A grid barrier of the persistent step whose wait bound runs out (bound 0: every block
    that is not the last to arrive gives up at once) ends the launch without trapping the
    device; ugks_batch_sync reports UGKS_ETIMEOUT, and with the bound restored and the
    state set again the batch steps correctly (the context stays usable)."""
    a, b, c, _ = mix_configs()
    pa, pb = prim_of(a, 50), prim_of(b, 51)
    ra = alone(U, a, pa, 3)
    with U.Batch(4) as B:
        sa, sb = B.admit(a), B.admit(b)
        B.instance(sa).init_maxwellian(*pa)
        B.instance(sb).init_maxwellian(*pb)
        B.set_wait_limit(0)
        B.step(3)  # 18 barriers: a block reaching one before the last block arrives gives up
        with pytest.raises(U.UGKSError) as e:
            B.sync()
        assert e.value.status == 4  # UGKS_ETIMEOUT
        B.sync()  # the flag was cleared
        B.set_wait_limit(8_000_000)
        B.instance(sa).init_maxwellian(*pa)
        B.instance(sb).init_maxwellian(*pb)
        # the parity of each instance is wherever the interrupted step left it; a state set
        # again and stepped from there must match the alone run
        B.step(3)
        B.sync()
        fa, Wa = B.instance(sa).get_state()
    assert np.array_equal(fa, ra[0]) and np.array_equal(Wa, ra[1])
