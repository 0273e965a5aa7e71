"""The seeded input generator: SplitMix64 as published (its first outputs for seed 0 and for
seed 1234567, the values quoted with the reference implementation), uniform doubles in
(0, 1], Box-Muller normals, and the channel initial state."""
import numpy as np

from paper_1810_08137_gb300 import inputs as I


def test_splitmix64_published_outputs():
    assert [int(x) for x in I.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x) for x in I.splitmix64(1234567, 3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_splitmix64_stream_offsets():
    z = I.splitmix64(42, 10)
    assert np.array_equal(I.splitmix64(42, 4, start=6), z[6:])


def test_uniform_and_normal_statistics():
    u = I.uniform01(7, 200000)
    assert u.min() > 0.0 and u.max() <= 1.0
    assert abs(u.mean() - 0.5) < 3e-3
    n = I.normal(8, 200000)
    assert abs(n.mean()) < 1e-2 and abs(n.std() - 1.0) < 1e-2


def test_channel_initial_state_recipe():
    cfg = I.workload_channel_small()
    rho, U, V, T = I.initial_prim(cfg, I.seed_for(1))
    assert rho.shape == (cfg.nc,)
    assert np.all(U == 0) and np.all(V == 0) and np.all(T == 1)
    assert abs(rho.mean() - 1.0) < 1e-3 and 5e-4 < rho.std() < 2e-3
    # the same seed gives the same state; another seed another one
    assert np.array_equal(rho, I.initial_prim(cfg, I.seed_for(1))[0])
    assert not np.array_equal(rho, I.initial_prim(cfg, I.seed_for(2))[0])
