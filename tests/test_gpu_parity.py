"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 path <= 1e-12 relative per macroscopic field per step (field-relative:
max|x - x_ref| / max|x_ref| per component of W); f to the same bound relative to max|f|.
FP32-f form: <= 1e-5 relative per field after 200 steps.
"""
import numpy as np
import pytest

from paper_1810_08137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def U():
    from paper_1810_08137_gb300 import build, ugks
    build.build()
    return ugks


def rel_fields(W, Wr):
    return np.max(np.abs(W - Wr), axis=1) / np.maximum(np.max(np.abs(Wr), axis=1), 1e-300)


def rel_f(f, fr):
    return np.max(np.abs(f - fr)) / np.max(np.abs(fr))


def periodic_cfg(**kw):
    base = dict(nx=4, ny=4, lx=1.0, ly=1.0, nu=5, nv=5, umin=-3.0, umax=3.0, vmin=-3.0,
                vmax=3.0, K=1, kn=0.05, bc=[I.BC(I.BC_PERIODIC)] * 4)
    base.update(kw)
    return I.Config(**base)


def random_state(oracle, cfg, seed, amp=0.2, flow=0.3):
    r = I.uniform01(seed, 4 * cfg.nc).reshape(4, cfg.nc)
    rho = 0.8 + 0.4 * r[0]
    Uf = flow * (2 * r[1] - 1)
    Vf = flow * (2 * r[2] - 1)
    T = 0.8 + 0.4 * r[3]
    f, W = oracle.init_maxwellian(cfg, rho, Uf, Vf, T)
    return f * I.perturbation(seed + 1, f.shape, amp), W


def one_step(U, cfg, f, W, prec=0, n=1):
    with U.Solver(cfg, prec) as s:
        s.set_state(f, W)
        s.step(n)
        return s.get_state()


CASES = {
    "periodic_4x4_v5x4": lambda: periodic_cfg(nu=5, nv=4),
    "periodic_13x7_v37": lambda: periodic_cfg(nx=13, ny=7, lx=1.3, ly=0.7, nu=37, nv=37, umin=-4,
                                              umax=4, vmin=-4, vmax=4, kn=0.02),
    "periodic_9x5_v33x6_K0": lambda: periodic_cfg(nx=9, ny=5, nu=33, nv=6, K=0, kn=0.5),
    "periodic_6x6_v8_K2": lambda: periodic_cfg(nx=6, ny=6, nu=8, nv=8, K=2, kn=2.0),
    "channel_11x6_v7_hotwall": lambda: _hotwall(),
    "walls_x_pressure_y_7x9_v9": lambda: _rotated(),
    "channel_1x3_v6": lambda: I.channel_config(nx=1, ny=3, n_vel=6),
    "channel_5x1_v9": lambda: I.channel_config(nx=5, ny=1, n_vel=9),
    "channel_40x20_v20": lambda: I.workload_channel_small(),
    # degenerate velocity grids of the FP32-f paired-row layout (each half of the v axis
    # padded to an even number of rows): a single v = 0 row, all v < 0, all v > 0, and an
    # asymmetric grid whose halves differ in size, with nu > 32
    "periodic_5x4_v6x1": lambda: periodic_cfg(nx=5, ny=4, nu=6, nv=1, vmin=0.0, vmax=0.0),
    "periodic_5x4_v5x7_vneg": lambda: periodic_cfg(nx=5, ny=4, nu=5, nv=7, vmin=-3.0, vmax=-0.5),
    "periodic_5x4_v5x6_vpos": lambda: periodic_cfg(nx=5, ny=4, nu=5, nv=6, vmin=0.5, vmax=3.0),
    "periodic_6x5_v35x8_asym": lambda: periodic_cfg(nx=6, ny=5, nu=35, nv=8, vmin=-3.0, vmax=1.5,
                                                    kn=0.1),
    # asymmetric grid with a v = 0 node away from the centre of the range (-2 + 5 * 0.4):
    # the host builds the grid without floating-point contraction, so the node is exactly 0
    # (H(0) = 1/2) on every host architecture, as in the oracle
    "periodic_5x4_v9x21_asym0": lambda: periodic_cfg(nx=5, ny=4, nu=9, nv=21, vmin=-6.0, vmax=2.0,
                                                     umin=-4.0, umax=4.0),
    # general viscosity laws (R3): variable hard sphere with omega = 0.81 and variable soft
    # sphere with omega = 0.75, alpha = 1.4 (tau through T^omega instead of the hard-sphere
    # shortcut), the latter in a channel at small Kn (dt/tau above 0.1 in many faces)
    "periodic_7x5_v9_vhs": lambda: periodic_cfg(nx=7, ny=5, nu=9, nv=9, kn=0.05, omega=0.81),
    "channel_9x6_v11_vss": lambda: _vss(),
}


def _vss():
    cfg = I.channel_config(nx=9, ny=6, n_vel=11, kn=0.01)
    cfg.omega, cfg.alpha = 0.75, 1.4
    return cfg


def _hotwall():
    cfg = I.channel_config(nx=11, ny=6, n_vel=7, vrange=3.5, kn=0.05)
    cfg.bc[2] = I.BC(I.BC_WALL, T=1.3, U=0.2)
    cfg.bc[3] = I.BC(I.BC_WALL, T=0.9, U=-0.1)
    return cfg


def _rotated():
    cfg = I.channel_config(nx=7, ny=9, n_vel=9, kn=0.1)
    cfg.bc = [I.BC(I.BC_WALL, T=1.1), I.BC(I.BC_WALL, T=1.0, U=0.1),
              I.BC(I.BC_PRESSURE, 1.15, 1.05), I.BC(I.BC_PRESSURE, 0.95, 1.0)]
    return cfg


@pytest.mark.parametrize("name", list(CASES))
def test_one_step_fp64_parity(U, oracle, name):
    cfg = CASES[name]()
    f, W = random_state(oracle, cfg, 101)
    fr, Wr = oracle.step(cfg, f, W, 1)
    fg, Wg = one_step(U, cfg, f, W)
    assert np.all(rel_fields(Wg, Wr) <= FP64_TOL), rel_fields(Wg, Wr)
    assert rel_f(fg, fr) <= FP64_TOL, rel_f(fg, fr)


@pytest.mark.parametrize("name", list(CASES))
def test_one_step_df64_parity(U, oracle, name):
    """DF64 form (double-FP32 f and per-velocity arithmetic): the FP64 tolerance."""
    cfg = CASES[name]()
    f, W = random_state(oracle, cfg, 101)
    fr, Wr = oracle.step(cfg, f, W, 1)
    fg, Wg = one_step(U, cfg, f, W, prec=U.DF64)
    print(f"df64 {name}: W {rel_fields(Wg, Wr)} f {rel_f(fg, fr):.2e}")
    assert np.all(rel_fields(Wg, Wr) <= FP64_TOL), rel_fields(Wg, Wr)
    assert rel_f(fg, fr) <= FP64_TOL, rel_f(fg, fr)


@pytest.mark.parametrize("name", list(CASES))
def test_one_step_fp32f_parity(U, oracle, name):
    """FP32-f form, one step from a non-equilibrium state, every edge-case configuration:
    per-field error <= 1e-6 relative, f <= 1e-5 relative to max|f|."""
    cfg = CASES[name]()
    f, W = random_state(oracle, cfg, 103)
    fr, Wr = oracle.step(cfg, f, W, 1)
    fg, Wg = one_step(U, cfg, f, W, prec=U.FP32F)
    ew, ef = rel_fields(Wg, Wr), rel_f(fg, fr)
    print(f"fp32f {name}: W {ew} f {ef:.2e}")
    assert np.all(ew <= 1e-6), ew
    assert ef <= 1e-5, ef


def test_init_maxwellian_parity(U, oracle):
    cfg = I.workload_channel_small()
    rho, Uf, Vf, T = I.initial_prim(cfg, I.seed_for(1))
    fr, Wr = oracle.init_maxwellian(cfg, rho, Uf, Vf, T)
    with U.Solver(cfg) as s:
        s.init_maxwellian(rho, Uf, Vf, T)
        fg, Wg = s.get_state()
    assert np.all(rel_fields(Wg, Wr) <= 1e-15)
    assert rel_f(fg, fr) <= 1e-15


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "df64"])
def test_channel_config1_200_steps_fp64(U, oracle, prec):
    """Channel 40x20 cells, 20^2 velocities, Kn 0.1, 200 steps from the seeded
    Maxwellian: per-step parity compounds over 200 steps; require 1e-11."""
    cfg = I.workload_channel_small()
    rho, Uf, Vf, T = I.initial_prim(cfg, I.seed_for(1))
    f0, W0 = oracle.init_maxwellian(cfg, rho, Uf, Vf, T)
    fr, Wr = oracle.step(cfg, f0, W0, cfg.steps)
    with U.Solver(cfg, prec) as s:
        s.init_maxwellian(rho, Uf, Vf, T)
        s.step(cfg.steps)
        fg, Wg = s.get_state()
    assert np.all(rel_fields(Wg, Wr) <= 1e-11), rel_fields(Wg, Wr)
    assert rel_f(fg, fr) <= 1e-11


def test_fp32f_form_200_steps(U, oracle):
    """FP32 storage of f, FP64 moments/W/face scalars: per-field error after 200 steps of
    the 40x20 channel against the FP64 oracle."""
    cfg = I.workload_channel_small()
    rho, Uf, Vf, T = I.initial_prim(cfg, I.seed_for(1))
    f0, W0 = oracle.init_maxwellian(cfg, rho, Uf, Vf, T)
    fr, Wr = oracle.step(cfg, f0, W0, cfg.steps)
    with U.Solver(cfg, U.FP32F) as s:
        s.init_maxwellian(rho, Uf, Vf, T)
        s.step(cfg.steps)
        W, prim = s.moments(prim=True)
    err = rel_fields(W, Wr)
    print(f"fp32f 200 steps: per-field error {err}")
    assert np.all(err <= FP32_TOL), err


def test_fp32f_one_step_random_state(U, oracle):
    cfg = CASES["periodic_13x7_v37"]()
    f, W = random_state(oracle, cfg, 102)
    fr, Wr = oracle.step(cfg, f, W, 1)
    fg, Wg = one_step(U, cfg, f, W, prec=U.FP32F)
    assert np.all(rel_fields(Wg, Wr) <= 1e-6), rel_fields(Wg, Wr)
    assert rel_f(fg, fr) <= 1e-5


def test_collisionless_exact_shift_gpu(U, oracle):
    nx = ny = 8
    cfg = periodic_cfg(nx=nx, ny=ny, nu=3, nv=3, umin=-1, umax=1, vmin=-1, vmax=1, kn=1e250,
                       dt=0.125, lx=1.0, ly=1.0)
    f, W = random_state(oracle, cfg, 5, amp=0.5)
    fg, _ = one_step(U, cfg, f, W)
    F = f.reshape(ny, nx, 3, 3, 2)
    G = fg.reshape(ny, nx, 3, 3, 2)
    tol = 1e-14 * np.max(np.abs(f))
    assert np.max(np.abs(G[:, :, 1, 2] - np.roll(F[:, :, 1, 2], 1, axis=1))) < tol
    assert np.max(np.abs(G[:, :, 1, 0] - np.roll(F[:, :, 1, 0], -1, axis=1))) < tol
    assert np.max(np.abs(G[:, :, 2, 1] - np.roll(F[:, :, 2, 1], 1, axis=0))) < tol
    assert np.max(np.abs(G[:, :, 0, 1] - np.roll(F[:, :, 0, 1], -1, axis=0))) < tol
    assert np.max(np.abs(G[:, :, 1, 1] - F[:, :, 1, 1])) < tol


def test_periodic_conservation_gpu(U, oracle):
    cfg = periodic_cfg(nx=16, ny=12, nu=12, nv=12, umin=-5, umax=5, vmin=-5, vmax=5, kn=0.02)
    f, W = random_state(oracle, cfg, 33)
    for prec in (U.FP64, U.FP32F, U.DF64):
        with U.Solver(cfg, prec) as s:
            s.set_state(f, W)
            s.step(10)
            W1 = s.moments()
        assert np.max(np.abs(W1.sum(axis=1) - W.sum(axis=1))) <= 1e-13 * cfg.nc * np.max(np.abs(W))


def test_checkpoint_resume_bitwise(U, oracle):
    cfg = CASES["channel_11x6_v7_hotwall"]()
    f, W = random_state(oracle, cfg, 7)
    with U.Solver(cfg) as s:
        s.set_state(f, W)
        s.step(5)
        fc, Wc = s.get_state()
        s.step(5)
        fa, Wa = s.get_state()
    with U.Solver(cfg) as s:
        s.set_state(fc, Wc)
        s.step(5)
        fb, Wb = s.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(Wa, Wb)


def test_residual_matches_definition(U, oracle):
    cfg = I.workload_channel_small()
    rho, Uf, Vf, T = I.initial_prim(cfg, I.seed_for(1))
    with U.Solver(cfg) as s:
        s.init_maxwellian(rho, Uf, Vf, T)
        assert np.all(s.residual() == 0)
        s.step(3)
        W0 = s.moments()
        s.step(1)
        W1 = s.moments()
        res = s.residual()
    ref = np.sqrt(np.mean((W1 - W0) ** 2, axis=1)) / np.max(np.abs(W1), axis=1)
    assert np.allclose(res, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("name", ["periodic_13x7_v37", "channel_40x20_v20", "periodic_5x4_v6x1"])
def test_state_bytes_predicts_allocation(U, name):
    """ugks_state_bytes (used for admission against an HBM budget) equals the device bytes
    ugks_create allocates, in every form."""
    cfg = CASES[name]()
    for prec in (U.FP64, U.FP32F, U.DF64):
        with U.Solver(cfg, prec) as s:
            assert s.device_bytes == U.state_bytes(cfg, prec), (prec, s.device_bytes)


def test_device_state_roundtrip(U, oracle):
    torch = pytest.importorskip("torch")
    cfg = CASES["periodic_13x7_v37"]()
    f, W = random_state(oracle, cfg, 9)
    fr, Wr = oracle.step(cfg, f, W, 1)
    fd = torch.tensor(f, device="cuda")
    Wd = torch.tensor(W, device="cuda")
    with U.Solver(cfg) as s:
        s.set_state_device(fd, Wd)
        s.step(1)
        fo = torch.empty_like(fd)
        Wo = torch.empty_like(Wd)
        s.get_state_device(fo, Wo)
        s.sync()
    assert np.all(rel_fields(Wo.cpu().numpy(), Wr) <= FP64_TOL)
    assert rel_f(fo.cpu().numpy(), fr) <= FP64_TOL


@pytest.mark.parametrize("name", ["periodic_13x7_v37", "channel_9x5_v21"])
def test_fp32f_state_through_pinned_host_buffers(U, oracle, name):
    """FP32-f form: set_state / get_state with page-locked host buffers (converted in place
    by the kernels) give bitwise the state of the staged path for pageable buffers.  The
    9x5 mesh with 21^2 velocities has staging halves that are not a multiple of 16 bytes
    before rounding."""
    import ctypes
    torch = pytest.importorskip("torch")
    cfg = (CASES[name]() if name in CASES else
           I.channel_config(nx=9, ny=5, n_vel=21, kn=0.05, rho_in=1.45))
    f, W = random_state(oracle, cfg, 11)
    with U.Solver(cfg, U.FP32F) as s:
        s.set_state(f, W)
        s.step(2)
        fa, Wa = s.get_state()
    pin_in = torch.empty(f.shape, dtype=torch.float64, pin_memory=True)
    pin_in.numpy()[:] = f
    pin_out = torch.empty(f.shape, dtype=torch.float64, pin_memory=True)
    Wb = np.empty_like(W)
    P = ctypes.POINTER(ctypes.c_double)
    with U.Solver(cfg, U.FP32F) as s:
        s.set_state(pin_in.numpy(), W)
        s.step(2)
        s._check(s._L.ugks_get_state(s._h, pin_out.numpy().ctypes.data_as(P), Wb.ctypes.data_as(P)))
    assert np.array_equal(pin_out.numpy(), fa)
    assert np.array_equal(Wb, Wa)


def test_numeric_failure_is_reported(U, oracle):
    """A state with negative density is caught by the cell kernel's check and surfaces as
    UGKS_ENUMERIC at the next synchronising call (no device trap)."""
    cfg = periodic_cfg(nx=4, ny=4, nu=6, nv=6)
    f, W = random_state(oracle, cfg, 3)
    W = W.copy()
    W[0, 5] = -1.0
    with U.Solver(cfg) as s:
        s.set_state(f, W)
        s.step(1)
        with pytest.raises(U.UGKSError) as e:
            s.sync()
        assert e.value.status == 5


def _sample_ids(cfg, n_random, seed):
    nx, ny = cfg.nx, cfg.ny
    edge = [0, nx - 1, (ny - 1) * nx, ny * nx - 1, nx // 2, (ny // 2) * nx, (ny // 2) * nx + nx - 1,
            (ny - 1) * nx + nx // 3, nx + 1, 2 * nx + 2]
    r = I.uniform01(seed, n_random)
    return sorted(set(edge + [int(x * (nx * ny)) for x in r]))


@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, 1e-5), (2, FP64_TOL)])
def test_full_size_800x400_sampled(U, oracle, prec, tol):
    """Mesh-sweep workload at full size (800x400 cells, 28^2 velocities), in the launch
    configuration the bench times: 20 steps from the seeded Maxwellian, then one more step
    checked on sampled cells against the oracle run on the same state."""
    cfg = I.workload_mesh_sweep(800)
    rho, Uf, Vf, T = I.initial_prim(cfg, I.seed_for(2, 800))
    ids = _sample_ids(cfg, 24, 55)
    with U.Solver(cfg, prec) as s:
        s.init_maxwellian(rho, Uf, Vf, T)
        s.step(20)
        f, W = s.get_state()
        s.step(1)
        f1, W1 = s.get_state()
    fo, Wo = oracle.step_cells(cfg, f, W, ids)
    Wg = W1[:, ids].T
    scale = np.max(np.abs(W1), axis=1)
    err = np.max(np.abs(Wg - Wo), axis=0) / scale
    assert np.all(err <= tol), err
    assert np.max(np.abs(f1[ids] - fo)) / np.max(np.abs(fo)) <= max(tol, 1e-12) * 10


@pytest.mark.parametrize("nvel", [101, 201])
@pytest.mark.parametrize("prec,tol", [(0, FP64_TOL), (1, 1e-5), (2, FP64_TOL)])
def test_large_velocity_full_mesh_sampled(U, oracle, nvel, prec, tol):
    """Large-velocity workload at full size (200x100 cells, nvel^2 velocities on
    [-20,20]^2, Kn 0.01), in the launch configuration the bench times: 5 steps from the
    seeded Maxwellian, then one more step checked on sampled cells against the oracle run on
    the same state."""
    cfg = I.workload_large_velocity(nvel)
    rho, Uf, Vf, T = I.initial_prim(cfg, I.seed_for(3, nvel))
    ids = _sample_ids(cfg, 12, 77)
    with U.Solver(cfg, prec) as s:
        s.init_maxwellian(rho, Uf, Vf, T)
        s.step(5)
        f, W = s.get_state()
        s.step(1)
        f1, W1 = s.get_state()
    fo, Wo = oracle.step_cells(cfg, f, W, ids)
    del f
    Wg = W1[:, ids].T
    scale = np.max(np.abs(W1), axis=1)
    err = np.max(np.abs(Wg - Wo), axis=0) / scale
    assert np.all(err <= tol), err
    assert np.max(np.abs(f1[ids] - fo)) / np.max(np.abs(fo)) <= max(tol, 1e-12) * 10


@pytest.mark.parametrize("name,steps", [("mesh_800x400_v28", 200), ("large_velocity_v101", 50),
                                        ("large_velocity_v201", 50)])
def test_fp32f_against_fp64_long_runs(U, name, steps):
    """Transitive parity of long runs at full size: the FP32-f form against the plain FP64
    form (whose every step matches the oracle to 1e-12, see the sampled full-size tests)
    from the same seeded Maxwellian, per-field error of W <= 1e-5 relative."""
    if name.startswith("mesh"):
        cfg = I.workload_mesh_sweep(800)
        prim = I.initial_prim(cfg, I.seed_for(2, 800))
    else:
        n = int(name.rsplit("_v", 1)[1])
        cfg = I.workload_large_velocity(n)
        prim = I.initial_prim(cfg, I.seed_for(3, n))
    Ws = []
    for prec in (U.FP64, U.FP32F):
        with U.Solver(cfg, prec) as s:
            s.init_maxwellian(*prim)
            s.step(steps)
            Ws.append(s.moments())
    err = rel_fields(Ws[1], Ws[0])
    print(f"{name} {steps} steps: FP32-f vs FP64 {err}")
    assert np.all(err <= 1e-5), err


def test_graph_replay_matches_direct_launches(U, oracle):
    """ugks_step replays captured graphs; with tracing on it launches the kernels directly.
    Both orders of work are the same, so the results must be bitwise identical."""
    cfg = CASES["channel_11x6_v7_hotwall"]()
    f, W = random_state(oracle, cfg, 77)
    out = []
    for prof in (False, True):
        for prec in (U.FP64, U.FP32F, U.DF64):
            with U.Solver(cfg, prec) as s:
                s.set_state(f, W)
                if prof:
                    s.profile(True)
                s.step(3)
                out.append(s.get_state())
    for a, b in ((0, 3), (1, 4), (2, 5)):
        assert np.array_equal(out[a][0], out[b][0]) and np.array_equal(out[a][1], out[b][1])


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, FP32_TOL)])
def test_large_velocity_space(U, oracle, prec, tol):
    """Velocity domain [-20,20]^2 (thermal speed small against the range, the paper's
    particle-like regime), 51^2 velocities (two u chunks of 32), Kn 0.01, inlet rho 1.05:
    200 steps from the seeded Maxwellian on a 12x6 channel, the stated tolerances."""
    cfg = I.workload_large_velocity(51).replace(nx=12, ny=6)
    rho, Uf, Vf, T = I.initial_prim(cfg, I.seed_for(3, 51))
    f0, W0 = oracle.init_maxwellian(cfg, rho, Uf, Vf, T)
    fr, Wr = oracle.step(cfg, f0, W0, 200)
    with U.Solver(cfg, prec) as s:
        s.init_maxwellian(rho, Uf, Vf, T)
        s.step(200)
        fg, Wg = s.get_state()
    err = rel_fields(Wg, Wr)
    print(f"large velocity space prec {prec}: {err}")
    assert np.all(err <= tol), err
    assert rel_f(fg, fr) <= 10 * tol


def test_fp32f_walk_wait_timeout_is_reported(U, oracle):
    """The FP32-f update walk waits (bounded) for the bulk copies of its face and cell
    records.  With the bound set to zero polls the wait runs out at once: the walk drains its
    copies in flight, records the failure and returns, and the next synchronising call reports
    UGKS_ETIMEOUT without trapping the device.  A new state clears it, and with the default
    bound the instance steps exactly as a fresh one."""
    cfg = CASES["channel_11x6_v7_hotwall"]()
    f, W = random_state(oracle, cfg, 61)
    with U.Solver(cfg, U.FP32F) as s:
        s.set_state(f, W)
        s.set_wait_limit(0)
        s.step(1)
        with pytest.raises(U.UGKSError) as e:
            s.sync()
        assert e.value.status == 4  # UGKS_ETIMEOUT
        s.set_wait_limit(1 << 22)
        s.set_state(f, W)
        s.step(2)
        fa, Wa = s.get_state()
    fb, Wb = one_step(U, cfg, f, W, prec=U.FP32F, n=2)
    assert np.array_equal(fa, fb) and np.array_equal(Wa, Wb)
