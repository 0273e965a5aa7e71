"""The allocation-free step entry point (ugks_step_noalloc) against the regular one.

Some callers cannot allocate device memory (a host framework that owns every device
allocation, or code where an allocation could block or fail at a bad time); they call
ugks_step_noalloc, which keeps its intermediates in a fixed array inside the library.
Two calls in a row must agree with ugks_create/ugks_set_state_device/ugks_step/
ugks_get_state_device within the FP64 tolerance of the parity tests (1e-12 per field), and
after both calls with two steps of the oracle.
This file sorts last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from paper_1810_08137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _state(cfg, seed):
    """Non-equilibrium FP64 state built here from seeded numbers (no oracle involved)."""
    r = I.uniform01(seed, 4 * cfg.nc).reshape(4, cfg.nc)
    rho, U, V, T = 0.8 + 0.4 * r[0], 0.3 * (2 * r[1] - 1), 0.3 * (2 * r[2] - 1), 0.8 + 0.4 * r[3]
    u = np.linspace(cfg.umin, cfg.umax, cfg.nu)
    v = np.linspace(cfg.vmin, cfg.vmax, cfg.nv)
    uq, vq = np.tile(u, cfg.nv), np.repeat(v, cfg.nu)
    lam = 1.0 / T
    gh = (rho * lam / np.pi)[:, None] * np.exp(
        -lam[:, None] * ((uq[None, :] - U[:, None]) ** 2 + (vq[None, :] - V[:, None]) ** 2))
    f = np.stack([gh, cfg.K / (2 * lam)[:, None] * gh], axis=2)
    f = f * I.perturbation(seed + 1, f.shape, 0.2)
    W = np.stack([rho, rho * U, rho * V, rho * (0.5 * (U * U + V * V) + (cfg.K + 2) * T / 4)])
    return f, W


def _rel(a, b):
    return np.max(np.abs(a - b), axis=-1) / np.max(np.abs(b), axis=-1)


def _case(name):
    if name == "channel_13x7_v11":  # pressure ends, one hot moving wall
        cfg = I.channel_config(nx=13, ny=7, n_vel=11, kn=0.05)
        cfg.bc[2] = I.BC(I.BC_WALL, T=1.1, U=0.05)
        return cfg
    # periodic both ways (its own ghost fill), an even grid without v = 0
    return I.Config(nx=8, ny=6, lx=1.0, ly=0.75, nu=10, nv=10, kn=0.02,
                    bc=[I.BC(I.BC_PERIODIC)] * 4)


@pytest.mark.parametrize("case", ["channel_13x7_v11", "periodic_8x6_v10"])
@pytest.mark.parametrize("side_stream", [False, True], ids=["default_stream", "side_stream"])
def test_noalloc_matches_regular_entry_point_twice(oracle, case, side_stream):
    torch = pytest.importorskip("torch")
    from paper_1810_08137_gb300 import build, ugks
    build.build()
    cfg = _case(case)
    f, W = _state(cfg, 2024)
    # the step it must take, from the oracle (the regular entry point is held to the same)
    f_ref, W_ref = oracle.step(cfg, f, W, 2)
    f_in = torch.tensor(f, device="cuda")
    W_in = torch.tensor(W, device="cuda")
    f_a, W_a = torch.empty_like(f_in), torch.empty_like(W_in)
    f_b, W_b = torch.empty_like(f_in), torch.empty_like(W_in)
    # the allocation-free call on the caller's stream (a side stream, or the legacy one)
    stream = torch.cuda.Stream() if side_stream else None
    handle = stream.cuda_stream if stream is not None else None
    torch.cuda.synchronize()
    with ugks.Solver(cfg) as s:
        s.set_state_device(f_in, W_in)
        for call in range(2):
            ugks.step_noalloc(cfg, f_in, W_in, f_a, W_a, stream=handle)
            s.step(1)
            s.get_state_device(f_b, W_b)
            s.sync()
            torch.cuda.synchronize()
            Wa, Wb = W_a.cpu().numpy(), W_b.cpu().numpy()
            fa, fb = f_a.cpu().numpy(), f_b.cpu().numpy()
            assert np.all(_rel(Wa, Wb) <= TOL), (call, _rel(Wa, Wb))
            assert np.max(np.abs(fa - fb)) <= TOL * np.max(np.abs(fb)), call
            assert not np.allclose(Wa, W_in.cpu().numpy())  # the state advanced
            f_in, W_in = f_a.clone(), W_a.clone()  # next call continues from this state
        # after both calls: the oracle's two steps, to the same tolerance
        assert np.all(_rel(Wa, W_ref) <= TOL), _rel(Wa, W_ref)
        assert np.max(np.abs(fa - f_ref)) <= TOL * np.max(np.abs(f_ref))


def test_noalloc_rejects_oversize_problem():
    torch = pytest.importorskip("torch")
    from paper_1810_08137_gb300 import build, ugks
    build.build()
    cfg = I.workload_mesh_sweep(400)  # 400x200 cells x 28^2: far beyond the fixed scratch
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ugks.UGKSError) as e:
        ugks.step_noalloc(cfg, x, x, x, x)
    assert e.value.status == 1
