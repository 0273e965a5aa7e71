"""Pins of the oracle's Shakhov model (Prandtl number != 1; the paper's Eq. 1 is the BGK
model, and the Shakhov equilibrium replaces its Maxwellian in the collision term):

* the Shakhov equilibrium carries the density, momentum and energy of its Maxwellian and
  the fraction 1 - Pr of the heat flux, on a fine wide velocity grid (closed forms; K = 0,
  1, 2 internal degrees of freedom);
* a uniform Maxwellian stays uniform (its heat flux is zero);
* a spatially uniform state relaxes its heat flux by the closed-form factor of the
  trapezoidal collision term, [(1 - x/2) + x (1 - Pr)] / (1 + x/2) per step, x = dt/tau;
* the interface fluxes equal a brute-force evaluation of the integral solution with the
  Shakhov factor stated in physical units and the internal variable integrated by
  quadrature (tests/bruteforce.py);
* a full step makes the residuals of Eq. 4 and of the implicit Eq. 3 with g+ in place of g
  vanish, the heat flux of f^n in g+^n and g+^{n+1};
* Pr -> 1 approaches the BGK step continuously.
"""
import math

import numpy as np
import pytest

from paper_1810_08137_gb300 import inputs as I
from tests import bruteforce as BF


def periodic_cfg(**kw):
    base = dict(nx=4, ny=4, lx=1.0, ly=1.0, nu=5, nv=5, umin=-3.0, umax=3.0, vmin=-3.0,
                vmax=3.0, K=1, kn=0.05, bc=[I.BC(I.BC_PERIODIC)] * 4, pr=2.0 / 3.0)
    base.update(kw)
    return I.Config(**base)


def random_state(oracle, cfg, seed, amp=0.2, flow=0.3):
    r = I.uniform01(seed, 4 * cfg.nc).reshape(4, cfg.nc)
    f, W = oracle.init_maxwellian(cfg, 0.8 + 0.4 * r[0], flow * (2 * r[1] - 1),
                                  flow * (2 * r[2] - 1), 0.8 + 0.4 * r[3])
    return f * I.perturbation(seed + 1, f.shape, amp), W


def fine_grid(n=161, vr=10.0):
    x = np.linspace(-vr, vr, n)
    w = np.full(n, x[1] - x[0])
    w[0] = w[-1] = w[0] / 2
    U, V = np.meshgrid(x, x)
    return U.reshape(-1), V.reshape(-1), np.outer(w, w).reshape(-1)


@pytest.mark.parametrize("K", [0, 1, 2])
@pytest.mark.parametrize("pr", [2.0 / 3.0, 0.5, 1.3])
def test_shakhov_equilibrium_moments(oracle, K, pr):
    u, v, w = fine_grid()
    rho, U, V, lam = 1.3, 0.2, -0.35, 0.8
    q = np.array([0.11, -0.07])
    g = oracle.shakhov_eq([rho, U, V, lam], K, pr, q, u, v)
    h, b = g[:, 0], g[:, 1]
    E = rho * (0.5 * (U * U + V * V) + (K + 2) / (4 * lam))
    mom = [np.sum(w * h), np.sum(w * u * h), np.sum(w * v * h),
           np.sum(w * (0.5 * (u * u + v * v) * h + 0.5 * b))]
    np.testing.assert_allclose(mom, [rho, rho * U, rho * V, E], rtol=1e-12, atol=1e-13)
    cu, cv = u - U, v - V
    e = (cu * cu + cv * cv) * h + b
    qg = 0.5 * np.array([np.sum(w * cu * e), np.sum(w * cv * e)])
    np.testing.assert_allclose(qg, (1 - pr) * q, rtol=1e-11, atol=1e-13)


def test_shakhov_uniform_maxwellian_preserved(oracle):
    cfg = periodic_cfg(nu=24, nv=24, umin=-6, umax=6, vmin=-6, vmax=6)
    n = cfg.nc
    f, W = oracle.init_maxwellian(cfg, np.full(n, 1.1), np.full(n, 0.2), np.full(n, -0.1),
                                  np.full(n, 0.9))
    f1, W1 = oracle.step(cfg, f, W, 3)
    assert np.max(np.abs(W1 - W)) < 1e-14 * np.max(np.abs(W))
    assert np.max(np.abs(f1 - f)) < 1e-8 * np.max(np.abs(f))  # heat flux of the grid ~1e-10


@pytest.mark.parametrize("K", [0, 1, 2])
@pytest.mark.parametrize("kn", [0.02, 0.5])
def test_shakhov_homogeneous_heat_flux_relaxation(oracle, K, kn):
    cfg = periodic_cfg(nx=3, ny=3, nu=81, nv=81, umin=-9, umax=9, vmin=-9, vmax=9, K=K, kn=kn)
    n = cfg.nc
    rho, U, V, T = 1.05, 0.15, -0.1, 1.1
    f, W = oracle.init_maxwellian(cfg, np.full(n, rho), np.full(n, U), np.full(n, V),
                                  np.full(n, T))
    # one cell's distribution with a heat flux: a Maxwellian times 1 + a polynomial that
    # is odd in the peculiar velocity, copied into every cell (spatially uniform)
    u, v, _ = oracle.vgrid(cfg)
    uq, vq = np.tile(u, cfg.nv), np.repeat(v, cfg.nu)
    cu, cv = uq - U, vq - V
    lam = 1 / T
    shape = 1 + 0.08 * (cu - 0.5 * cv) * (lam * (cu * cu + cv * cv) - 2.0)
    f = f * shape[None, :, None]
    q0 = oracle.heat_flux(cfg, f[0], W[:, 0])
    assert np.min(np.abs(q0)) > 1e-3
    f1, W1 = oracle.step(cfg, f, W, 1)
    np.testing.assert_array_equal(W1, W)  # identical faces: the fluxes cancel exactly
    q1 = oracle.heat_flux(cfg, f1[4], W1[:, 4])
    x = oracle.dt(cfg) / oracle.tau(cfg, rho, lam)
    ratio = ((1 - x / 2) + x * (1 - cfg.pr)) / (1 + x / 2)
    np.testing.assert_allclose(q1, ratio * q0, rtol=1e-10, atol=1e-14)


def _compare_fluxes(oracle, cfg, f, W):
    dt = oracle.dt(cfg)
    Fx, Fy, fx, fy = oracle.fluxes(cfg, f, W)
    bx, by, bfx, bfy = BF.fluxes(cfg, dt, f, W)
    sF = max(np.max(np.abs(bx)), np.max(np.abs(by)))
    sf = max(np.max(np.abs(bfx)), np.max(np.abs(bfy)))
    assert np.max(np.abs(Fx - bx)) < 1e-11 * sF
    assert np.max(np.abs(Fy - by)) < 1e-11 * sF
    assert np.max(np.abs(fx - bfx)) < 1e-11 * sf
    assert np.max(np.abs(fy - bfy)) < 1e-11 * sf


@pytest.mark.parametrize("K,kn,pr", [(1, 0.05, 2.0 / 3.0), (0, 0.3, 0.5), (2, 0.01, 0.72)])
def test_shakhov_bruteforce_periodic_4x4(oracle, K, kn, pr):
    cfg = periodic_cfg(nu=5, nv=4, K=K, kn=kn, pr=pr)
    f, W = random_state(oracle, cfg, 31)
    _compare_fluxes(oracle, cfg, f, W)


def test_shakhov_bruteforce_channel_4x4(oracle):
    cfg = I.channel_config(nx=4, ny=4, n_vel=5, vrange=3.0, kn=0.1)
    cfg.pr = 2.0 / 3.0
    cfg.bc[2] = I.BC(I.BC_WALL, T=1.2, U=0.1)
    f, W = random_state(oracle, cfg, 32, flow=0.2)
    _compare_fluxes(oracle, cfg, f, W)


def _shakhov_red(cfg, Wc, q, uq, vq):
    """g+ (h, b) of W with heat flux q: the Shakhov factor of tests/bruteforce.py integrated
    over the internal variable by Gauss-Hermite quadrature; and tau."""
    K = cfg.K
    rho = Wc[0]
    U, V = Wc[1] / rho, Wc[2] / rho
    lam = (K + 2) * rho / (4 * (Wc[3] - 0.5 * rho * (U * U + V * V)))
    gh = rho * lam / math.pi * np.exp(-lam * ((uq - U) ** 2 + (vq - V) ** 2))
    if K > 0:
        x, wx = np.polynomial.hermite.hermgauss(8)
        comps = np.meshgrid(*([x / math.sqrt(lam)] * K), indexing="ij")
        xi2 = sum(c.reshape(-1) ** 2 for c in comps)
        wxi = np.prod([c.reshape(-1) for c in np.meshgrid(*([wx / math.sqrt(math.pi)] * K),
                                                            indexing="ij")], axis=0)
    else:
        xi2, wxi = np.zeros(1), np.ones(1)
    S = BF.shakhov_s(cfg.pr, K, rho, U, V, lam, q, uq[:, None], vq[:, None], xi2[None, :])
    h = gh * ((1 + S) * wxi).sum(axis=1)
    b = gh * ((1 + S) * xi2 * wxi).sum(axis=1)
    return np.stack([h, b], axis=1), BF.tau_of(cfg, rho, lam)


@pytest.mark.parametrize("case", ["periodic", "channel"])
def test_shakhov_step_satisfies_eq3_and_eq4(oracle, case):
    if case == "periodic":
        cfg = periodic_cfg(nu=5, nv=4, kn=0.02)
    else:
        cfg = I.channel_config(nx=4, ny=4, n_vel=5, vrange=3.0, kn=0.02)
        cfg.pr = 2.0 / 3.0
    f, W = random_state(oracle, cfg, 33)
    dt = oracle.dt(cfg)
    f1, W1 = oracle.step(cfg, f, W, 1)
    Fx, Fy, fx, fy = BF.fluxes(cfg, dt, f, W)
    nx, ny = cfg.nx, cfg.ny
    dx, dy = cfg.lx / nx, cfg.ly / ny
    u, wu = BF.axis(cfg.nu, cfg.umin, cfg.umax)
    v, wv = BF.axis(cfg.nv, cfg.vmin, cfg.vmax)
    uq, vq = np.tile(u, cfg.nv), np.repeat(v, cfg.nu)
    wq = np.outer(wv, wu).reshape(-1)
    assert np.max(np.abs(W1 - W)) > 1e-4
    for c in range(cfg.nc):
        i, j = c % nx, c // nx
        xw, xe = j * (nx + 1) + i, j * (nx + 1) + i + 1
        ys, yn = j * nx + i, (j + 1) * nx + i
        r4 = W1[:, c] - W[:, c] - (Fx[xw] - Fx[xe]) / dx - (Fy[ys] - Fy[yn]) / dy
        assert np.max(np.abs(r4)) < 1e-12 * np.max(np.abs(W))
        U, V = W[1, c] / W[0, c], W[2, c] / W[0, c]
        cu, cv = uq - U, vq - V
        e = (cu * cu + cv * cv) * f[c, :, 0] + f[c, :, 1]
        qn = 0.5 * np.array([np.sum(wq * cu * e), np.sum(wq * cv * e)])
        g1, t1 = _shakhov_red(cfg, W1[:, c], qn, uq, vq)
        g0, t0 = _shakhov_red(cfg, W[:, c], qn, uq, vq)
        r3 = (f1[c] - f[c] - (fx[xw] - fx[xe]) / dx - (fy[ys] - fy[yn]) / dy
              - dt / 2 * ((g1 - f1[c]) / t1 + (g0 - f[c]) / t0))
        assert np.max(np.abs(r3)) < 1e-11 * np.max(np.abs(f))


def test_shakhov_tends_to_bgk(oracle):
    cfg = periodic_cfg(nu=6, nv=6, kn=0.05)
    f, W = random_state(oracle, cfg, 34)
    fb, Wb = oracle.step(cfg.replace(pr=1.0), f, W, 2)
    fs, Ws = oracle.step(cfg.replace(pr=1.0 - 1e-7), f, W, 2)
    fs2, _ = oracle.step(cfg.replace(pr=2.0 / 3.0), f, W, 2)
    d = np.max(np.abs(fs - fb)) / np.max(np.abs(fb))
    d2 = np.max(np.abs(fs2 - fb)) / np.max(np.abs(fb))
    assert 0 < d < 1e-7 * 10 and d2 > 1e4 * d  # continuous in Pr, and the model matters
