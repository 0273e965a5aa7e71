"""Brute-force UGKS interface fluxes for tiny meshes, written independently of the oracle.

Where the oracle uses closed forms, this module integrates numerically:
  * the time integrals of the integral solution (Eq. 2) by nested Gauss-Legendre rules
    (no Mt1..Mt5 formulas),
  * the Maxwellian moments by Gauss-Hermite / half-line Gauss-Legendre quadrature in
    (u, v, xi) (no half-range moment recursions),
  * the micro-slope systems by assembling the 4x4 moment matrix by quadrature and
    calling numpy.linalg.solve,
  * the reduced h and b components by quadrature over the internal variable xi.
The discrete-velocity parts (interface values, W0, the free-transport sums) are sums over
the same discrete grid, as the scheme defines them.  Periodic index handling uses
numpy.roll, and the channel boundaries are implemented from their definitions.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial.hermite import hermgauss
from numpy.polynomial.legendre import leggauss

WALL, PERIODIC, PRESSURE = 1, 0, 2


def vanleer(s1, s2):
    out = np.zeros_like(s1)
    m = s1 * s2 > 0
    out[m] = 2 * s1[m] * s2[m] / (s1[m] + s2[m])
    return out


def axis(n, lo, hi):
    if n == 1:
        return np.array([0.5 * (lo + hi)]), np.array([1.0])
    x = np.linspace(lo, hi, n)
    h = (hi - lo) / (n - 1)
    w = np.full(n, h)
    w[0] = w[-1] = h / 2
    return x, w


def tau_of(cfg, rho, lam):
    a, om = cfg.alpha, cfg.omega
    mu_ref = 5 * (a + 1) * (a + 2) * math.sqrt(math.pi) / (4 * a * (5 - 2 * om) * (7 - 2 * om)) * cfg.kn
    return mu_ref * (1.0 / lam) ** om / (rho / (2 * lam))


class Quad:
    """Quadrature of the normalised Maxwellian (density 1) in (un, ut, xi^K).  The un
    axis is split at 0 into two half-line Gauss-Legendre rules."""

    def __init__(self, Un, Ut, lam, K, n_half=40, n_t=28, n_xi=8):
        sig = 1 / math.sqrt(2 * lam)
        L = abs(Un) + 16 * sig
        x, w = leggauss(n_half)
        up = (x + 1) / 2 * L
        wp = w * L / 2
        un = np.concatenate([-up[::-1], up])
        wun = np.concatenate([wp[::-1], wp]) * np.sqrt(lam / math.pi) * np.exp(-lam * (un - Un) ** 2)
        xh, wh = hermgauss(n_t)
        ut = Ut + xh / math.sqrt(lam)
        wut = wh / math.sqrt(math.pi)
        xx, wx = hermgauss(n_xi)
        xi_nodes = [np.zeros(1)]
        xi_w = np.ones(1)
        comps = []
        for _ in range(K):
            comps.append(xx / math.sqrt(lam))
        if K > 0:
            grids = np.meshgrid(*comps, indexing="ij")
            wgr = np.meshgrid(*([wx / math.sqrt(math.pi)] * K), indexing="ij")
            xi2 = sum(g.reshape(-1) ** 2 for g in grids)
            xi_w = np.prod([g.reshape(-1) for g in wgr], axis=0)
        else:
            xi2 = np.zeros(1)
        U, T, X = np.meshgrid(un, ut, xi2, indexing="ij")
        WU, WT, WX = np.meshgrid(wun, wut, xi_w, indexing="ij")
        self.un, self.ut, self.xi2 = U.reshape(-1), T.reshape(-1), X.reshape(-1)
        self.w = (WU * WT * WX).reshape(-1)
        self.pos = self.un > 0
        del xi_nodes

    def psi(self):
        return np.stack([np.ones_like(self.un), self.un, self.ut,
                         0.5 * (self.un ** 2 + self.ut ** 2 + self.xi2)])


def apsi(a, un, ut, xi2):
    return a[0] + a[1] * un + a[2] * ut + 0.5 * a[3] * (un ** 2 + ut ** 2 + xi2)


def time_weights(dt, tau, n=24):
    """Nested Gauss-Legendre sums of the Eq. 2 weights over t in [0,dt], t' in [0,t]:
    C0 = int int e^{-(t-t')/tau}/tau, C1 = same times (t-t'), C2 = same times t',
    D0 = int e^{-t/tau}, D1 = int t e^{-t/tau}."""
    x, w = leggauss(n)
    t = (x + 1) / 2 * dt
    wt = w * dt / 2
    C0 = C1 = C2 = 0.0
    for ti, wi in zip(t, wt):
        tp = (x + 1) / 2 * ti
        wtp = w * ti / 2
        k = np.exp(-(ti - tp) / tau) / tau * wtp * wi
        C0 += k.sum()
        C1 += (k * (ti - tp)).sum()
        C2 += (k * tp).sum()
    D0 = (wt * np.exp(-t / tau)).sum()
    D1 = (wt * t * np.exp(-t / tau)).sum()
    return C0, C1, C2, D0, D1


def shakhov_s(pr, K, rho, Un, Ut, lam, q, un, ut, xi2):
    """Shakhov factor S of g+ = g (1 + S) at (un, ut, |xi|^2), stated in physical terms:
    S = (1 - Pr) (c . q) / ((D + 2) p RT) (c_t^2 / RT - (D + 2)), D = 2 + K, RT = 1/(2 lam),
    p = rho RT, c_t^2 = |c|^2 + |xi|^2 (the internal variable integrated by quadrature)."""
    RT = 1.0 / (2.0 * lam)
    p = rho * RT
    D = 2 + K
    cn, ct = un - Un, ut - Ut
    return (1.0 - pr) * (cn * q[0] + ct * q[1]) / ((D + 2) * p * RT) * (
        (cn ** 2 + ct ** 2 + xi2) / RT - (D + 2))


def ugks_face(cfg, dt, unq, utq, wq, f_up, sn_up, st_up, W0, WL, WR, delta, St, K):
    """Brute-force macroscopic (rotated frame) and micro flux at one interface.  With a
    Prandtl number pr != 1 (Shakhov model) the zeroth-order equilibrium term carries the
    Shakhov factor of the interface heat flux (that of the upwind values about the
    interface velocity)."""
    rho0 = W0[0]
    Un, Ut = W0[1] / rho0, W0[2] / rho0
    lam = (K + 2) * rho0 / (4 * (W0[3] - 0.5 * rho0 * (Un ** 2 + Ut ** 2)))
    tau = tau_of(cfg, rho0, lam)
    Q = Quad(Un, Ut, lam, K)
    psi = Q.psi()
    M = np.einsum("in,jn,n->ij", psi, psi, Q.w)
    aL = np.linalg.solve(M, (W0 - WL) / (rho0 * delta / 2))
    aR = np.linalg.solve(M, (WR - W0) / (rho0 * delta / 2))
    b = np.linalg.solve(M, St / rho0)
    a_of_u = np.where(Q.pos[None, :], aL[:, None], aR[:, None])
    pa = (a_of_u[0] + a_of_u[1] * Q.un + a_of_u[2] * Q.ut
          + 0.5 * a_of_u[3] * (Q.un ** 2 + Q.ut ** 2 + Q.xi2))
    pb = apsi(b, Q.un, Q.ut, Q.xi2)
    sA = -np.einsum("in,n->i", psi, Q.w * (Q.un * pa + Q.ut * pb))
    A = np.linalg.solve(M, sA)
    pA = apsi(A, Q.un, Q.ut, Q.xi2)
    C0, C1, C2, D0, D1 = time_weights(dt, tau)
    pr = getattr(cfg, "pr", 1.0)
    q0 = np.zeros(2)
    if pr != 1.0:
        cn, ct = unq - Un, utq - Ut
        e = (cn ** 2 + ct ** 2) * f_up[:, 0] + f_up[:, 1]
        q0 = 0.5 * np.array([np.sum(wq * cn * e), np.sum(wq * ct * e)])
    # equilibrium part: g0 [1 + S + (a.psi) x' + (b.psi) y' + (A.psi) t'], x' = -un s,
    # y' = -ut s, the Shakhov factor S on the zeroth-order term only
    S_q = shakhov_s(pr, K, rho0, Un, Ut, lam, q0, Q.un, Q.ut, Q.xi2)
    eq = C0 * (1.0 + S_q) - C1 * Q.un * pa - C1 * Q.ut * pb + C2 * pA
    Feq = rho0 * np.einsum("in,n->i", psi, Q.w * Q.un * eq)
    # free transport, discrete sums
    d = unq[:, None] * sn_up + utq[:, None] * st_up  # (nq, 2)
    fm = D0 * f_up - D1 * d
    e2 = 0.5 * (unq ** 2 + utq ** 2)
    wu = wq * unq
    Fft = np.array([np.sum(wu * fm[:, 0]), np.sum(wu * unq * fm[:, 0]), np.sum(wu * utq * fm[:, 0]),
                    np.sum(wu * (e2 * fm[:, 0] + 0.5 * fm[:, 1]))])
    F = Feq + Fft
    # micro flux at the discrete velocities: reduce over xi by quadrature
    xx, wx = hermgauss(8)
    if K > 0:
        comps = np.meshgrid(*([xx / math.sqrt(lam)] * K), indexing="ij")
        xi2 = sum(c.reshape(-1) ** 2 for c in comps)
        wxi = np.prod([c.reshape(-1) for c in np.meshgrid(*([wx / math.sqrt(math.pi)] * K),
                                                            indexing="ij")], axis=0)
    else:
        xi2, wxi = np.zeros(1), np.ones(1)
    u = unq[:, None]
    v = utq[:, None]
    g0 = rho0 * (lam / math.pi) * np.exp(-lam * ((u - Un) ** 2 + (v - Ut) ** 2))  # (nq,1)
    aq = np.where(unq[:, None] > 0, aL[None, :], np.where(unq[:, None] < 0, aR[None, :],
                                                          0.5 * (aL + aR)[None, :]))
    X = xi2[None, :]
    paq = aq[:, 0:1] + aq[:, 1:2] * u + aq[:, 2:3] * v + 0.5 * aq[:, 3:4] * (u ** 2 + v ** 2 + X)
    S_d = shakhov_s(pr, K, rho0, Un, Ut, lam, q0, u, v, X)
    eqq = C0 * (1.0 + S_d) - C1 * u * paq - C1 * v * apsi(b, u, v, X) + C2 * apsi(A, u, v, X)
    h_eq = (g0 * eqq * wxi[None, :]).sum(axis=1)
    b_eq = (g0 * eqq * X * wxi[None, :]).sum(axis=1)
    ft = np.stack([unq * (h_eq + fm[:, 0]), unq * (b_eq + fm[:, 1])], axis=1)
    return F, ft


def wall_face(cfg, dt, unq, utq, wq, f_face, interior_high, Tw, Uw, K):
    lam = 1.0 / Tw
    gw = (lam / math.pi) * np.exp(-lam * ((utq - Uw) ** 2 + unq ** 2))
    inc = unq < 0 if interior_high else unq > 0
    out = unq > 0 if interior_high else unq < 0
    rhow = -np.sum((wq * unq * f_face[:, 0])[inc]) / np.sum((wq * unq * gw)[out])
    fw = np.zeros_like(f_face)
    fw[inc] = f_face[inc]
    fw[out, 0] = rhow * gw[out]
    fw[out, 1] = K / (2 * lam) * rhow * gw[out]
    ft = dt * unq[:, None] * fw
    e2 = 0.5 * (unq ** 2 + utq ** 2)
    F = np.array([np.sum(wq * ft[:, 0]), np.sum(wq * unq * ft[:, 0]), np.sum(wq * utq * ft[:, 0]),
                  np.sum(wq * (e2 * ft[:, 0] + 0.5 * ft[:, 1]))])
    return F, ft


def fluxes(cfg, dt, f, W):
    """All face fluxes of the mesh, same storage order as the oracle's orc_fluxes.
    Every side may be periodic (paired), a diffuse wall or a pressure ghost."""
    nx, ny, nq, K = cfg.nx, cfg.ny, cfg.nq, cfg.K
    dx, dy = cfg.lx / nx, cfg.ly / ny
    u, wu = axis(cfg.nu, cfg.umin, cfg.umax)
    v, wv = axis(cfg.nv, cfg.vmin, cfg.vmax)
    uq = np.tile(u, cfg.nv)
    vq = np.repeat(v, cfg.nu)
    wq = np.outer(wv, wu).reshape(-1)
    F = f.reshape(ny, nx, nq, 2)
    Wc = W.reshape(4, ny, nx)
    kinds = [b.kind for b in cfg.bc]
    # extended arrays with two ghost layers: (ny+4, nx+4)
    fe = np.zeros((ny + 4, nx + 4, nq, 2))
    We = np.zeros((4, ny + 4, nx + 4))
    fe[2:-2, 2:-2] = F
    We[:, 2:-2, 2:-2] = Wc
    for side, cols in ((0, (1, 0)), (1, (nx + 2, nx + 3))):
        for l, col in enumerate(cols):
            if kinds[side] == PERIODIC:
                src = (nx + col - 2) % nx + 2 if side == 0 else (col - 2 - nx) + 2
                fe[2:-2, col] = fe[2:-2, src]
                We[:, 2:-2, col] = We[:, 2:-2, src]
            elif kinds[side] == PRESSURE:
                adj = 2 if side == 0 else nx + 1
                bc = cfg.bc[side]
                lam = 1.0 / bc.T
                for j in range(2, ny + 2):
                    Ua = We[1, j, adj] / We[0, j, adj]
                    Va = We[2, j, adj] / We[0, j, adj]
                    gh = bc.rho * lam / math.pi * np.exp(-lam * ((uq - Ua) ** 2 + (vq - Va) ** 2))
                    fe[j, col, :, 0] = gh
                    fe[j, col, :, 1] = K / (2 * lam) * gh
                    We[:, j, col] = [bc.rho, bc.rho * Ua, bc.rho * Va,
                                     bc.rho * (0.5 * (Ua ** 2 + Va ** 2) + (K + 2) / (4 * lam))]
            else:
                adj = 2 if side == 0 else nx + 1
                fe[2:-2, col] = fe[2:-2, adj]
                We[:, 2:-2, col] = We[:, 2:-2, adj]
    # y sides over every column, the x-ghost columns included (corners): periodic image,
    # zero-gradient copy next to a wall, or a pressure Maxwellian with the velocity of the
    # cell (or x-ghost) next to it in the same column
    for side, rows in ((2, (1, 0)), (3, (ny + 2, ny + 3))):
        for row in rows:
            if kinds[side] == PERIODIC:
                src = (ny + row - 2) % ny + 2 if side == 2 else (row - 2 - ny) + 2
                fe[row] = fe[src]
                We[:, row] = We[:, src]
            elif kinds[side] == WALL:
                adj = 2 if side == 2 else ny + 1
                fe[row] = fe[adj]
                We[:, row] = We[:, adj]
            else:
                adj = 2 if side == 2 else ny + 1
                bc = cfg.bc[side]
                lam = 1.0 / bc.T
                for col in range(nx + 4):
                    Ua = We[1, adj, col] / We[0, adj, col]
                    Va = We[2, adj, col] / We[0, adj, col]
                    gh = bc.rho * lam / math.pi * np.exp(-lam * ((uq - Ua) ** 2 + (vq - Va) ** 2))
                    fe[row, col, :, 0] = gh
                    fe[row, col, :, 1] = K / (2 * lam) * gh
                    We[:, row, col] = [bc.rho, bc.rho * Ua, bc.rho * Va,
                                       bc.rho * (0.5 * (Ua ** 2 + Va ** 2) + (K + 2) / (4 * lam))]
    sx = np.zeros_like(fe)
    sy = np.zeros_like(fe)
    sx[:, 1:-1] = vanleer((fe[:, 1:-1] - fe[:, :-2]) / dx, (fe[:, 2:] - fe[:, 1:-1]) / dx)
    sy[1:-1] = vanleer((fe[1:-1] - fe[:-2]) / dy, (fe[2:] - fe[1:-1]) / dy)
    if kinds[0] == PRESSURE:
        sx[:, :2] = 0; sy[:, :2] = 0
    if kinds[1] == PRESSURE:
        sx[:, -2:] = 0; sy[:, -2:] = 0
    if kinds[2] == PRESSURE:
        sx[:2] = 0; sy[:2] = 0
    if kinds[3] == PRESSURE:
        sx[-2:] = 0; sy[-2:] = 0

    def face(un, ut, fL, snL, stL, WL, fR, snR, stR, WR, delta):
        H = np.where(un > 0, 1.0, np.where(un < 0, 0.0, 0.5))[:, None]
        f_up = H * (fL + snL * delta / 2) + (1 - H) * (fR - snR * delta / 2)
        sn = H * snL + (1 - H) * snR
        st = H * stL + (1 - H) * stR
        e2 = 0.5 * (un ** 2 + ut ** 2)
        W0 = np.array([np.sum(wq * f_up[:, 0]), np.sum(wq * un * f_up[:, 0]),
                       np.sum(wq * ut * f_up[:, 0]), np.sum(wq * (e2 * f_up[:, 0] + 0.5 * f_up[:, 1]))])
        St = np.array([np.sum(wq * st[:, 0]), np.sum(wq * un * st[:, 0]), np.sum(wq * ut * st[:, 0]),
                       np.sum(wq * (e2 * st[:, 0] + 0.5 * st[:, 1]))])
        return ugks_face(cfg, dt, un, ut, wq, f_up, sn, st, W0, WL, WR, delta, St, K)

    Fx = np.zeros(((nx + 1) * ny, 4))
    fx = np.zeros(((nx + 1) * ny, nq, 2))
    for j in range(ny):
        for i in range(-1, nx):
            n = j * (nx + 1) + i + 1
            J, IL, IR = j + 2, i + 2, i + 3
            if i == -1 and kinds[0] == WALL:
                bc = cfg.bc[0]  # gas on the high side of the face: interior value f - s dx/2
                f_face = fe[J, IR] - sx[J, IR] * dx / 2
                Fx[n], fx[n] = wall_face(cfg, dt, uq, vq, wq, f_face, True, bc.T, bc.U, K)
            elif i == nx - 1 and kinds[1] == WALL:
                bc = cfg.bc[1]  # gas on the low side: f + s dx/2
                f_face = fe[J, IL] + sx[J, IL] * dx / 2
                Fx[n], fx[n] = wall_face(cfg, dt, uq, vq, wq, f_face, False, bc.T, bc.U, K)
            else:
                Fx[n], fx[n] = face(uq, vq, fe[J, IL], sx[J, IL], sy[J, IL], We[:, J, IL],
                                    fe[J, IR], sx[J, IR], sy[J, IR], We[:, J, IR], dx)
    rot = [0, 2, 1, 3]
    Fy = np.zeros((nx * (ny + 1), 4))
    fy = np.zeros((nx * (ny + 1), nq, 2))
    for j in range(-1, ny):
        for i in range(nx):
            n = (j + 1) * nx + i
            I, JL, JR = i + 2, j + 2, j + 3
            if j == -1 and kinds[2] == WALL:
                bc = cfg.bc[2]
                f_face = fe[JR, I] - sy[JR, I] * dy / 2
                Fr, fy[n] = wall_face(cfg, dt, vq, uq, wq, f_face, True, bc.T, bc.U, K)
            elif j == ny - 1 and kinds[3] == WALL:
                bc = cfg.bc[3]
                f_face = fe[JL, I] + sy[JL, I] * dy / 2
                Fr, fy[n] = wall_face(cfg, dt, vq, uq, wq, f_face, False, bc.T, bc.U, K)
            else:
                Fr, fy[n] = face(vq, uq, fe[JL, I], sy[JL, I], sx[JL, I], We[rot, JL, I],
                                 fe[JR, I], sy[JR, I], sx[JR, I], We[rot, JR, I], dy)
            Fy[n] = Fr[rot]
    return Fx, Fy, fx, fy
