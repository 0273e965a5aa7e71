"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of the oracle's C source (a single textual
replacement at a unique anchor), compiles the copy into a temporary library, routes the
oracle binding to it, and checks that at least one named pin then fails.  The mistakes are
the kind a restatement of the scheme could make: a wrong factor in the viscosity law, a
max in place of a sum in the CFL rule, a flipped side at a wall, a dropped or mis-signed
term of the interface flux (Eq. 2 time integrals, compatibility condition, internal
degrees of freedom), the wrong collision time in the implicit update (Eq. 3).
Everything runs on the CPU; nothing here touches the CUDA library.
"""
import os

import pytest

from oracle import oracle as O
from tests import test_oracle_pins as T
from tests import test_oracle_shakhov as TS

SRC = open(O.SRC).read()


def _pin_tau(o):
    T.test_tau_hard_sphere_closed_form(o)


def _pin_vhs(o):
    T.test_tau_vhs_law(o, 0.81)


def _pin_dt(o):
    T.test_dt_hand_values(o)


def _pin_walls_x(o):
    T.test_bruteforce_walls_x_pressure_y_4x4(o)


def _pin_bf_periodic(o):
    T.test_bruteforce_periodic_4x4(o, 0.1)


def _pin_bf_k2(o):
    T.test_bruteforce_periodic_internal_dof(o, 2)


def _pin_bf_channel(o):
    T.test_bruteforce_channel_4x4(o)


def _pin_eq3(o):
    T.test_step_satisfies_eq3_and_eq4(o, "channel")


def _pin_muscl(o):
    T.test_collisionless_half_cell_van_leer(o)


def _pin_moments(o):
    T.test_maxwellian_discrete_moments_match_closed_forms(o, 4.0, 28, 2e-5, 1)


def _pin_mt(o):
    T.test_mt_against_time_quadrature(o, 1.0)


def _pin_shk_moments(o):
    TS.test_shakhov_equilibrium_moments(o, 2, 2.0 / 3.0)


def _pin_shk_relax(o):
    TS.test_shakhov_homogeneous_heat_flux_relaxation(o, 1, 0.5)


def _pin_shk_bf(o):
    TS.test_shakhov_bruteforce_periodic_4x4(o, 1, 0.05, 2.0 / 3.0)


def _pin_shk_eq3(o):
    TS.test_shakhov_step_satisfies_eq3_and_eq4(o, "channel")


# (name, anchor in ugks_oracle.c, replacement, pin that must fail)
MUTATIONS = [
    ("mu_ref (5-2w)(7-2w) -> (5-w)(7-w)", "(5.0 - 2.0 * om) * (7.0 - 2.0 * om)",
     "(5.0 - om) * (7.0 - om)", _pin_tau),
    ("p = rho/(2 lam) -> rho/lam", "double p = rho / (2.0 * lam);", "double p = rho / lam;",
     _pin_tau),
    ("T^omega -> T^(1/2)", "pow(T, om)", "pow(T, 0.5)", _pin_vhs),
    ("CFL: max instead of sum", "c->cfl / (um / dx + vm / dy)", "c->cfl / fmax(um / dx, vm / dy)",
     _pin_dt),
    ("x-wall W: gas side flipped", "cell_f(x, 0, j), wk->snR, 1, ORC_W",
     "cell_f(x, 0, j), wk->snR, 0, ORC_W", _pin_walls_x),
    ("x-wall E: slope sign flipped", "cell_f(x, i, j), wk->snL, 0, ORC_E",
     "cell_f(x, i, j), wk->snL, 1, ORC_E", _pin_walls_x),
    ("y-pressure ghost W from the second row",
     "fill_ghost(x, i, -l, ORC_S, i, kS == ORC_BC_PERIODIC ? ny - l : 0);",
     "fill_ghost(x, i, -l, ORC_S, i, kS == ORC_BC_PERIODIC ? ny - l : (ny > 1 ? 1 : 0));",
     _pin_walls_x),
    ("Mt5 sign in the macroscopic flux", "Mt[3] * Sf[i] - Mt[4] * Ss[i]",
     "Mt[3] * Sf[i] + Mt[4] * Ss[i]", _pin_bf_periodic),
    ("a_L and a_R swapped in the compatibility condition",
     "mom_pq(&g, 1, 1, 0, &psi, &pL) + mom_pq(&g, 2, 1, 0, &psi, &pR)",
     "mom_pq(&g, 1, 1, 0, &psi, &pR) + mom_pq(&g, 2, 1, 0, &psi, &pL)", _pin_bf_periodic),
    ("tangential term dropped from the compatibility condition",
     "mom_pq(&g, 2, 1, 0, &psi, &pR) +\n              mom_pq(&g, 0, 0, 1, &psi, &pB));",
     "mom_pq(&g, 2, 1, 0, &psi, &pR));", _pin_bf_periodic),
    ("xi^4 moment dropped", "g->xi[4] = (K * K + 2.0 * K) / (4.0 * lam * lam);", "g->xi[4] = 0.0;",
     _pin_bf_k2),
    ("H(0) = 1 instead of 1/2", "double H = un[q] > 0.0 ? 1.0 : (un[q] < 0.0 ? 0.0 : 0.5);",
     "double H = un[q] >= 0.0 ? 1.0 : 0.0;", _pin_bf_periodic),
    ("Mt3 sign", "Mt[2] * mom_pq(&g, 0, 1, 0, &psi, &pA)", "-Mt[2] * mom_pq(&g, 0, 1, 0, &psi, &pA)",
     _pin_bf_periodic),
    ("normal slope over dx instead of dx/2", "sL[k] = (W0[k] - WL[k]) / (rho0 * delta / 2.0);",
     "sL[k] = (W0[k] - WL[k]) / (rho0 * delta);", _pin_bf_periodic),
    ("tau^n in place of tau^{n+1} in the implicit factor",
     "fnew[n] = rhs / (1.0 + dt / (2.0 * tn1));", "fnew[n] = rhs / (1.0 + dt / (2.0 * tn));",
     _pin_eq3),
    ("wall b = K/2 h instead of K/(2 lam_w) h", "fb = K / (2.0 * lamw) * fh;", "fb = K / 2.0 * fh;",
     _pin_bf_channel),
    ("van Leer without the factor 2", "2.0 * s1 * s2 / (s1 + s2)", "s1 * s2 / (s1 + s2)", _pin_muscl),
    ("equilibrium flux moment <psi> instead of <un psi>", "Mt[0] * mom_p(&g, 0, 1, 0, &psi)",
     "Mt[0] * mom_p(&g, 0, 0, 0, &psi)", _pin_bf_periodic),
    ("Maxwellian b = K/2 h at set-up", "f[o + 1] = c->K / (2.0 * lam) * gh;", "f[o + 1] = c->K / 2.0 * gh;",
     _pin_moments),
    ("Mt4 limit: e^{-x} dropped", "c4 = em / x;", "c4 = 1.0 / x;", _pin_mt),
    # Shakhov model (Prandtl number != 1)
    ("Shakhov: D + 2 taken as 5 whatever K", "double d2 = K + 4.0;", "double d2 = 5.0;",
     _pin_shk_moments),
    ("Shakhov: <xi^4> term of the b factor dropped", "*sb = alpha * cq * ((c2 - d2) * xi2 + 2.0 * lam * xi4);",
     "*sb = alpha * cq * (c2 - d2) * xi2;", _pin_shk_moments),
    ("Shakhov: heat flux without the b part", "double e = (cu * cu + cv * cv) * f[2 * k] + f[2 * k + 1];",
     "double e = (cu * cu + cv * cv) * f[2 * k];", _pin_shk_relax),
    ("Shakhov: g+^{n+1} with W^n", "shakhov_factor(pn1, K, c->pr, qn, uq[q], vq[q], &sh, &sb);",
     "shakhov_factor(pn, K, c->pr, qn, uq[q], vq[q], &sh, &sb);", _pin_shk_eq3),
    ("Shakhov: interface heat flux about U = 0",
     "heat_flux(nq, w, un, ut, sc->fup, prim0[1], prim0[2], q0);",
     "heat_flux(nq, w, un, ut, sc->fup, 0.0, 0.0, q0);", _pin_shk_bf),
    ("Shakhov: macroscopic flux without the Shakhov part",
     "Feq[i] += rho0 * Mt[0] * mom_pb(&g, 0, 1, 0, &psi, &S0);", "Feq[i] += 0.0;", _pin_shk_bf),
]


@pytest.fixture(scope="module")
def oracle_ready(oracle):
    return oracle


@pytest.mark.parametrize("name,anchor,repl,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(oracle_ready, tmp_path, name, anchor, repl, pin):
    assert SRC.count(anchor) == 1, f"anchor not unique in the oracle source: {anchor!r}"
    src = tmp_path / "mutant.c"
    src.write_text(SRC.replace(anchor, repl))
    lib = O.compile_source(str(src), str(tmp_path / f"libmutant{os.getpid()}.so"))
    # the unmodified oracle passes the pin ...
    pin(oracle_ready)
    # ... and the copy with the planted mistake does not
    with O.use_library(lib):
        with pytest.raises(AssertionError):
            pin(oracle_ready)
