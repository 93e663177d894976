"""Pins of the oracle's thermo and temperature solve (Eq. 10; calculate_T of Table 1).

* NASA-7 tables: cp, h, s continuous at T_mid; dh/dT = cp and ds/dT = cp/T
  (thermodynamic consistency, by finite differences); h(298.15) and s(298.15) equal
  the formation enthalpy and standard entropy the tables are anchored to;
* de/dT at fixed composition equals cv;
* Newton: closed form for a single constant-cp species; agreement with bisection;
  residual |e(T) - e| <= 1e-12 |e|.
"""
import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W

R_U = 8.31446261815324
MECH = M.build(0)
O = oracle.Oracle(MECH)


@pytest.mark.parametrize("k", range(M.N_SPECIES))
def test_nasa_continuity_at_tmid(k):
    Tm = MECH["T_mid"][k]
    below = np.nextafter(Tm, 0.0)
    for f in (O.cp_R, O.h_RT, O.s_R):
        lo, hi = f(k, below), f(k, Tm)
        assert abs(lo - hi) <= 1e-10 * max(1.0, abs(hi)), (f.__name__, lo, hi)


@pytest.mark.parametrize("k", range(M.N_SPECIES))
@pytest.mark.parametrize("T", [350.0, 700.0, 1500.0, 2600.0, 4000.0])
def test_thermo_consistency(k, T):
    d = 1e-3 * T
    h = lambda t: O.h_RT(k, t) * R_U * t
    s = lambda t: O.s_R(k, t) * R_U
    cp = O.cp_R(k, T) * R_U
    assert (h(T + d) - h(T - d)) / (2 * d) == pytest.approx(cp, rel=1e-6)
    assert (s(T + d) - s(T - d)) / (2 * d) == pytest.approx(cp / T, rel=1e-6)


@pytest.mark.parametrize("k", range(M.N_SPECIES))
def test_reference_state_anchors(k):
    _, _, hf, s0, _, _ = M._SPECIES[k]
    T = 298.15
    assert O.h_RT(k, T) * R_U * T == pytest.approx(hf, abs=1e-6)
    assert O.s_R(k, T) * R_U == pytest.approx(s0, rel=1e-12)


def test_cv_is_de_dT():
    r = W.reactors(16, seed=5)
    for i in range(16):
        Y = r["Y"][:, i]
        for T in (600.0, 1400.0, 2500.0):
            d = 1e-3 * T
            de = (O.e_mix(Y, T + d) - O.e_mix(Y, T - d)) / (2 * d)
            assert de == pytest.approx(O.cv_mix(Y, T), rel=1e-6)


def _single_species(a1, a6):
    coeffs = np.zeros((1, 7))
    coeffs[0, 0] = a1
    coeffs[0, 5] = a6
    return M.custom(["X"], [0.028014], [[0, 0, 2]], coeffs, coeffs.copy(), [])


@pytest.mark.parametrize("a1,a6,T", [(3.5, -1043.5, 900.0), (4.2, 2000.0, 2450.0), (2.5, 0.0, 310.0)])
def test_newton_closed_form_constant_cp(a1, a6, T):
    mech = _single_species(a1, a6)
    o = oracle.Oracle(mech)
    Wk = 0.028014
    e = R_U / Wk * ((a1 - 1.0) * T + a6)
    rc, Tn, it = o.T_from_e(np.array([1.0]), e, 1500.0)
    assert rc == 0
    assert Tn == pytest.approx((e * Wk / R_U - a6) / (a1 - 1.0), rel=1e-13)
    assert it <= 3  # linear e(T): Newton is exact after one update, confirmed by the next


def test_newton_vs_bisection_and_residual():
    rng = np.random.default_rng(11)
    r = W.reactors(64, seed=6)
    for i in range(64):
        Y = r["Y"][:, i].copy()
        # add radicals so every species matters
        Y[3:8] += rng.uniform(0, 0.02, 5)
        Y /= Y.sum()
        T = rng.uniform(300.0, 3500.0)
        e = O.e_mix(Y, T)
        rc, Tn, it = O.T_from_e(Y, e, rng.uniform(400.0, 3000.0))
        assert rc == 0 and it > 0
        rcb, Tb = O.T_from_e_bisect(Y, e)
        assert rcb == 0
        assert Tn == pytest.approx(T, rel=1e-11)
        assert abs(Tn - Tb) < 1e-8
        assert abs(O.e_mix(Y, Tn) - e) <= 1e-12 * abs(e) + 1e-9


def test_newton_nan_guess_and_out_of_range():
    r = W.reactors(1, seed=7)
    Y = r["Y"][:, 0]
    e = O.e_mix(Y, 1234.0)
    rc, Tn, _ = O.T_from_e(Y, e, float("nan"))
    assert rc == 0 and Tn == pytest.approx(1234.0, rel=1e-12)
    # an energy below e(200 K) has no root in the bracket
    rc, _, _ = O.T_from_e(Y, O.e_mix(Y, 150.0), 1000.0)
    rcb, _ = O.T_from_e_bisect(Y, O.e_mix(Y, 150.0))
    assert rcb == 3
