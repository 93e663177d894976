"""Pins of the oracle's comparator schemes (conventional explicit RK with full k-storage).

The paper measures its two-register scheme (Eq. 21) against standard explicit RK that
keeps every stage derivative (RKF45, its ref. [36]; Sec. 2.2.3, Sec. 4.2.2).  The oracle
holds two such schemes, each pinned here against the mathematics rather than itself:

* scheme 1, the RK4(3)5[2R+]C tableau in Butcher form with full k-storage: its A is the
  exact rational tableau of the published coefficients (a_ij = b_j for j < i-1); one step
  on y' = lambda y equals R(h lambda) y and the error register (R - Rhat)(h lambda) y, and
  it matches the two-register form of the same method on chemistry to rounding (equal
  step counts);
* scheme 2, Fehlberg's RKF45: the tableau is Fehlberg's rationals (golden fixture), which
  satisfy every order condition to order 4 (propagated weights) and 5 (error weights)
  exactly, the z^5 term of its stability polynomial is 1/104; one step on y' = lambda y
  equals that polynomial; fixed-step slopes are 4 and 5 on y' = -y^2; on chemistry it
  conserves elements and energy to 1e-12 and lands within the tolerance of the Eq. 21
  result.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W
from tests import _tableau

LS = _tableau.load()
RKF = _tableau.load_rkf45()


def test_full_storage_tableau_is_the_exact_one():
    s, A, b, bh, expo = oracle.butcher(1)
    assert s == 5 and expo == 0.25
    for i in range(5):
        for j in range(5):
            assert A[i, j] == float(LS["A"][i][j]), (i, j)
        assert b[i] == float(LS["b"][i]) and bh[i] == float(LS["bh"][i])


def test_rkf45_tableau_and_order_conditions():
    s, A, b, bh, expo = oracle.butcher(2)
    assert s == 6 and expo == 0.2
    for i in range(6):
        for j in range(6):
            assert A[i, j] == float(RKF["A"][i][j]), (i, j)
        assert b[i] == float(RKF["b"][i]) and bh[i] == float(RKF["bh"][i])
    for w in (RKF["b"], RKF["bh"]):
        for k, v in _tableau.order_residuals(w, RKF["A"], RKF["c"]).items():
            assert v == 0, k
    for k, v in _tableau.order5_residuals(RKF["bh"], RKF["A"], RKF["c"]).items():
        assert v == 0, k
    # the propagated solution is fourth order only
    assert max(abs(v) for v in _tableau.order5_residuals(RKF["b"], RKF["A"], RKF["c"]).values()) > Fr(1, 10 ** 4)
    assert [float(x) for x in RKF["c"]] == [0.0, 0.25, 0.375, 12.0 / 13.0, 1.0, 0.5]
    # stability polynomial of the fourth-order solution: 1 + z + ... + z^4/24 + z^5/104
    v = [Fr(1)] * 6
    coef = []
    for _ in range(6):
        coef.append(sum(RKF["b"][i] * v[i] for i in range(6)))
        v = [sum(RKF["A"][i][j] * v[j] for j in range(6)) for i in range(6)]
    assert coef == [1, Fr(1, 2), Fr(1, 6), Fr(1, 24), Fr(1, 104), 0]


@pytest.mark.parametrize("scheme,tab", [(1, LS), (2, RKF)])
@pytest.mark.parametrize("z", [-0.3, -1.0, -2.5, 0.7])
def test_one_step_linear(scheme, tab, z):
    lam = -987.25
    h = z / lam
    y0 = 0.731
    y, E = oracle.linear_step_scheme(scheme, np.array([[lam]]), h, np.array([y0]))
    zf = Fr(h) * Fr(lam)
    R = _tableau.stability(zf, tab["b"], tab["A"])
    Rh = _tableau.stability(zf, tab["bh"], tab["A"])
    assert y[0] == pytest.approx(float(R * Fr(y0)), rel=1e-14, abs=1e-300)
    assert E[0] == pytest.approx(float((R - Rh) * Fr(y0)), rel=1e-9, abs=1e-16)


def test_full_storage_step_equals_two_register_step():
    rng = np.random.default_rng(2)
    M_ = rng.standard_normal((6, 6)) * 300.0
    y0 = rng.standard_normal(6)
    y2, E2 = oracle.linear_step(M_, 1e-3, y0)
    y1, E1 = oracle.linear_step_scheme(1, M_, 1e-3, y0)
    np.testing.assert_allclose(y1, y2, rtol=1e-13, atol=1e-15 * np.abs(y0).max())
    np.testing.assert_allclose(E1, E2, rtol=1e-9, atol=1e-15 * np.abs(y0).max())


@pytest.mark.parametrize("scheme,embedded,order", [(1, False, 4.0), (1, True, 3.0),
                                                   (2, False, 4.0), (2, True, 5.0)])
def test_convergence_order_quadratic(scheme, embedded, order):
    # y' = -y^2, y(0) = 1 -> y(1) = 1/2
    Ns = [8, 16, 32, 64]
    errs = [abs(oracle.quadratic_fixed_scheme(scheme, 1.0, 1.0 / N, N, embedded) - 0.5) for N in Ns]
    slopes = -np.diff(np.log(errs)) / np.log(2.0)
    if order == 5.0:
        # the fifth-order solution approaches its rate from above (5.95, 5.54, 5.29 here);
        # a wrong weight would leave it at 4 or below
        assert np.all(np.diff(slopes) < 0) and abs(slopes[-1] - order) < 0.35, slopes
    else:
        assert abs(slopes[-1] - order) < 0.15, slopes


@pytest.fixture(scope="module")
def reactors():
    mech = M.build(0)
    o = oracle.Oracle(mech)
    r = W.reactors(384, seed=0)
    rho, e = o.state_from_TPY(r["T"], r["p"], r["Y"])
    base = o.integrate(rho, e, r["Y"], r["T"], 1e-7)
    return mech, o, r, rho, e, base


def test_full_storage_matches_two_register_on_chemistry(reactors):
    mech, o, r, rho, e, base = reactors
    full = o.integrate(rho, e, r["Y"], r["T"], 1e-7, scheme=1)
    assert np.all(full["status"] == 0)
    edge = (base["margin"] < 1e-7) | (full["margin"] < 1e-7)
    np.testing.assert_array_equal(full["nsteps"][~edge], base["nsteps"][~edge])
    relT = np.abs(full["T"] - base["T"]) / base["T"]
    assert relT[~edge].max() <= 1e-10
    assert np.abs(full["Y"] - base["Y"]).max(axis=0)[~edge].max() <= 1e-12


def test_rkf45_on_chemistry(reactors):
    mech, o, r, rho, e, base = reactors
    out = o.integrate(rho, e, r["Y"], r["T"], 1e-7, scheme=2)
    assert np.all(out["status"] == 0)
    # invariants of any RK method on this system: element mass fractions and energy
    El = np.asarray(mech["ncomp"], float).T * np.array([M.ATOMIC_MASS[x] for x in M.ELEMENTS])[:, None] \
        / np.asarray(mech["W"])[None, :]
    np.testing.assert_allclose(El @ out["Y"], El @ r["Y"], rtol=0, atol=1e-12)
    for i in range(0, 384, 37):
        assert abs(o.e_mix(out["Y"][:, i], out["T"][i]) - e[i]) <= 1e-12 * abs(e[i])
    # both integrate the same ODE to rtol 1e-6: their answers agree to the tolerance
    assert np.max(np.abs(out["T"] - base["T"]) / base["T"]) <= 1e-4
    # RKF45 takes fewer (six-stage, higher-order) steps than the five-stage scheme here
    assert out["nsteps"].sum() < 2 * base["nsteps"].sum()
