"""Pins of the oracle on the 13-species / 27-reaction mechanism (the paper's mechanism
size, Sec. 5.2.3): the synthetic H2-O2 structure with argon, helium, CO and CO2 as
colliders and collider-specific third-body channels.

* every reaction balances H, O, N (integers); the colliders take part in none, so
  the production rates leave them exactly unchanged;
* noble gases have cp = 5/2 R exactly, so the temperature of pure argon or helium is the
  closed form T = T_ref + (e - e_ref) / (3/2 R / W);
* a third-body channel whose only collider is argon (or helium) runs at [M] = c_Ar
  (c_He): its rate of progress is proportional to that concentration alone;
* the integrator conserves sum Y, the element mass fractions and e to 1e-12 and the
  colliders' mass fractions exactly, through ignition;
* at long times every reaction is in detailed balance (q_f = q_r).
"""
import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W

R_U = 8.31446261815324
MECH = M.build13(0)
O = oracle.Oracle(MECH)
SP = list(M.SPECIES13)
COLL = [SP.index(x) for x in ("AR", "HE", "CO", "CO2")]
AMASS = np.array([M.ATOMIC_MASS[e] for e in M.ELEMENTS])


def test_structure_and_balance():
    assert len(MECH["W"]) == 13 and len(MECH["A"]) == 27
    nu = MECH["nu_r"] - MECH["nu_f"]
    assert np.all(nu @ MECH["ncomp"] == 0)
    assert np.all(MECH["nu_f"][:, COLL] == 0) and np.all(MECH["nu_r"][:, COLL] == 0)
    # molar masses of the colliders: standard atomic weights
    np.testing.assert_allclose(MECH["W"][COLL], [39.948e-3, 4.0026e-3, 28.010e-3, 44.009e-3], rtol=1e-12)


def test_wdot_leaves_colliders_unchanged_and_conserves():
    r = W.reactors13(64, seed=3)
    rng = np.random.default_rng(4)
    for i in range(64):
        Y = r["Y"][:, i].copy()
        Y[3:8] += rng.uniform(0.0, 0.03, 5)
        Y /= Y.sum()
        w = O.wdot(rng.uniform(0.1, 3.0), rng.uniform(800.0, 3000.0), Y)
        assert np.all(w[COLL] == 0.0)
        scale = np.abs(w * MECH["W"]).max()
        assert abs(np.dot(MECH["W"], w)) <= 1e-13 * scale
        assert np.all(np.abs(MECH["ncomp"].T @ w) * AMASS.max() <= 1e-13 * scale)


@pytest.mark.parametrize("name", ["AR", "HE"])
@pytest.mark.parametrize("T", [300.0, 1234.5, 2800.0])
def test_noble_gas_temperature_closed_form(name, T):
    k = SP.index(name)
    for a in (MECH["nasa_lo"][k], MECH["nasa_hi"][k]):
        np.testing.assert_allclose(a[:5], [2.5, 0, 0, 0, 0], atol=1e-12)
    Y = np.zeros(13)
    Y[k] = 1.0
    W_ = MECH["W"][k]
    e_ref = O.e_mix(Y, 1000.0)
    e = e_ref + 1.5 * R_U / W_ * (T - 1000.0)
    rc, Tn, _ = O.T_from_e(Y, e, 1500.0)
    assert rc == 0 and Tn == pytest.approx(T, rel=1e-12)


@pytest.mark.parametrize("coll,j", [("AR", 21), ("HE", 22), ("AR", 23), ("HE", 24)])
def test_collider_specific_channel_rate(coll, j):
    k = SP.index(coll)
    other = SP.index("HE" if coll == "AR" else "AR")
    T, rho = 1800.0, 1.3
    base = np.zeros(13)
    base[SP.index("H2")] = 0.02
    base[SP.index("O")] = 0.01
    base[SP.index("O2")] = 0.05
    qs = []
    for ya, yo in ((0.3, 0.0), (0.6, 0.0), (0.3, 0.6)):
        Y = base.copy()
        Y[k] = ya
        Y[other] = yo
        Y[SP.index("N2")] = 1.0 - Y.sum()
        qf, qr = O.progress(rho, T, Y)
        qs.append(qf[j])
    # doubling c_coll doubles the forward progress; the other noble gas adds nothing
    assert qs[1] == pytest.approx(2.0 * qs[0], rel=1e-13)
    assert qs[2] == pytest.approx(qs[0], rel=1e-13)


def test_integrator_invariants_through_ignition():
    r = W.reactors13(24, seed=9)
    r["T"][:] = np.linspace(1300.0, 2000.0, 24)
    rho, e = O.state_from_TPY(r["T"], r["p"], r["Y"])
    out = O.integrate(rho, e, r["Y"], r["T"], 5e-5)
    assert np.all(out["status"] == 0)
    assert np.all(out["T"] > r["T"] + 300.0)
    np.testing.assert_allclose(out["Y"].sum(axis=0), 1.0, rtol=0, atol=1e-12)
    Z = (MECH["ncomp"] * AMASS[None, :] / MECH["W"][:, None]).T
    np.testing.assert_allclose(Z @ out["Y"], Z @ r["Y"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(out["Y"][COLL], r["Y"][COLL])
    for i in range(24):
        assert abs(O.e_mix(out["Y"][:, i], out["T"][i]) - e[i]) <= 1e-12 * abs(e[i])


def test_detailed_balance_at_long_times():
    r = W.reactors13(1, seed=5)
    r["T"][:] = 1800.0
    r["p"][:] = 101325.0
    rho, e = O.state_from_TPY(r["T"], r["p"], r["Y"])
    out = O.integrate(rho, e, r["Y"], r["T"], 1e-3, rtol=1e-10, atol=1e-18, max_steps=1000000)
    assert out["status"][0] == 0 and out["T"][0] > 2500.0
    qf, qr = O.progress(rho[0], out["T"][0], out["Y"][:, 0])
    assert np.max(np.abs(qf - qr) / np.maximum(qf, qr)) < 1e-7
