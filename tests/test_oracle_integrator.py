"""Pins of the oracle's whole-cell integration (Eq. 14, 20-22; Sec. 2.2.3).

* invariants the source term fixes (Eq. 14: only the partial densities change, every
  reaction conserves elements): sum Y = 1 and element mass fractions to 1e-12, and
  e(T_out, Y_out) = e to 1e-12 relative, both over one dt and through ignition;
* tolerance proportionality against a tight-tolerance run;
* step-halving: the fixed-step solution at a point of the ignition front converges at
  fourth order (differences shrink ~16x per halving);
* long-time state: detailed balance q_f = q_r for every reaction, and the ideal-gas
  chemical potentials are a combination of element potentials (true equilibrium);
* per-cell status codes for the documented failure modes.
"""
import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W

R_U = 8.31446261815324
P_REF = 101325.0
MECH = M.build(0)
O = oracle.Oracle(MECH)
AMASS = np.array([M.ATOMIC_MASS[e] for e in M.ELEMENTS])


def _elements(Y):
    """Element mass fractions Z_e = sum_k n_ke A_e Y_k / W_k."""
    return (MECH["ncomp"] * AMASS[None, :] / MECH["W"][:, None]).T @ Y


def _setup(r):
    rho, e = O.state_from_TPY(r["T"], r["p"], r["Y"])
    return rho, e


def _check_invariants(out, Y0, e):
    assert np.all(out["status"] == 0)
    np.testing.assert_allclose(out["Y"].sum(axis=0), 1.0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(_elements(out["Y"]), _elements(Y0), rtol=0, atol=1e-12)
    e_out = np.array([O.e_mix(out["Y"][:, i], out["T"][i]) for i in range(out["T"].size)])
    np.testing.assert_allclose(e_out, e, rtol=1e-12)


def test_invariants_reactors_one_dt():
    r = W.reactors(4096, seed=0)
    rho, e = _setup(r)
    out = O.integrate(rho, e, r["Y"], r["T"], 1e-7)
    _check_invariants(out, r["Y"], e)
    assert out["nsteps"].max() > 1  # some cells need several attempts


def test_invariants_through_ignition():
    r = W.reactors(16, seed=9)
    rho, e = _setup(r)
    out = O.integrate(rho, e, r["Y"], r["T"], 5e-5)
    _check_invariants(out, r["Y"], e)
    assert np.all(out["T"] > r["T"] + 300.0)  # every cell ignited


def test_tolerance_proportionality():
    r = W.reactors(512, seed=0)
    rho, e = _setup(r)
    ref = O.integrate(rho, e, r["Y"], r["T"], 1e-7, rtol=1e-13, atol=1e-20)
    errs = []
    for rtol in (1e-6, 1e-8):
        out = O.integrate(rho, e, r["Y"], r["T"], 1e-7, rtol=rtol, atol=rtol * 1e-4)
        errs.append(max(np.max(np.abs(out["T"] - ref["T"]) / ref["T"]),
                        np.max(np.abs(out["Y"] - ref["Y"]))))
    assert errs[0] <= 10 * 1e-6
    # two decades of rtol buy at least ~(10^2)^(4/5) / 2 of accuracy
    assert errs[0] / errs[1] > 20.0


def test_step_halving_in_the_ignition_front():
    Y = W.mass_from_mole(W.h2_air_mole(np.array([1.0])))
    T0 = 1200.0
    rho, e = O.state_from_TPY(np.array([T0]), np.array([P_REF]), Y)
    tstar = 3.07e-5  # inside the steepest part of the temperature rise
    Ts = []
    for N in (1000, 2000, 4000):
        rc, _, trace = O.chem_fixed(rho[0], e[0], Y[:, 0], T0, tstar / N, N)
        assert rc == 0
        Ts.append(trace[-1])
    assert Ts[-1] > T0 + 200.0
    d = np.diff(Ts)
    assert 12.0 < d[0] / d[1] < 22.0, d


@pytest.mark.parametrize("T0,patm,tend", [(1800.0, 1.0, 1e-3), (1500.0, 0.3, 3e-3)])
def test_long_time_equilibrium(T0, patm, tend):
    Y = W.mass_from_mole(W.h2_air_mole(np.array([1.0])))
    rho, e = O.state_from_TPY(np.array([T0]), np.array([patm * P_REF]), Y)
    out = O.integrate(rho, e, Y, np.array([T0]), tend, rtol=1e-10, atol=1e-18, max_steps=1000000)
    assert out["status"][0] == 0
    T, Yf = out["T"][0], out["Y"][:, 0]
    qf, qr = O.progress(rho[0], T, Yf)
    assert np.max(np.abs(qf - qr) / np.maximum(qf, qr)) < 1e-7
    # element potentials: mu_k / RT = g_k / RT + ln(c_k R T / p_ref) = sum_e lambda_e n_ke
    c = rho[0] * Yf / MECH["W"]
    live = c > 1e-12 * c.max()
    mu = np.array([O.h_RT(k, T) - O.s_R(k, T) + np.log(c[k] * R_U * T / P_REF)
                   for k in range(M.N_SPECIES) if live[k]])
    A = MECH["ncomp"][live].astype(float)
    lam, *_ = np.linalg.lstsq(A, mu, rcond=None)
    assert np.max(np.abs(A @ lam - mu)) < 1e-6
    assert T > T0 + 900.0


def test_status_codes():
    r = W.reactors(6, seed=4)
    rho, e = _setup(r)
    Y = r["Y"].copy()
    rho[1] = np.nan                          # non-finite input
    e[2] = -5e7                              # no positive temperature has this energy
    out = O.integrate(rho, e, Y, r["T"], 1e-7)
    assert out["status"][0] == 0
    assert out["status"][1] == 4
    assert out["status"][2] == 3
    out = O.integrate(rho[3:], e[3:], Y[:, 3:], r["T"][3:], 1e-4, max_steps=3)
    assert np.all(out["status"] == 1) and np.all(out["nsteps"] == 3)


def test_initial_step_option():
    r = W.reactors(64, seed=0)
    rho, e = _setup(r)
    a = O.integrate(rho, e, r["Y"], r["T"], 1e-7)
    b = O.integrate(rho, e, r["Y"], r["T"], 1e-7, h0=np.full(64, 1e-9))
    np.testing.assert_allclose(a["T"], b["T"], rtol=1e-8)
    assert np.all(b["nsteps"] >= 1)


def test_rejected_attempts_restore_the_temperature_start():
    """A long first step on hot burnt gas (2870-2910 K, 7-9 atm) is rejected several
    times; the trial stages of those attempts reach temperatures where the extrapolated
    NASA-7 e(T) has another root (~14,500 K).  A rejection returns the cell to its
    accepted state, the Newton starting temperature included, so one call over 2e-7 s
    must land where 40 calls over 5e-9 s land (without the restore the cell ran to
    20,600 K and stopped with h underflow)."""
    b = W.amr_batch(nboxes=40, seed=22, edges=(2, 3, 4))
    idx = np.array([87, 104, 163, 367])
    T0, p, Y0 = b["T"][idx], b["p"][idx], b["Y"][:, idx]
    rho, e = O.state_from_TPY(T0, p, Y0)
    one = O.integrate(rho, e, Y0, T0, 2e-7)
    Y, T = Y0.copy(), T0.copy()
    for _ in range(40):
        r = O.integrate(rho, e, Y, T, 5e-9)
        Y, T = r["Y"], r["T"]
        assert np.all(r["status"] == 0)
    assert np.all(one["status"] == 0)
    assert np.all(one["T"] < 3100.0)
    np.testing.assert_allclose(one["T"], T, rtol=1e-6)
    np.testing.assert_allclose(one["Y"], Y, atol=1e-6)
