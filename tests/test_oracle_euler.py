"""Pins of the oracle's 1D reactive Euler step and Strang splitting (Sec. 2.2.1): the
operator on either side of the chemistry.

* Sod's shock tube for a single inert species of constant c_p (gamma = 1.4) against the
  exact Riemann solution (Toro, "Riemann Solvers and Numerical Methods for Fluid
  Dynamics", ch. 4: the pressure function solved by Newton, then sampled at x/t): the L1
  density error is small and falls with resolution;
* a reflecting box conserves total mass, energy and the mass of every species to
  rounding; a uniform moving state stays uniform (free-stream preservation);
* Strang splitting: for a gas at rest the split step equals two chemistry half-steps;
  on a smooth reacting, moving mixture its error falls ~4x per halving of dt (second
  order in time).
"""
import math

import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W

R_U = 8.31446261815324


def _inert(gamma=1.4, Wm=0.028):
    a1 = gamma / (gamma - 1.0)  # cp / R
    nasa = [[a1, 0.0, 0.0, 0.0, 0.0, -1000.0, 3.0]]
    return M.custom(["X"], [Wm], [[0, 0, 2]], nasa, nasa, [])


def exact_riemann(rhoL, uL, pL, rhoR, uR, pR, g, xi):
    """Exact solution of the ideal-gas Riemann problem sampled at xi = x / t."""
    cL, cR = math.sqrt(g * pL / rhoL), math.sqrt(g * pR / rhoR)

    def fk(p, rk, pk, ck):
        if p > pk:
            A, B = 2.0 / ((g + 1.0) * rk), (g - 1.0) / (g + 1.0) * pk
            q = math.sqrt(A / (p + B))
            return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (B + p))
        r = (p / pk) ** ((g - 1.0) / (2.0 * g))
        return 2.0 * ck / (g - 1.0) * (r - 1.0), 1.0 / (rk * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))

    p = 0.5 * (pL + pR)
    for _ in range(100):
        fL, dL = fk(p, rhoL, pL, cL)
        fR, dR = fk(p, rhoR, pR, cR)
        pn = max(p - (fL + fR + uR - uL) / (dL + dR), 1e-12 * p)
        if abs(pn - p) <= 1e-14 * p:
            p = pn
            break
        p = pn
    us = 0.5 * (uL + uR) + 0.5 * (fk(p, rhoR, pR, cR)[0] - fk(p, rhoL, pL, cL)[0])
    out = np.zeros((len(xi), 3))
    for i, s in enumerate(xi):
        if s <= us:  # left of the contact
            if p > pL:
                SL = uL - cL * math.sqrt((g + 1) / (2 * g) * p / pL + (g - 1) / (2 * g))
                out[i] = (rhoL, uL, pL) if s <= SL else (
                    rhoL * ((p / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pL + 1)), us, p)
            else:
                cs = cL * (p / pL) ** ((g - 1) / (2 * g))
                if s <= uL - cL:
                    out[i] = (rhoL, uL, pL)
                elif s >= us - cs:
                    out[i] = (rhoL * (p / pL) ** (1 / g), us, p)
                else:
                    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    out[i] = (rhoL * (c / cL) ** (2 / (g - 1)), 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s),
                              pL * (c / cL) ** (2 * g / (g - 1)))
        else:
            if p > pR:
                SR = uR + cR * math.sqrt((g + 1) / (2 * g) * p / pR + (g - 1) / (2 * g))
                out[i] = (rhoR, uR, pR) if s >= SR else (
                    rhoR * ((p / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pR + 1)), us, p)
            else:
                cs = cR * (p / pR) ** ((g - 1) / (2 * g))
                if s >= uR + cR:
                    out[i] = (rhoR, uR, pR)
                elif s <= us + cs:
                    out[i] = (rhoR * (p / pR) ** (1 / g), us, p)
                else:
                    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    out[i] = (rhoR * (c / cR) ** (2 / (g - 1)), 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s),
                              pR * (c / cR) ** (2 * g / (g - 1)))
    return out


def _run(o, U, dx, tend, cfl=0.5, bc=(0, 0)):
    t = 0.0
    while t < tend * (1 - 1e-12):
        dt = min(cfl * dx / o.euler1d_max_speed(U), tend - t)
        rc, U = o.euler1d_step(U, dx, dt, bc)
        assert rc == 0
        t += dt
    return U


def test_exact_riemann_solver_sanity():
    # the textbook Sod values: p* = 0.30313, u* = 0.92745, rho*L = 0.42632, rho*R = 0.26557
    s = exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4, [0.5, 1.2])
    assert s[0][2] == pytest.approx(0.30313, abs=2e-5) and s[0][1] == pytest.approx(0.92745, abs=2e-5)
    assert s[0][0] == pytest.approx(0.42632, abs=2e-5) and s[1][0] == pytest.approx(0.26557, abs=2e-5)


def test_sod_against_exact_solution():
    m = _inert()
    o = oracle.Oracle(m)
    Rg = R_U / 0.028
    errs = []
    for n in (200, 400):
        x = (np.arange(n) + 0.5) / n
        rho = np.where(x < 0.5, 1.0, 0.125)
        p = np.where(x < 0.5, 1e5, 1e4)
        U = o.conserved_from_prim(rho, np.zeros(n), p / (rho * Rg), np.ones((1, n)))
        tend = 5e-4
        U = _run(o, U, 1.0 / n, tend)
        ex = exact_riemann(1.0, 0.0, 1e5, 0.125, 0.0, 1e4, 1.4, (x - 0.5) / tend)
        errs.append(np.mean(np.abs(U["rho"] - ex[:, 0])))
        u = U["rhou"] / U["rho"]
        assert np.mean(np.abs(u - ex[:, 1])) <= 0.03 * np.max(np.abs(ex[:, 1]))
    assert errs[1] <= 8e-3, errs
    assert errs[1] <= 0.7 * errs[0], errs


def _random_mixture(n, seed):
    mech = M.build(0)
    r = W.reactors(n, seed=seed)
    x = np.linspace(0.0, 2 * np.pi, n)
    T = 1100.0 + 150.0 * np.sin(x)
    rho = 1.0 + 0.2 * np.cos(2 * x)
    u = 50.0 * np.sin(3 * x)
    return mech, rho, u, T, r["Y"]


def test_reflecting_box_conserves():
    mech, rho, u, T, Y = _random_mixture(128, 3)
    o = oracle.Oracle(mech)
    U0 = o.conserved_from_prim(rho, u, T, Y)
    U = _run(o, dict(U0), 1e-3, 2e-5, bc=(1, 1))
    assert np.sum(U["rho"]) == pytest.approx(np.sum(U0["rho"]), rel=1e-13)
    assert np.sum(U["rhoE"]) == pytest.approx(np.sum(U0["rhoE"]), rel=1e-13)
    np.testing.assert_allclose(U["rhoY"].sum(axis=1), U0["rhoY"].sum(axis=1), rtol=1e-13)
    assert np.max(np.abs(U["rho"] - U0["rho"])) > 1e-3  # the flow did move


def test_free_stream_preserved():
    mech = M.build(0)
    o = oracle.Oracle(mech)
    n = 64
    Y = np.repeat(W.reactors(1, seed=1)["Y"], n, axis=1)
    U0 = o.conserved_from_prim(np.full(n, 0.8), np.full(n, 120.0), np.full(n, 1400.0), Y)
    rc, U = o.euler1d_step(U0, 1e-3, 1e-7)
    assert rc == 0
    for k in ("rho", "rhou", "rhoE", "rhoY"):
        np.testing.assert_allclose(U[k], U0[k], rtol=1e-13)


def test_strang_at_rest_is_two_chemistry_half_steps():
    mech = M.build(0)
    o = oracle.Oracle(mech)
    n = 16
    r = W.reactors(1, seed=2)
    Y = np.repeat(r["Y"], n, axis=1)
    T = np.full(n, 1500.0)
    rho = np.full(n, 0.5)
    U0 = o.conserved_from_prim(rho, np.zeros(n), T, Y)
    rc, U = o.strang_step(U0, 1e-3, 2e-6)
    assert rc == 0
    e = U0["rhoE"] / rho
    a = o.integrate(rho, e, Y, T, 1e-6)
    b = o.integrate(rho, e, a["Y"], a["T"], 1e-6)
    np.testing.assert_allclose(U["rhoY"] / rho, b["Y"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(U["rhoE"], U0["rhoE"], rtol=1e-15)
    assert np.max(np.abs(b["Y"] - Y)) > 1e-6  # the chemistry did act


def test_strang_second_order_in_time():
    mech, rho, u, T, Y = _random_mixture(48, 5)
    T = T + 400.0                                  # reacting over the interval
    o = oracle.Oracle(mech)
    U0 = o.conserved_from_prim(rho, u, T, Y)
    dx, tend = 2e-3, 2e-6

    def run(nsteps):
        U = dict(U0)
        for _ in range(nsteps):
            rc, U = o.strang_step(U, dx, tend / nsteps, rtol=1e-11, atol=1e-16)
            assert rc == 0
        return U

    ref = run(64)
    e = [np.max(np.abs(run(k)["rhoY"] - ref["rhoY"])) for k in (4, 8)]
    assert 3.0 < e[0] / e[1] < 5.5, e
