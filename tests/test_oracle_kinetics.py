"""Pins of the oracle's kinetics (Eq. 15-16, Sec. 2.1.2; third-body and fall-off forms).

* every reaction of the synthetic mechanism balances the elements (integer check), so
  the production rates conserve elements and mass: sum_k n_ke wdot_k = 0 and
  sum_k W_k wdot_k = 0;
* the Arrhenius form is recovered by regression of ln k on (1, ln T, 1/T);
* Lindemann limits k -> k0 [M] and k -> k_inf; Troe F equals F_cent at the centre of
  the fall-off curve and reduces to alpha when T*** -> 0, T* -> inf;
* [M] with unit efficiencies is the total concentration p / (R_u T);
* an isomerisation A <=> B with equal enthalpies relaxes in closed form, with
  K_c = exp(Delta s / R);
* a dissociation H2 <=> 2H reaches the ideal-gas chemical-potential balance
  mu_H2 = 2 mu_H, which fixes the (p_ref / R_u T)^(sum nu) factor of K_c.
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


def _random_states(n, seed):
    rng = np.random.default_rng(seed)
    r = W.reactors(n, seed=seed)
    Y = r["Y"].copy()
    Y[3:8] += rng.uniform(0.0, 0.03, (5, n))
    Y /= Y.sum(axis=0, keepdims=True)
    T = rng.uniform(600.0, 3200.0, n)
    rho = rng.uniform(0.05, 5.0, n)
    return rho, T, Y


def test_element_balance_every_reaction():
    nu = MECH["nu_r"] - MECH["nu_f"]
    np.testing.assert_array_equal(nu @ MECH["ncomp"], 0)
    # the structure of a 9-species / 21-reaction H2-O2 mechanism
    assert nu.shape == (21, 9)
    assert (MECH["rtype"] == 1).sum() == 4 and (MECH["rtype"] == 2).sum() == 2


def test_wdot_conserves_elements_and_mass():
    rho, T, Y = _random_states(200, 21)
    for i in range(200):
        w = O.wdot(rho[i], T[i], Y[:, i])
        scale_e = np.abs(w)[:, None] * MECH["ncomp"]
        assert np.all(np.abs(MECH["ncomp"].T @ w) <= 1e-12 * scale_e.sum(axis=0) + 1e-300)
        assert abs(MECH["W"] @ w) <= 1e-12 * (MECH["W"] @ np.abs(w)) + 1e-300
        assert np.any(w != 0.0)


def _one_reaction(rx, species=("H", "O2", "O", "OH")):
    idx = [M.SPECIES.index(s) for s in species]
    sub = {i: j for j, i in enumerate(idx)}
    r = dict(rx)
    r["nu_f"] = {sub[k]: v for k, v in rx["nu_f"].items()}
    r["nu_r"] = {sub[k]: v for k, v in rx["nu_r"].items()}
    if "eff" in rx:
        r["eff"] = {sub[k]: v for k, v in rx["eff"].items()}
    return M.custom(list(species), MECH["W"][idx], MECH["ncomp"][idx], MECH["nasa_lo"][idx],
                    MECH["nasa_hi"][idx], [r])


def test_arrhenius_regression():
    H, O2, Ox, OH = (M.SPECIES.index(s) for s in ("H", "O2", "O", "OH"))
    A, b, Ea = 3.7e8, 0.63, 71234.0
    mech = _one_reaction({"nu_f": {H: 1, O2: 1}, "nu_r": {Ox: 1, OH: 1}, "A": A, "b": b, "Ea": Ea,
                          "reversible": False})
    o = oracle.Oracle(mech)
    Ts = np.linspace(700.0, 3000.0, 25)
    lnk = np.array([np.log(o.rate_constants(T, np.ones(4))[0][0]) for T in Ts])
    X = np.stack([np.ones_like(Ts), np.log(Ts), 1.0 / Ts], axis=1)
    coef, *_ = np.linalg.lstsq(X, lnk, rcond=None)
    assert np.exp(coef[0]) == pytest.approx(A, rel=1e-8)
    assert coef[1] == pytest.approx(b, rel=1e-9)
    assert -coef[2] * R_U == pytest.approx(Ea, rel=1e-9)


def _falloff_mech(troe=()):
    H, O2, HO2 = (M.SPECIES.index(s) for s in ("H", "O2", "HO2"))
    return _one_reaction({"nu_f": {H: 1, O2: 1}, "nu_r": {HO2: 1}, "type": "troe", "A": 5.0e6,
                          "A0": 2.0e3, "troe": troe, "reversible": False},
                         species=("H", "O2", "HO2"))


def test_lindemann_limits():
    o = oracle.Oracle(_falloff_mech())
    A_inf, A0 = 5.0e6, 2.0e3
    for Mc in (1e-6, 1e-4):
        kf = o.rate_constants(1500.0, np.array([Mc / 3] * 3))[0][0]
        Pr = A0 * Mc / A_inf  # k = k0 [M] / (1 + Pr): relative deviation Pr
        assert kf == pytest.approx(A0 * Mc, rel=2.0 * Pr)
        assert kf < A0 * Mc
    kf = o.rate_constants(1500.0, np.array([1e12] * 3))[0][0]
    assert kf == pytest.approx(A_inf, rel=1e-8)
    # exactly in between: Pr = 1 gives k_inf / 2
    Mc = A_inf / A0
    kf = o.rate_constants(1500.0, np.array([Mc / 3] * 3))[0][0]
    assert kf == pytest.approx(A_inf / 2, rel=1e-12)


@pytest.mark.parametrize("alpha", [0.3, 0.55, 0.8])
def test_troe_centre_and_fcent_reduction(alpha):
    o = oracle.Oracle(_falloff_mech(troe=(alpha, 1e-30, 1e30)))
    # F_cent = alpha; at log10 Pr = -c = 0.4 + 0.67 log10 F_cent the Troe factor is F_cent
    Pr = 10.0 ** (0.4 + 0.67 * np.log10(alpha))
    assert o.troe_F(0, 1700.0, Pr) == pytest.approx(alpha, rel=1e-13)
    # away from the centre the broadening factor moves toward 1 but stays below it
    for Pr2 in (Pr * 1e-3, Pr * 1e3):
        F = o.troe_F(0, 1700.0, Pr2)
        assert alpha < F < 1.0


@pytest.mark.parametrize("alpha,T3,T1,T2,fcent", [
    (0.0, 180.0, 1e30, 0.0, lambda T: np.exp(-T / 180.0)),      # T*** term alone
    (1.0, 1e-30, 2500.0, 0.0, lambda T: np.exp(-T / 2500.0)),   # T* term alone
    (0.0, 1e-30, 1e30, 5000.0, lambda T: np.exp(-5000.0 / T)),  # T** term alone
])
def test_troe_fcent_terms(alpha, T3, T1, T2, fcent):
    troe = (alpha, T3, T1, T2) if T2 else (alpha, T3, T1)
    o = oracle.Oracle(_falloff_mech(troe=troe))
    for T in (800.0, 1600.0, 2600.0):
        Fc = fcent(T)
        Pr = 10.0 ** (0.4 + 0.67 * np.log10(Fc))
        assert o.troe_F(0, T, Pr) == pytest.approx(Fc, rel=1e-12)


@pytest.mark.parametrize("alpha", [0.35, 0.7])
def test_troe_half_width(alpha):
    # the broadening term f1 = x / (n - 0.14 x), x = log10 Pr + c, reaches 1 (F = sqrt(F_cent))
    # at x = n / 1.14 above the centre and -1 at x = -n / 0.86 below it
    o = oracle.Oracle(_falloff_mech(troe=(alpha, 1e-30, 1e30)))
    lf = np.log10(alpha)
    c, n = -0.4 - 0.67 * lf, 0.75 - 1.27 * lf
    for x in (n / 1.14, -n / 0.86):
        assert o.troe_F(0, 1500.0, 10.0 ** (x - c)) == pytest.approx(np.sqrt(alpha), rel=1e-12)


def test_third_body_zero_efficiency_species():
    H, H2, N2 = (M.SPECIES.index(s) for s in ("H", "H2", "N2"))
    sp = ("H", "H2", "N2")
    tb = _one_reaction({"nu_f": {H: 2}, "nu_r": {H2: 1}, "type": "tb", "A": 1e2, "b": -1.0,
                        "eff": {N2: 0.0}, "reversible": True}, species=sp)
    el = _one_reaction({"nu_f": {H: 2}, "nu_r": {H2: 1}, "type": "elem", "A": 1e2, "b": -1.0,
                        "reversible": True}, species=sp)
    otb, oel = oracle.Oracle(tb), oracle.Oracle(el)
    T, p = 1900.0, 2.0 * P_REF
    X = np.array([0.02, 0.28, 0.70])
    Y = (X * MECH["W"][[H, H2, N2]] / (X * MECH["W"][[H, H2, N2]]).sum())[:, None]
    rho, _ = otb.state_from_TPY(np.array([T]), np.array([p]), Y)
    ratio = otb.wdot(rho[0], T, Y[:, 0])[:2] / oel.wdot(rho[0], T, Y[:, 0])[:2]
    # [M] excludes N2: total concentration times (1 - X_N2)
    np.testing.assert_allclose(ratio, p / (R_U * T) * (1.0 - X[2]), rtol=1e-12)


def test_third_body_unit_efficiency_is_total_concentration():
    H, H2, N2 = (M.SPECIES.index(s) for s in ("H", "H2", "N2"))
    sp = ("H", "H2", "N2")
    tb = _one_reaction({"nu_f": {H: 2}, "nu_r": {H2: 1}, "type": "tb", "A": 1e2, "b": -1.0,
                        "reversible": True}, species=sp)
    el = _one_reaction({"nu_f": {H: 2}, "nu_r": {H2: 1}, "type": "elem", "A": 1e2, "b": -1.0,
                        "reversible": True}, species=sp)
    otb, oel = oracle.Oracle(tb), oracle.Oracle(el)
    T, p = 2200.0, 3.3 * P_REF
    Y = np.array([[0.01], [0.2], [0.79]])
    rho, _ = otb.state_from_TPY(np.array([T]), np.array([p]), Y)
    wt = otb.wdot(rho[0], T, Y[:, 0])
    we = oel.wdot(rho[0], T, Y[:, 0])
    assert wt[2] == 0.0 and we[2] == 0.0  # N2 is inert
    np.testing.assert_allclose(wt[:2] / we[:2], p / (R_U * T), rtol=1e-12)


def _isomer_mech(delta_s, A):
    a = MECH["nasa_lo"][M.SPECIES.index("OH")].copy()
    ah = MECH["nasa_hi"][M.SPECIES.index("OH")].copy()
    b_lo, b_hi = a.copy(), ah.copy()
    b_lo[6] += delta_s
    b_hi[6] += delta_s
    return M.custom(["A", "B"], [0.017007, 0.017007], [[1, 1, 0], [1, 1, 0]],
                    [a, b_lo], [ah, b_hi],
                    [{"nu_f": {0: 1}, "nu_r": {1: 1}, "A": A, "b": 0.0, "Ea": 0.0}])


@pytest.mark.parametrize("delta_s", [0.7, -1.3])
def test_isomerisation_relaxation_closed_form(delta_s):
    A = 2.0e5
    o = oracle.Oracle(_isomer_mech(delta_s, A))
    Kc = np.exp(delta_s)
    kf, kr = A, A / Kc
    Yeq = kr / (kf + kr)
    T0, p = 1300.0, P_REF
    Y0 = np.array([[0.9], [0.1]])
    rho, e = o.state_from_TPY(np.array([T0]), np.array([p]), Y0)
    for t in (2e-6, 5e-6, 1.5e-5):
        out = o.integrate(rho, e, Y0, np.array([T0]), t, rtol=1e-10, atol=1e-14)
        YA = Yeq + (0.9 - Yeq) * np.exp(-(kf + kr) * t)
        assert out["status"][0] == 0
        assert out["Y"][0, 0] == pytest.approx(YA, rel=1e-8)
        assert out["T"][0] == pytest.approx(T0, rel=1e-12)


def test_dissociation_chemical_potential_balance():
    H, H2, N2 = (M.SPECIES.index(s) for s in ("H", "H2", "N2"))
    sp = ("H2", "H", "N2")
    mech = _one_reaction({"nu_f": {H2: 1}, "nu_r": {H: 2}, "A": 1e9, "b": 0.0, "Ea": 0.0},
                         species=sp)
    o = oracle.Oracle(mech)
    T0, p = 3600.0, 0.2 * P_REF
    Y0 = np.array([[0.3], [0.0], [0.7]])
    rho, e = o.state_from_TPY(np.array([T0]), np.array([p]), Y0)
    out = o.integrate(rho, e, Y0, np.array([T0]), 2e-6, rtol=1e-10, atol=1e-16)
    assert out["status"][0] == 0
    T = out["T"][0]
    Wk = MECH["W"][[H2, H, N2]]
    c = rho[0] * out["Y"][:, 0] / Wk
    mu = [o.h_RT(k, T) - o.s_R(k, T) + np.log(c[k] * R_U * T / P_REF) for k in range(2)]
    assert mu[0] == pytest.approx(2.0 * mu[1], abs=1e-7)
    # and the dissociation cooled the gas (endothermic), as energy conservation demands
    assert T < T0 - 10.0
