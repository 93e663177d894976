"""Equilibrium exponents of the mixed-precision right-hand sides against the oracle.

The reverse rate of each reversible reaction is k_r = k_f / K_c (Sec. 2.2.3), with
ln(1 / K_c,j) = sum_k nu_jk g_k / (R_u T) + (sum_k nu_jk) ln(R_u T / p_ref).  The mixed
variant evaluates the Gibbs functions and ln T in fp64 and adds them as fp32 hi/lo pairs
(the hi parts on a 2^-12 grid, whose sums are exact), so its ln(1 / K_c) is the fp64 sum
rounded once to fp32 up to the lo parts' own rounding.  The error test's all-fp32 form is
an estimator and only has to stay within a loose multiple of the fp32 rounding of its
terms.  The oracle's value is ln(k_r / k_f) of its fp64 rate coefficients, over
300-3500 K and on both sides of the NASA-7 range switch.
"""
import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
# lo parts: the split truncates each fp64 term to the 2^-12 grid, so |lo| < 2^-12, carried
# with relative error 2^-24; at most five of them (two products, two reactants,
# ln(R_u T / p_ref)) are summed in fp32
LO_ABS = 5 * 2.0 ** -36 + 4 * U32 * 5 * 2.0 ** -12
FP64_ABS = 1e-12  # the two sides' fp64 evaluation orders of the Gibbs sums


def _temperatures(mech):
    t_mid = float(mech["T_mid"][0])
    edge = [np.nextafter(t_mid, 0.0), t_mid, np.nextafter(t_mid, 1e9)]
    return np.concatenate([np.linspace(300.0, 3500.0, 3201), edge])


def _oracle_ln_inv_kc(O, mech, T):
    R = len(mech["A"])
    c = np.full(len(mech["W"]), 1.0)
    out = np.full((T.size, R), np.nan)
    for i, t in enumerate(T):
        kf, kr = O.rate_constants(float(t), c)
        with np.errstate(divide="ignore"):
            out[i] = np.log(kr) - np.log(kf)
    return out


def _term_sums(mech, T):
    """Sum of |terms| of g_k / (R_u T) in the NASA-7 form, [n, S]: the scale of each
    species' fp32 evaluation error."""
    lo, hi = np.asarray(mech["nasa_lo"]), np.asarray(mech["nasa_hi"])
    t_mid = float(mech["T_mid"][0])
    a = np.where((T >= t_mid)[:, None, None], hi[None], lo[None])
    t = T[:, None]
    terms = [a[..., 0] * (1.0 - np.log(t)), a[..., 1] * t / 2, a[..., 2] * t ** 2 / 6,
             a[..., 3] * t ** 3 / 12, a[..., 4] * t ** 4 / 20, a[..., 5] / t, a[..., 6]]
    return sum(np.abs(x) for x in terms)


@pytest.fixture(scope="module", params=[9, 13], ids=["h2o2_9", "h2o2_13"])
def case(request):
    import torch
    from paper_2506_02602_gb300 import chem
    mech = M.build(0) if request.param == 9 else M.build13(0)
    T = _temperatures(mech)
    ctx = chem.Context(mech, variant="mixed")
    Td = torch.tensor(T, dtype=torch.float64, device="cuda")
    got = {f: ctx.ln_inv_kc(Td, form=f).cpu().numpy() for f in (0, 1)}
    ctx.close()
    ref = _oracle_ln_inv_kc(oracle.Oracle(mech), mech, T)
    rev = np.asarray(mech["reversible"]).astype(bool)
    return mech, T, got, ref, rev


def test_mixed_form_is_the_fp64_sum_rounded_once(case):
    mech, T, got, ref, rev = case
    g, r = got[0][:, rev], ref[:, rev]
    ok = np.isfinite(r)
    assert ok.mean() > 0.99, "oracle rate coefficients under/overflowed on too many points"
    err = np.abs(g - r)[ok]
    tol = U32 * np.abs(r[ok]) + LO_ABS + FP64_ABS
    assert np.all(err <= tol), f"worst ratio {np.max(err / tol):.3g}"
    # beyond the one fp32 rounding of the result, what is left is the lo parts' error
    excess = err - U32 * np.abs(r[ok])
    print(f"\nln(1/Kc) mixed: max |err| {err.max():.3g}, max beyond one fp32 rounding "
          f"{max(excess.max(), 0.0):.3g}, max |ln(1/Kc)| {np.abs(r[ok]).max():.3g}")


def test_all_fp32_form_within_its_estimator_bound(case):
    mech, T, got, ref, rev = case
    nu = np.abs(np.asarray(mech["nu_r"]) - np.asarray(mech["nu_f"])).astype(np.float64)
    dnu = np.abs((np.asarray(mech["nu_r"]) - np.asarray(mech["nu_f"])).sum(axis=1)).astype(np.float64)
    scale = _term_sums(mech, T) @ nu.T + dnu[None] * (np.abs(np.log(T))[:, None] + 30.0)
    g, r, s = got[1][:, rev], ref[:, rev], scale[:, rev]
    ok = np.isfinite(r)
    err = np.abs(g - r)[ok]
    tol = 64 * U32 * s[ok]
    assert np.all(err <= tol), f"worst ratio {np.max(err / tol):.3g}"
    print(f"\nln(1/Kc) fp32: max |err| {err.max():.3g}, max err / scale {np.max(err / s[ok]):.3g}")


def test_every_exponent_is_finite(case):
    """Irreversible reactions' exponents are formed too (they are never used); both forms
    give finite values for every reaction at every temperature."""
    _, _, got, _, _ = case
    assert np.isfinite(got[0]).all() and np.isfinite(got[1]).all()
