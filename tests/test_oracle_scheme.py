"""Pins of the oracle's integrator against what the scheme fixes (Sec. 2.2.3, Eq. 21-22).

* the coefficients it uses are the published rationals of RK4(3)5[2R+]C, which satisfy
  every order condition up to order 4 (main) / 3 (embedded) to far below fp64 rounding;
* one step on y' = lambda y equals R(h lambda) y, with R the stability polynomial of
  the exact tableau, and the error register equals (R - Rhat)(h lambda) y;
* the adaptive trajectory on y' = lambda y follows Eq. 22 exactly;
* fixed-step convergence slopes are 4 (main) and 3 (embedded) on y' = -y^2.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from tests import _tableau

TAB = _tableau.load()


def test_coefficients_are_the_published_rationals():
    a, b, bh = oracle.lsrk_coefficients()
    for x, q in zip(a, TAB["sub"]):
        assert x == float(q)
    for x, q in zip(b, TAB["b"]):
        assert x == float(q)
    for x, q in zip(bh, TAB["bh"]):
        assert x == float(q)


def test_order_conditions_exact():
    A, c = TAB["A"], TAB["c"]
    rb = _tableau.order_residuals(TAB["b"], A, c)
    for k, v in rb.items():
        assert abs(v) < Fr(1, 10 ** 20), (k, float(v))
    rh = _tableau.order_residuals(TAB["bh"], A, c)
    for k in ("1", "c", "c2", "Ac"):
        assert abs(rh[k]) < Fr(1, 10 ** 20), (k, float(rh[k]))
    # the embedded scheme is genuinely third order: some order-4 condition fails
    assert max(abs(rh[k]) for k in ("c3", "cAc", "Ac2", "AAc")) > Fr(1, 1000)
    # the row sums are the published abscissae c = (0, 0.22502, 0.59527, 0.57675, 0.84550)
    np.testing.assert_allclose([float(x) for x in c], [0, 0.22502, 0.59527, 0.57675, 0.84550],
                               atol=1e-5)


def test_stability_polynomial_coefficients():
    # R(z) = sum_k z^k / k! up to k = 4; z^5 coefficient b^T A^4 1 ~ 1/206
    A, b = TAB["A"], TAB["b"]
    v = [Fr(1)] * 5
    coefs = []
    for _ in range(5):
        coefs.append(sum(b[i] * v[i] for i in range(5)))
        v = [sum(A[i][j] * v[j] for j in range(5)) for i in range(5)]
    for k, (cf, fact) in enumerate(zip(coefs, [1, 2, 6, 24])):
        assert abs(cf - Fr(1, fact)) < Fr(1, 10 ** 20)
    assert abs(float(1 / coefs[4]) - 206.0) < 1e-9


@pytest.mark.parametrize("z", [-0.3, -1.0, -2.5, -4.0, 0.7])
def test_one_step_real_linear(z):
    lam = -1234.5
    h = z / lam
    y0 = 0.731
    y, E = oracle.linear_step(np.array([[lam]]), h, np.array([y0]))
    zf = Fr(h) * Fr(lam)
    R = _tableau.stability(zf, TAB["b"], TAB["A"])
    Rh = _tableau.stability(zf, TAB["bh"], TAB["A"])
    assert y[0] == pytest.approx(float(R * Fr(y0)), rel=1e-14, abs=1e-300)
    assert E[0] == pytest.approx(float((R - Rh) * Fr(y0)), rel=1e-9, abs=1e-16)


@pytest.mark.parametrize("z", [complex(-1.0, 1.5), complex(-0.2, 2.8), complex(-3.0, 0.5)])
def test_one_step_complex_linear(z):
    # y' = lambda y with complex lambda, as the real 2x2 system [[re, -im], [im, re]]
    h = 1e-3
    lam = z / h
    M = np.array([[lam.real, -lam.imag], [lam.imag, lam.real]])
    y0 = complex(0.6, -0.3)
    y, E = oracle.linear_step(M, h, np.array([y0.real, y0.imag]))
    # exact stability polynomial in complex arithmetic: evaluate coefficients exactly, then z
    A, b, bh = TAB["A"], TAB["b"], TAB["bh"]

    def R_complex(w):
        v = [Fr(1)] * 5
        val = complex(1.0)
        zk = complex(1.0)
        for _ in range(5):
            zk = zk * (h * lam)
            val += float(sum(w[i] * v[i] for i in range(5))) * zk
            v = [sum(A[i][j] * v[j] for j in range(5)) for i in range(5)]
        return val

    expect = R_complex(b) * y0
    err = (R_complex(b) - R_complex(bh)) * y0
    assert abs(complex(y[0], y[1]) - expect) < 1e-14 * abs(expect)
    assert abs(complex(E[0], E[1]) - err) < 1e-12 * abs(y0)


def _controller_reference(lam, y0, dt, rtol, atol, h0=None, max_steps=10000):
    """Eq. 22 trajectory on the scalar y' = lam y from the exact stability polynomials."""
    t, h, y = 0.0, (h0 or dt), y0
    hs, acc = [], []
    while dt - t > 1e-12 * dt and len(hs) < max_steps:
        h = min(h, dt - t)
        zf = Fr(h) * Fr(lam)
        R = float(_tableau.stability(zf, TAB["b"], TAB["A"]))
        Rh = float(_tableau.stability(zf, TAB["bh"], TAB["A"]))
        ynew = R * y
        e = (R - Rh) * y
        err = abs(e) / (rtol * max(abs(y), abs(ynew)) + atol)
        fac = 5.0 if err == 0 else min(5.0, max(0.2, 0.9 * (1.0 / err) ** 0.25))
        hs.append(h)
        acc.append(err <= 1.0)
        if err <= 1.0:
            t += h
            y = ynew
        h *= fac
    return np.array(hs), np.array(acc), y


# lam * dt stays near -20 or above: far deeper decay puts y below atol, where every step
# sits on the stability boundary and accept/reject becomes a rounding coin-flip.
@pytest.mark.parametrize("lam,dt,rtol,atol", [(-1e3, 1e-2, 1e-6, 1e-10), (-5e4, 4e-4, 1e-4, 1e-8),
                                              (-10.0, 1e-2, 1e-8, 1e-12), (-2e5, 1e-4, 1e-6, 1e-10)])
def test_controller_trajectory_linear(lam, dt, rtol, atol):
    y0 = 1.0
    out = oracle.linear_integrate(np.array([[lam]]), np.array([y0]), dt, rtol, atol)
    hs, acc, y = _controller_reference(lam, y0, dt, rtol, atol)
    assert out["status"] == 0
    assert len(out["h"]) == len(hs)
    np.testing.assert_array_equal(out["acc"], acc)
    # E = (R - Rhat) y is a small difference of O(1) numbers, so its float value carries
    # ~1e-16 / (rtol) relative rounding; h follows err^(-1/4): 1e-6 bounds the drift, a
    # logic error moves h by O(1).
    np.testing.assert_allclose(out["h"], hs, rtol=1e-6)
    assert out["y"][0] == pytest.approx(y, rel=1e-8, abs=1e-300)
    # the controller both rejects and grows on this problem
    assert acc.sum() > 0


def _controller_reference_diag(lams, y0, dt, rtol, atol, max_steps=10000):
    """Eq. 22 trajectory on the diagonal system y_i' = lam_i y_i: WRMS over the n
    components with |u_i| = max(|y_n,i|, |y_n+1,i|)."""
    lams, y = np.asarray(lams, float), np.asarray(y0, float).copy()
    t, h = 0.0, dt
    hs, acc = [], []
    while dt - t > 1e-12 * dt and len(hs) < max_steps:
        h = min(h, dt - t)
        R = np.array([float(_tableau.stability(Fr(h) * Fr(l), TAB["b"], TAB["A"])) for l in lams])
        Rh = np.array([float(_tableau.stability(Fr(h) * Fr(l), TAB["bh"], TAB["A"])) for l in lams])
        ynew = R * y
        e = (R - Rh) * y
        w = e / (rtol * np.maximum(np.abs(y), np.abs(ynew)) + atol)
        err = np.sqrt(np.mean(w * w))
        fac = 5.0 if err == 0 else min(5.0, max(0.2, 0.9 * (1.0 / err) ** 0.25))
        hs.append(h)
        acc.append(err <= 1.0)
        if err <= 1.0:
            t += h
            y = ynew
        h *= fac
    return np.array(hs), np.array(acc), y


def test_controller_trajectory_diagonal_system():
    # one growing component that dominates the error norm (so the max(|y_n|, |y_n+1|)
    # weight picks y_n+1) and three decaying ones (where it picks y_n); the mean over n
    # and both weights shape the step sequence
    lams = [2000.0, -300.0, -50.0, -800.0]
    y0 = [1.0, 1.0, 0.5, 0.1]
    dt, rtol, atol = 2e-3, 1e-6, 1e-10
    out = oracle.linear_integrate(np.diag(lams), np.array(y0), dt, rtol, atol)
    hs, acc, y = _controller_reference_diag(lams, y0, dt, rtol, atol)
    assert out["status"] == 0
    assert len(out["h"]) == len(hs)
    np.testing.assert_array_equal(out["acc"], acc)
    np.testing.assert_allclose(out["h"], hs, rtol=1e-6)
    np.testing.assert_allclose(out["y"], y, rtol=1e-8)


def test_controller_rejects_then_shrinks():
    # a first step far beyond the stability limit must be rejected and shrunk by 1/5
    out = oracle.linear_integrate(np.array([[-1e6]]), np.array([1.0]), 1e-4, 1e-6, 1e-10)
    assert not out["acc"][0]
    assert out["h"][1] == pytest.approx(0.2 * out["h"][0], rel=1e-15)
    assert out["status"] == 0


def test_step_limits_report_status():
    # max-steps limit
    out = oracle.linear_integrate(np.array([[-1e3]]), np.array([1.0]), 1.0, 1e-10, 1e-14, max_steps=5)
    assert out["status"] == 1 and out["nacc"] + out["nrej"] == 5


@pytest.mark.parametrize("embedded,order", [(False, 4.0), (True, 3.0)])
def test_convergence_order_quadratic(embedded, order):
    # y' = -y^2, y(0) = 1 -> y(1) = 1/2
    errs = []
    Ns = [8, 16, 32, 64]
    for N in Ns:
        y = oracle.quadratic_fixed(1.0, 1.0 / N, N, embedded)
        errs.append(abs(y - 0.5))
    slopes = -np.diff(np.log(errs)) / np.log(2.0)
    assert abs(slopes[-1] - order) < 0.1, slopes
    assert abs(slopes[-2] - order) < 0.15, slopes
