"""Pins of the surrogate's FP64 CPU reference (oracle/mlp.py).

* gradients of the MSE loss for every weight and bias match central finite differences;
* GELU: GELU(x) - GELU(-x) = x (Phi(x) + Phi(-x) = 1), GELU(0) = 0, derivative by finite
  differences, asymptotes GELU(x) -> x and -> 0;
* Box-Cox: the inverse undoes the transform, and small lam gives ln y + lam ln^2 y / 2;
* forward: a hand-built 2-3-3-1 network whose hidden pre-activations land on 0, +-1, 2
  and +-10, so the output is a closed form in the normal-table values Phi(1), Phi(2)
  (a dropped bias, a transposed hidden weight or a GELU on the output layer each change
  it by far more than rounding);
* Adam: the first bias-corrected step is lr * sign(g) (up to eps), and with a constant
  gradient every later step is lr * sign(g) as well (the bias corrections undo the
  moments' warm-up exactly);
* projection: E Y'' = E Y0 to rounding, idempotent, and the correction is the weighted
  least-squares one (KKT stationarity: (Y'' - Y') / w lies in the row space of E).
"""
import math

import numpy as np
import pytest

from chem_inputs import mechanism as M
from oracle import mlp

SIZES = [12, 7, 6, 5, 9]


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = mlp.init_params(SIZES, seed=2)
    for p in params:
        p["b"] = rng.standard_normal(p["b"].shape) * 0.1
    x = rng.standard_normal((11, 12))
    t = rng.standard_normal((11, 9))

    def loss():
        y, _ = mlp.forward(params, x)
        return mlp.mse(y, t)[0]

    y, pre = mlp.forward(params, x)
    _, dy = mlp.mse(y, t)
    grads = mlp.backward(params, pre, dy)
    h = 1e-6
    for i, p in enumerate(params):
        for key in ("W", "b"):
            flat = p[key].reshape(-1)
            gflat = grads[i][key].reshape(-1)
            for j in rng.choice(flat.size, min(6, flat.size), replace=False):
                old = flat[j]
                flat[j] = old + h
                lp = loss()
                flat[j] = old - h
                lm = loss()
                flat[j] = old
                fd = (lp - lm) / (2 * h)
                assert gflat[j] == pytest.approx(fd, rel=1e-6, abs=1e-9), (i, key, j)


def test_gelu_identities():
    x = np.linspace(-6, 6, 241)
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-14)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([12.0]))[0] == pytest.approx(12.0, rel=1e-15)
    assert abs(mlp.gelu(np.array([-12.0]))[0]) < 1e-30
    h = 1e-5
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, rtol=1e-8, atol=1e-10)
    # GELU(1) = Phi(1) = (1 + erf(1/sqrt 2)) / 2
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)


def test_boxcox_inverse_and_log_limit():
    y = np.array([1e-20, 1e-10, 1e-4, 0.01, 0.3, 0.99, 1.0])
    for lam in (0.05, 0.1, 0.25):
        # conditioning 1/lam near y -> 0: (1 + lam z) carries ~1e-16, raised to 1/lam
        np.testing.assert_allclose(mlp.boxcox_inv(mlp.boxcox(y, lam), lam), y, rtol=1e-10)
    # small lam: (y^lam - 1)/lam = ln y + lam ln^2 y / 2 + O(lam^2)
    lam = 1e-6
    ly = np.log(y)
    np.testing.assert_allclose(mlp.boxcox(y, lam), ly + lam * ly ** 2 / 2, rtol=1e-8, atol=1e-9)


# standard normal distribution function, Abramowitz & Stegun Table 26.1
PHI_1 = 0.8413447460685429
PHI_2 = 0.9772498680518208


def _hand_network():
    """2 -> 3 -> 3 -> 1 with weights chosen so that, at x = (1, 2), the first hidden
    pre-activations are (0, 10, -10) and the second's are (1, -1, 2)."""
    W1 = np.array([[-2.0, 9.0, -11.0],
                   [0.5, 0.0, 0.0]])
    b1 = np.array([1.0, 1.0, 1.0])
    # rows = inputs of the layer: only row 1 meets a non-zero activation (GELU(10) = 10);
    # the matrix is not symmetric, so using its transpose changes the result
    W2 = np.array([[0.3, 0.7, -0.2],
                   [0.05, -0.15, 0.15],
                   [0.4, 0.9, 0.6]])
    b2 = np.array([0.5, 0.5, 0.5])
    W3 = np.array([[1.0], [2.0], [-1.0]])
    b3 = np.array([0.25])
    return [{"W": W1, "b": b1}, {"W": W2, "b": b2}, {"W": W3, "b": b3}]


def test_forward_closed_form():
    params = _hand_network()
    y, pre = mlp.forward(params, np.array([[1.0, 2.0]]))
    # hidden layer 1: z = (0, 10, -10); GELU(0) = 0, GELU(10) = 10 (Phi(10) = 1 - 7.6e-24),
    # GELU(-10) = -7.6e-23
    np.testing.assert_allclose(pre[0][1][0], [0.0, 10.0, -10.0], atol=1e-15)
    # hidden layer 2: z = 10 * (0.05, -0.15, 0.15) + 0.5 = (1, -1, 2)
    np.testing.assert_allclose(pre[1][1][0], [1.0, -1.0, 2.0], atol=1e-14)
    # output (no activation): GELU(1) + 2 GELU(-1) - GELU(2) + 1/4 with GELU(x) = x Phi(x)
    # and Phi(-1) = 1 - Phi(1)
    want = PHI_1 + 2.0 * (-(1.0 - PHI_1)) - 2.0 * PHI_2 + 0.25
    assert y.shape == (1, 1)
    assert y[0, 0] == pytest.approx(want, rel=1e-14, abs=1e-15)


def test_forward_closed_form_detects_plausible_mistakes():
    x = np.array([[1.0, 2.0]])
    want = mlp.forward(_hand_network(), x)[0][0, 0]
    bad = []
    p = _hand_network(); p[0]["b"] = np.zeros(3); bad.append(p)            # first bias dropped
    p = _hand_network(); p[1]["b"] = np.zeros(3); bad.append(p)            # hidden bias dropped
    p = _hand_network(); p[2]["b"] = np.zeros(1); bad.append(p)            # output bias dropped
    p = _hand_network(); p[1]["W"] = p[1]["W"].T.copy(); bad.append(p)     # transposed weight
    for q in bad:
        assert abs(mlp.forward(q, x)[0][0, 0] - want) > 1e-2
    # GELU applied after the output layer as well
    assert abs(mlp.gelu(np.array([want]))[0] - want) > 1e-2


def test_adam_constant_gradient_steps_are_sign_steps():
    params = [{"W": np.array([[1.0, -2.0]]), "b": np.array([0.5])}]
    grads = [{"W": np.array([[3.0, -0.25]]), "b": np.array([-7.0])}]
    st = {}
    step = lambda g: 0.01 * g / (abs(g) + 1e-8)  # lr mhat / (sqrt(vhat) + eps) at mhat = g
    for t in range(1, 6):
        mlp.adam_step(params, grads, st, lr=0.01)
        # m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so mhat = g and vhat = g^2
        np.testing.assert_allclose(params[0]["W"], [[1.0 - t * step(3.0), -2.0 - t * step(-0.25)]],
                                   rtol=1e-13)
        np.testing.assert_allclose(params[0]["b"], [0.5 - t * step(-7.0)], rtol=1e-13)


def test_adam_first_step_is_sign_step():
    params = [{"W": np.array([[1.0, -2.0]]), "b": np.array([0.5])}]
    grads = [{"W": np.array([[3.0, -0.25]]), "b": np.array([-7.0])}]
    st = {}
    mlp.adam_step(params, grads, st, lr=0.01)
    np.testing.assert_allclose(params[0]["W"], [[0.99, -1.99]], rtol=1e-9)
    np.testing.assert_allclose(params[0]["b"], [0.51], rtol=1e-9)


def test_projection_conserves_elements_and_is_least_squares():
    m = M.build(0)
    E = mlp.element_matrix(m["W"], m["ncomp"], [M.ATOMIC_MASS[e] for e in M.ELEMENTS])
    rng = np.random.default_rng(4)
    for _ in range(20):
        Y0 = rng.dirichlet(np.ones(9))
        Yp = np.clip(Y0 + 1e-3 * rng.standard_normal(9), 1e-9, None)
        Y2 = mlp.project(Yp, Y0, E)
        np.testing.assert_allclose(E @ Y2, E @ Y0, rtol=0, atol=1e-15)
        assert abs(Y2.sum() - Y0.sum()) < 1e-14   # element mass fractions sum to sum Y
        np.testing.assert_allclose(mlp.project(Y2, Y0, E), Y2, atol=1e-16)
        w = np.maximum(Yp, 1e-12)
        step = (Y2 - Yp) / w
        coef, *_ = np.linalg.lstsq(E.T, step, rcond=None)
        np.testing.assert_allclose(E.T @ coef, step, atol=1e-9 * max(1.0, np.abs(step).max()))
