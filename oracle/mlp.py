"""Plain FP64 CPU reference of the learned surrogate (test infrastructure only).

The paper proposes learning the chemical source term only as future work (Sec. 7); the
surrogate's definition here follows the benchmark specification: a multilayer perceptron
12 -> 256 -> 256 -> 256 -> 9 with GELU activations, trained with mean-squared error and
Adam on (state, dt) -> state pairs produced by the integrator, whose inputs and outputs
use Box-Cox-transformed mass fractions, followed by a projection that restores element
conservation.  Each function here is the textbook definition written out in numpy fp64:

  GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2              (Hendrycks & Gimpel 2016)
  Box-Cox(y) = (y^lam - 1) / lam                                (Box & Cox 1964)
  Adam: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
        w <- w - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)  (Kingma & Ba 2015)
  projection: the Y'' closest to Y' in the norm sum_k d_k^2 / w_k with E Y'' = E Y0,
        Y'' = Y' - W E^T (E W E^T)^{-1} (E Y' - E Y0)            (weighted least squares)

No blocking or fusion: a numpy matmul is one step.
"""
from __future__ import annotations

import math

import numpy as np

SQRT1_2 = 1.0 / math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)
_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x * SQRT1_2))


def gelu_grad(x):
    """d GELU / dx = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + _erf(x * SQRT1_2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def init_params(sizes, seed=0):
    """He-style initialisation (normal, std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        params.append({"W": rng.standard_normal((fi, fo)) * math.sqrt(2.0 / fi), "b": np.zeros(fo)})
    return params


def forward(params, x):
    """y = W_L^T GELU(... GELU(W_1^T x + b_1) ...) + b_L for a batch x [B, in].
    Returns the output and the per-layer pre-activations (kept for backward)."""
    pre = []
    h = x
    for i, p in enumerate(params):
        z = h @ p["W"] + p["b"]
        pre.append((h, z))
        h = gelu(z) if i < len(params) - 1 else z
    return h, pre


def mse(y, t):
    """Mean over batch and outputs of (y - t)^2, and its gradient w.r.t. y."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(params, pre, dy):
    """Gradients of the loss for every W, b given dL/dy (chain rule layer by layer)."""
    grads = [None] * len(params)
    g = dy
    for i in range(len(params) - 1, -1, -1):
        h, z = pre[i]
        if i < len(params) - 1:
            g = g * gelu_grad(z)
        grads[i] = {"W": h.T @ g, "b": g.sum(axis=0)}
        g = g @ params[i]["W"].T
    return grads


def adam_step(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v per tensor and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for i, (p, g) in enumerate(zip(params, grads)):
        for key in ("W", "b"):
            m = state.setdefault(("m", i, key), np.zeros_like(p[key]))
            v = state.setdefault(("v", i, key), np.zeros_like(p[key]))
            m *= b1
            m += (1.0 - b1) * g[key]
            v *= b2
            v += (1.0 - b2) * g[key] ** 2
            mhat = m / (1.0 - b1 ** t)
            vhat = v / (1.0 - b2 ** t)
            p[key] -= lr * mhat / (np.sqrt(vhat) + eps)


def boxcox(y, lam, floor=1e-30):
    """Box-Cox transform of mass fractions, floored at `floor` (no negatives enter)."""
    y = np.maximum(np.asarray(y, dtype=np.float64), floor)
    return (y ** lam - 1.0) / lam


def boxcox_inv(z, lam):
    """Inverse Box-Cox; arguments below the transform's range map to zero."""
    base = np.maximum(1.0 + lam * np.asarray(z, dtype=np.float64), 0.0)
    return base ** (1.0 / lam)


def element_matrix(W, ncomp, atomic_mass):
    """E [elements, species]: element mass fraction per unit species mass fraction,
    E_ek = n_ke A_e / W_k, so E Y is the vector of element mass fractions."""
    return (np.asarray(ncomp, dtype=np.float64) * np.asarray(atomic_mass)[None, :] /
            np.asarray(W)[:, None]).T


def project(Yp, Y0, E, wfloor=1e-12):
    """Weighted least-squares projection of Yp [S] onto {Y : E Y = E Y0}, weights
    w_k = max(Yp_k, wfloor) (small species move least)."""
    w = np.maximum(Yp, wfloor)
    r = E @ Yp - E @ Y0
    EW = E * w[None, :]
    lam = np.linalg.solve(EW @ E.T, r)
    return Yp - w * (E.T @ lam)
