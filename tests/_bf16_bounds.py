"""Element-wise bounds for the surrogate network's BF16 tensor-core arithmetic against the
FP64 oracle (oracle/mlp.py) on the same BF16-valued weights and inputs.

Two kinds of check use them.

* End to end (outputs and every gradient element of one forward/backward pass): the GPU
  rounds each hidden activation and each backward gradient to BF16 (unit roundoff
  u = 2^-8) and accumulates in FP32, so its result differs from the FP64 oracle's by
  rounding errors carried through three hidden layers.  Each output or gradient element
  is a dot product s = sum_i a_i b_i of the oracle's own FP64 operands; the bound is
  2 u sum_i |a_i| |b_i| = 2^-7 sum |a| |b|.  It is not a worst-case bound (the worst case
  grows like (1.13 * sum_i |w_i|)^depth and is useless for 256-wide layers) but a
  calibrated one: a CPU emulation of the GPU's rounding schedule (emulate_gpu) stays below
  0.2 of it on outputs and 0.65 on gradients, and a swapped pair of weight columns
  exceeds it by ~8x.
* Layer by layer (chem_surrogate_trace): every GEMM and elementwise kernel is checked on
  the GPU's own inputs to that stage, where the bound is rigorous: an FP32 dot product of
  length K is within (K + 8) 4 u_f32 sum |a| |b| of the exact one (u_f32 = 2^-24), and a
  BF16-rounded value within u of the FP32 value it rounds (plus that value's own FP32
  evaluation error).  A single wrong weight fails it.

GELU'(x) = Phi(x) + x phi(x) peaks at 1.1289; GELU and GELU' are evaluated on the GPU in
FP32 with Phi from the rational approximation of Abramowitz & Stegun 7.1.26 (absolute
error of erf at most 1.5e-7, so of Phi at most 7.5e-8 = 1.26 u_f32) and exp; with the FP32
rounding of the polynomial the absolute errors stay within a few u_f32 (|value| + |x|),
and the checks allow 8 u_f32 (|value| + |x|).
"""
from __future__ import annotations

import numpy as np

from oracle import mlp

U_BF16 = 2.0 ** -8
U_F32 = 2.0 ** -24
E2E = 2.0 ** -7


def acc_bound(K):
    """Relative bound of an FP32 dot product of length K (sequential summation, with room
    for the tensor cores' own accumulation order)."""
    return (K + 8) * 4.0 * U_F32


def e2e_reference(params, x, t):
    """Oracle outputs and loss gradients with the end-to-end element bounds.
    Returns (y, Dy, grads, Dgrads) with grads / Dgrads lists of {"W", "b"} like
    mlp.backward (W as [in, out])."""
    y, pre = mlp.forward(params, x)
    h_last = pre[-1][0]
    W, b = params[-1]["W"], params[-1]["b"]
    Dy = E2E * (np.abs(h_last) @ np.abs(W) + np.abs(b))
    _, dy = mlp.mse(y, t)
    grads = mlp.backward(params, pre, dy)
    Dg = [None] * len(params)
    g = dy
    for i in range(len(params) - 1, -1, -1):
        h, z = pre[i]
        if i < len(params) - 1:
            g = g * mlp.gelu_grad(z)
        Dg[i] = {"W": E2E * (np.abs(h).T @ np.abs(g)), "b": E2E * np.abs(g).sum(axis=0)}
        g = g @ params[i]["W"].T
    return y, Dy, grads, Dg


def emulate_gpu(params, x, t=None, plant=None):
    """CPU emulation of the GPU's rounding schedule (BF16 activations and gradients, FP32
    accumulation), for calibrating the end-to-end bound.  plant(name, array) may return a
    modified array for one stage (a planted mistake).  Returns y, or (y, grads) with t."""
    import torch
    bf = lambda a: torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    hook = plant or (lambda name, a: a)
    L = len(params)
    hs, zs = [], []
    h = np.asarray(x, dtype=np.float64)
    for i, p in enumerate(params):
        W = hook(f"W{i}", p["W"])
        z = f32(f32(h.astype(np.float32) @ W.astype(np.float32)) + p["b"].astype(np.float32))
        hs.append(h)
        zs.append(z)
        h = bf(f32(mlp.gelu(z))) if i < L - 1 else z
    y = h
    if t is None:
        return y
    g = bf(f32(2.0 * (y - t) / y.size))
    grads = [None] * L
    for i in range(L - 1, -1, -1):
        grads[i] = {"W": f32(hs[i].T.astype(np.float32) @ g.astype(np.float32)),
                    "b": f32(g.astype(np.float32).sum(axis=0))}
        if i == 0:
            break
        dh = f32(g.astype(np.float32) @ params[i]["W"].T.astype(np.float32))
        g = bf(f32(dh * hook(f"gelu_grad{i - 1}", mlp.gelu_grad(zs[i - 1]))))
    return y, grads


def check_dot(name, got, a, b, bias=None):
    """got ~ a @ b (+ bias) element by element, within the FP32 accumulation bound of
    the stage (a, b: the GPU's own operands, exactly representable)."""
    ref = a @ b
    mag = np.abs(a) @ np.abs(b)
    if bias is not None:
        ref = ref + bias
        mag = mag + np.abs(bias)
    tol = acc_bound(a.shape[-1]) * mag + 1e-30
    bad = np.abs(got - ref) > tol
    assert not bad.any(), f"{name}: {bad.sum()} of {bad.size} elements outside the FP32 bound, " \
                          f"worst ratio {np.max(np.abs(got - ref) / tol):.3g}"


def check_bf16_of(name, got, exact, eval_err):
    """got == bf16(v) where v is an FP32 evaluation of `exact` with absolute error at most
    eval_err: |got - exact| <= u (|exact| + eval_err) + eval_err."""
    tol = U_BF16 * (np.abs(exact) + eval_err) + eval_err + 1e-38
    bad = np.abs(got - exact) > tol
    assert not bad.any(), f"{name}: {bad.sum()} of {bad.size} elements outside the BF16 bound, " \
                          f"worst ratio {np.max(np.abs(got - exact) / tol):.3g}"


def gelu_eval_err(z):
    """Absolute error bound of an FP32 GELU(z) = z Phi(z) with Phi within 7.5e-8 of exact."""
    return 8.0 * U_F32 * (np.abs(mlp.gelu(z)) + np.abs(z))


def gelu_grad_eval_err(dh, z):
    """Absolute error bound of FP32 dh * GELU'(z), GELU'(z) = Phi(z) + z phi(z)."""
    return 16.0 * U_F32 * np.abs(dh) * (np.abs(mlp.gelu_grad(z)) + 1.0 + np.abs(z))
