"""CPU checks of the element bounds the GPU network tests use (tests/_bf16_bounds.py).

* a CPU emulation of the GPU's rounding schedule (BF16 activations and gradients, FP32
  accumulation) meets the end-to-end bound on a seeded 12-256-256-256-9 network, with
  margin (outputs below 0.3 of it, gradients below 0.8);
* mistakes the bound must catch fail it: a swapped pair of weight columns (end to end),
  and one wrong weight or a 2 % error in GELU' (layer by layer, on the stage's inputs);
* the layer-by-layer checks accept the stage computed in FP32 and rounded to BF16.
"""
import numpy as np
import pytest

from oracle import mlp
from tests import _bf16_bounds as BB

torch = pytest.importorskip("torch")


def _net(seed=5):
    rng = np.random.default_rng(seed + 1)
    params = mlp.init_params([12, 256, 256, 256, 9], seed=seed)
    bf = lambda a: torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    for p in params:
        p["W"] = bf(p["W"])
        p["b"] = np.asarray(0.1 * rng.standard_normal(p["b"].shape), np.float32).astype(np.float64)
    x = bf(rng.standard_normal((512, 12)))
    t = rng.standard_normal((512, 9))
    return params, x, t


def test_emulated_gpu_meets_end_to_end_bound():
    params, x, t = _net()
    y, Dy, g, Dg = BB.e2e_reference(params, x, t)
    ye, ge = BB.emulate_gpu(params, x, t)
    assert np.max(np.abs(ye - y) / Dy) < 0.3
    for l in range(4):
        for k in ("W", "b"):
            assert np.max(np.abs(ge[l][k] - g[l][k]) / (Dg[l][k] + 1e-300)) < 0.8, (l, k)


def test_end_to_end_bound_catches_swapped_columns():
    params, x, t = _net()
    y, Dy, _, _ = BB.e2e_reference(params, x, t)

    def swap(name, a):
        if name == "W1":
            a = a.copy()
            a[:, [3, 7]] = a[:, [7, 3]]
        return a

    ye = BB.emulate_gpu(params, x, plant=swap)
    assert np.max(np.abs(ye - y) / Dy) > 2.0


def test_stage_checks_accept_fp32_bf16_and_catch_single_errors():
    rng = np.random.default_rng(3)
    bf = lambda a: torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    H = bf(rng.standard_normal((64, 256)))
    W = bf(0.09 * rng.standard_normal((256, 256)))
    b = np.asarray(0.1 * rng.standard_normal(256), np.float32).astype(np.float64)
    Z = (torch.tensor(H, dtype=torch.float32) @ torch.tensor(W.T, dtype=torch.float32)
         + torch.tensor(b, dtype=torch.float32)).double().numpy()
    BB.check_dot("Z", Z, H, W.T, b)
    Hn = torch.nn.functional.gelu(torch.tensor(Z, dtype=torch.float32)).to(torch.bfloat16).double().numpy()
    BB.check_bf16_of("H", Hn, mlp.gelu(Z), BB.gelu_eval_err(Z))
    Wbad = W.copy()
    Wbad[10, 20] = W[11, 20]                  # one weight read from the neighbouring row
    Zbad = Z + H @ (Wbad - W).T
    with pytest.raises(AssertionError):
        BB.check_dot("Z", Zbad, H, W.T, b)
    dH = rng.standard_normal((64, 256))
    G = bf(dH * mlp.gelu_grad(Z) * 1.02)      # GELU' off by 2 %
    with pytest.raises(AssertionError):
        BB.check_bf16_of("G", G, dH * mlp.gelu_grad(Z), BB.gelu_grad_eval_err(dH, Z))
