"""GPU checks of the learned surrogate (chem_surrogate_*), against the FP64 CPU MLP
oracle (oracle/mlp.py) and the integrator.

* one forward/backward pass of the BF16 tensor-core network matches the FP64 oracle on
  the same weights and batch within BF16 bounds (outputs and every gradient tensor,
  relative 2e-2 in norm; padding gradients exactly zero);
* training on integrator-generated pairs lowers the loss; parameters and the saved file
  round-trip exactly;
* inference: accepted cells conserve the element mass fractions to 1e-12 (fp64
  projection) and energy exactly (T solved from e); rejected cells are integrated by the
  same arithmetic as chem_integrate (bit-identical); mask and statistics agree;
* what the network gains: on a million held-out states at dt = 1e-9 s the surrogate
  path (network, error test, fallback) is faster than plain integration of the same cells and
  within 1e-3 relative on T of it.
"""
import numpy as np
import pytest

from chem_inputs import mechanism as M
from oracle import mlp

pytestmark = pytest.mark.gpu

MECH = M.build(0)


@pytest.fixture(scope="module")
def lib():
    from paper_2506_02602_gb300 import build, chem
    build.build()
    return chem


def _to_gpu_layout(params):
    """Oracle layers (W [in, out], b [out]) of 12-256-256-256-9 -> the library's padded
    flat layout (W [N x K] per layer, input padded to 16, output to 16)."""
    N = [256, 256, 256, 16]
    K = [16, 256, 256, 256]
    flat = []
    for l, p in enumerate(params):
        Wg = np.zeros((N[l], K[l]))
        Wg[: p["W"].shape[1], : p["W"].shape[0]] = p["W"].T
        bg = np.zeros(N[l])
        bg[: p["b"].size] = p["b"]
        flat += [Wg.ravel(), bg]
    return np.concatenate(flat).astype(np.float32)


def _from_gpu_layout(flat):
    N = [256, 256, 256, 16]
    K = [16, 256, 256, 256]
    out, o = [], 0
    for l in range(4):
        W = flat[o: o + N[l] * K[l]].reshape(N[l], K[l]); o += N[l] * K[l]
        b = flat[o: o + N[l]]; o += N[l]
        out.append((W, b))
    return out


def test_forward_backward_matches_fp64_oracle(lib):
    import torch
    ctx = lib.Context(MECH, "fp64")
    params = mlp.init_params([12, 256, 256, 256, 9], seed=5)
    rng = np.random.default_rng(6)
    for p in params:
        p["b"] = 0.1 * rng.standard_normal(p["b"].shape)
    # round the weights to bf16 first so both sides use the same values
    flat = _to_gpu_layout(params)
    flat_bf = torch.tensor(flat).to(torch.bfloat16).to(torch.float32).numpy()
    got = _from_gpu_layout(flat_bf.astype(np.float64))
    for l, p in enumerate(params):
        W, b = got[l]
        p["W"] = W[: p["W"].shape[1], : p["W"].shape[0]].T.copy()
        p["b"] = b[: p["b"].size].copy()
    ctx.surrogate_params(flat_bf)
    B = 512
    X = np.zeros((B, 16)); X[:, :12] = rng.standard_normal((B, 12))
    Tt = np.zeros((B, 16)); Tt[:, :9] = rng.standard_normal((B, 9))
    Xb = torch.tensor(X, dtype=torch.float32).to(torch.bfloat16).to(torch.float32)
    Y, g, loss = ctx.surrogate_grad(Xb.cuda(), torch.tensor(Tt, dtype=torch.float32).cuda())
    Yo, pre = mlp.forward(params, Xb.numpy().astype(np.float64)[:, :12])
    lo, dy = mlp.mse(Yo, Tt[:, :9])
    go = mlp.backward(params, pre, dy)
    Yg = Y.cpu().numpy()
    # the one-kernel mma.sync forward: same fragments, K order and epilogue -> same numbers
    Yf = ctx.surrogate_forward(Xb.cuda(), impl=ctx.FWD_FUSED).cpu().numpy()
    np.testing.assert_array_equal(Yf, Yg)
    Yf2 = ctx.surrogate_forward(Xb[:333].contiguous().cuda(), impl=ctx.FWD_FUSED).cpu().numpy()  # ragged tile
    np.testing.assert_array_equal(Yf2, Yg[:333])
    np.testing.assert_array_equal(ctx.surrogate_forward(Xb.cuda(), impl=ctx.FWD_LAYERS).cpu().numpy(), Yg)
    # the tcgen05 kernel inference uses: the tensor cores sum the K products in their own
    # order, so FP32 sums differ in the last bits and a BF16 activation can round the
    # other way; the outputs agree to BF16 level, and with the FP64 oracle as above
    for rows in (B, 333, 129, 1):
        Yt, err = ctx.surrogate_forward(Xb[:rows].contiguous().cuda(), check=True)
        Yt = Yt.cpu().numpy()
        assert err == 0
        assert np.linalg.norm(Yt - Yg[:rows]) <= 5e-3 * np.linalg.norm(Yg[:rows]), rows
        assert np.all(Yt[:, 9:] == 0.0)
    Yt = ctx.surrogate_forward(Xb.cuda()).cpu().numpy()
    assert np.linalg.norm(Yt[:, :9] - Yo) <= 2e-2 * np.linalg.norm(Yo)
    assert np.linalg.norm(Yg[:, :9] - Yo) <= 2e-2 * np.linalg.norm(Yo)
    assert np.all(Yg[:, 9:] == 0.0)
    assert loss == pytest.approx(lo, rel=2e-2)
    gg = _from_gpu_layout(g.astype(np.float64))
    for l in range(4):
        W, b = gg[l]
        ref_W, ref_b = go[l]["W"].T, go[l]["b"]
        live_W = W[: ref_W.shape[0], : ref_W.shape[1]]
        assert np.linalg.norm(live_W - ref_W) <= 2e-2 * np.linalg.norm(ref_W), l
        assert np.linalg.norm(b[: ref_b.size] - ref_b) <= 2e-2 * np.linalg.norm(ref_b), l
        pad = W.copy(); pad[: ref_W.shape[0], : ref_W.shape[1]] = 0.0
        assert np.all(pad == 0.0) and np.all(b[ref_b.size:] == 0.0)
    ctx.close()


@pytest.fixture(scope="module")
def trained(lib, tmp_path_factory):
    from paper_2506_02602_gb300 import surrogate
    ctx = lib.Context(MECH, "fp64")
    gen = lib.Context(MECH, "fp64", max_steps=4000)
    st = surrogate.trajectory_states(gen, 2048, seed=3)
    pairs = surrogate.make_pairs(ctx, st, seed=3, max_pairs=60000)
    loss = ctx.surrogate_train(pairs["rho"], pairs["e"], pairs["Y0"], pairs["dt"], pairs["Y1"],
                               T0=pairs["T0"], epochs=20, batch=2048, lr=2e-3, seed=1, dt_power=1.0)
    held = surrogate.trajectory_states(gen, 256, seed=97)
    gen.close()
    path = tmp_path_factory.mktemp("sur") / "net.bin"
    ctx.surrogate_save(str(path))
    yield ctx, loss, held, path
    ctx.close()


def test_training_lowers_loss_and_roundtrips(lib, trained):
    ctx, loss, held, path = trained
    assert np.all(np.isfinite(loss)) and loss[-1] < 0.5 * loss[0], loss
    p = ctx.surrogate_params()
    ctx2 = lib.Context(MECH, "fp64")
    ctx2.surrogate_load(str(path))
    np.testing.assert_array_equal(ctx2.surrogate_params(), p)
    ctx2.close()


def test_inference_invariants_and_fallback(lib, trained):
    import torch
    ctx, _, held, _ = trained
    n = held["T"].numel()
    Y, T = held["Y"].clone(), held["T"].clone()
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ns = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    stats = torch.zeros(lib.STATS_WORDS, dtype=torch.int64, device="cuda")
    ctx.surrogate_infer(held["rho"], held["e"], Y, T, 1e-8, status=st, nsteps=ns, mask=mask, stats=stats,
                        gate={"max_dT": 10.0})
    # the plain integrator on the same states
    Yr, Tr = held["Y"].clone(), held["T"].clone()
    nsr = torch.empty(n, dtype=torch.int32, device="cuda")
    str_ = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.integrate(held["rho"], held["e"], Yr, Tr, 1e-8, nsteps=nsr, status=str_)
    torch.cuda.synchronize()
    fb = mask.cpu().numpy().astype(bool)
    s = st.cpu().numpy()
    sr = str_.cpu().numpy()
    assert 0 < fb.sum() < n  # both paths exercised
    # a fallback cell reports CHEM_CELL_SURROGATE, or the integrator's own failure code
    np.testing.assert_array_equal(s[fb], np.where(sr[fb] == 0, lib.CELL_SURROGATE, sr[fb]))
    assert np.all(s[~fb] == lib.CELL_OK)
    assert np.all(ns.cpu().numpy()[~fb] == 0)
    Yg, Tg = Y.cpu().numpy(), T.cpu().numpy()
    np.testing.assert_array_equal(Yg[:, fb], Yr.cpu().numpy()[:, fb])
    np.testing.assert_array_equal(Tg[fb], Tr.cpu().numpy()[fb])
    np.testing.assert_array_equal(ns.cpu().numpy()[fb], nsr.cpu().numpy()[fb])
    # accepted cells: element mass fractions and energy
    E = mlp.element_matrix(MECH["W"], MECH["ncomp"], [M.ATOMIC_MASS[x] for x in M.ELEMENTS])
    Y0 = held["Y"].cpu().numpy()
    acc = ~fb
    np.testing.assert_allclose(E @ Yg[:, acc], E @ Y0[:, acc], rtol=0, atol=1e-12)
    import oracle
    o = oracle.Oracle(MECH)
    e = held["e"].cpu().numpy()
    for i in np.flatnonzero(acc)[:200]:
        assert abs(o.e_mix(Yg[:, i], Tg[i]) - e[i]) <= 1e-12 * abs(e[i]) + 1e-5
    sv = stats.cpu().numpy()
    assert sv[0] == n and sv[5 + lib.CELL_SURROGATE] == (fb & (sr == 0)).sum() and sv[5 + 0] == acc.sum()


def test_trained_network_gains_over_plain_integration(lib, trained):
    import time

    import torch
    from paper_2506_02602_gb300 import surrogate
    ctx, _, held, _ = trained
    cells = surrogate.draw_cells(held, 1 << 20, seed=5)
    n = cells["T"].numel()
    dt = 1e-9
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")

    def best(fn):
        out = float("inf")
        for _ in range(4):
            Y, T = cells["Y"].clone(), cells["T"].clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn(Y, T)
            torch.cuda.synchronize()
            out = min(out, time.perf_counter() - t0)
        return out, Y, T

    tp, Yp, Tp = best(lambda Y, T: ctx.integrate(cells["rho"], cells["e"], Y, T, dt))
    ts, Ys, Ts = best(lambda Y, T: ctx.surrogate_infer(cells["rho"], cells["e"], Y, T, dt, mask=mask))
    rel = ((Ts - Tp).abs() / Tp).max().item()
    fb = (mask != 0).float().mean().item()
    print(f"plain {n / tp:.3e} cells/s, surrogate {n / ts:.3e} cells/s, fallback {fb:.4f}, max rel T {rel:.2e}")
    assert rel <= 1e-3
    assert fb < 0.5
    assert ts < tp
