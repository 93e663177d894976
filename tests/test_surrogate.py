"""GPU checks of the learned surrogate (chem_surrogate_*), against the FP64 CPU MLP
oracle (oracle/mlp.py) and the integrator.

* one forward/backward pass of the BF16 network matches the FP64 oracle on the same
  weights and batch element by element: every output and every gradient element within
  2^-7 sum |a| |b| of its dot product (tests/_bf16_bounds.py: a bound calibrated on a CPU
  emulation of the GPU's rounding schedule); padding gradients exactly zero;
* layer by layer (chem_surrogate_trace): every GEMM, GELU, loss gradient and GELU'
  stage matches the oracle's arithmetic on the GPU's own stage inputs within rigorous
  FP32 accumulation and BF16 rounding bounds, element by element;
* one Adam step (chem_surrogate_adam) matches oracle/mlp.adam_step element by element
  at FP32 rounding; the fp64 projection (chem_surrogate_project) matches mlp.project
  element by element at 1e-14;
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
from tests import _bf16_bounds as BB

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


def _bf16_network(ctx, seed=5):
    """Oracle parameters rounded to bf16 (weights) and fp32 (biases), uploaded to ctx;
    returns the oracle's params (fp64 copies of the same values) and the flat vector."""
    import torch
    params = mlp.init_params([12, 256, 256, 256, 9], seed=seed)
    rng = np.random.default_rng(seed + 1)
    for p in params:
        p["b"] = 0.1 * rng.standard_normal(p["b"].shape)
    flat = _to_gpu_layout(params)
    flat_bf = torch.tensor(flat).to(torch.bfloat16).to(torch.float32).numpy()
    got = _from_gpu_layout(flat_bf.astype(np.float64))
    for l, p in enumerate(params):
        W, b = got[l]
        p["W"] = W[: p["W"].shape[1], : p["W"].shape[0]].T.copy()
        p["b"] = b[: p["b"].size].copy()
    ctx.surrogate_params(flat_bf)
    return params, flat_bf


def _batch(B, seed=6):
    import torch
    rng = np.random.default_rng(seed)
    X = np.zeros((B, 16)); X[:, :12] = rng.standard_normal((B, 12))
    Tt = np.zeros((B, 16)); Tt[:, :9] = rng.standard_normal((B, 9))
    Xb = torch.tensor(X, dtype=torch.float32).to(torch.bfloat16).to(torch.float32)
    return Xb, torch.tensor(Tt, dtype=torch.float32)


def test_forward_backward_elementwise_vs_fp64_oracle(lib):
    ctx = lib.Context(MECH, "fp64")
    params, _ = _bf16_network(ctx)
    B = 512
    Xb, Tt = _batch(B)
    Y, g, loss = ctx.surrogate_grad(Xb.cuda(), Tt.cuda())
    x64, t64 = Xb.numpy().astype(np.float64)[:, :12], Tt.numpy().astype(np.float64)[:, :9]
    Yo, Dy, go, Dg = BB.e2e_reference(params, x64, t64)
    Yg = Y.cpu().numpy()
    # outputs, element by element
    ratio = np.abs(Yg[:, :9] - Yo) / Dy
    assert ratio.max() <= 1.0, ratio.max()
    assert np.all(Yg[:, 9:] == 0.0)
    lo = mlp.mse(Yo, t64)[0]
    assert loss == pytest.approx(lo, rel=1e-2)
    # every gradient element of every tensor; padding gradients exactly zero
    gg = _from_gpu_layout(g.astype(np.float64))
    for l in range(4):
        W, b = gg[l]
        ref_W, ref_b = go[l]["W"].T, go[l]["b"]
        live_W = W[: ref_W.shape[0], : ref_W.shape[1]]
        rW = np.abs(live_W - ref_W) / (Dg[l]["W"].T + 1e-30)
        rb = np.abs(b[: ref_b.size] - ref_b) / (Dg[l]["b"] + 1e-30)
        assert rW.max() <= 1.0 and rb.max() <= 1.0, (l, rW.max(), rb.max())
        pad = W.copy(); pad[: ref_W.shape[0], : ref_W.shape[1]] = 0.0
        assert np.all(pad == 0.0) and np.all(b[ref_b.size:] == 0.0)
    # the layer-by-layer forward is the training pass's own (the same tcgen05 GEMMs)
    np.testing.assert_array_equal(ctx.surrogate_forward(Xb.cuda(), impl=ctx.FWD_LAYERS).cpu().numpy(), Yg)
    # the one-kernel mma.sync forward (the legacy tensor path, kept as a check): its own
    # summation order, the same element bound against the oracle, full and ragged tiles
    for rows in (B, 333):
        Yf = ctx.surrogate_forward(Xb[:rows].contiguous().cuda(), impl=ctx.FWD_FUSED).cpu().numpy()
        assert np.max(np.abs(Yf[:, :9] - Yo[:rows]) / Dy[:rows]) <= 1.0, rows
    # the tcgen05 kernel inference uses sums the K products in the tensor cores' own
    # order; its outputs meet the same element bound against the oracle, on full and
    # ragged tiles
    for rows in (B, 333, 129, 1):
        Yt, err = ctx.surrogate_forward(Xb[:rows].contiguous().cuda(), check=True)
        Yt = Yt.cpu().numpy()
        assert err == 0
        ratio = np.abs(Yt[:, :9] - Yo[:rows]) / Dy[:rows]
        assert ratio.max() <= 1.0, (rows, ratio.max())
        assert np.all(Yt[:, 9:] == 0.0)
    ctx.close()


def test_tcgen05_network_with_many_tiles_per_cta(lib):
    """The inference kernel keeps two 128-row tiles in flight per CTA (one epilogue group
    each) over a persistent grid: on 3 tiles per SM plus a ragged end (pairs, a lone last
    tile, a partial tile) every output meets the element bound against the oracle, and a
    row's result does not depend on which CTA, group or position processed it."""
    import torch
    ctx = lib.Context(MECH, "fp64")
    params, _ = _bf16_network(ctx, seed=11)
    big = 152 * 128 * 3 + 77
    Xb, _ = _batch(big, seed=12)
    Xd = Xb.cuda()
    Y, err = ctx.surrogate_forward(Xd, check=True)
    assert err == 0
    Y = Y.cpu().numpy()
    x64 = Xb.numpy().astype(np.float64)[:, :12]
    Yo, Dy, _, _ = BB.e2e_reference(params, x64, np.zeros((big, 9)))
    ratio = np.abs(Y[:, :9] - Yo) / Dy
    assert ratio.max() <= 1.0, ratio.max()
    assert np.all(Y[:, 9:] == 0.0)
    for r0, r1 in ((0, 512), (300 * 128, 301 * 128), (big - 77 - 128, big)):
        Ys = ctx.surrogate_forward(Xd[r0:r1].contiguous()).cpu().numpy()
        np.testing.assert_array_equal(Ys, Y[r0:r1])
    ctx.close()


def test_every_network_stage_elementwise(lib):
    """chem_surrogate_trace: each stage against the oracle's arithmetic on the GPU's own
    inputs to that stage (rigorous FP32 / BF16 bounds, element by element)."""
    ctx = lib.Context(MECH, "fp64")
    _, flat = _bf16_network(ctx, seed=11)
    B = 384
    Xb, Tt = _batch(B, seed=12)
    tr = ctx.surrogate_trace(Xb.cuda(), Tt.cuda())
    layers = _from_gpu_layout(flat.astype(np.float64))      # W [N x K], b [N]
    X = Xb.numpy().astype(np.float64)
    T = Tt.numpy().astype(np.float64)
    Hin = [X] + [tr["H"][l].astype(np.float64) for l in range(3)]
    Z = [tr["Z"][l].astype(np.float64) for l in range(3)]
    # forward: Z_l = H_{l-1} W_l^T + b_l, H_l = bf16(GELU(Z_l)), Y = H_2 W_3^T + b_3
    for l in range(3):
        W, b = layers[l]
        BB.check_dot(f"Z{l}", Z[l], Hin[l], W.T, b)
        BB.check_bf16_of(f"H{l}", Hin[l + 1], mlp.gelu(Z[l]), BB.gelu_eval_err(Z[l]))
    W3, b3 = layers[3]
    Y = tr["Y"].astype(np.float64)
    BB.check_dot("Y", Y, Hin[3], W3.T, b3)
    # loss gradient: G_3 = bf16(2 (Y - T) / (9 B)) on the 9 live outputs, zero padding
    G3 = tr["G3"].astype(np.float64)
    d = 2.0 * (Y[:, :9] - T[:, :9]) / (9 * B)
    BB.check_bf16_of("G3", G3[:, :9], d, 8.0 * BB.U_F32 * np.abs(d))
    assert np.all(G3[:, 9:] == 0.0)
    assert tr["loss"] == pytest.approx(float(np.mean((Y[:, :9] - T[:, :9]) ** 2)), rel=1e-5)
    # backward: dW_l = G_l^T H_{l-1}, db_l = sum_m G_l, dH_{l-1} = G_l W_l,
    # G_{l-1} = bf16(dH_{l-1} GELU'(Z_{l-1}))
    grads = _from_gpu_layout(tr["grad"].astype(np.float64))
    G = [tr["G"][l].astype(np.float64) for l in range(3)] + [G3]
    dH = [tr["dH"][l].astype(np.float64) for l in range(3)]
    ones = np.ones((1, B))
    for l in range(3, -1, -1):
        W, _ = layers[l]
        gW, gb = grads[l]
        BB.check_dot(f"dW{l}", gW, G[l].T, Hin[l])
        BB.check_dot(f"db{l}", gb[None, :], ones, G[l])
        if l == 0:
            break
        BB.check_dot(f"dH{l - 1}", dH[l - 1], G[l], W)
        BB.check_bf16_of(f"G{l - 1}", G[l - 1], dH[l - 1] * mlp.gelu_grad(Z[l - 1]),
                         BB.gelu_grad_eval_err(dH[l - 1], Z[l - 1]))
    # the trace's gradient is the one chem_surrogate_grad returns
    _, g2, _ = ctx.surrogate_grad(Xb.cuda(), Tt.cuda())
    np.testing.assert_array_equal(g2, tr["grad"])
    ctx.close()


def test_adam_step_matches_oracle(lib):
    ctx = lib.Context(MECH, "fp64")
    n = int(lib.load().chem_surrogate_param_count())
    rng = np.random.default_rng(21)
    p0 = (0.05 * rng.standard_normal(n)).astype(np.float32)
    g1 = (1e-3 * rng.standard_normal(n)).astype(np.float32)
    g2 = (1e-3 * rng.standard_normal(n)).astype(np.float32)
    g1[::97] = 0.0                                  # no gradient: no move
    g2[::89] = 1e-9                                 # gradients near eps
    ctx.surrogate_params(p0)
    lr = 2e-3
    ctx.surrogate_adam(g1, lr)
    p1 = ctx.surrogate_params()
    ctx.surrogate_adam(g2, lr)
    p2 = ctx.surrogate_params()
    ref = [{"W": p0.astype(np.float64), "b": np.zeros(0)}]
    st = {}
    for got, g in ((p1, g1), (p2, g2)):
        mlp.adam_step(ref, [{"W": g.astype(np.float64), "b": np.zeros(0)}], st, lr=lr)
        want = ref[0]["W"]
        # fp32 parameters (2 roundings per step) and an fp32 update (|update| <= lr / (1 - b1)
        # relative error ~1e-6, the fp32 b1 and b2 constants included)
        tol = 4.0 * 2.0 ** -24 * np.abs(want) + 1e-6 * lr * 10.0
        assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want) / tol)
    np.testing.assert_array_equal(p1[::97], p0[::97])
    ctx.close()


def test_projection_matches_oracle(lib):
    import torch
    ctx = lib.Context(MECH, "fp64")
    E = mlp.element_matrix(MECH["W"], MECH["ncomp"], [M.ATOMIC_MASS[x] for x in M.ELEMENTS])
    rng = np.random.default_rng(8)
    n = 3001                                          # several blocks and a ragged tail
    Y0 = rng.dirichlet(np.full(9, 0.5), size=n).T.copy()
    Y0[:, :50] = rng.dirichlet(np.full(9, 0.05), size=50).T   # many tiny species
    Yp = Y0 * (1.0 + 1e-3 * rng.standard_normal((9, n))) + 1e-6 * rng.standard_normal((9, n))
    Yp[:, 100:120] = np.abs(Yp[:, 100:120])
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    got = ctx.surrogate_project(dev(Y0), dev(Yp)).cpu().numpy()
    want = np.stack([mlp.project(Yp[:, i], Y0[:, i], E) for i in range(n)], axis=1)
    err = np.abs(got - want)
    assert err.max() <= 1e-14, err.max()
    np.testing.assert_allclose(E @ got, E @ Y0, rtol=0, atol=1e-14)
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
