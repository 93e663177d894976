"""GPU parity of the plain FP64 integrator against the CPU oracle, through the C ABI.

Tolerance: 1e-8 relative on T and 1e-10 absolute on Y per cell (the FP64 bar), the
same attempted-step counts and status codes (integers: bit-exact).  Both sides run the
same algorithm in fp64; they differ only in rounding order (FMA contraction, mixture
coefficients, G_k products), which moves ||e|| by ~1e-11 at most, so only cells whose
oracle decision sat within 1e-7 of the accept threshold may diverge; those are counted
and held to an rtol-level bound.
"""
import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W
from tests._gpu import compare, run_device, sensitivity, to_dev

pytestmark = pytest.mark.gpu

MECH = M.build(0)
O = oracle.Oracle(MECH)


@pytest.fixture(scope="module")
def ctx():
    from paper_2506_02602_gb300 import build, chem
    build.build()
    c = chem.Context(MECH, "fp64")
    yield c
    c.close()


def _state(r):
    rho, e = O.state_from_TPY(r["T"], r["p"], r["Y"])
    return rho, e


@pytest.mark.parametrize("dt", [1e-7, 1e-6])
def test_reactors(ctx, dt):
    r = W.reactors(4096, seed=0)
    rho, e = _state(r)
    ref = O.integrate(rho, e, r["Y"], r["T"], dt)
    gpu = run_device(ctx, rho, e, r["Y"], r["T"], dt)
    res = compare(gpu, ref)
    print(dt, res)


def test_reactors_through_ignition(ctx):
    # over 10 us many cells ignite; a cell caught mid-ignition at the end of dt amplifies
    # rounding differences along the chain-branching radical pool, so where the oracle's
    # own sensitivity shows that amplification (tests._gpu.sensitivity) the cell gets the
    # method's rtol-level bound; all others the strict one
    r = W.reactors(4096, seed=0)
    rho, e = _state(r)
    ref = O.integrate(rho, e, r["Y"], r["T"], 1e-5)
    cond = sensitivity(O, rho, e, r["Y"], r["T"], 1e-5)
    gpu = run_device(ctx, rho, e, r["Y"], r["T"], 1e-5)
    ill = (cond[0] > 1e-11) | (cond[1] > 1e-11) | cond[2]
    dY = np.abs(gpu["Y"] - ref["Y"]).max(axis=0)
    worst = np.argsort(np.where(ill, -1.0, dY))[::-1][:5]
    for i in worst:  # diagnostics of the worst well-conditioned cells
        print("cell", i, "dY %.2e dT/T %.2e" % (dY[i], abs(gpu["T"][i] - ref["T"][i]) / ref["T"][i]),
              "T0 %.1f p %.3g" % (r["T"][i], r["p"][i]), "T1 %.1f" % ref["T"][i],
              "steps gpu/or", gpu["nsteps"][i], ref["nsteps"][i], "margin %.2e" % ref["margin"][i],
              "cond %.2e %.2e" % (cond[0][i], cond[1][i]))
    # rtol-level bound for the ill-conditioned class, tightened to 1e-6 (measured on
    # GB300: 9.0e-8 on T, 1.5e-7 on Y)
    res = compare(gpu, ref, cond=cond, loose_T=1e-6, loose_Y=1e-6)
    print(res)
    # the loose class (ill-conditioned plus knife-edge cells) is bounded at the measured
    # share plus margin: 2797 of 4096 cells (68.3 %) on GB300
    loose = res["edge"] + res["ill_conditioned"]
    assert loose <= 0.72 * res["n"], res
    assert res["strict"] + loose == res["n"]


@pytest.mark.parametrize("n,ld", [(1, 1), (31, 40), (33, 33), (127, 200), (129, 129), (1000, 1003)])
def test_ragged_sizes_and_padding(ctx, n, ld):
    r = W.reactors(n, seed=12)
    rho, e = _state(r)
    ref = O.integrate(rho, e, r["Y"], r["T"], 3e-7)
    gpu = run_device(ctx, rho, e, r["Y"], r["T"], 3e-7, ld=ld)
    compare(gpu, ref)
    assert np.all(gpu["Ypad"] == 0.0)  # padding between ncells and ldY is untouched


def test_empty_call_is_a_noop(ctx):
    import torch
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    Y = torch.zeros((9, 0), dtype=torch.float64, device="cuda")
    ctx.integrate(z, z, Y, z, 1e-7, ncells=0)
    torch.cuda.synchronize()


def test_argument_errors(ctx):
    from paper_2506_02602_gb300 import chem
    r = W.reactors(8, seed=1)
    rho, e = _state(r)
    args = (to_dev(rho), to_dev(e), to_dev(r["Y"]), to_dev(r["T"]))
    for dt, rtol, atol in [(0.0, 1e-6, 1e-10), (1e-7, 0.0, 1e-10), (1e-7, 1e-6, -1.0),
                           (float("nan"), 1e-6, 1e-10)]:
        with pytest.raises(chem.ChemError) as ei:
            ctx.integrate(*args, dt, rtol, atol)
        assert ei.value.code == chem.ERR_INVALID


def test_edge_cases_status_codes(ctx):
    r = W.reactors(64, seed=4)
    rho, e = _state(r)
    Y = r["Y"].copy()
    rho[1] = np.nan          # non-finite input -> status 4, Y untouched
    e[2] = -5e7              # no temperature root -> status 3
    Y[0, 3] = np.inf         # non-finite Y -> status 4
    rho[4] = -1.0            # non-positive density -> status 4
    ref = O.integrate(rho, e, Y, r["T"], 1e-7)
    gpu = run_device(ctx, rho, e, Y, r["T"], 1e-7)
    assert list(gpu["status"][:5]) == [0, 4, 3, 4, 4]
    np.testing.assert_array_equal(gpu["Y"][:, 1], Y[:, 1])
    assert np.isnan(gpu["T"][1]) and np.isnan(gpu["T"][2])
    ok = np.ones(64, bool)
    ok[1:5] = False
    compare({k: v[..., ok] for k, v in gpu.items() if k != "Ypad"},
            {k: v[..., ok] for k, v in ref.items()})


def test_max_steps_limit():
    from paper_2506_02602_gb300 import chem
    c = chem.Context(MECH, "fp64", max_steps=3)
    r = W.reactors(32, seed=3)
    rho, e = _state(r)
    ref = O.integrate(rho, e, r["Y"], r["T"], 1e-5, max_steps=3)
    gpu = run_device(c, rho, e, r["Y"], r["T"], 1e-5)
    c.close()
    assert np.all(gpu["status"] == 1) and np.all(gpu["nsteps"] == 3)
    np.testing.assert_allclose(gpu["Y"], ref["Y"], rtol=0, atol=1e-10)


def test_carried_step_size(ctx):
    r = W.reactors(512, seed=6)
    rho, e = _state(r)
    h0 = np.full(512, 2e-9)
    ref = O.integrate(rho, e, r["Y"], r["T"], 1e-6, h0=h0)
    gpu = run_device(ctx, rho, e, r["Y"], r["T"], 1e-6, h=h0)
    compare(gpu, ref)
    assert np.all(gpu["h"] > 0.0) and np.all(np.isfinite(gpu["h"]))


def test_stats_match_per_cell_outputs(ctx):
    r = W.reactors(3000, seed=8)
    rho, e = _state(r)
    rho[7] = np.nan
    gpu = run_device(ctx, rho, e, r["Y"], r["T"], 1e-6, stats=True)
    s = gpu["stats"]
    cells, acc, rej, rhs, mx = s[:5]
    hist = s[5:13]
    assert cells == 3000
    assert acc + rej == gpu["nsteps"].sum()
    assert mx == gpu["nsteps"].max()
    assert rhs >= 5 * (acc + rej) - 5 * 3000 and rhs <= 5 * (acc + rej)
    np.testing.assert_array_equal(hist[:6], np.bincount(gpu["status"], minlength=6)[:6])


def test_state_from_TPY_matches_oracle(ctx):
    r = W.reactors(1000, seed=2)
    T, p, Y = to_dev(r["T"]), to_dev(r["p"]), to_dev(r["Y"])
    rho, e = ctx.state_from_TPY(T, p, Y)
    ro, eo = _state(r)
    np.testing.assert_allclose(rho.cpu().numpy(), ro, rtol=1e-14)
    np.testing.assert_allclose(e.cpu().numpy(), eo, rtol=1e-12, atol=1e-6)


def test_host_entry_matches_device_entry(ctx):
    r = W.reactors(777, seed=5)
    rho, e = _state(r)
    dev = run_device(ctx, rho, e, r["Y"], r["T"], 1e-6)
    Y = np.ascontiguousarray(r["Y"].copy())
    T = r["T"].copy()
    st = np.zeros(777, np.int32)
    ns = np.zeros(777, np.int32)
    ctx.integrate_host(rho, e, Y, T, 1e-6, status=st, nsteps=ns)
    np.testing.assert_array_equal(Y, dev["Y"])
    np.testing.assert_array_equal(T, dev["T"])
    np.testing.assert_array_equal(st, dev["status"])
    np.testing.assert_array_equal(ns, dev["nsteps"])


def test_host_entry_pipeline_matches_device_entry(ctx):
    # 2^18 + 7 cells: the chunked copy/compute pipeline of the host entry (4 chunks,
    # the last one ragged), with a padded Y pitch and the carried step h
    d = W.detonation_slice(nx=512, ny=512)
    n = 512 * 512 + 7
    T0 = np.concatenate([d["T"], d["T"][:7]])
    p = np.concatenate([d["p"], d["p"][:7]])
    Y0 = np.concatenate([d["Y"], d["Y"][:, :7]], axis=1)
    import torch
    rho_d, e_d = ctx.state_from_TPY(to_dev(T0), to_dev(p), to_dev(Y0))
    rho, e = rho_d.cpu().numpy(), e_d.cpu().numpy()
    h0 = np.full(n, 1e-10)
    dev = run_device(ctx, rho, e, Y0, T0, 2e-9, h=h0, ld=n + 5)
    ld = n + 5
    Y = np.zeros((Y0.shape[0], ld))
    Y[:, :n] = Y0
    T, h = T0.copy(), h0.copy()
    st = np.zeros(n, np.int32)
    ns = np.zeros(n, np.int32)
    ctx.integrate_host(rho, e, Y, T, 2e-9, h=h, status=st, nsteps=ns)
    np.testing.assert_array_equal(Y[:, :n], dev["Y"])
    np.testing.assert_array_equal(Y[:, n:], 0.0)  # padding untouched
    np.testing.assert_array_equal(T, dev["T"])
    np.testing.assert_array_equal(h, dev["h"])
    np.testing.assert_array_equal(st, dev["status"])
    np.testing.assert_array_equal(ns, dev["nsteps"])


def test_detonation_slice_full_size_sampled(ctx):
    # the full 1024 x 1024 slice in the benchmark's launch configuration; the oracle
    # integrates a seeded sample of cells one by one
    d = W.detonation_slice()
    import torch
    T, p, Y = to_dev(d["T"]), to_dev(d["p"]), to_dev(d["Y"])
    rho, e = ctx.state_from_TPY(T, p, Y)
    T0 = T.clone()
    n = T.numel()
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    ns = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.integrate(rho, e, Y, T, 2e-9, status=st, nsteps=ns)
    torch.cuda.synchronize()
    rng = np.random.default_rng(99)
    idx = np.sort(np.concatenate([rng.choice(n, 3000, replace=False),
                                  np.arange(0, 1024), np.arange(n - 1024, n)]))
    idx = np.unique(idx)
    rho_s, e_s = rho.cpu().numpy()[idx], e.cpu().numpy()[idx]
    ref = O.integrate(rho_s, e_s, d["Y"][:, idx], T0.cpu().numpy()[idx], 2e-9)
    gpu = {"Y": Y.cpu().numpy()[:, idx], "T": T.cpu().numpy()[idx], "status": st.cpu().numpy()[idx],
           "nsteps": ns.cpu().numpy()[idx]}
    res = compare(gpu, ref)
    print(res, "steps max", ns.max().item())
    assert np.all(st.cpu().numpy() == 0)


def test_amr_batch_sample(ctx):
    b = W.amr_batch()
    rng = np.random.default_rng(5)
    idx = np.concatenate([np.flatnonzero(b["cls"] == c)[:300] for c in (0, 1, 2)])
    r = {"T": b["T"][idx], "p": b["p"][idx], "Y": b["Y"][:, idx]}
    rho, e = _state(r)
    ref = O.integrate(rho, e, r["Y"], r["T"], 1e-7)
    gpu = run_device(ctx, rho, e, r["Y"], r["T"], 1e-7)
    compare(gpu, ref)
    # cold inert cells take one step; the ignition front needs many (hot equilibrated
    # cells are stiff for an explicit method and need many too)
    cold = b["T"][idx[:300]] < 400.0
    assert np.all(ref["nsteps"][:300][cold] == 1)
    assert ref["nsteps"][600:].mean() > 10.0


def test_paper_thread_divergence_field(ctx):
    # Eq. 27-28 profile (Sec. 4.2.2) with the divergent smoothness alpha = 0.1
    f = W.eq27_profile(0.1, ny=256, nxz=8)
    rho, e = _state(f)
    ref = O.integrate(rho, e, f["Y"], f["T"], 1e-5)
    gpu = run_device(ctx, rho, e, f["Y"], f["T"], 1e-5)
    compare(gpu, ref)
