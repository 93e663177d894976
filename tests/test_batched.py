"""GPU checks of the batched persistent integrator (chem_integrate_batched).

* parity with the oracle on a ragged three-level batch: the oracle integrates every box
  substep by substep, carrying the step size and temperature guess, exactly as the
  persistent kernel's lanes do (same 1e-8 / 1e-10 / equal-steps bar as the one-pass
  kernel);
* the persistent kernel's per-cell arithmetic is the one-pass kernel's: with one
  substep per box the results are bit-identical to chem_integrate, whatever the queue
  order (stiffness-sorted, natural, cost hint) and with or without graph replay; the
  other compiled shapes agree to rounding;
* statistics, argument errors, and a full-size AMR batch checked on sampled cells;
* the autotuner leaves the caller's state alone, returns options that give the same
  results, and answers from its cache the second time.
"""
import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W
from tests._gpu import compare, to_dev

pytestmark = pytest.mark.gpu

MECH = M.build(0)
O = oracle.Oracle(MECH)


@pytest.fixture(scope="module", params=["fp64", "mixed"])
def ctx(request):
    from paper_2506_02602_gb300 import build, chem
    build.build()
    c = chem.Context(MECH, request.param)
    yield c
    c.close()


def _batch(nboxes, seed, edges=(2, 3, 4)):
    b = W.amr_batch(nboxes=nboxes, seed=seed, edges=edges)
    rho, e = O.state_from_TPY(b["T"], b["p"], b["Y"])
    b["rho"], b["e"] = rho, e
    return b


def _oracle_batch(b, rtol=1e-6, atol=1e-10):
    """The oracle, box by box and substep by substep, carrying h and T."""
    n = b["T"].size
    Y, T = b["Y"].copy(), b["T"].copy()
    h = np.full(n, np.nan)
    status = np.zeros(n, np.int32)
    nsteps = np.zeros(n, np.int32)
    margin = np.full(n, np.inf)
    off = b["box_offset"]
    for j in range(len(off) - 1):
        s = slice(off[j], off[j + 1])
        for _ in range(int(b["box_nsub"][j])):
            live = status[s] == 0
            r = O.integrate(b["rho"][s], b["e"][s], Y[:, s], T[s], float(b["box_dt"][j]), rtol, atol,
                            h0=h[s])
            # cells that stopped keep their state (a stopped cell does no further substeps)
            Y[:, s] = np.where(live, r["Y"], Y[:, s])
            T[s] = np.where(live, r["T"], T[s])
            h[s] = np.where(live, r["h"], h[s])
            nsteps[s] += np.where(live, r["nsteps"], 0)
            margin[s] = np.where(live, np.minimum(margin[s], r["margin"]), margin[s])
            status[s] = np.where(live, r["status"], status[s])
    return {"Y": Y, "T": T, "status": status, "nsteps": nsteps, "margin": margin, "h": h}


def _run_batched(ctx, b, **kw):
    import torch
    n = b["T"].size
    Y, T = to_dev(b["Y"]), to_dev(b["T"])
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ns = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    off = torch.tensor(b["box_offset"], dtype=torch.int64, device="cuda")
    dt = torch.tensor(b["box_dt"], dtype=torch.float64, device="cuda")
    nsub = torch.tensor(b["box_nsub"], dtype=torch.int32, device="cuda")
    ctx.integrate_batched(to_dev(b["rho"]), to_dev(b["e"]), Y, T, off, dt, nsub, status=st, nsteps=ns, **kw)
    torch.cuda.synchronize()
    return {"Y": Y.cpu().numpy(), "T": T.cpu().numpy(), "status": st.cpu().numpy(),
            "nsteps": ns.cpu().numpy()}


def test_batched_parity_with_substeps(ctx):
    b = _batch(30, seed=21)
    ref = _oracle_batch(b)
    gpu = _run_batched(ctx, b)
    if ctx.variant == "fp64":
        res = compare(gpu, ref)
        print(res)
    else:
        # mixed: 1e-5 relative on T (its stated bar) and, on every mass fraction, the
        # integration tolerance's scale rtol |Y| + atol <= 1e-6
        assert np.all(gpu["status"] == ref["status"])
        assert np.max(np.abs(gpu["T"] - ref["T"]) / ref["T"]) <= 1e-5
        assert np.max(np.abs(gpu["Y"] - ref["Y"])) <= 1e-6
    assert np.all(b["box_nsub"][b["box_dt"] < 1e-7] > 1)  # substeps were exercised


def test_single_substep_matches_one_pass_bitwise(ctx):
    import torch
    from paper_2506_02602_gb300 import chem
    b = _batch(40, seed=22)
    b["box_nsub"][:] = 1
    b["box_dt"][:] = 2e-7
    n = b["T"].size
    Y, T = to_dev(b["Y"]), to_dev(b["T"])
    ns = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.integrate(to_dev(b["rho"]), to_dev(b["e"]), Y, T, 2e-7, nsteps=ns)
    torch.cuda.synchronize()
    one = {"Y": Y.cpu().numpy(), "T": T.cpu().numpy(), "nsteps": ns.cpu().numpy()}
    hint = torch.tensor(one["nsteps"], dtype=torch.int32, device="cuda")
    for kw in (dict(), dict(order=chem.ORDER_NATURAL), dict(cost_hint=hint), dict(ctas_per_sm=1),
               dict(use_graph=True), dict(use_graph=True)):
        gpu = _run_batched(ctx, b, **kw)
        np.testing.assert_array_equal(gpu["Y"], one["Y"])
        np.testing.assert_array_equal(gpu["T"], one["T"])
        np.testing.assert_array_equal(gpu["nsteps"], one["nsteps"])
    for s in range(1, chem.BATCH_SHAPES):
        _agree_to_rounding(_run_batched(ctx, b, shape=s), one)


def _agree_to_rounding(a, b):
    """Another compiled shape: same algorithm, multiply-adds contracted differently, so
    rounding-level differences in 99 % of the cells; the rest are ill-conditioned at
    this long step (ignition in progress at its end: a rounding-seeded change of the
    step sequence moves the ignition time), and are only held to 1e-2 on T."""
    relT = np.abs(a["T"] - b["T"]) / b["T"]
    assert np.all(a["status"] == 0)
    assert np.quantile(relT, 0.99) <= 1e-10
    assert relT.max() <= 1e-2


def test_graph_recaptures_on_new_arguments(ctx):
    b1 = _batch(10, seed=23)
    b2 = _batch(14, seed=24)
    r1 = _run_batched(ctx, b1, use_graph=True)
    r2 = _run_batched(ctx, b2, use_graph=True)
    r1b = _run_batched(ctx, b1, use_graph=True)
    np.testing.assert_array_equal(r1["Y"], r1b["Y"])
    assert r2["Y"].shape[1] == b2["T"].size and np.all(r2["status"] == 0)


def test_batched_stats(ctx):
    import torch
    from paper_2506_02602_gb300 import chem
    b = _batch(20, seed=25)
    n = b["T"].size
    stats = torch.zeros(chem.STATS_WORDS, dtype=torch.int64, device="cuda")
    Y, T = to_dev(b["Y"]), to_dev(b["T"])
    ns = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.integrate_batched(to_dev(b["rho"]), to_dev(b["e"]), Y, T,
                          torch.tensor(b["box_offset"], device="cuda"),
                          torch.tensor(b["box_dt"], device="cuda"),
                          torch.tensor(b["box_nsub"], dtype=torch.int32, device="cuda"),
                          nsteps=ns, stats=stats)
    torch.cuda.synchronize()
    s = stats.cpu().numpy()
    assert s[0] == n and s[1] + s[2] == ns.sum().item() and s[4] == ns.max().item()
    assert s[5] == n  # every cell ok


def test_batched_argument_errors(ctx):
    import torch
    from paper_2506_02602_gb300 import chem
    b = _batch(4, seed=26)
    off = torch.tensor(b["box_offset"], device="cuda")
    dt = torch.tensor(b["box_dt"], device="cuda")
    nsub = torch.tensor(b["box_nsub"], dtype=torch.int32, device="cuda")
    args = (to_dev(b["rho"]), to_dev(b["e"]), to_dev(b["Y"]), to_dev(b["T"]))
    with pytest.raises(chem.ChemError):
        ctx.integrate_batched(*args, off, dt, nsub, order=7)
    with pytest.raises(chem.ChemError):
        ctx.integrate_batched(*args, off, dt, nsub, rtol=0.0)
    with pytest.raises(chem.ChemError):
        ctx.integrate_batched(*args, off, dt.to(torch.float32), nsub)


def test_amr_batch_full_size_sampled(ctx):
    # the full 256-box batch (3.46M cells) in one persistent launch; the oracle chains
    # the substeps of a seeded sample of cells drawn from every class
    b = W.amr_batch()
    gpu = _run_batched(ctx, {**b, **dict(zip(("rho", "e"), O.state_from_TPY(b["T"], b["p"], b["Y"])))})
    assert np.all(gpu["status"] == 0)
    rng = np.random.default_rng(8)
    idx = np.concatenate([rng.choice(np.flatnonzero(b["cls"] == c), 300, replace=False) for c in (0, 1, 2)])
    boxes = np.searchsorted(b["box_offset"], idx, side="right") - 1
    sub = {"T": b["T"][idx], "p": b["p"][idx], "Y": b["Y"][:, idx],
           "box_offset": np.arange(idx.size + 1), "box_dt": b["box_dt"][boxes],
           "box_nsub": b["box_nsub"][boxes]}
    sub["rho"], sub["e"] = O.state_from_TPY(sub["T"], sub["p"], sub["Y"])
    ref = _oracle_batch(sub)
    g = {"Y": gpu["Y"][:, idx], "T": gpu["T"][idx], "status": gpu["status"][idx], "nsteps": gpu["nsteps"][idx]}
    if ctx.variant == "fp64":
        print(compare(g, ref))
    else:
        assert np.max(np.abs(g["T"] - ref["T"]) / ref["T"]) <= 1e-5


def test_autotune_batched(ctx, tmp_path):
    import torch
    from paper_2506_02602_gb300 import chem
    b = _batch(40, seed=25)
    n = b["T"].size
    rho, e = to_dev(b["rho"]), to_dev(b["e"])
    Y, T = to_dev(b["Y"]), to_dev(b["T"])
    off = torch.tensor(b["box_offset"], dtype=torch.int64, device="cuda")
    dts = torch.tensor(b["box_dt"], dtype=torch.float64, device="cuda")
    nsub = torch.tensor(b["box_nsub"], dtype=torch.int32, device="cuda")
    cache = tmp_path / "tune.txt"
    best, table = ctx.autotune_batched(rho, e, Y, T, off, dts, nsub, cache_path=str(cache))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Y.cpu().numpy(), b["Y"])  # caller's state untouched
    np.testing.assert_array_equal(T.cpu().numpy(), b["T"])
    assert len(table) >= chem.BATCH_SHAPES + 2 and all(r["ms"] > 0 for r in table)
    assert {r["shape"] for r in table} == set(range(chem.BATCH_SHAPES))
    fastest = min(r["ms"] for r in table)
    assert any(r["ms"] == fastest and r["shape"] == best["shape"] for r in table)
    for s in range(chem.BATCH_SHAPES):
        blk, regs, per = ctx.batch_shape_info(s)
        assert blk in (64, 128, 256) and 0 < regs <= 255 and per >= 1
    ref = _run_batched(ctx, b)
    tuned = _run_batched(ctx, b, **best)
    if best["shape"] == 0:
        for k in ("Y", "T", "nsteps"):
            np.testing.assert_array_equal(tuned[k], ref[k])
    else:
        _agree_to_rounding(tuned, ref)
    again, table2 = ctx.autotune_batched(rho, e, Y, T, off, dts, nsub, cache_path=str(cache))
    assert table2 == [] and again == best
    assert len(cache.read_text().splitlines()) == 1
