"""GPU checks of the full hybrid on the reactive shock-bubble field (a 48^3 version of the
256^3 workload): AMR-like levels with 2^l substeps, the surrogate (trained here on the
field's own state family) with its error test and the persistent work-stealing
integrator for the cells it rejects, against plain FP64 batched integration, itself
checked against the oracle on sampled cells.  The one-call batched surrogate
(chem_surrogate_infer_batched) gives the per-box, per-substep loop's results bit for bit,
with consistent statistics."""
import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W
from tests._gpu import to_dev

pytestmark = pytest.mark.gpu

MECH = M.build(0)
O = oracle.Oracle(MECH)


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2506_02602_gb300 import build, chem, surrogate
    build.build()
    b = W.shock_bubble(48)
    rho, e = O.state_from_TPY(b["T"], b["p"], b["Y"])
    b["rho"], b["e"] = rho, e
    gen = chem.Context(MECH, "fp64", max_steps=4000)
    st = surrogate.trajectory_states(gen, 1024, seed=5, starts=W.bubble_trajectory_starts(1024, seed=5))
    gen.close()
    hyb = chem.Context(MECH, "mixed")
    pairs = surrogate.make_pairs(hyb, st, seed=5, dt_lo=1e-9, dt_hi=1e-8)
    hyb.surrogate_train(pairs["rho"], pairs["e"], pairs["Y0"], pairs["dt"], pairs["Y1"], T0=pairs["T0"],
                        epochs=30, batch=2048, lr=2e-3, seed=1, dt_power=1.0)
    plain = chem.Context(MECH, "fp64")
    n = b["T"].size
    Y, T = to_dev(b["Y"]), to_dev(b["T"])
    ns = torch.empty(n, dtype=torch.int32, device="cuda")
    st_ = torch.empty(n, dtype=torch.int32, device="cuda")
    plain.integrate_batched(to_dev(rho), to_dev(e), Y, T, torch.tensor(b["box_offset"], device="cuda"),
                            to_dev(b["box_dt"]), torch.tensor(b["box_nsub"], device="cuda"),
                            status=st_, nsteps=ns)
    torch.cuda.synchronize()
    ref = {"Y": Y.cpu().numpy(), "T": T.cpu().numpy(), "status": st_.cpu().numpy(), "nsteps": ns.cpu().numpy()}
    yield b, hyb, ref
    hyb.close()
    plain.close()


def test_plain_batched_matches_oracle_on_sampled_cells(setup):
    b, _, ref = setup
    assert np.all(ref["status"] == 0)
    rng = np.random.default_rng(11)
    off = b["box_offset"]
    for box in range(len(off) - 1):
        idx = np.sort(rng.choice(np.arange(off[box], off[box + 1]), 24, replace=False))
        Y, T = b["Y"][:, idx].copy(), b["T"][idx].copy()
        h = np.full(idx.size, np.nan)
        for _ in range(int(b["box_nsub"][box])):
            r = O.integrate(b["rho"][idx], b["e"][idx], Y, T, float(b["box_dt"][box]), h0=h)
            Y, T, h = r["Y"], r["T"], r["h"]
        np.testing.assert_allclose(ref["T"][idx], T, rtol=1e-8)
        np.testing.assert_allclose(ref["Y"][:, idx], Y, rtol=0, atol=1e-10)


def test_hybrid_against_plain_fp64(setup):
    import torch
    from paper_2506_02602_gb300 import surrogate
    b, hyb, ref = setup
    n = b["T"].size
    Y, T = to_dev(b["Y"]), to_dev(b["T"])
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    surrogate.hybrid_levels(hyb, to_dev(b["rho"]), to_dev(b["e"]), Y, T, b["box_offset"], b["box_dt"],
                            b["box_nsub"], status=st, mask=mask)
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    assert np.all((s == 0) | (s == 5))
    Yh, Th = Y.cpu().numpy(), T.cpu().numpy()
    rel = np.abs(Th - ref["T"]) / ref["T"]
    fb = mask.cpu().numpy() != 0
    reasons = np.bincount(mask.cpu().numpy(), minlength=7) / n
    print(f"cells {n}, fallback {fb.mean():.4f} {np.round(reasons, 4)}, max rel T {rel.max():.2e}, "
          f"accepted {rel[~fb].max(initial=0):.2e}")
    assert rel.max() <= 1e-3
    assert fb.mean() < 0.5  # the surrogate takes most of the field
    # element mass fractions conserved in every cell (projection or integrator)
    E = np.array([[M.ATOMIC_MASS[el] * MECH["ncomp"][k][j] for k in range(M.N_SPECIES)]
                  for j, el in enumerate(M.ELEMENTS)])
    E = E / E.sum(axis=0, keepdims=True)
    np.testing.assert_allclose(E @ Yh, E @ b["Y"], rtol=0, atol=1e-12)


def test_batched_surrogate_equals_per_box_loop(setup):
    import torch
    from paper_2506_02602_gb300 import chem, surrogate
    b, hyb, _ = setup
    n = b["T"].size
    dev_rho, dev_e = to_dev(b["rho"]), to_dev(b["e"])
    Y1, T1 = to_dev(b["Y"]), to_dev(b["T"])
    st1 = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    m1 = torch.empty(n, dtype=torch.uint8, device="cuda")
    surrogate.hybrid_levels(hyb, dev_rho, dev_e, Y1, T1, b["box_offset"], b["box_dt"], b["box_nsub"],
                            status=st1, mask=m1)
    Y2, T2 = to_dev(b["Y"]), to_dev(b["T"])
    st2 = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    m2 = torch.empty(n, dtype=torch.uint8, device="cuda")
    stats = torch.zeros(chem.STATS_WORDS, dtype=torch.int64, device="cuda")
    hyb.surrogate_infer_batched(dev_rho, dev_e, Y2, T2, torch.tensor(b["box_offset"], device="cuda"),
                                to_dev(b["box_dt"]), torch.tensor(b["box_nsub"], dtype=torch.int32, device="cuda"),
                                status=st2, mask=m2, stats=stats)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Y2.cpu().numpy(), Y1.cpu().numpy())
    np.testing.assert_array_equal(T2.cpu().numpy(), T1.cpu().numpy())
    np.testing.assert_array_equal(st2.cpu().numpy(), st1.cpu().numpy())
    np.testing.assert_array_equal(m2.cpu().numpy(), m1.cpu().numpy())
    sv = stats.cpu().numpy()
    subs = int((np.diff(b["box_offset"]) * np.asarray(b["box_nsub"])).sum())
    assert sv[0] == subs                           # cell-substeps
    assert sv[5 + 0] + sv[5 + 5] + sv[5 + 1:5 + 5].sum() == subs
    # a box table that does not cover the cells is refused before any launch
    bad = torch.tensor(np.asarray(b["box_offset"]) - 1, device="cuda")
    with pytest.raises(chem.ChemError) as ei:
        hyb.surrogate_infer_batched(dev_rho, dev_e, Y2, T2, bad, to_dev(b["box_dt"]),
                                    torch.tensor(b["box_nsub"], dtype=torch.int32, device="cuda"))
    assert ei.value.code == chem.ERR_INVALID
