"""GPU parity of the conventional explicit comparators (full k-storage) against the
oracle's same schemes, through the C ABI.

The paper measures its two-register scheme (Eq. 21) against standard explicit RK that
keeps every stage derivative (Sec. 2.2.3, Sec. 4.2.2).  chem_options.scheme selects the
comparators: the RK4(3)5 tableau in Butcher form with all five k_i kept, and Fehlberg's
RKF45.  Each must match the oracle's scheme on the 4096-reactor workload and a
detonation-slice sample at the FP64 bar (1e-8 relative on T, 1e-10 absolute on Y, equal
attempted-step counts outside knife-edge cells) in every compiled block shape, including
a ragged cell count with padded planes; the mixed-precision comparators meet 1e-5 on T
against the FP64 ones.  The batched and surrogate calls refuse a comparator context.
"""
import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W
from tests._gpu import compare, run_device

pytestmark = pytest.mark.gpu

MECH = M.build(0)
O = oracle.Oracle(MECH)
SCH = {"full": 1, "rkf45": 2}


@pytest.fixture(scope="module")
def lib():
    from paper_2506_02602_gb300 import build, chem
    build.build()
    return chem


@pytest.fixture(scope="module")
def reactors():
    r = W.reactors(4096, seed=0)
    rho, e = O.state_from_TPY(r["T"], r["p"], r["Y"])
    return r, rho, e


@pytest.mark.parametrize("scheme", ["full", "rkf45"])
@pytest.mark.parametrize("block", [128, 256, 64])
def test_comparator_matches_oracle_reactors(lib, reactors, scheme, block):
    r, rho, e = reactors
    ref = O.integrate(rho, e, r["Y"], r["T"], 1e-7, scheme=SCH[scheme])
    ctx = lib.Context(MECH, "fp64", scheme=scheme, block_size=block)
    gpu = run_device(ctx, rho, e, r["Y"], r["T"], 1e-7)
    res = compare(gpu, ref)
    print(scheme, block, res)
    ctx.close()


@pytest.mark.parametrize("scheme", ["full", "rkf45"])
def test_comparator_ragged_and_slice(lib, scheme):
    d = W.detonation_slice(64, 32, seed=1)
    n = 2000                               # not a multiple of any block, planes padded
    idx = np.random.default_rng(3).choice(d["T"].size, n, replace=False)
    T0, p0, Y0 = d["T"][idx], d["p"][idx], d["Y"][:, idx]
    rho, e = O.state_from_TPY(T0, p0, Y0)
    ref = O.integrate(rho, e, Y0, T0, 2e-9, scheme=SCH[scheme])
    ctx = lib.Context(MECH, "fp64", scheme=scheme)
    gpu = run_device(ctx, rho, e, Y0, T0, 2e-9, ld=n + 37)
    compare(gpu, ref)
    assert np.all(gpu["Ypad"] == 0.0)
    ctx.close()


@pytest.mark.parametrize("scheme", ["full", "rkf45"])
def test_mixed_comparator_vs_fp64(lib, reactors, scheme):
    r, rho, e = reactors
    c64 = lib.Context(MECH, "fp64", scheme=scheme)
    cmx = lib.Context(MECH, "mixed", scheme=scheme)
    a = run_device(c64, rho, e, r["Y"], r["T"], 1e-7)
    b = run_device(cmx, rho, e, r["Y"], r["T"], 1e-7)
    assert np.all(b["status"] == 0)
    assert np.max(np.abs(b["T"] - a["T"]) / a["T"]) <= 1e-5
    c64.close()
    cmx.close()


def test_batched_and_surrogate_refuse_comparators(lib):
    import torch
    ctx = lib.Context(MECH, "fp64", scheme="full")
    x = torch.ones(8, dtype=torch.float64, device="cuda")
    Y = torch.full((9, 8), 1.0 / 9.0, dtype=torch.float64, device="cuda")
    off = torch.tensor([0, 8], dtype=torch.int64, device="cuda")
    dt = torch.tensor([1e-7], dtype=torch.float64, device="cuda")
    nsub = torch.tensor([1], dtype=torch.int32, device="cuda")
    with pytest.raises(lib.ChemError) as ei:
        ctx.integrate_batched(x, x, Y, x, off, dt, nsub)
    assert ei.value.code == lib.ERR_UNSUPPORTED
    with pytest.raises(lib.ChemError) as ei:
        ctx.integrate_batched_noalloc(x, x, Y, x, off, dt, nsub)
    assert ei.value.code == lib.ERR_UNSUPPORTED
    ctx.close()
