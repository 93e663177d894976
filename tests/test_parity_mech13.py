"""GPU parity of the 13-species / 27-reaction mechanism (the paper's mechanism size,
Sec. 5.2.3) against the oracle, through the C ABI of libchem_h2o2_13.so (the same kernel
sources compiled for the generated 13-species structure).

* plain FP64 on 4096 independent reactors (N2 / Ar / He diluted H2-O2 with CO and CO2
  traces) at dt 1e-7 and 1e-6 s: 1e-8 relative on T, 1e-10 absolute on Y, equal
  attempted steps and statuses outside knife-edge cells; colliders bit-unchanged;
* a ragged sample of the 13-species detonation slice with padded planes;
* mixed precision within 1e-5 relative on T of FP64;
* the persistent batched kernel (one box, one substep) equals the one-pass kernel bit
  for bit;
* the full-storage comparator matches the oracle's scheme;
* the surrogate entry points answer CHEM_ERR_UNSUPPORTED.
"""
import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W
from tests._gpu import compare, run_device, to_dev

pytestmark = pytest.mark.gpu

MECH = M.build13(0)
O = oracle.Oracle(MECH)
COLL = [9, 10, 11, 12]


@pytest.fixture(scope="module")
def lib():
    from paper_2506_02602_gb300 import build, chem
    build.build()
    return chem


@pytest.fixture(scope="module")
def reactors():
    r = W.reactors13(4096, seed=0, mech=MECH)
    rho, e = O.state_from_TPY(r["T"], r["p"], r["Y"])
    return r, rho, e


@pytest.mark.parametrize("dt", [1e-7, 1e-6])
def test_fp64_matches_oracle(lib, reactors, dt):
    r, rho, e = reactors
    ctx = lib.Context(MECH, "fp64")
    ref = O.integrate(rho, e, r["Y"], r["T"], dt)
    gpu = run_device(ctx, rho, e, r["Y"], r["T"], dt)
    res = compare(gpu, ref)
    print(dt, res)
    np.testing.assert_array_equal(gpu["Y"][COLL], r["Y"][COLL])
    ctx.close()


def test_slice_sample_ragged(lib):
    d = W.detonation_slice13(64, 32, seed=1, mech=MECH)
    idx = np.random.default_rng(5).choice(d["T"].size, 1500, replace=False)
    T0, p0, Y0 = d["T"][idx], d["p"][idx], d["Y"][:, idx]
    rho, e = O.state_from_TPY(T0, p0, Y0)
    ref = O.integrate(rho, e, Y0, T0, 2e-9)
    ctx = lib.Context(MECH, "fp64")
    gpu = run_device(ctx, rho, e, Y0, T0, 2e-9, ld=1531)
    compare(gpu, ref)
    assert np.all(gpu["Ypad"] == 0.0)
    ctx.close()


def test_mixed_vs_fp64(lib, reactors):
    r, rho, e = reactors
    a = run_device(lib.Context(MECH, "fp64"), rho, e, r["Y"], r["T"], 1e-6)
    b = run_device(lib.Context(MECH, "mixed"), rho, e, r["Y"], r["T"], 1e-6)
    assert np.all(b["status"] == 0)
    assert np.max(np.abs(b["T"] - a["T"]) / a["T"]) <= 1e-5


def test_batched_one_substep_equals_one_pass(lib, reactors):
    import torch
    r, rho, e = reactors
    ctx = lib.Context(MECH, "fp64")
    a = run_device(ctx, rho, e, r["Y"], r["T"], 1e-7)
    n = rho.size
    Y, T = to_dev(r["Y"]), to_dev(r["T"])
    ns = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.integrate_batched(to_dev(rho), to_dev(e), Y, T, to_dev(np.array([0, n]), torch.int64),
                          to_dev(np.array([1e-7])), to_dev(np.array([1]), torch.int32), nsteps=ns)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Y.cpu().numpy(), a["Y"])
    np.testing.assert_array_equal(T.cpu().numpy(), a["T"])
    np.testing.assert_array_equal(ns.cpu().numpy(), a["nsteps"])
    ctx.close()


def test_full_storage_comparator(lib, reactors):
    r, rho, e = reactors
    ref = O.integrate(rho, e, r["Y"], r["T"], 1e-7, scheme=1)
    ctx = lib.Context(MECH, "fp64", scheme="full", block_size=256)
    compare(run_device(ctx, rho, e, r["Y"], r["T"], 1e-7), ref)
    ctx.close()


def test_surrogate_is_unsupported(lib):
    ctx = lib.Context(MECH, "fp64")
    with pytest.raises(lib.ChemError) as ei:
        ctx.surrogate_params()
    assert ei.value.code == lib.ERR_UNSUPPORTED
    ctx.close()
