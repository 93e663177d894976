"""The benchmark's per-workload oracle timing (bench.oracle_config), on the CPU.

Each workload's cpu_baseline times the oracle on a seeded stratified sample and
extrapolates every stratum's time to the workload by the stratum's weight.  These checks
run it on a small two-stratum sample of reactors: the reported rate is the workload's
cells over the extrapolated time, the extrapolation is labelled, and the comparison with
given temperatures is the largest relative difference on the sampled cells (zero against
the oracle's own result).
"""
import numpy as np

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W


def test_stratified_extrapolation_and_sample_comparison():
    import bench
    r = W.reactors(96, seed=0)
    mech = M.build(0)
    o = oracle.Oracle(mech)
    rho, e = o.state_from_TPY(r["T"], r["p"], r["Y"])
    idx = np.arange(96)
    smp = {"rho": rho, "e": e, "Y": r["Y"], "T": r["T"],
           "strata": [{"idx": idx[:64], "dt": 1e-8, "nsub": 1, "weight": 6400},
                      {"idx": idx[64:], "dt": 2e-8, "nsub": 2, "weight": 320}]}
    # the workload's own temperatures: the oracle run of every stratum in full
    ref = np.array(r["T"], dtype=float)
    for st in smp["strata"]:
        Y, T, h = r["Y"][:, st["idx"]].copy(), r["T"][st["idx"]].copy(), np.full(st["idx"].size, np.nan)
        for _ in range(st["nsub"]):
            out = o.integrate(rho[st["idx"]], e[st["idx"]], Y, T, st["dt"], bench.RTOL, bench.ATOL, h0=h)
            Y, T, h = out["Y"], out["T"], out["h"]
        ref[st["idx"]] = T
    res = bench.oracle_config("two strata", smp, True, 60.0, {"self": ref})
    a = res["all_cores"]
    assert a["workload_cells"] == 6720 and a["extrapolated"] and a["sample_cells"] <= 96
    assert a["value"] > 0 and a["all_status_ok"]
    # the rate is the workload's cells over the per-stratum extrapolated time
    assert 0 < a["value"] * a["seconds"] < 6720 * 1.0001
    assert res["one_core"]["cores"] == 1
    assert res["vs_gpu_on_sample"]["self"] == 0.0
    assert res["config"] == "two strata"
