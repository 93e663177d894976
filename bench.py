"""Benchmark: chemistry cells integrated per second over one hydro dt.

Workload: the uniform 2D detonation slice, 1024 x 1024 = 1,048,576 cells, seeded 1D
detonation-like profile extruded with +-2 % noise (chem_inputs.workloads.detonation_slice,
seed 1), dt = 2e-9 s, rtol 1e-6, atol 1e-10, fp64 state.  A step is one integration of
every cell over dt (the whole hot path: temperature solves, rates, low-storage RK
stages, step control), from the same pristine state each time; the restore copy and
an L2 flush (a 256 MB write, the inputs are 96 MB < 129 MB L2) are inside the timed
region, so the reported rate slightly understates the kernel.

Variants: plain fp64, mixed precision (fp32 rates and stages, fp64 temperature solve,
Gibbs terms, registers and control) and the hybrid (the learned surrogate with its
error test, mixed-precision integration of the cells it rejects), each timed over K
steps; the headline is the fastest variant whose error against the FP64 result meets
its stated bound (mixed: 1e-5, hybrid: 1e-3 relative on T).  Every variant's rate,
error and roofline fraction is in "variants".

The shock-bubble leg ("shock_bubble") is the full hybrid on the 256^3 reactive
shock-bubble field (chem_inputs.workloads.shock_bubble: 16.7M cells, AMR-like levels
with 2^l substeps of 1e-8 / 2^l s): the surrogate, trained on the field's own state
family (workloads.bubble_trajectory_starts), with its error test and the persistent
work-stealing integrator (mixed precision) for the cells it rejects, per level,
against plain fp64 and mixed batched integration of the whole field in one persistent
launch.

The Eq. 27 leg ("eq27") is the paper's own thread-divergence benchmark (Sec. 4.2.2,
Eq. 27-28, Tables 4-5): 65,536 cells of H2 : O2 : N2 = 1 : 2 : 7 at 1 atm with the
smooth (alpha = 1) and the divergent (alpha = 0.1) temperature profile, 100 successive
steps of 1e-5 s (h and the temperature carried), timed as 100 chem_integrate calls and
as one persistent launch with 100 substeps; the paper's V100 times (4.40 s and 5.12 s,
its 13-species mechanism) are context, not a like-for-like target.

The surrogate leg ("surrogate") is the learned part's own workload: 48,000 seeded 0D
ignition trajectories (phi U[0.5, 2], T0 U[900, 2200] K, p U[1, 30] atm) recorded by the
GPU integrator, 2M (state, dt ~ logU[1e-9, 1e-7] s) -> state training pairs from 90 % of
them, training on the GPU (batch 4096), and inference on 16,777,216 cells drawn from the
held-out 10 %, against plain fp64 and mixed integration of the same cells.

Legs of one run (rank 0 prints one JSON line):
  surrogate data generation, training and inference (above; skipped by --no-surrogate,
            which also drops the hybrid variant);
  value     device-resident throughput (cells/s) of the headline variant;
  e2e       the same through chem_integrate_host: host buffers (pinned), H2D + D2H
            copies inside the timed region;
  roofline  credited FP64 flops per launch / CUDA-event launch time vs the FP64 peak;
  cpu_baseline  the CPU oracle on a bounded sample of the same workload (rank 0, N=1).
--impl reference runs only the oracle (the deliberately slow plain CPU program).
Under torchrun each rank integrates its own full slice (independent cells, weak
scaling, no collective on the data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DT, RTOL, ATOL = 2e-9, 1e-6, 1e-10
METRIC = "chem cells/s per hydro dt at stated error vs FP64; learned+batched vs plain"
WORKLOAD = "detonation slice 1024x1024 (1,048,576 cells), H2-air 9 sp / 21 rx, dt=2e-9 s, rtol 1e-6, atol 1e-10"


def _jsonable(o):
    """numpy scalars and arrays in the JSON line as plain numbers and lists."""
    if isinstance(o, np.generic):
        return o.item()
    if isinstance(o, np.ndarray):
        return o.tolist()
    raise TypeError(f"not serialisable: {type(o).__name__}")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-amr", action="store_true", help="skip the AMR-batch comparison leg")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned surrogate (leg and variant)")
    ap.add_argument("--sur-traj", type=int, default=48000)
    ap.add_argument("--sur-epochs", type=int, default=100)
    ap.add_argument("--sur-cells", type=int, default=1 << 24)
    ap.add_argument("--no-bubble", action="store_true", help="skip the shock-bubble hybrid leg")
    ap.add_argument("--no-eq27", action="store_true", help="skip the Eq. 27 divergence benchmark leg")
    ap.add_argument("--no-mech13", action="store_true", help="skip the 13-species mechanism leg")
    ap.add_argument("--no-znd", action="store_true", help="skip the 1D Strang-split detonation leg")
    ap.add_argument("--no-cpu-configs", action="store_true",
                    help="skip the oracle timings of configs 0, 2, 3 and 4")
    ap.add_argument("--no-comparators", action="store_true",
                    help="skip the full-storage / RKF45 comparator leg")
    ap.add_argument("--bubble-n", type=int, default=256)
    ap.add_argument("--cpu-sample", type=int, default=131072)
    ap.add_argument("--ref-sample", type=int, default=32768)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def max_over_ranks(vals, world, device):
    """Element-wise maximum of a list of floats over all ranks (the slowest rank's
    timings); the identity for one rank."""
    if world <= 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_rate(world, cells_per_rank, steps, elapsed):
    """Whole-job throughput: every rank integrates its own cells_per_rank each step
    (weak scaling), timed by the slowest rank."""
    return world * cells_per_rank * steps / elapsed


# ----------------------------------------------------------------- clocks sampler
class Clocks:
    """nvidia-smi sampling during the timed region (every 200 ms)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------- CPU oracle leg
def cpu_oracle(sample_cells: int, nx: int, ny: int, gpu_out=None):
    """Time the CPU oracle on a seeded sample of the workload; optionally compare the
    GPU result on the same cells (parity of the benchmarked run)."""
    import oracle
    from chem_inputs import mechanism, workloads
    d = workloads.detonation_slice(nx, ny, seed=1)
    n = d["T"].size
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(n, min(sample_cells, n), replace=False))
    o = oracle.Oracle(mechanism.build(0))
    rho, e = o.state_from_TPY(d["T"][idx], d["p"][idx], d["Y"][:, idx])
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = o.integrate(rho, e, d["Y"][:, idx], d["T"][idx], DT, RTOL, ATOL, nthreads=cores)
    el = time.perf_counter() - t0
    res = {"value": idx.size / el, "unit": "cells/s", "cores": cores, "kind": "oracle",
           "sample": f"{idx.size} cells drawn uniformly (seed 2024) from the {n}-cell slice, "
                     f"plain fp64 C, OpenMP over cells, {el:.2f} s wall"}
    # one core, on the first 8192 cells of the same sample
    m = min(8192, idx.size)
    t0 = time.perf_counter()
    o.integrate(rho[:m], e[:m], d["Y"][:, idx[:m]], d["T"][idx[:m]], DT, RTOL, ATOL, nthreads=1)
    res["single_core"] = {"value": m / (time.perf_counter() - t0), "unit": "cells/s", "cores": 1,
                          "sample": f"the first {m} cells of the sample"}
    parity = None
    if gpu_out is not None:
        Yg, Tg = gpu_out["Y"][:, idx], gpu_out["T"][idx]
        edge = ref["margin"] < 1e-7
        relT = np.abs(Tg - ref["T"]) / ref["T"]
        absY = np.abs(Yg - ref["Y"]).max(axis=0)
        parity = {"cells": int(idx.size), "knife_edge_cells": int(edge.sum()),
                  "max_rel_T": float(relT[~edge].max()), "max_abs_Y": float(absY[~edge].max()),
                  "steps_equal": bool(np.array_equal(gpu_out["nsteps"][idx][~edge], ref["nsteps"][~edge]))}
    return res, parity


def _oracle_strata(o, smp, nthreads, frac=1.0, carry_h=True):
    """The oracle on each stratum of a sample (a leading fraction of its cells): nsub
    substeps of the stratum's dt, h carried between substeps when carry_h.  Returns per
    stratum the wall seconds, cell count, stratum weight (its cells in the whole
    workload), cell indices and final T."""
    out = []
    for st in smp["strata"]:
        idx = st["idx"][: max(1, int(round(len(st["idx"]) * frac)))]
        Y, T = smp["Y"][:, idx].copy(), smp["T"][idx].copy()
        h = np.full(idx.size, np.nan)
        t0 = time.perf_counter()
        for _ in range(st["nsub"]):
            r = o.integrate(smp["rho"][idx], smp["e"][idx], Y, T, st["dt"], RTOL, ATOL,
                            h0=h if carry_h else None, nthreads=nthreads)
            Y, T, h = r["Y"], r["T"], r["h"]
        out.append({"seconds": time.perf_counter() - t0, "cells": int(idx.size), "weight": int(st["weight"]),
                    "idx": idx, "T": T, "status": r["status"]})
    return out


def oracle_config(name, smp, carry_h, budget_s, gpu_T=None):
    """cpu_baseline of one configuration: the oracle (as it stands, OpenMP over cells) on
    a seeded stratified sample, all host cores and one core, each stratum's time
    extrapolated to the workload by its weight (labelled "extrapolated" when the sample
    is not the whole workload).  A 1/16 pilot sizes the sample to about budget_s of
    all-core work.  gpu_T: {label: GPU temperatures of the workload's cells} compared on
    the sampled cells (max relative difference)."""
    import oracle
    from chem_inputs import mechanism
    o = oracle.Oracle(smp.get("mech") or mechanism.build(0))
    cores = os.cpu_count() or 1
    pilot = sum(r["seconds"] for r in _oracle_strata(o, smp, cores, 1.0 / 16.0, carry_h))
    frac = float(min(1.0, budget_s / max(16.0 * pilot, 1e-9)))
    res = {}
    for label, nthreads, f in (("all_cores", cores, frac), ("one_core", 1, frac / 16.0)):
        rs = _oracle_strata(o, smp, nthreads, f, carry_h)
        cells = sum(r["cells"] for r in rs)
        total = sum(r["weight"] for r in rs)
        t_extra = sum(r["weight"] * r["seconds"] / r["cells"] for r in rs)
        res[label] = {"value": total / t_extra, "unit": "cells/s", "cores": nthreads, "kind": "oracle",
                      "sample_cells": cells, "workload_cells": total,
                      "extrapolated": cells < total,
                      "sample": f"{cells} of {total} cells, stratified ({len(rs)} strata), seeded; "
                                f"per-stratum time x stratum size",
                      "seconds": sum(r["seconds"] for r in rs)}
        if label == "all_cores":
            ok = all(np.all(r["status"] == 0) for r in rs)
            res[label]["all_status_ok"] = bool(ok)
            if gpu_T:
                idx = np.concatenate([r["idx"] for r in rs])
                To = np.concatenate([r["T"] for r in rs])
                res["vs_gpu_on_sample"] = {k: float(np.max(np.abs(v[idx] - To) / To)) for k, v in gpu_T.items()}
    res["config"] = name
    return res


def cpu_baselines(args, reactors_state, amr_sample, sur_sample, bubble_sample):
    """The oracle on every workload (rank 0, N = 1): the 4096 reactors whole; the AMR
    batch, the surrogate's held-out cells and the shock-bubble field on seeded stratified
    samples (extrapolated); the detonation slice is the headline cpu_baseline."""
    from chem_inputs import mechanism, workloads
    out = {}
    if reactors_state is not None:
        r = reactors_state
        smp = {"rho": r["rho"], "e": r["e"], "Y": r["Y"], "T": r["T"],
               "strata": [{"idx": np.arange(r["T"].size), "dt": 1e-7, "nsub": 1, "weight": r["T"].size}]}
        out["reactors_4096"] = oracle_config("4096 reactors, dt 1e-7 s", smp, True, 10.0,
                                            {"fp64": r["gpu_T"]})
    if amr_sample:
        out["amr_batch_256_boxes"] = oracle_config("AMR-like batch, 256 boxes, 3 levels", amr_sample, True, 15.0,
                                                  {amr_sample["variant"]: amr_sample["gpu_T"]})
    if sur_sample is not None:
        for dt in SUR_DTS:
            smp = dict(sur_sample)
            n = smp["T"].size if dt < 1e-7 else min(smp["T"].size, 16384)
            smp["strata"] = [{"idx": np.arange(n), "dt": dt, "nsub": 1, "weight": args.sur_cells}]
            out[f"surrogate_heldout_cells_dt={dt:g}"] = oracle_config(
                f"held-out surrogate cells, dt {dt:g} s (uniform sample)", smp, True, 10.0)
    if bubble_sample is not None:
        out["shock_bubble_256cubed"] = oracle_config(
            "256^3 shock-bubble field, 4 levels, dt 1e-8 s", bubble_sample, False, 15.0,
            {"plain_fp64": bubble_sample["gpu_T_plain"], "hybrid": bubble_sample["gpu_T_hybrid"]})
    return out


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores: W untimed and K timed steps, each one
    integration of a bounded seeded sample of the workload from the same state."""
    if rank != 0:
        return
    import oracle
    from chem_inputs import mechanism, workloads
    d = workloads.detonation_slice(args.nx, args.ny, seed=1)
    n = d["T"].size
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(n, min(args.ref_sample, n), replace=False))
    o = oracle.Oracle(mechanism.build(0))
    rho, e = o.state_from_TPY(d["T"][idx], d["p"][idx], d["Y"][:, idx])
    cores = os.cpu_count() or 1
    run = lambda: o.integrate(rho, e, d["Y"][:, idx], d["T"][idx], DT, RTOL, ATOL, nthreads=cores)
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    el = time.perf_counter() - t0
    res = {"value": idx.size * args.steps / el, "unit": "cells/s", "cores": cores, "kind": "oracle",
           "sample": f"{idx.size} cells drawn uniformly (seed 2024) from the {n}-cell slice per step, "
                     f"{args.steps} timed steps, plain fp64 C, OpenMP over cells"}
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": "cells/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "variant": "cpu oracle"},
            "cpu_baseline": res,
            "e2e": {"value": res["value"], "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line, default=_jsonable), flush=True)


# ----------------------------------------------------------------- GPU leg
VARIANTS = (("fp64", 0.0), ("mixed", 1e-5), ("hybrid", 1e-3))  # (variant, stated error bound on T vs FP64)
MLP_FLOPS_PER_ROW = 2 * (16 * 256 + 256 * 256 * 2 + 256 * 16)  # padded 16-256-256-256-16 network
# DRAM bytes (read + write) per cell of one k_lsrk launch (dram__bytes_read.sum +
# dram__bytes_write.sum), from an ncu capture of the 131,072-cell slice, scaled by the
# cell count; to be set to None whenever the kernel changes until it is captured again.
# fp64: 12.84 MB per 131,072-cell launch (mean of 4 launches of the current kernel);
# mixed (32 warps per SM, spilling): 12.75 MB read + 7.75 MB written (spill lines evicted
# from L2), mean of 4 launches of the current kernel
TRAFFIC_PER_CELL = {"fp64": 12.841984e6 / 131072, "mixed": 20.507712e6 / 131072}


def _bf16_peak():
    """Measured dense BF16 peak (TFLOP/s, cuBLAS burst) of this GPU model."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


BF16_PEAK_TFLOPS, BF16_PEAK_KIND = _bf16_peak()


def timed(fn, reps, stream):
    """Best CUDA-event time (ms) of fn() over reps calls, after one untimed call."""
    import torch
    fn()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


FALLBACK_REASONS = ("range", "residual", "negative", "temperature", "reactive", "error")


def fallback_reasons(mask):
    """Fraction of cells per rejection reason of chem_surrogate_infer's fallback mask."""
    import torch
    counts = torch.bincount(mask.long().flatten(), minlength=7).cpu().numpy()
    n = max(int(mask.numel()), 1)
    return {name: float(counts[i + 1]) / n for i, name in enumerate(FALLBACK_REASONS)}


# The conventional explicit comparators (full k-storage) and the one-pass block shape
# each runs fastest in on GB300 (measured over 64 / 128 / 256 threads per block).
COMPARATORS = {"fp64": (("lsrk", 128), ("full", 128), ("rkf45", 128)),
               "mixed": (("lsrk", 64), ("full", 64), ("rkf45", 64))}


def comparators_leg(mech, rho, e, Y0, T0, Y, T, nsteps, flush, steps, stream):
    """The paper's comparison of its two-register scheme with standard explicit RK that
    keeps every stage derivative (Sec. 2.2.3, Sec. 4.2.2), on the benchmark slice: the
    same RK4(3)5 tableau with full k-storage and Fehlberg's RKF45, one-pass launches,
    each the median of `steps` CUDA-event-timed launches from the pristine state (L2
    flushed), with the compiled kernel's registers and spills."""
    import torch
    from paper_2506_02602_gb300 import build, chem
    n = T0.numel()
    out = {}
    for variant, cfgs in COMPARATORS.items():
        base = None
        for scheme, block in cfgs:
            ctx = chem.Context(mech, variant, scheme=scheme, block_size=block)
            ts = []
            for k in range(steps + 1):
                Y.copy_(Y0)
                T.copy_(T0)
                flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.integrate(rho, e, Y, T, DT, RTOL, ATOL, nsteps=nsteps, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                if k:
                    ts.append(a.elapsed_time(b))
            ms = float(np.median(ts))
            if base is None:
                base = ms
            out[f"{variant} {scheme}"] = {"block": block, "ms": ms, "cells_per_s": n / (ms * 1e-3),
                                          "attempted_steps": int(nsteps.sum()),
                                          "time_vs_lsrk": ms / base}
            ctx.close()
    out["registers"] = build.kernel_resources("4chem6k_lsrkI")
    return out


def mech13_leg(steps, dev, stream, flush, ref9):
    """The 13-species / 27-reaction mechanism (the paper's mechanism size, Sec. 5.2.3) on
    the 13-species detonation slice (workloads.detonation_slice13: the benchmark slice
    with its N2 split into N2 / Ar / He and CO, CO2 traces), through libchem_h2o2_13.so:
    fp64 and mixed one-pass launches, median of `steps` CUDA-event-timed launches from the
    pristine state (L2 flushed), credited flops against the FP64 peak, and the compiled
    kernels' registers and spills beside the 9-species ones (the register budget of the
    paper's Sec. 4.1.2 at its own species count)."""
    import torch
    from chem_inputs import mechanism, workloads
    from paper_2506_02602_gb300 import build, chem, roofline
    m13 = mechanism.build13(0)
    d = workloads.detonation_slice13(mech=m13)
    n = d["T"].size
    T0 = torch.tensor(d["T"], dtype=torch.float64, device=dev)
    Y0 = torch.tensor(d["Y"], dtype=torch.float64, device=dev)
    out = {"workload": f"13-species detonation slice, {n} cells, dt={DT:g} s", "cells": n}
    ctx0 = chem.Context(m13, "fp64")
    rho, e = ctx0.state_from_TPY(T0, torch.tensor(d["p"], dtype=torch.float64, device=dev), Y0)
    ctx0.close()
    Y, T = Y0.clone(), T0.clone()
    ns = torch.empty(n, dtype=torch.int32, device=dev)
    res = {}
    for variant in ("fp64", "mixed"):
        ctx = chem.Context(m13, variant)
        ts = []
        for k in range(steps + 1):
            Y.copy_(Y0)
            T.copy_(T0)
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.integrate(rho, e, Y, T, DT, RTOL, ATOL, nsteps=ns, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            if k:
                ts.append(a.elapsed_time(b))
        ms = float(np.median(ts))
        steps_tot = int(ns.sum())
        if variant == "fp64":
            flops = roofline.launch_flops(steps_tot, n, m13)
        else:
            flops = roofline.launch_flops_mixed_fp64(steps_tot, n, m13)
        achieved = flops / (ms * 1e-3) / 1e9
        res[variant] = {"ms": ms, "cells_per_s": n / (ms * 1e-3), "attempted_steps": steps_tot,
                        "credited_gflop_per_launch": flops / 1e9, "achieved_gflops": achieved,
                        "frac_of_fp64_peak": achieved / roofline.FP64_PEAK_GFLOPS}
        ctx.close()
        if ref9 is not None and variant in ref9:
            res[variant]["cells_per_s_9sp"] = ref9[variant]["value"]
            res[variant]["frac_9sp"] = ref9[variant]["roofline"]["frac"]
    out.update(res)
    out["step_flops"] = {"9sp": roofline.step_flops(mechanism.build(0)), "13sp": roofline.step_flops(m13)}
    out["registers_13sp"] = build.kernel_resources("4chem6k_lsrkI", build.LIBS["h2o2_13"]["build"])
    return out


def znd_leg(mech, dev, stream, n=2048, dx=25e-6, t_end=2e-5, cfl=0.45):
    """The split scheme end to end (Sec. 2.2.1): a 1D detonation in stoichiometric H2-air
    at 300 K and 1 atm, initiated by a driver of the same mixture at 3000 K and 30 atm in
    the left 4 % of a closed tube (wall at the left, transmissive at the right), advanced
    by chem_strang_step at the CFL limit (chem_euler1d_max_speed) for t_end.  Reported:
    the front's speed (a linear fit of the position where T first exceeds 1500 K, from the
    right, over the second half of the run), the peak pressure and temperature behind
    it, the step count and the wall time.  Qualitative context for the shape of the paper's Table 13 (its values
    are for Burke's mechanism in a full solver)."""
    import torch
    from chem_inputs import workloads
    from paper_2506_02602_gb300 import chem
    ctx = chem.Context(mech, "fp64")
    f64 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x = (np.arange(n) + 0.5) * dx
    drv = x < 0.04 * n * dx
    Y = np.repeat(workloads.mass_from_mole(workloads.h2_air_mole(np.array([1.0]))), n, axis=1)
    T0 = np.where(drv, 3000.0, 300.0)
    p0 = np.where(drv, 30.0, 1.0) * workloads.ATM
    Tg, Yg = f64(T0), f64(Y)
    rho, e = ctx.state_from_TPY(Tg, f64(p0), Yg)
    U = {"rho": rho, "rhou": torch.zeros_like(rho), "rhoE": rho * e, "rhoY": rho[None, :] * Yg,
         "T": Tg.clone()}
    st = torch.zeros(n, dtype=torch.int32, device=dev)
    t, steps, hist = 0.0, 0, []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while t < t_end * (1 - 1e-12):
        dt = min(cfl * dx / ctx.euler1d_max_speed(U, stream=stream), t_end - t)
        ctx.strang_step(U, dx, dt, (1, 0), RTOL, ATOL, status=st, stream=stream)
        t += dt
        steps += 1
        if steps % 50 == 0:
            T = U["T"].cpu().numpy()
            hot = np.flatnonzero(T > 1500.0)
            hist.append((t, float(x[hot[-1]]) if hot.size else 0.0))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    T = U["T"].cpu().numpy()
    rho_h = U["rho"].cpu().numpy()
    Yh = (U["rhoY"] / U["rho"][None, :]).cpu().numpy()
    p = rho_h * 8.31446261815324 * T * (Yh / np.asarray(mech["W"])[:, None]).sum(axis=0)
    h = np.array(hist)
    half = h[h[:, 0] >= 0.5 * t_end]
    speed = float(np.polyfit(half[:, 0], half[:, 1], 1)[0]) if len(half) > 2 else None
    ctx.close()
    return {"cells": n, "dx_m": dx, "t_end_s": t_end, "steps": steps, "wall_s": wall,
            "cell_steps_per_s": n * steps / wall,
            "per_step": "a CFL reduction (synchronous) + chemistry dt/2, Euler dt, chemistry dt/2; "
                        "2048 cells are a latency case, not a throughput one",
            "front_speed_m_s": speed, "front_position_m": float(h[-1, 1]) if len(h) else None,
            "peak_pressure_atm": float(p.max() / 101325.0), "peak_T_K": float(T.max()),
            "all_status_ok": bool((st == 0).all()),
            "note": "synthetic 9-species mechanism; H2-air CJ speed is about 1970 m/s for real kinetics"}


def eq27_leg(mech, dev, stream):
    """The Eq. 27 thread-divergence benchmark (module docstring)."""
    import torch
    from chem_inputs import workloads
    from paper_2506_02602_gb300 import chem
    out = {"cells": 65536, "steps": 100, "dt": 1e-5,
           "paper_v100_s": {"alpha=1": 4.4032, "alpha=0.1": 5.1225},
           "paper_note": "the paper's V100 runs: LSRK about 3x faster than RKF45 and 6x than CVODE"}
    for variant in ("fp64", "mixed"):
        # the comparators on the same field: 100 one-pass calls each
        for scheme, block in COMPARATORS[variant][1:]:
            ctx = chem.Context(mech, variant, scheme=scheme, block_size=block)
            for alpha in (1.0, 0.1):
                w = workloads.eq27_profile(alpha)
                f64 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
                T0, Y0 = f64(w["T"]), f64(w["Y"])
                rho, e = ctx.state_from_TPY(T0, f64(w["p"]), Y0)
                Y, T = Y0.clone(), T0.clone()
                h = torch.empty(T0.numel(), dtype=torch.float64, device=dev)

                def calls():
                    Y.copy_(Y0); T.copy_(T0); h.fill_(float("nan"))
                    for _ in range(100):
                        ctx.integrate(rho, e, Y, T, 1e-5, RTOL, ATOL, h=h, stream=stream)

                out[f"{variant} {scheme} alpha={alpha:g}"] = {"calls_s": timed(calls, 1, stream) * 1e-3}
            ctx.close()
        ctx = chem.Context(mech, variant)
        for alpha in (1.0, 0.1):
            w = workloads.eq27_profile(alpha)
            n = w["T"].size
            f64 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
            T0, Y0 = f64(w["T"]), f64(w["Y"])
            rho, e = ctx.state_from_TPY(T0, f64(w["p"]), Y0)
            Y, T = Y0.clone(), T0.clone()
            h = torch.empty(n, dtype=torch.float64, device=dev)
            st = torch.empty(n, dtype=torch.int32, device=dev)

            def calls():
                Y.copy_(Y0); T.copy_(T0); h.fill_(float("nan"))
                for _ in range(100):
                    ctx.integrate(rho, e, Y, T, 1e-5, RTOL, ATOL, h=h, status=st, stream=stream)

            off = torch.tensor([0, n], dtype=torch.int64, device=dev)
            bdt = torch.tensor([1e-5], dtype=torch.float64, device=dev)
            bsub = torch.tensor([100], dtype=torch.int32, device=dev)

            def persistent():
                Y.copy_(Y0); T.copy_(T0); h.fill_(float("nan"))
                ctx.integrate_batched(rho, e, Y, T, off, bdt, bsub, RTOL, ATOL, h=h, status=st, stream=stream)

            t_calls = timed(calls, 1, stream)
            Tc, ok_c = T.clone(), bool((st == 0).all())
            t_pers = timed(persistent, 1, stream)
            for scheme, _ in COMPARATORS[variant][1:]:
                r = out[f"{variant} {scheme} alpha={alpha:g}"]
                r["time_vs_lsrk_calls"] = r["calls_s"] / (t_calls * 1e-3)
            out[f"{variant} alpha={alpha:g}"] = {
                "calls_s": t_calls * 1e-3, "persistent_s": t_pers * 1e-3,
                "cell_substeps_per_s": n * 100 / (min(t_calls, t_pers) * 1e-3),
                "all_ok": ok_c and bool((st == 0).all()),
                "max_rel_T_calls_vs_persistent": float(((T - Tc).abs() / Tc).max()),
                "T_final_range_K": [float(T.min()), float(T.max())]}
        ctx.close()
    return out


def shock_bubble_leg(args, mech, dev, stream, flush):
    """The full hybrid on the shock-bubble field (module docstring): "learned + batched
    against plain", each path timed as the median of K steps (CUDA events, state restored
    and L2 flushed before each): plain fp64 and mixed batched integration of every level
    and substep in one persistent launch, and the hybrid in one chem_surrogate_infer_batched
    call (network, error test and one persistent fallback launch per substep round); the
    per-box Python loop of chem_surrogate_infer calls is timed beside it.  Returns the
    summary and a level-stratified host sample of the field for the oracle."""
    import torch
    from chem_inputs import workloads
    from paper_2506_02602_gb300 import chem, surrogate
    out = {}
    t0 = time.perf_counter()
    b = workloads.shock_bubble(args.bubble_n)
    n = b["T"].size
    plain = chem.Context(mech, "fp64")
    mixed = chem.Context(mech, "mixed")
    f64 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    T0, Y0 = f64(b["T"]), f64(b["Y"])
    rho, e = plain.state_from_TPY(T0, f64(b["p"]), Y0)
    del b["p"]
    off = torch.tensor(b["box_offset"], dtype=torch.int64, device=dev)
    bdt = f64(b["box_dt"])
    nsub = torch.tensor(b["box_nsub"], dtype=torch.int32, device=dev)
    subs = int((np.diff(b["box_offset"]) * np.asarray(b["box_nsub"])).sum())
    out["field"] = {"cells": int(n), "cell_substeps": subs,
                    "levels": [int(x) for x in np.diff(b["box_offset"])][::-1],
                    "box_dt": [float(x) for x in b["box_dt"]][::-1], "setup_s": time.perf_counter() - t0}
    # surrogate for this field's state family
    t0 = time.perf_counter()
    gen = chem.Context(mech, "fp64", max_steps=4000)
    starts = workloads.bubble_trajectory_starts(16000, seed=5)
    st = surrogate.trajectory_states(gen, 16000, seed=5, starts=starts)
    gen.close()
    pairs = surrogate.make_pairs(plain, st, seed=5, dt_lo=1e-9, dt_hi=1e-8, max_pairs=2_000_000)
    hyb = chem.Context(mech, "mixed")
    loss = hyb.surrogate_train(pairs["rho"], pairs["e"], pairs["Y0"], pairs["dt"], pairs["Y1"], T0=pairs["T0"],
                               epochs=60, batch=4096, lr=1e-3, seed=1, dt_power=1.0)
    torch.cuda.synchronize()
    out["train"] = {"trajectories": 16000, "pairs": int(pairs["T0"].numel()), "epochs": 60,
                    "loss_first_last": [float(loss[0]), float(loss[-1])], "seconds": time.perf_counter() - t0}
    del pairs, st
    Y, T = Y0.clone(), T0.clone()
    mask = torch.empty(n, dtype=torch.uint8, device=dev)
    K = max(3, args.steps)

    def med(fn, reps):
        ts = []
        for k in range(reps + 1):
            Y.copy_(Y0)
            T.copy_(T0)
            flush.fill_(1.0)
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            c.record(stream)
            torch.cuda.synchronize()
            if k:
                ts.append(a.elapsed_time(c))
        return float(np.median(ts)), len(ts)

    t_plain, k1 = med(lambda: plain.integrate_batched(rho, e, Y, T, off, bdt, nsub, RTOL, ATOL, stream=stream), K)
    Yr, Tr = Y.clone(), T.clone()
    t_mixed, k2 = med(lambda: mixed.integrate_batched(rho, e, Y, T, off, bdt, nsub, RTOL, ATOL, stream=stream), K)
    rel_m = float(((T - Tr).abs() / Tr).max())
    t_hyb, k3 = med(lambda: hyb.surrogate_infer_batched(rho, e, Y, T, off, bdt, nsub, RTOL, ATOL, mask=mask,
                                                        stream=stream), K)
    rel = (T - Tr).abs() / Tr
    fb = float((mask != 0).float().mean())
    reasons = fallback_reasons(mask)
    Yh, Th = Y.clone(), T.clone()
    t_loop, _ = med(lambda: surrogate.hybrid_levels(hyb, rho, e, Y, T, b["box_offset"], b["box_dt"], b["box_nsub"],
                                                    RTOL, ATOL, mask=mask, stream=stream), 3)
    same = bool(torch.equal(Y, Yh) and torch.equal(T, Th))
    out["steps_timed"] = K
    out["plain_fp64"] = {"cells_per_s": n / (t_plain * 1e-3), "ms_per_step": t_plain}
    out["mixed"] = {"cells_per_s": n / (t_mixed * 1e-3), "ms_per_step": t_mixed, "max_rel_T": rel_m}
    out["hybrid"] = {"cells_per_s": n / (t_hyb * 1e-3), "ms_per_step": t_hyb, "max_rel_T": float(rel.max()),
                     "entry": "chem_surrogate_infer_batched",
                     "fallback_frac_last_substep": fb, "fallback_reasons_last_substep": reasons,
                     "speedup_vs_plain_fp64": t_plain / t_hyb, "speedup_vs_mixed": t_mixed / t_hyb,
                     "per_box_loop_ms_per_step": t_loop, "per_box_loop_identical": same}
    out["stated_error_T"] = 1e-3
    # the oracle's sample: 16,384 cells per level (stratified), host arrays
    rng = np.random.default_rng(44)
    offh = b["box_offset"]
    samp = []
    for lv in range(len(offh) - 1):
        a0, a1 = int(offh[lv]), int(offh[lv + 1])
        idx = np.sort(rng.choice(np.arange(a0, a1), min(16384, a1 - a0), replace=False))
        samp.append({"idx": idx, "dt": float(b["box_dt"][lv]), "nsub": int(b["box_nsub"][lv]),
                     "weight": a1 - a0})
    sample = {"rho": rho.cpu().numpy(), "e": e.cpu().numpy(), "Y": b["Y"], "T": b["T"], "strata": samp,
              "gpu_T_plain": Tr.cpu().numpy(), "gpu_T_hybrid": Th.cpu().numpy()}
    for c in (plain, mixed, hyb):
        c.close()
    return out, sample


SUR_DTS = (1e-9, 1e-8, 1e-7)


def surrogate_leg(args, mech, dev, stream, flush):
    """Data generation, training and inference of the learned surrogate (module docstring).
    Trajectories are split three ways by whole trajectories: 80 % train, 10 % validation
    (the error test's thresholds are tuned there, per dt, surrogate.tune_gate) and 10 %
    held out (reported).  Per dt of 1e-9, 1e-8 and 1e-7 s: the held-out cells (16.7M at
    the two smaller dt, 4.2M at 1e-7 s, where plain fp64 integration is slow) with plain
    fp64, mixed and surrogate integration, each timed as the median of K launches (L2
    flushed), errors against plain fp64.  Returns the leg's summary, a mixed-precision
    context holding the trained network and a host sample of held-out cells for the oracle."""
    import tempfile

    import torch
    from paper_2506_02602_gb300 import chem, surrogate
    out = {}
    gen = chem.Context(mech, "fp64", max_steps=4000)
    plain = chem.Context(mech, "fp64")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = surrogate.trajectory_states(gen, args.sur_traj, seed=3)
    tr_all, held = surrogate.split_by_trajectory(st, 0.1, seed=3)
    tr, val = surrogate.split_by_trajectory(tr_all, 1.0 / 9.0, seed=4)
    pairs = surrogate.make_pairs(plain, tr, seed=3, max_pairs=2_000_000)
    torch.cuda.synchronize()
    out["data"] = {"trajectories": args.sur_traj, "states": int(st["T"].numel()),
                   "train_pairs": int(pairs["T0"].numel()), "validation_states": int(val["T"].numel()),
                   "heldout_states": int(held["T"].numel()),
                   "split": "by whole trajectory: 80 % train, 10 % validation (gate tuning), 10 % held out",
                   "seconds": time.perf_counter() - t0}
    gen.close()
    del st, tr_all
    hyb = chem.Context(mech, "mixed")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = hyb.surrogate_train(pairs["rho"], pairs["e"], pairs["Y0"], pairs["dt"], pairs["Y1"], T0=pairs["T0"],
                               epochs=args.sur_epochs, batch=4096, lr=1e-3, seed=1, dt_power=1.0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    steps = (pairs["T0"].numel() // 4096) * args.sur_epochs
    out["train"] = {"epochs": args.sur_epochs, "batch": 4096, "adam_steps": int(steps), "seconds": t_train,
                    "loss_first_last": [float(loss[0]), float(loss[-1])],
                    "samples_per_s": steps * 4096 / t_train,
                    "tflops": 3 * MLP_FLOPS_PER_ROW * steps * 4096 / t_train / 1e12}
    del pairs, tr
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "net.bin")
        hyb.surrogate_save(path)
        hyb64 = chem.Context(mech, "fp64")
        hyb64.surrogate_load(path)
    mixed = chem.Context(mech, "mixed")
    # the error test's thresholds per dt, on 1M validation cells
    vcells = surrogate.draw_cells(val, 1 << 20, seed=4)
    gates = {}
    out["gate_tuning"] = {"on": f"{vcells['T'].numel()} validation cells (trajectories not trained on "
                                f"and not reported)", "bound": "max rel T <= 1e-3 / 1.5 over all cells"}
    for dt in SUR_DTS:
        g, table = surrogate.tune_gate(hyb, plain, vcells, dt)
        gates[dt] = g
        out["gate_tuning"][f"dt={dt:g}"] = {"chosen": g, "candidates": table}
    del vcells, val
    # the fused network alone on rows of the batch size (the MLP kernel's tensor-pipe roofline)
    Xf = torch.zeros(1 << 22, 16, dtype=torch.float32, device=dev)
    Xf[:, :12].normal_()
    t_mlp = timed(lambda: hyb.surrogate_forward(Xf, stream=stream), 3, stream)
    out["mlp_kernel"] = {"rows": int(Xf.shape[0]), "ms": t_mlp,
                         "tflops": Xf.shape[0] * MLP_FLOPS_PER_ROW / (t_mlp * 1e-3) / 1e12}
    del Xf
    cells_all = surrogate.draw_cells(held, args.sur_cells, seed=3)
    # a host sample for the oracle (its cpu_baseline on this workload)
    rng = np.random.default_rng(33)
    pick = torch.tensor(np.sort(rng.choice(cells_all["T"].numel(), 65536, replace=False)), device=dev)
    oracle_sample = {k: (v[:, pick] if k == "Y" else v[pick]).cpu().numpy()
                     for k, v in cells_all.items() if k in ("rho", "e", "Y", "T")}
    out["inference"] = {}
    K = max(3, min(args.steps, 10))
    for dt in SUR_DTS:
        n = cells_all["T"].numel() if dt < 1e-7 else min(cells_all["T"].numel(), 1 << 22)
        cells = {k: (v[:, :n] if k == "Y" else v[:n]).contiguous() for k, v in cells_all.items()}
        Y, T = cells["Y"].clone(), cells["T"].clone()
        mask = torch.empty(n, dtype=torch.uint8, device=dev)

        def reset():
            Y.copy_(cells["Y"])
            T.copy_(cells["T"])
            flush.fill_(1.0)

        def med(fn, reps):
            ts = []
            for k in range(reps + 1):
                reset()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                if k:
                    ts.append(a.elapsed_time(b))
            return float(np.median(ts))

        r = {"cells": n, "gate": gates[dt]}
        reps_int = K if dt < 1e-7 else 2
        t = med(lambda: plain.integrate(cells["rho"], cells["e"], Y, T, dt, RTOL, ATOL, stream=stream), reps_int)
        Yr, Tr = Y.clone(), T.clone()
        r["plain_fp64"] = {"cells_per_s": n / (t * 1e-3), "ms": t}
        t = med(lambda: mixed.integrate(cells["rho"], cells["e"], Y, T, dt, RTOL, ATOL, stream=stream), reps_int)
        r["mixed"] = {"cells_per_s": n / (t * 1e-3), "ms": t,
                      "max_rel_T": float(((T - Tr).abs() / Tr).max())}
        for name, ctx in (("surrogate_fp64_fallback", hyb64), ("surrogate_mixed_fallback", hyb)):
            t = med(lambda: ctx.surrogate_infer(cells["rho"], cells["e"], Y, T, dt, RTOL, ATOL, mask=mask,
                                                gate=gates[dt], stream=stream), K)
            rel = (T - Tr).abs() / Tr
            fb = mask.bool()
            r[name] = {"cells_per_s": n / (t * 1e-3), "ms": t, "fallback_frac": float(fb.float().mean()),
                       "fallback_reasons": fallback_reasons(mask),
                       "p999_rel_T": float(torch.quantile(rel[::4].float(), 0.999)),  # every 4th cell
                       "max_rel_T": float(rel.max()),
                       "max_rel_T_accepted": float(rel[~fb].max()) if bool((~fb).any()) else 0.0,
                       "max_abs_Y": float((Y - Yr).abs().max()),
                       "meets_1e-3": float(rel.max()) <= 1e-3,
                       "meets_fallback_0.5pct": float(fb.float().mean()) <= 5e-3,
                       "speedup_vs_plain_fp64": r["plain_fp64"]["ms"] / t,
                       "speedup_vs_mixed": r["mixed"]["ms"] / t}
        out["inference"][f"dt={dt:g}"] = r
        del Yr, Tr, Y, T, cells
    out["heldout_cells"] = int(cells_all["T"].numel())
    out["stated_error_T"] = 1e-3
    out["fallback_target"] = 5e-3
    del cells_all, held
    for c in (plain, hyb64, mixed):
        c.close()
    return out, hyb, oracle_sample


def amr_leg(ctx, steps, dev, sample=None):
    """Ragged AMR-like batch (256 boxes, edges {8,16,24,32}^3, 3 levels with 2^l substeps
    of 1e-7/2^l s, heavy-tailed stiffness): the persistent work-stealing launch, with the
    options chem_autotune_batched picks on this batch, against the plain path of one
    chem_integrate launch per box and substep on 8 streams (one stream per box, round
    robin).  Both run the same per-cell arithmetic; compiled shapes may contract
    multiply-adds differently, so the line reports how far the two agree: the largest
    relative difference in T and the share of cells whose T and Y are bit-identical."""
    import torch
    from chem_inputs import workloads
    b = workloads.amr_batch()
    n = b["T"].size
    T0 = torch.tensor(b["T"], dtype=torch.float64, device=dev)
    p0 = torch.tensor(b["p"], dtype=torch.float64, device=dev)
    Y0 = torch.tensor(b["Y"], dtype=torch.float64, device=dev)
    rho, e = ctx.state_from_TPY(T0, p0, Y0)
    off_h = b["box_offset"]
    off = torch.tensor(off_h, dtype=torch.int64, device=dev)
    dts = torch.tensor(b["box_dt"], dtype=torch.float64, device=dev)
    nsub = torch.tensor(b["box_nsub"], dtype=torch.int32, device=dev)
    Y, T = Y0.clone(), T0.clone()
    h = torch.empty(n, dtype=torch.float64, device=dev)
    ns = torch.empty(n, dtype=torch.int32, device=dev)
    streams = [torch.cuda.Stream(dev) for _ in range(8)]

    def persistent(**opts):
        Y.copy_(Y0); T.copy_(T0); h.fill_(float("nan"))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.integrate_batched(rho, e, Y, T, off, dts, nsub, RTOL, ATOL, h=h, nsteps=ns, **opts)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    # the autotuner on this batch (its own copies of the state; no cache file)
    h.fill_(float("nan"))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tuned, table = ctx.autotune_batched(rho, e, Y0, T0, off, dts, nsub, RTOL, ATOL, h=h)
    t_tune = time.perf_counter() - t0
    persistent()
    t_default = min(persistent() for _ in range(steps))

    def per_box():
        Y.copy_(Y0); T.copy_(T0); h.fill_(float("nan"))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in range(len(off_h) - 1):
            a, z = int(off_h[j]), int(off_h[j + 1])
            st = streams[j % len(streams)]
            for _ in range(int(b["box_nsub"][j])):
                ctx.integrate(rho[a:z], e[a:z], Y[:, a:z], T[a:z], float(b["box_dt"][j]), RTOL, ATOL,
                              h=h[a:z], stream=st, ncells=z - a)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    persistent(**tuned)
    tp = min(persistent(**tuned) for _ in range(steps))
    Yp, Tp, steps_p = Y.cpu().numpy(), T.cpu().numpy(), ns.cpu().numpy()
    per_box()
    tb = min(per_box() for _ in range(steps))
    Yb, Tb = Y.cpu().numpy(), T.cpu().numpy()
    same = (Tb == Tp) & np.all(Yb == Yp, axis=0)
    max_rel_T = float(np.max(np.abs(Tb - Tp) / np.abs(Tp)))
    subs = int((b["box_nsub"].astype(np.int64) * np.diff(off_h)).sum())
    if sample is not None:
        # the oracle's sample, stratified by (stiffness class, level): up to 7,282 cells per
        # stratum (65,536 over the 9 strata), with the GPU result of those cells
        rng = np.random.default_rng(55)
        lev = np.repeat(np.asarray(b["box_level"]), np.diff(off_h))
        boxid = np.repeat(np.arange(len(off_h) - 1), np.diff(off_h))
        strata = []
        for c in range(3):
            for lv in range(3):
                cand = np.flatnonzero((b["cls"] == c) & (lev == lv))
                if cand.size == 0:
                    continue
                idx = np.sort(rng.choice(cand, min(7282, cand.size), replace=False))
                strata.append({"idx": idx, "dt": float(b["box_dt"][boxid[idx[0]]]),
                               "nsub": int(b["box_nsub"][boxid[idx[0]]]), "weight": int(cand.size),
                               "class": c, "level": lv})
        sample.update({"rho": rho.cpu().numpy(), "e": e.cpu().numpy(), "Y": b["Y"], "T": b["T"],
                       "strata": strata, "gpu_T": Tp, "variant": ctx.variant})
    return {"workload": f"AMR-like batch: 256 boxes, {n} cells, {subs} cell-substeps, 3 levels",
            "variant": ctx.variant,
            "persistent_cells_per_s": n / tp, "persistent_ms": 1e3 * tp,
            "autotuned": {"options": tuned, "default_options_ms": 1e3 * t_default, "tuned_ms": 1e3 * tp,
                          "tuning_s": t_tune,
                          "candidates": [{k: r[k] for k in ("shape", "block", "regs", "ctas_per_sm", "order",
                                                            "use_graph", "ms")} for r in table]},
            "per_box_cells_per_s": n / tb, "per_box_ms": 1e3 * tb,
            "speedup": tb / tp, "cell_substeps_per_s": subs / tp,
            "attempted_steps": int(steps_p.sum()), "max_steps": int(steps_p.max()),
            "vs_per_box": {"max_rel_T": max_rel_T, "bit_identical_frac": float(same.mean())}}


def run_ours(args, rank, world, local):
    import torch
    from chem_inputs import mechanism, workloads
    from paper_2506_02602_gb300 import build, chem, roofline

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mech = mechanism.build(0)
    stream = torch.cuda.current_stream(dev)
    sur, ctxs, sur_sample = None, {}, None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    variants = [(v, b) for v, b in VARIANTS if v != "hybrid" or not args.no_surrogate]
    if not args.no_surrogate:
        sur, ctxs["hybrid"], sur_sample = surrogate_leg(args, mech, dev, stream, flush)
    d = workloads.detonation_slice(args.nx, args.ny, seed=1)
    n = d["T"].size
    S = d["Y"].shape[0]
    ctxs.update({v: chem.Context(mech, v) for v, _ in variants if v != "hybrid"})
    T0 = torch.tensor(d["T"], dtype=torch.float64, device=dev)
    p0 = torch.tensor(d["p"], dtype=torch.float64, device=dev)
    Y0 = torch.tensor(d["Y"], dtype=torch.float64, device=dev)
    rho, e = ctxs["fp64"].state_from_TPY(T0, p0, Y0)
    Y, T = Y0.clone(), T0.clone()
    status = torch.empty(n, dtype=torch.int32, device=dev)
    nsteps = torch.empty(n, dtype=torch.int32, device=dev)
    fbmask = torch.empty(n, dtype=torch.uint8, device=dev)

    def step(ctx, ev0=None, ev1=None):
        Y.copy_(Y0)
        T.copy_(T0)
        flush.fill_(1.0)
        if ev0 is not None:
            ev0.record(stream)
        if ctx is ctxs.get("hybrid"):
            ctx.surrogate_infer(rho, e, Y, T, DT, RTOL, ATOL, status=status, nsteps=nsteps, mask=fbmask,
                                stream=stream)
        else:
            ctx.integrate(rho, e, Y, T, DT, RTOL, ATOL, status=status, nsteps=nsteps, stream=stream)
        if ev1 is not None:
            ev1.record(stream)

    clocks = Clocks(local)
    clocks.start()
    res = {}
    for v, _ in variants:
        ctx = ctxs[v]
        for _ in range(args.warmup):
            step(ctx)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            step(ctx, *evs[k])
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        elapsed = time.perf_counter() - t0
        times = [a.elapsed_time(b) for a, b in evs]
        kernel_ms, kernel_med = float(np.mean(times)), float(np.median(times))
        elapsed, kernel_ms, kernel_med = max_over_ranks([elapsed, kernel_ms, kernel_med], world, dev)
        ns = nsteps.cpu().numpy()
        res[v] = {"elapsed": elapsed, "kernel_ms": kernel_ms, "kernel_ms_median": kernel_med, "nsteps": ns,
                  "status": status.cpu().numpy(), "Y": Y.cpu().numpy(), "T": T.cpu().numpy()}
        if v == "hybrid":
            res[v]["fallback_frac"] = float((fbmask != 0).float().mean())
            res[v]["fallback_reasons"] = fallback_reasons(fbmask)
    # the FMA-pipe probe (chem_diag_fma_peak) under the same clock sampling: measured fp64
    # and fp32 FMA throughput beside the unit-count peak the roofline divides by
    f64, _ = chem.fma_peak(0, 152 * 8, 256, 1000, stream=stream)
    f32, _ = chem.fma_peak(1, 152 * 8, 256, 40000, stream=stream)
    probe = {"fp64_gflops": f64, "fp32_gflops": f32, "fp64_unit_peak_gflops": roofline.FP64_PEAK_GFLOPS,
             "fp32_unit_peak_gflops": roofline.FP32_PEAK_GFLOPS,
             "fp64_probe_over_unit_peak": f64 / roofline.FP64_PEAK_GFLOPS,
             "launch": "1216 blocks x 256 threads, 8 independent all-register FMA chains per thread"}
    clk = clocks.stop()

    ref = res["fp64"]
    summary = {}
    for v, bound in variants:
        r = res[v]
        relT = float(np.max(np.abs(r["T"] - ref["T"]) / ref["T"]))
        absY = float(np.max(np.abs(r["Y"] - ref["Y"])))
        if v == "fp64":
            flops = roofline.launch_flops(int(r["nsteps"].sum()), n, mech)
            note = "fp64 pipe; credited flops (exp/log = 20) / CUDA-event launch time"
        elif v == "mixed":
            flops = roofline.launch_flops_mixed_fp64(int(r["nsteps"].sum()), n, mech)
            note = "fp64 pipe; credited fp64 part only (temperature solve, Gibbs, hi/lo splits for ln Kc, fp64 registers, control)"
        if v == "hybrid":
            # the fused network kernel, timed alone on the surrogate leg's rows
            mk = sur["mlp_kernel"]
            rl = {"bound": "tensor", "achieved": mk["tflops"], "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                  "frac": mk["tflops"] / BF16_PEAK_TFLOPS, "traffic": None,
                  "note": "the network's tcgen05 BF16 kernel, timed alone on "
                          f"{mk['rows']} rows; peak = measured cuBLAS bf16 burst"}
        else:
            achieved = flops / (r["kernel_ms"] * 1e-3) / 1e9
            tpc = TRAFFIC_PER_CELL.get(v)
            rl = {"bound": "alu", "achieved": achieved, "peak": roofline.FP64_PEAK_GFLOPS,
                  "unit": "GFLOP/s", "frac": achieved / roofline.FP64_PEAK_GFLOPS,
                  "traffic": None if tpc is None else tpc * n, "note": note +
                  "; traffic = ncu DRAM bytes per cell on a 131,072-cell slice x cells"}
        summary[v] = {
            "value": job_rate(world, n, args.steps, r["elapsed"]), "ms_per_step": 1e3 * r["elapsed"] / args.steps,
            "kernel_ms": r["kernel_ms"], "kernel_ms_median": r["kernel_ms_median"], "stated_error_T": bound,
            "error_vs_fp64_gpu": {"max_rel_T": relT, "max_abs_Y": absY},
            "meets_stated_error": relT <= bound if v != "fp64" else True,
            "attempted_steps": int(r["nsteps"].sum()), "max_steps": int(r["nsteps"].max()),
            "status_ok": int((r["status"] == 0).sum()),
            "roofline": rl,
        }
        if v == "hybrid":
            summary[v]["fallback_frac"] = r["fallback_frac"]
            summary[v]["fallback_reasons"] = r["fallback_reasons"]
    ok = [v for v, _ in variants if summary[v]["meets_stated_error"]]
    head = max(ok, key=lambda v: summary[v]["value"])
    H = summary[head]

    # end to end through the host-buffer entry point (pinned host memory), headline variant
    ctx = ctxs[head]
    pin = lambda a: torch.tensor(a, dtype=torch.float64).pin_memory()
    h_rho, h_e = pin(rho.cpu().numpy()), pin(e.cpu().numpy())
    h_Y0, h_T0 = d["Y"].copy(), d["T"].copy()
    h_Y, h_T = pin(h_Y0), pin(h_T0)
    h_st = torch.empty(n, dtype=torch.int32).pin_memory()
    h_ns = torch.empty(n, dtype=torch.int32).pin_memory()
    hY, hT = h_Y.numpy(), h_T.numpy()

    d_rho, d_e = torch.empty_like(rho), torch.empty_like(e)
    d_Y, d_T = torch.empty_like(Y), torch.empty_like(T)

    def e2e_step():
        """One step through the host-buffer path; returns its wall time.  Restoring the
        host inputs (a benchmark artefact: an application hands over new data) is
        outside the timed part; the host-device copies are inside."""
        hY[...] = h_Y0
        hT[...] = h_T0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if head == "hybrid":  # no host entry point for the surrogate: copies in the timed region
            d_rho.copy_(h_rho, non_blocking=True)
            d_e.copy_(h_e, non_blocking=True)
            d_Y.copy_(h_Y, non_blocking=True)
            d_T.copy_(h_T, non_blocking=True)
            ctx.surrogate_infer(d_rho, d_e, d_Y, d_T, DT, RTOL, ATOL, status=status, nsteps=nsteps,
                                stream=stream)
            h_Y.copy_(d_Y, non_blocking=True)
            h_T.copy_(d_T, non_blocking=True)
            h_st.copy_(status, non_blocking=True)
            h_ns.copy_(nsteps, non_blocking=True)
            torch.cuda.synchronize()
        else:
            ctx.integrate_host(h_rho.numpy(), h_e.numpy(), hY, hT, DT, RTOL, ATOL,
                               status=h_st.numpy(), nsteps=h_ns.numpy(), stream=stream)
        return time.perf_counter() - t0

    e2e_step()
    if world > 1:
        torch.distributed.barrier()
    e2e_el = sum(e2e_step() for _ in range(args.steps))
    e2e_el, = max_over_ranks([e2e_el], world, dev)
    e2e_match = bool(np.array_equal(hY, res[head]["Y"]) and np.array_equal(hT, res[head]["T"]))

    # 4096 independent reactors, dt 1e-7 s (the parity workload): plain fp64 one-pass
    # launches, median of K; the same states are the oracle's sample of this workload
    r0 = workloads.reactors(4096, seed=0)
    T0r = torch.tensor(r0["T"], dtype=torch.float64, device=dev)
    Y0r = torch.tensor(r0["Y"], dtype=torch.float64, device=dev)
    rho_r, e_r = ctxs["fp64"].state_from_TPY(T0r, torch.tensor(r0["p"], dtype=torch.float64, device=dev), Y0r)
    Yr_, Tr_ = Y0r.clone(), T0r.clone()
    ts0 = []
    for k in range(max(3, args.steps) + 1):
        Yr_.copy_(Y0r)
        Tr_.copy_(T0r)
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctxs["fp64"].integrate(rho_r, e_r, Yr_, Tr_, 1e-7, RTOL, ATOL, stream=stream)
        b_.record(stream)
        torch.cuda.synchronize()
        if k:
            ts0.append(a.elapsed_time(b_))
    reactors = {"workload": "4096 reactors, phi U[0.5,2], T0 U[1000,2000] K, p U[0.5,5] atm, dt 1e-7 s",
               "variant": "fp64", "ms": float(np.median(ts0)), "cells_per_s": 4096 / (float(np.median(ts0)) * 1e-3),
               "note": "4096 cells fill 32 of 152 SMs' worth of 128-thread blocks: latency, not throughput"}
    reactors_state = {"rho": rho_r.cpu().numpy(), "e": e_r.cpu().numpy(), "Y": r0["Y"], "T": r0["T"],
                      "gpu_T": Tr_.cpu().numpy()}

    mech13 = None
    if not args.no_mech13:
        mech13 = mech13_leg(max(3, min(args.steps, 5)), dev, stream, flush,
                            {v: summary[v] for v in ("fp64", "mixed") if v in summary})

    comparators = None
    if not args.no_comparators:
        comparators = comparators_leg(mech, rho, e, Y0, T0, Y, T, nsteps, flush, max(3, min(args.steps, 5)),
                                      stream)

    eq27 = None
    if not args.no_eq27:
        eq27 = eq27_leg(mech, dev, stream)

    znd = None
    if not args.no_znd:
        znd = znd_leg(mech, dev, stream)

    bubble, bubble_sample = None, None
    if not args.no_bubble:
        bubble, bubble_sample = shock_bubble_leg(args, mech, dev, stream, flush)

    amr, amr_sample = None, {}
    if not args.no_amr:
        # the batching gain in both precisions: persistent launch against per-box launches
        amr = {v: amr_leg(ctxs[v], max(2, min(args.steps, 3)), dev, amr_sample if v == "fp64" else None)
               for v in ("fp64", "mixed")}

    line = None
    if rank == 0:
        cpu, parity = (None, {})
        if world == 1 and not args.no_cpu_baseline:
            cpu, parity[head] = cpu_oracle(args.cpu_sample, args.nx, args.ny,
                                           {"Y": res[head]["Y"], "T": res[head]["T"],
                                            "nsteps": res[head]["nsteps"]})
        cpu_cfgs = None
        if world == 1 and not args.no_cpu_baseline and not args.no_cpu_configs:
            cpu_cfgs = cpu_baselines(args, reactors_state, amr_sample, sur_sample, bubble_sample)
        line = {
            "metric": METRIC, "value": H["value"], "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": H["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "f32+f64", "hybrid": "bf16+f32+f64"}[head],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "variant": head, "cells": n,
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"{world} independent slices (one per GPU)"},
            "kernel_ms": H["kernel_ms"],
            "roofline": H["roofline"],
            "variants": {v: {k: x for k, x in summary[v].items() if k != "roofline"} |
                         {"roofline_frac": summary[v]["roofline"]["frac"]} for v in summary},
            "e2e": {"value": job_rate(world, n, args.steps, e2e_el), "unit": "cells/s",
                    "h2d_bytes_per_step": n * (3 + S) * 8,
                    "d2h_bytes_per_step": n * (1 + S) * 8 + 2 * n * 4,
                    "matches_device_path": e2e_match},
            "gpu_launches": args.steps * sum(1 if v != "hybrid" else 4 for v, _ in variants),
            "amr_batch": amr,
            "surrogate": sur,
            "shock_bubble": bubble,
            "eq27": eq27,
            "comparators": comparators,
            "znd_1d_strang": znd,
            "mech13": mech13,
            "reactors_4096": reactors,
            "clocks": clk,
            "fma_probe": probe,
            "cpu_baseline": cpu,
            "cpu_baseline_configs": cpu_cfgs,
            "parity_vs_oracle_sample": parity,
        }
        print(json.dumps(line, default=_jsonable), flush=True)
    for c in ctxs.values():
        c.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return line


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
