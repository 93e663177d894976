"""Training data and evaluation of the learned surrogate.

Data recipe (0D ignition trajectories): initial states phi ~ U[0.5, 2], T0 ~ U[900, 2200] K,
p ~ U[1, 30] atm (chem_inputs.workloads.trajectory_starts).  Every trajectory is integrated
on the GPU with the FP64 integrator over a logarithmic time grid, recording the initial
state and the state at each grid point up to its ignition (first time T exceeds
T0 + 400 K); the grid interval holding the ignition is then re-recorded at a fine
per-trajectory spacing, followed by a short post-ignition window (trajectory_states).
Each recorded state then gets a step dt ~ log-uniform [1e-9, 1e-7] s and is integrated
over it (the batched integrator, one box per cell), giving a (state, dt) -> state pair.

Everything that computes runs in libchem's kernels; torch gathers and stores arrays.
"""
from __future__ import annotations

import numpy as np

from chem_inputs import workloads


def trajectory_states(ctx, ntraj, seed=3, nstage=48, t0=1e-9, t_end=3e-3, nfine=16, post=5e-6,
                      npost=8, device="cuda", starts=None):
    """States along ntraj ignition trajectories (dict of CUDA tensors rho, e, Y [S, m], T,
    plus the trajectory id and time of each state).

    Pass 1 records the initial state, integrates every trajectory over a logarithmic time
    grid (one dt for all) and records the states until the grid interval [t_lo, t_hi] in
    which T first exceeds
    T0 + 400 K, or the integration stops at ctx's step limit (the interval is stiff).
    Pass 2 restarts each such trajectory at t_lo and records nfine equal sub-intervals of
    its own [t_lo, t_hi] (the ignition transient), then npost intervals of post / npost
    past t_hi (the burnt state is stiff for an explicit method, so the recorded
    post-ignition window is kept short).  A trajectory stops at the first pass-2
    integration that does not end with status 0; only status-0 states are recorded.
    Pass ctx a step limit of a few thousand (Context(..., max_steps=4000)): the cost of
    every call is its stiffest cell's step count, run serially.  starts (optional): the
    initial states {T, p, Y} (default: workloads.trajectory_starts(ntraj, seed))."""
    import torch
    s = workloads.trajectory_starts(ntraj, seed=seed) if starts is None else starts
    ntraj = len(s["T"])
    f64 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)
    T0 = f64(s["T"])
    rho, e = ctx.state_from_TPY(T0, f64(s["p"]), f64(s["Y"]))
    Y, T = f64(s["Y"]), T0.clone()
    tgrid = t0 * (t_end / t0) ** (np.arange(nstage + 1) / nstage)
    active = torch.arange(ntraj, device=device)
    out = {"rho": [], "e": [], "Y": [], "T": [], "traj": [], "t": []}

    def record(idx, r, en, Ya, Ta, t):
        out["rho"].append(r); out["e"].append(en); out["Y"].append(Ya); out["T"].append(Ta)
        out["traj"].append(idx); out["t"].append(t)

    # the initial states (radical free) are states of the trajectories too
    record(active.clone(), rho, e, Y.clone(), T.clone(), torch.zeros_like(T))
    ign_idx, ign_lo, ign_hi = [], [], []
    for j in range(nstage):
        if active.numel() == 0:
            break
        dt = float(tgrid[j + 1] - tgrid[j])
        r_a, e_a = rho[active], e[active]
        Y_a, T_a = Y[:, active].contiguous(), T[active].clone()
        st = torch.empty(active.numel(), dtype=torch.int32, device=device)
        ctx.integrate(r_a, e_a, Y_a, T_a, dt, status=st)
        good = st == 0
        ign = (good & (T_a > T0[active] + 400.0)) | (st == 1)
        keep = good & ~ign
        record(active[keep], r_a[keep], e_a[keep], Y_a[:, keep], T_a[keep],
               torch.full_like(T_a[keep], tgrid[j + 1]))
        ign_idx.append(active[ign])            # state stays at t_lo = tgrid[j]
        ign_lo.append(torch.full_like(T_a[ign], tgrid[j]))
        ign_hi.append(torch.full_like(T_a[ign], tgrid[j + 1]))
        Y[:, active[keep]], T[active[keep]] = Y_a[:, keep], T_a[keep]
        active = active[keep]
    idx = torch.cat(ign_idx) if ign_idx else torch.empty(0, dtype=torch.int64, device=device)
    if idx.numel():
        t_lo, t_hi = torch.cat(ign_lo), torch.cat(ign_hi)
        r_i, e_i = rho[idx].contiguous(), e[idx].contiguous()
        Y_i, T_i = Y[:, idx].contiguous(), T[idx].clone()
        t = t_lo.clone()
        fine = (t_hi - t_lo) / nfine
        for k in range(nfine + npost):
            m = idx.numel()
            if m == 0:
                break
            dt_i = fine if k < nfine else torch.full_like(fine, post / npost)
            st = torch.empty(m, dtype=torch.int32, device=device)
            ctx.integrate_batched(r_i, e_i, Y_i, T_i, torch.arange(m + 1, dtype=torch.int64, device=device),
                                  dt_i.contiguous(), torch.ones(m, dtype=torch.int32, device=device),
                                  status=st)
            t = t + dt_i
            good = st == 0
            record(idx[good], r_i[good], e_i[good], Y_i[:, good], T_i[good], t[good])
            if not bool(good.all()):
                idx, r_i, e_i, t, fine = idx[good], r_i[good], e_i[good], t[good], fine[good]
                Y_i, T_i = Y_i[:, good].contiguous(), T_i[good].clone()
    return {k: (torch.cat(v, dim=1) if k == "Y" else torch.cat(v)) for k, v in out.items()}


def make_pairs(ctx, states, seed=3, dt_lo=1e-9, dt_hi=1e-7, max_pairs=None, max_dT=None):
    """(state, dt) -> state pairs: each state advanced over its own log-uniform dt
    (pairs whose integration did not end with status 0 are dropped, and with max_dT
    those whose temperature changes by more than max_dT K)."""
    import torch
    n = states["T"].numel()
    rng = np.random.default_rng(seed + 7)
    idx = np.arange(n)
    if max_pairs is not None and max_pairs < n:
        idx = np.sort(rng.choice(n, max_pairs, replace=False))
    idx_t = torch.tensor(idx, device=states["T"].device)
    rho, e = states["rho"][idx_t].contiguous(), states["e"][idx_t].contiguous()
    Y0, T0 = states["Y"][:, idx_t].contiguous(), states["T"][idx_t].contiguous()
    m = idx.size
    dt = workloads.log_uniform_dt(m, dt_lo, dt_hi, seed=seed)
    dev = rho.device
    Y1, T1 = Y0.clone(), T0.clone()
    dt = torch.tensor(dt, dtype=torch.float64, device=dev)
    st = torch.empty(m, dtype=torch.int32, device=dev)
    ctx.integrate_batched(rho, e, Y1, T1, torch.arange(m + 1, dtype=torch.int64, device=dev), dt,
                          torch.ones(m, dtype=torch.int32, device=dev), status=st)
    good = st == 0   # a pair whose integration failed is not a sample of the map
    if max_dT is not None:   # keep the mildly reactive pairs only
        good &= (T1 - T0).abs() <= max_dT
    return {"rho": rho[good].contiguous(), "e": e[good].contiguous(), "Y0": Y0[:, good].contiguous(),
            "T0": T0[good].contiguous(), "dt": dt[good].contiguous(), "Y1": Y1[:, good].contiguous(),
            "T1": T1[good].contiguous()}


def split_by_trajectory(states, heldout=0.1, seed=3):
    """(train, held-out) state sets; a seeded fraction of whole trajectories is held out."""
    import torch
    traj = states["traj"]
    ntraj = int(traj.max().item()) + 1 if traj.numel() else 0
    rng = np.random.default_rng(seed + 11)
    held = torch.tensor(rng.random(ntraj) < heldout, device=traj.device)[traj]

    def take(m):
        return {k: (v[:, m].contiguous() if k == "Y" else v[m].contiguous()) for k, v in states.items()}
    return take(~held), take(held)


def draw_cells(states, n, seed=3):
    """n cells drawn with replacement (seeded) from a state set, as contiguous planes."""
    import torch
    m = states["T"].numel()
    idx = torch.tensor(np.random.default_rng(seed + 13).integers(0, m, n), device=states["T"].device)
    return {k: (v[:, idx].contiguous() if k == "Y" else v[idx].contiguous()) for k, v in states.items()}


def evaluate(ctx_sur, ctx_ref, states, dt, rtol=1e-6, atol=1e-10, gate=None, reps=3):
    """Surrogate (with fallback) against the reference integrator on the same states and
    dt: max relative T error, fallback fraction, and throughput of both (cells/s)."""
    import time

    import torch
    from paper_2506_02602_gb300 import chem
    n = states["T"].numel()
    dev = states["T"].device
    mask = torch.empty(n, dtype=torch.uint8, device=dev)
    stats = torch.zeros(chem.STATS_WORDS, dtype=torch.int64, device=dev)

    def run(fn):
        best = float("inf")
        for _ in range(reps):
            Y, T = states["Y"].clone(), states["T"].clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn(Y, T)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return Y, T, best

    Ys, Ts, ts = run(lambda Y, T: ctx_sur.surrogate_infer(states["rho"], states["e"], Y, T, dt, rtol, atol,
                                                          mask=mask, stats=stats, gate=gate))
    Yr, Tr, tr = run(lambda Y, T: ctx_ref.integrate(states["rho"], states["e"], Y, T, dt, rtol, atol))
    relT = ((Ts - Tr).abs() / Tr).cpu().numpy()
    fb = mask.cpu().numpy().astype(bool)
    return {"cells": n, "dt": dt, "fallback_frac": float(fb.mean()),
            "max_rel_T": float(relT.max()), "max_rel_T_accepted": float(relT[~fb].max(initial=0.0)),
            "p99_rel_T": float(np.quantile(relT, 0.99)),
            "max_abs_Y": float((Ys - Yr).abs().max().item()),
            "surrogate_cells_per_s": n / ts, "integrator_cells_per_s": n / tr, "speedup": tr / ts,
            "stats": stats.cpu().numpy().tolist()}


ERR_TOL_GRID = (3e-4, 4e-4, 5e-4, 6e-4, 8e-4)
RATE_MAX_GRID = (1.0, 1.5, 2.0)


def tune_gate(ctx_sur, ctx_ref, states, dt, bound=1e-3, margin=1.5, rtol=1e-6, atol=1e-10,
              err_grid=ERR_TOL_GRID, rate_grid=RATE_MAX_GRID):
    """The error test's thresholds for step dt, chosen on validation states (trajectories
    neither trained on nor reported): among (err_tol, rate_max) pairs whose largest
    relative T error over all cells, against the reference integrator, stays within
    bound / margin, the one with the fewest fallbacks (ties: the smaller err_tol).
    Returns (gate dict, table of every candidate)."""
    import torch
    n = states["T"].numel()
    dev = states["T"].device
    Yr, Tr = states["Y"].clone(), states["T"].clone()
    ctx_ref.integrate(states["rho"], states["e"], Yr, Tr, dt, rtol, atol)
    mask = torch.empty(n, dtype=torch.uint8, device=dev)
    table, best = [], None
    for et in err_grid:
        for rm in rate_grid:
            gate = {"err_tol": et, "rate_max": rm}
            Y, T = states["Y"].clone(), states["T"].clone()
            ctx_sur.surrogate_infer(states["rho"], states["e"], Y, T, dt, rtol, atol, mask=mask, gate=gate)
            rel = float(((T - Tr).abs() / Tr).max())
            fb = float((mask != 0).float().mean())
            table.append({"err_tol": et, "rate_max": rm, "max_rel_T": rel, "fallback_frac": fb})
            if rel <= bound / margin and (best is None or fb < best[1] - 1e-12):
                best = (gate, fb)
    if best is None:  # nothing meets the bound: the strictest test
        best = ({"err_tol": min(err_grid), "rate_max": min(rate_grid)}, None)
    return best[0], table


def hybrid_levels(ctx, rho, e, Y, T, box_offset, box_dt, box_nsub, rtol=1e-6, atol=1e-10, gate=None,
                  status=None, nsteps=None, mask=None, stream=None):
    """One hydro step of a level-ordered field with the surrogate: for each box (cells
    box_offset[b] .. box_offset[b+1], host arrays) box_nsub[b] chem_surrogate_infer calls
    of box_dt[b] on that slice of the state (in place).  status / nsteps / mask receive
    the last substep's values."""
    import torch
    for b in range(len(box_dt)):
        a, z = int(box_offset[b]), int(box_offset[b + 1])
        if z <= a:
            continue
        sl = slice(a, z)
        for _ in range(int(box_nsub[b])):
            ctx.surrogate_infer(rho[sl], e[sl], Y[:, sl], T[sl], float(box_dt[b]), rtol, atol,
                                status=None if status is None else status[sl],
                                nsteps=None if nsteps is None else nsteps[sl],
                                mask=None if mask is None else mask[sl], gate=gate, stream=stream)
