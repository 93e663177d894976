"""Credited floating-point work of the integrator, for the roofline.

The work of one launch is credited from the algorithm, not from what the hardware ran:
per attempted RK step, five right-hand-side evaluations plus the register updates and
the WRMS norm of Eq. 21-22; per cell, the final temperature solve.  Each right-hand
side is counted from the mechanism structure in the formulation the kernels use:

  Newton on mixture coefficients sum_k Y_k ec_k / W_k (assembly + 2 iterations), ln T,
  1/T, per species the NASA-7 Gibbs function (one combined polynomial) and
  G_k = exp(-g_k/RT) with its reciprocal, per reaction the
  Arrhenius exponential, the products of the law of mass action (Eq. 16) with the
  equilibrium-constant factors, the third-body sums, the Troe fall-off terms, and the
  conversion F_k = W_k wdot_k / rho.

Add, multiply, compare-free min/max and divide count 1 flop, an FMA 2, and every
exp / log / exp10 / log10 / sqrt is credited a fixed TRANSCENDENTAL flops.  The FP64
pipe of GB300 spends about 20 FMA slots (40 flops) on a library exp, so this credit is
conservative: the reported fraction understates the FP64 pipe's busy time, which the
ncu summary reports separately.
"""
from __future__ import annotations

TRANSCENDENTAL = 20

# compiled reaction structure of the 9-species mechanism: (n_reactants, n_products, type,
# troe_n); type 0/1/2 = elementary / third body / fall-off.  Mirrors csrc/mech_h2o2_9.cuh;
# a mechanism dict given to the functions below supplies its own.
_RX = [
    (2, 2, 0, 0), (2, 2, 0, 0), (2, 2, 0, 0), (2, 2, 0, 0),
    (1, 2, 1, 0), (2, 1, 1, 0), (2, 1, 1, 0), (2, 1, 1, 0),
    (2, 1, 2, 4),
    (2, 2, 0, 0), (2, 2, 0, 0), (2, 2, 0, 0), (2, 2, 0, 0), (2, 2, 0, 0), (2, 2, 0, 0),
    (1, 2, 2, 3),
    (2, 2, 0, 0), (2, 2, 0, 0), (2, 2, 0, 0), (2, 2, 0, 0), (2, 2, 0, 0),
]
NSP = 9
NEWTON_ITERS = 2
# stages of each integration scheme (chem_scheme): the two-register RK4(3)5, the same
# tableau with full k-storage, RKF45
STAGES = {0: 5, 1: 5, 2: 6}


def _structure(mech):
    """(species count, reaction structure list) of mech, or of the 9-species mechanism."""
    if mech is None:
        return NSP, _RX
    rx = [(int(sum(mech["nu_f"][j])), int(sum(mech["nu_r"][j])), int(mech["rtype"][j]),
           int(mech["troe_n"][j]) if int(mech["rtype"][j]) == 2 else 0) for j in range(len(mech["A"]))]
    return len(mech["W"]), rx


def newton_flops(iters: int = NEWTON_ITERS, nsp: int = NSP) -> int:
    assembly = 6 * nsp * 2 + 4 + 1        # 6 mixture coefficients x nsp FMAs, c_v scalings, - e/R
    per_iter = 5 * 2 + 4 * 2 + 2 + 1      # e(T) and c_v(T) Horner, reciprocal x residual, update
    return assembly + iters * per_iter


def rhs_flops(mech: dict | None = None) -> int:
    """Credited flops of one right-hand side.  ``mech`` (chem_inputs layout) gives the
    structure, marks temperature-independent rates (no exponential) and third-body
    efficiency lists (the 9-species structure with all efficiencies counted when None)."""
    T = TRANSCENDENTAL
    nsp, rxs = _structure(mech)
    f = newton_flops(nsp=nsp)
    f += 2 * nsp                               # concentrations rho Y_k / W_k
    f += T + 1 + 2 + 1 + 1 + (nsp - 1)         # ln T, 1/T, RT/p, p/RT, 1 - ln T, total conc.
    f += nsp * (12 + T + 1 + 1)                # g/RT (6 FMAs), G = exp(-g), 1/G, c/G
    for j, (nr, npr, typ, troe_n) in enumerate(rxs):
        kconst = mech is not None and mech["b"][j] == 0.0 and mech["Ea"][j] == 0.0
        f += 0 if kconst else T + 4            # Arrhenius exponential
        f += (nr - 1) + 1                      # prod c_reactants, times k_f
        f += (nr - 1) + (1 if nr != npr else 0) + (npr - 1) + 2  # prod G, prod c/G, (RT/p)^dnu, FMA
        f += nr + npr                          # production-rate updates
        if typ != 0:                           # [M]: one FMA per efficiency != 1
            f += 2 * (nsp if mech is None else int(sum(abs(x - 1.0) > 0 for x in mech["eff"][j])))
        if typ == 1:
            f += 1
        if typ == 2:
            f += T + 4 + 2                     # k0, Pr
            f += (3 if troe_n == 4 else 2) * (T + 2) + 3  # F_cent
            f += 3 * T + 4 + 1 + 3 + 3 + 4     # log10 F_cent, log10 Pr, exp10, Troe algebra
    f += 2 * nsp                               # F_k = W_k wdot_k / rho
    return f


def step_flops(mech: dict | None = None, scheme: int = 0) -> int:
    """Credited flops of one attempted step: the scheme's right-hand sides, its register
    updates (Eq. 21 for scheme 0: h a, h b, h e and 3 FMAs per component and stage; the
    full-storage schemes: one FMA per tableau coefficient and component for the stage
    inputs, the solution and the error) and the Eq. 22 control."""
    nsp, _ = _structure(mech)
    s = STAGES[scheme]
    if scheme == 0:
        updates = s * (3 + nsp * 3 * 2)
    else:
        ncoef = s * (s - 1) // 2               # strictly lower A
        updates = nsp * 2 * (ncoef + 2 * s) + s
    wrms = nsp * (2 + 1 + 2 + 1 + 2) + 2 + T_SQRT
    control = 2 * T_SQRT + 1 + 3 + 1
    return s * rhs_flops(mech) + updates + wrms + control


T_SQRT = TRANSCENDENTAL


def cell_flops(mech: dict | None = None) -> int:
    """Per-cell work outside the step loop: 1/rho, e/R and the final temperature solve."""
    return 2 + newton_flops(nsp=_structure(mech)[0])


def launch_flops(total_attempted_steps: int, ncells: int, mech: dict | None = None, scheme: int = 0) -> float:
    """Credited flops of one launch from the attempted-step total the kernel reports."""
    return float(total_attempted_steps) * step_flops(mech, scheme) + float(ncells) * cell_flops(mech)


def rhs_flops_mixed_fp64(mech: dict | None = None) -> int:
    """The part of one mixed-precision right-hand side that stays fp64: the temperature
    solve, ln T, 1/T, the Gibbs functions and ln(R T / p), and the split of each of those
    into the fp32 hi / lo parts from which ln(1/K_c) is summed in fp32 (one fp64
    subtraction each; the sums themselves are fp32 and not credited)."""
    T = TRANSCENDENTAL
    nsp, _ = _structure(mech)
    f = newton_flops(nsp=nsp)
    f += T + 1 + 1 + 1                         # ln T, 1/T, 1 - ln T, ln(R T / p)
    f += nsp * 12                              # g_k / RT: 6 FMAs each
    f += nsp + 1                               # x - hi of the splits
    return f


def step_flops_mixed_fp64(mech: dict | None = None, scheme: int = 0) -> int:
    """fp64 credited flops of one mixed-precision attempted step: the right-hand sides'
    fp64 part, the fp64 solution and error registers (scheme 0: 2 FMAs per component and
    stage; full storage: one FMA per weight and component for each) and the fp64 WRMS
    norm and control."""
    nsp, _ = _structure(mech)
    s = STAGES[scheme]
    updates = s * (2 + nsp * 2 * 2)
    wrms = nsp * (2 + 1 + 2 + 1 + 2) + 2 + T_SQRT
    control = 2 * T_SQRT + 1 + 3 + 1
    return s * rhs_flops_mixed_fp64(mech) + updates + wrms + control


def launch_flops_mixed_fp64(total_attempted_steps: int, ncells: int, mech: dict | None = None,
                            scheme: int = 0) -> float:
    return float(total_attempted_steps) * step_flops_mixed_fp64(mech, scheme) + float(ncells) * cell_flops(mech)


# FP64 peak of GB300 derived from unit counts and clocks: 152 SMs x 2 FP64 FMA lanes per
# clock per SM (measured: 1192.8 GFLOP/s at ~1.96 GHz) x 2 flops x 2.070 GHz max clock.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
# FP32: 152 SMs x 128 FMA lanes x 2 flops x 2.070 GHz (measured 72.9 TFLOP/s at ~1.96 GHz)
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.070
