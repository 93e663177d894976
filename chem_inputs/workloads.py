"""Seeded synthetic cell states for the chemistry workloads: input data only.

Every generator returns temperature T [n] (K), pressure p [n] (Pa) and mass fractions
Y [S, n] (species planes, structure-of-arrays), plus workload-specific extras.  The
conversion to the integrator's conserved state (rho, e) is thermo arithmetic and is
left to each side: the oracle has its own, the GPU library has chem_state_from_TPY.

Randomness comes from numpy's PCG64 seeded per workload.  Compositions are built
from mole fractions, X_H2 : X_O2 : X_N2 = 2 phi : 1 : 3.76 for hydrogen-air at
equivalence ratio phi, converted with the molar masses.  Radicals are zero unless a
recipe seeds them.  The shapes follow the paper's workloads: independent reactors, a
detonation-like slice, a ragged AMR-like batch of boxes with heavy-tailed stiffness,
and the temperature profile of Eq. 27-28 (Sec. 4.2.2).
"""
from __future__ import annotations

import numpy as np

from . import mechanism as _mech

ATM = 101325.0
IDX = {name: k for k, name in enumerate(_mech.SPECIES)}


def _rng(seed):
    return np.random.default_rng(np.random.PCG64(seed))


def _W():
    return np.array([sum(n * _mech.ATOMIC_MASS[el] for n, el in zip(comp, _mech.ELEMENTS))
                     for _, comp, *_ in _mech._SPECIES])


def mass_from_mole(X):
    """Mass fractions from mole fractions; X has the species on axis 0."""
    X = np.asarray(X, dtype=np.float64)
    W = _W().reshape((-1,) + (1,) * (X.ndim - 1))
    m = X * W
    return m / m.sum(axis=0, keepdims=True)


def h2_air_mole(phi):
    """Mole fractions [S, n] of hydrogen-air at equivalence ratio phi [n]."""
    phi = np.atleast_1d(np.asarray(phi, dtype=np.float64))
    X = np.zeros((len(_mech.SPECIES), phi.size))
    X[IDX["H2"]] = 2.0 * phi
    X[IDX["O2"]] = 1.0
    X[IDX["N2"]] = 3.76
    return X / X.sum(axis=0, keepdims=True)


def burnt_mole():
    """Mole fractions of a partly dissociated burnt stoichiometric H2-air state (~2900 K)."""
    X = np.zeros(len(_mech.SPECIES))
    X[IDX["H2O"]] = 0.30
    X[IDX["N2"]] = 0.63
    X[IDX["OH"]] = 0.025
    X[IDX["H2"]] = 0.025
    X[IDX["O2"]] = 0.008
    X[IDX["H"]] = 0.006
    X[IDX["O"]] = 0.004
    X[IDX["HO2"]] = 2e-5
    X[IDX["H2O2"]] = 2e-6
    return X / X.sum()


def reactors(n=4096, seed=0):
    """Independent constant-volume reactors: phi ~ U[0.5, 2], T0 ~ U[1000, 2000] K,
    p0 ~ U[0.5, 5] atm, fresh hydrogen-air, no radicals."""
    r = _rng(seed)
    phi = r.uniform(0.5, 2.0, n)
    T = r.uniform(1000.0, 2000.0, n)
    p = r.uniform(0.5, 5.0, n) * ATM
    Y = mass_from_mole(h2_air_mole(phi))
    return {"T": T, "p": p, "Y": Y, "phi": phi}


def detonation_slice(nx=1024, ny=1024, seed=1):
    """Uniform 2D slice: a 1D detonation-like profile along x, extruded along y with
    +-2 % noise on T and p.  Cell index = y * nx + x.

    x < 0.25: pre-shock fresh stoichiometric H2-air, 300 K, 1 atm.
    0.25 <= x < 0.45: post-shock induction zone, T 1200 -> 1600 K, 25 atm, fresh
        mixture with H, O, OH seeds growing log-linearly from 1e-9 to 1e-5 (mole).
    next 200 cells: exponential reaction zone, state blended toward the burnt state
        with weight 1 - exp(-5 s), s in [0, 1).
    rest: burnt, partly dissociated state at 2900 K, 25 atm.
    """
    r = _rng(seed)
    S = len(_mech.SPECIES)
    xf = (np.arange(nx) + 0.5) / nx
    T1 = np.empty(nx)
    p1 = np.full(nx, 25.0 * ATM)
    X1 = np.empty((S, nx))
    fresh = h2_air_mole(np.array([1.0]))[:, 0]
    burnt = burnt_mole()
    i_shock = int(round(0.25 * nx))
    i_rz = int(round(0.45 * nx))
    rz_len = min(200, nx - i_rz)
    for i in range(nx):
        if i < i_shock:
            T1[i], p1[i], X1[:, i] = 300.0, ATM, fresh
        elif i < i_rz:
            s = (i - i_shock) / max(1, i_rz - i_shock)
            x = fresh.copy()
            seed_frac = 10.0 ** (-9.0 + 4.0 * s)
            for nm in ("H", "O", "OH"):
                x[IDX[nm]] = seed_frac
            T1[i], X1[:, i] = 1200.0 + 400.0 * s, x / x.sum()
        elif i < i_rz + rz_len:
            s = (i - i_rz) / rz_len
            w = 1.0 - np.exp(-5.0 * s)
            x = fresh.copy()
            for nm in ("H", "O", "OH"):
                x[IDX[nm]] = 1e-5
            x = (1.0 - w) * x / x.sum() + w * burnt
            T1[i], X1[:, i] = 1600.0 + 1300.0 * w, x / x.sum()
        else:
            T1[i], X1[:, i] = 2900.0, burnt
    Y1 = mass_from_mole(X1)
    T = np.tile(T1, ny) * (1.0 + 0.02 * r.uniform(-1.0, 1.0, nx * ny))
    p = np.tile(p1, ny) * (1.0 + 0.02 * r.uniform(-1.0, 1.0, nx * ny))
    Y = np.tile(Y1, (1, ny))
    return {"T": T, "p": p, "Y": Y, "nx": nx, "ny": ny}


def amr_batch(nboxes=256, seed=2, edges=(8, 16, 24, 32), nlevels=3, dt0=1e-7):
    """Ragged AMR-like batch: cubic boxes of edge drawn from ``edges``, level = box
    index mod nlevels, level l advanced by 2^l substeps of dt0 / 2^l.

    Per-cell stiffness classes, drawn independently per cell:
      90 % inert: half cold fresh mixture at 300 K / 1 atm, half burnt at 2700-3000 K;
       8 % moderate: fresh, 1100-1300 K, 1-10 atm;
       2 % ignition front: fresh with H and OH seeds (mass fraction ~1e-4),
           1500-2000 K, 1-10 atm.
    Returns T, p, Y for the flattened cells plus box_offset [nboxes+1], box_level,
    box_dt, box_nsub and the class of each cell (0 inert, 1 moderate, 2 front).
    """
    r = _rng(seed)
    e = r.choice(np.asarray(edges), nboxes)
    ncell = e.astype(np.int64) ** 3
    off = np.concatenate([[0], np.cumsum(ncell)])
    n = int(off[-1])
    level = np.arange(nboxes) % nlevels
    u = r.uniform(0.0, 1.0, n)
    cls = np.where(u < 0.90, 0, np.where(u < 0.98, 1, 2)).astype(np.int8)
    T = np.empty(n)
    p = np.empty(n)
    S = len(_mech.SPECIES)
    X = np.zeros((S, n))
    fresh = h2_air_mole(np.array([1.0]))[:, 0]
    burnt = burnt_mole()
    inert = cls == 0
    cold = inert & (r.uniform(0.0, 1.0, n) < 0.5)
    hot = inert & ~cold
    T[cold], p[cold] = 300.0, ATM
    X[:, cold] = fresh[:, None]
    T[hot] = r.uniform(2700.0, 3000.0, hot.sum())
    p[hot] = r.uniform(1.0, 10.0, hot.sum()) * ATM
    X[:, hot] = burnt[:, None]
    mod = cls == 1
    T[mod] = r.uniform(1100.0, 1300.0, mod.sum())
    p[mod] = r.uniform(1.0, 10.0, mod.sum()) * ATM
    X[:, mod] = fresh[:, None]
    fr = cls == 2
    T[fr] = r.uniform(1500.0, 2000.0, fr.sum())
    p[fr] = r.uniform(1.0, 10.0, fr.sum()) * ATM
    X[:, fr] = fresh[:, None]
    Y = mass_from_mole(X)
    # radical seeds for the ignition front, as mass fractions, then renormalise
    Y[IDX["H"], fr] = 1e-4 * r.uniform(0.5, 1.5, fr.sum())
    Y[IDX["OH"], fr] = 1e-4 * r.uniform(0.5, 1.5, fr.sum())
    Y /= Y.sum(axis=0, keepdims=True)
    return {"T": T, "p": p, "Y": Y, "cls": cls, "box_offset": off, "box_level": level,
            "box_dt": dt0 / 2.0 ** level, "box_nsub": (2 ** level).astype(np.int32)}


def eq27_profile(alpha, ny=256, nxz=256, T_low=1000.0, T_high=1600.0, p=ATM):
    """The reaction benchmark field of Sec. 4.2.2 (Eq. 27-28): T varies along y only,
    uniform composition H2 : O2 : N2 = 1 : 2 : 7 (mole), constant pressure.

    T(y) = T_b + T_r tanh(k (y - y_m)/L) + A exp(-8 ((y - y_m)/L)^2) cos(2 pi f y / L)
    with T_b, T_r the mean and half-range of [T_low, T_high], y_m = L/2,
    k = 6/alpha, f = 4/alpha, A = 50/alpha.  Cells are ordered with y fastest, so
    the profile varies across the lanes of a warp.  n = ny * nxz cells.
    """
    L = 1.0
    y = (np.arange(ny) + 0.5) / ny * L
    ym = 0.5 * L
    Tb, Tr = 0.5 * (T_high + T_low), 0.5 * (T_high - T_low)
    k, f, A = 6.0 / alpha, 4.0 / alpha, 50.0 / alpha
    Ty = Tb + Tr * np.tanh(k * (y - ym) / L) + A * np.exp(-8.0 * ((y - ym) / L) ** 2) * np.cos(2 * np.pi * f * y / L)
    T = np.tile(Ty, nxz)
    X = np.zeros(len(_mech.SPECIES))
    X[IDX["H2"]], X[IDX["O2"]], X[IDX["N2"]] = 1.0, 2.0, 7.0
    Y = np.tile(mass_from_mole(X / X.sum())[:, None], (1, T.size))
    return {"T": T, "p": np.full(T.size, p), "Y": Y}


def trajectory_starts(ntraj, seed=3):
    """Initial states for 0D ignition trajectories: phi ~ U[0.5, 2],
    T0 ~ U[900, 2200] K, p ~ U[1, 30] atm, fresh H2-air."""
    r = _rng(seed)
    phi = r.uniform(0.5, 2.0, ntraj)
    T = r.uniform(900.0, 2200.0, ntraj)
    p = r.uniform(1.0, 30.0, ntraj) * ATM
    return {"T": T, "p": p, "Y": mass_from_mole(h2_air_mole(phi)), "phi": phi}


def log_uniform_dt(n, lo=1e-9, hi=1e-7, seed=3):
    """Step sizes drawn log-uniformly in [lo, hi]."""
    r = _rng(seed + 1000)
    return np.exp(r.uniform(np.log(lo), np.log(hi), n))


def _bubble_mole(f):
    """Mole fractions across the bubble interface: a fraction f of stoichiometric H2-O2
    diluted by 70 % N2 (H2 : O2 : N2 = 0.2 : 0.1 : 0.7), the rest N2."""
    f = np.asarray(f, dtype=np.float64)
    X = np.zeros((len(_mech.SPECIES),) + f.shape)
    X[IDX["H2"]] = 0.2 * f
    X[IDX["O2"]] = 0.1 * f
    X[IDX["N2"]] = 0.7 * f + (1.0 - f)
    return X


def shock_bubble(n=256, seed=4, dt=1e-8, fractions=(0.25, 0.08, 0.02)):
    """Reactive shock-bubble field on n^3 cells (cell index (z n + y) n + x before the
    level ordering below).  A sphere of radius 48 n/256 cells centred in the box holds
    stoichiometric H2-O2 diluted 70 % by mole with N2, with a tanh interface of width
    3 n/256 cells, in N2.  The half domain x < n/2 is shock-compressed (1500 K, 20 atm),
    the rest is at 300 K, 1 atm; T and p carry +-0.5 % seeded noise.

    AMR-like levels: cells are ranked by their distance to the two fronts (the shock
    plane and the bubble surface, where the gradients are); the nearest fractions[2]
    of the cells are level 3, the next up to fractions[1] level 2, up to fractions[0]
    level 1, the rest level 0.  Level l takes 2^l substeps of dt / 2^l.  The cells are
    returned ordered by level (stable within a level), one box per level: box_offset,
    box_dt, box_nsub as in amr_batch; `perm` maps a returned cell to its grid index."""
    r = _rng(seed)
    s = n / 256.0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x, y, z = x.ravel() + 0.5, y.ravel() + 0.5, z.ravel() + 0.5
    c = n / 2.0
    rad = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    del y, z
    R, w = 48.0 * s, 3.0 * s
    f = 0.5 * (1.0 - np.tanh((rad - R) / w))
    shocked = x < c
    N = x.size
    T = np.where(shocked, 1500.0, 300.0) * (1.0 + 0.005 * r.uniform(-1.0, 1.0, N))
    p = np.where(shocked, 20.0, 1.0) * ATM * (1.0 + 0.005 * r.uniform(-1.0, 1.0, N))
    Y = mass_from_mole(_bubble_mole(f))
    dist = np.minimum(np.abs(x - c), np.abs(rad - R))
    del x, rad
    order = np.argsort(dist, kind="stable")
    level = np.zeros(N, dtype=np.int32)
    n3, n2, n1 = (int(round(fr * N)) for fr in (fractions[2], fractions[1], fractions[0]))
    level[order[:n1]] = 1
    level[order[:n2]] = 2
    level[order[:n3]] = 3
    perm = np.argsort(-level, kind="stable")  # level 3 first: the stiffest boxes lead
    counts = np.bincount(level, minlength=4)[::-1]
    box_offset = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    levels = np.arange(3, -1, -1)
    return {"T": T[perm], "p": p[perm], "Y": np.ascontiguousarray(Y[:, perm]), "level": level[perm],
            "perm": perm, "box_offset": box_offset, "box_dt": dt / 2.0 ** levels,
            "box_nsub": (2 ** levels).astype(np.int32), "fuel": f[perm]}


def bubble_trajectory_starts(ntraj, seed=5):
    """Initial states of the shock-bubble field's family for surrogate training: fuel
    fraction f across the interface (a quarter pure N2, f = 0; a quarter log-uniform in
    [1e-12, 1], the tanh tail of the interface; the rest U[0, 1]); half shocked (1500 K,
    20 atm), half not (300 K, 1 atm); +-2 % uniform noise on T and p."""
    r = _rng(seed)
    u = r.uniform(0.0, 1.0, ntraj)
    f = np.where(u < 0.25, 0.0, np.where(u < 0.5, 10.0 ** r.uniform(-12.0, 0.0, ntraj),
                                         r.uniform(0.0, 1.0, ntraj)))
    shocked = r.uniform(0.0, 1.0, ntraj) < 0.5
    T = np.where(shocked, 1500.0, 300.0) * (1.0 + 0.02 * r.uniform(-1.0, 1.0, ntraj))
    p = np.where(shocked, 20.0, 1.0) * ATM * (1.0 + 0.02 * r.uniform(-1.0, 1.0, ntraj))
    return {"T": T, "p": p, "Y": mass_from_mole(_bubble_mole(f)), "fuel": f}


def reactors13(n=4096, seed=0, mech=None):
    """Independent constant-volume reactors for the 13-species mechanism (species order
    mechanism.SPECIES13): phi ~ U[0.5, 2], T0 ~ U[1000, 2000] K, p0 ~ U[0.5, 5] atm, fresh
    H2-O2 with a diluent whose N2 : Ar : He split is Dirichlet(1, 1, 1) per cell, 3.76 moles
    of diluent per mole of O2 (air-like), and traces of CO and CO2 (mole fractions
    U[0, 1e-3] each) as extra colliders; no radicals.  The paper's detonation runs
    dilute H2 : O2 with argon (2 : 1 : 7, Sec. 5.3); this recipe spans N2, Ar and He."""
    from . import mechanism as m13
    mech = mech or m13.build13(0)
    idx = {name: k for k, name in enumerate(m13.SPECIES13)}
    r = _rng(seed)
    phi = r.uniform(0.5, 2.0, n)
    T = r.uniform(1000.0, 2000.0, n)
    p = r.uniform(0.5, 5.0, n) * ATM
    split = r.dirichlet(np.ones(3), n).T
    X = np.zeros((len(m13.SPECIES13), n))
    X[idx["H2"]] = 2.0 * phi
    X[idx["O2"]] = 1.0
    X[idx["N2"]] = 3.76 * split[0]
    X[idx["AR"]] = 3.76 * split[1]
    X[idx["HE"]] = 3.76 * split[2]
    X[idx["CO"]] = r.uniform(0.0, 1e-3, n) * (2.0 * phi + 4.76)
    X[idx["CO2"]] = r.uniform(0.0, 1e-3, n) * (2.0 * phi + 4.76)
    X /= X.sum(axis=0, keepdims=True)
    m = X * np.asarray(mech["W"])[:, None]
    Y = m / m.sum(axis=0, keepdims=True)
    return {"T": T, "p": p, "Y": Y, "phi": phi}


def detonation_slice13(nx=1024, ny=1024, seed=1, mech=None):
    """The detonation slice (detonation_slice: same T, p and profile) for the 13-species
    mechanism: in every cell the N2 mole fraction is split into N2 : Ar : He by a
    Dirichlet(1, 1, 1) draw (the paper's detonations are argon-diluted, Sec. 5.3), CO and
    CO2 traces (mole fractions U[0, 1e-4]) are added, and the mass fractions recomputed
    with the 13 molar masses."""
    from . import mechanism as m13
    mech = mech or m13.build13(0)
    d = detonation_slice(nx, ny, seed)
    n = d["T"].size
    r = _rng(seed + 1000)
    W9 = _W()
    X9 = d["Y"] / W9[:, None]
    X9 /= X9.sum(axis=0, keepdims=True)
    X = np.zeros((len(m13.SPECIES13), n))
    X[:9] = X9
    split = r.dirichlet(np.ones(3), n).T
    n2 = X9[IDX["N2"]]
    X[IDX["N2"]] = n2 * split[0]
    X[9] = n2 * split[1]
    X[10] = n2 * split[2]
    X[11] = r.uniform(0.0, 1e-4, n)
    X[12] = r.uniform(0.0, 1e-4, n)
    X /= X.sum(axis=0, keepdims=True)
    m = X * np.asarray(mech["W"])[:, None]
    return {"T": d["T"], "p": d["p"], "Y": m / m.sum(axis=0, keepdims=True)}
