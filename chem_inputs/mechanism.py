"""Seeded synthetic H2/O2/N2 reaction mechanisms: input data only.

The paper names a detailed hydrogen mechanism (Sec. 5.2.3) but prints none of its
coefficients.  This module builds mechanisms with the same structure.  ``build`` gives
the 9-species / 21-reaction one below; ``build13`` the 13-species / 27-reaction one of
the paper's size (``build13``'s docstring).  The 9-species mechanism has:

* 9 species: H2, O2, H2O, H, O, OH, HO2, H2O2, N2 (N2 inert);
* 21 reversible reactions of the usual hydrogen-oxidation classes: chain branching
  and propagation, four third-body reactions, two Troe fall-off reactions, HO2/H2O2
  chemistry and two duplicate pairs (Eq. 15 form, reverse rate from the equilibrium
  constant as stated in Sec. 2.1.2);
* NASA-7 thermo tables for each species (the e(T) relation of Eq. 10).

Each rate parameter is drawn, from the seed, in a band around a rounded
order-of-magnitude centre for its reaction class.  Each thermo table is a NASA-7 fit
of a seeded vibrational (Einstein-oscillator) heat-capacity model, anchored at rounded
textbook formation enthalpies and entropies.  None of these numbers is the paper's
mechanism, so absolute chemistry values cannot be compared with the paper.

Units are SI throughout: kg/mol, J/mol, J/(mol K), mol/m^3, s.  An Arrhenius rate
constant is k = A T^b exp(-Ea/(R_u T)) with A in (m^3/mol)^(order-1)/s, where the
order counts the reactant molecularity plus one for a third body (or for the
low-pressure limit of a fall-off reaction).

This module only constructs data.  It never evaluates a rate, a production rate, a
temperature solve or an integrator step, so both the oracle and the GPU path may
read what it returns.  The returned mechanism is a plain dict of numpy arrays
(see ``build``); each side marshals it into its own structure.
"""
from __future__ import annotations

import numpy as np

ELEMENTS = ("H", "O", "N")
ATOMIC_MASS = {"H": 1.008e-3, "O": 15.999e-3, "N": 14.007e-3}  # kg/mol

# name, (H, O, N), formation enthalpy at 298.15 K [J/mol], standard entropy [J/(mol K)],
# translational+rotational cp/R, vibrational temperatures [K]  (rounded textbook values)
_SPECIES = (
    ("H2",   (2, 0, 0),       0.0, 130.7, 3.5, (6300.0,)),
    ("O2",   (0, 2, 0),       0.0, 205.1, 3.5, (2250.0,)),
    ("H2O",  (2, 1, 0), -241800.0, 188.8, 4.0, (2300.0, 5250.0, 5400.0)),
    ("H",    (1, 0, 0),  218000.0, 114.7, 2.5, ()),
    ("O",    (0, 1, 0),  249200.0, 161.1, 2.5, ()),
    ("OH",   (1, 1, 0),   37300.0, 183.7, 3.5, (5350.0,)),
    ("HO2",  (1, 2, 0),   12000.0, 229.0, 4.0, (1600.0, 2000.0, 5000.0)),
    ("H2O2", (2, 2, 0), -136100.0, 232.7, 4.0, (500.0, 1250.0, 1950.0, 2000.0, 5200.0, 5200.0)),
    ("N2",   (0, 0, 2),       0.0, 191.6, 3.5, (3350.0,)),
)
SPECIES = tuple(s[0] for s in _SPECIES)

T_LO, T_MID, T_HI = 200.0, 1000.0, 6000.0
T_REF = 298.15

# Reaction table: equation, type, centre (log10 A in mol-cm-s units, b, Ea in kJ/mol),
# low-pressure centre for fall-off, third-body efficiency overrides, duplicate flag.
# type: "elem" elementary, "tb" third body (+M), "troe" fall-off (+M).
_REACTIONS = (
    ("H+O2=O+OH",        "elem", (14.3, 0.0, 69.0), None, None, False),
    ("O+H2=H+OH",        "elem", (4.7, 2.7, 26.0), None, None, False),
    ("H2+OH=H2O+H",      "elem", (8.3, 1.5, 14.0), None, None, False),
    ("OH+OH=O+H2O",      "elem", (4.5, 2.4, -9.0), None, None, False),
    ("H2+M=H+H+M",       "tb",   (19.7, -1.4, 436.0), None, {"H2": 2.5, "H2O": 12.0}, False),
    ("O+O+M=O2+M",       "tb",   (15.8, -0.5, 0.0), None, {"H2": 2.5, "H2O": 12.0}, False),
    ("O+H+M=OH+M",       "tb",   (18.7, -1.0, 0.0), None, {"H2": 2.5, "H2O": 12.0}, False),
    ("H+OH+M=H2O+M",     "tb",   (22.6, -2.0, 0.0), None, {"H2": 0.7, "H2O": 3.7}, False),
    ("H+O2(+M)=HO2(+M)", "troe", (12.7, 0.44, 0.0), (20.8, -1.7, 2.0),
     {"H2": 2.0, "H2O": 11.0, "O2": 0.8}, False),
    ("HO2+H=H2+O2",      "elem", (6.4, 2.1, -6.0), None, None, False),
    ("HO2+H=OH+OH",      "elem", (13.9, 0.0, 1.0), None, None, False),
    ("HO2+O=O2+OH",      "elem", (13.3, 0.0, 0.0), None, None, False),
    ("HO2+OH=H2O+O2",    "elem", (13.5, 0.0, -2.0), None, None, False),
    ("HO2+HO2=H2O2+O2",  "elem", (11.1, 0.0, -7.0), None, None, True),
    ("HO2+HO2=H2O2+O2",  "elem", (14.6, 0.0, 50.0), None, None, True),
    ("H2O2(+M)=OH+OH(+M)", "troe", (12.3, 0.9, 204.0), (24.4, -2.3, 203.0),
     {"H2": 3.7, "H2O": 7.5}, False),
    ("H2O2+H=H2O+OH",    "elem", (13.4, 0.0, 17.0), None, None, False),
    ("H2O2+H=HO2+H2",    "elem", (13.7, 0.0, 33.0), None, None, False),
    ("H2O2+O=OH+HO2",    "elem", (7.0, 2.0, 17.0), None, None, False),
    ("H2O2+OH=HO2+H2O",  "elem", (12.2, 0.0, 1.0), None, None, True),
    ("H2O2+OH=HO2+H2O",  "elem", (13.9, 0.0, 30.0), None, None, True),
)
# Four-parameter Troe form for the first fall-off reaction, three-parameter for the second.
_TROE_NPARAM = {"H+O2(+M)=HO2(+M)": 4, "H2O2(+M)=OH+OH(+M)": 3}

N_SPECIES = len(_SPECIES)
N_REACTIONS = len(_REACTIONS)

# The 13-species extension: the colliders of the paper's mechanism size (argon, helium,
# carbon monoxide and dioxide; Sec. 5.2.3 names 13 species and 27 reactions).  They take
# part in no reaction; they enter the third-body concentrations with their own
# efficiencies.  Their elements beyond H, O, N (Ar, He, C) are carried in the molar mass
# only (the element counts cover H, O, N).  Columns as _SPECIES, plus the mass of the
# untracked elements (kg/mol); noble gases have cp = 5/2 R exactly (no vibrational or
# electronic term).
_SPECIES13_EXTRA = (
    ("AR",  (0, 0, 0),       0.0, 154.8, 2.5, (), 39.948e-3),
    ("HE",  (0, 0, 0),       0.0, 126.2, 2.5, (), 4.0026e-3),
    ("CO",  (0, 1, 0), -110500.0, 197.7, 3.5, (3100.0,), 12.011e-3),
    ("CO2", (0, 2, 0), -393500.0, 213.8, 3.5, (960.0, 960.0, 1930.0, 3380.0), 12.011e-3),
)
SPECIES13 = SPECIES + tuple(s[0] for s in _SPECIES13_EXTRA)
_COLLIDERS13 = {"AR": 0.7, "HE": 0.7, "CO": 1.9, "CO2": 3.8}
# The 27 reactions: the 21 above (their third-body reactions with the 13-species
# efficiencies) and six collider-specific or duplicate channels, as a detailed hydrogen
# mechanism lists them: dissociation and recombination with Ar and He as the only
# collision partner, recombination to water with water as the partner, and the second
# HO2 + OH channel.  "{X}" in the efficiency dict sets the default of every species not
# named.
_REACTIONS13_EXTRA = (
    ("H2+M=H+H+M",       "tb",   (18.9, -1.1, 436.0), None, {"*": 0.0, "AR": 1.0}, False),
    ("H2+M=H+H+M",       "tb",   (18.9, -1.1, 436.0), None, {"*": 0.0, "HE": 1.0}, False),
    ("O+O+M=O2+M",       "tb",   (13.8, 0.0, -7.5), None, {"*": 0.0, "AR": 1.0}, False),
    ("O+O+M=O2+M",       "tb",   (13.8, 0.0, -7.5), None, {"*": 0.0, "HE": 1.0}, False),
    ("H+OH+M=H2O+M",     "tb",   (21.9, -1.8, 0.0), None, {"*": 0.0, "H2O": 1.0}, False),
    ("HO2+OH=H2O+O2",    "elem", (15.8, -1.0, 0.0), None, None, True),
)
# third-body reactions of the 21 whose Ar / He channels are separate reactions above
_SEPARATE13 = {"H2+M=H+H+M", "O+O+M=O2+M"}


def _parse_side(side: str, species=SPECIES) -> dict[int, int]:
    """'H+O2(+M)' -> {species index: stoichiometric coefficient}, ignoring M."""
    side = side.replace("(+M)", "")
    nu: dict[int, int] = {}
    for tok in side.split("+"):
        tok = tok.strip()
        if not tok or tok == "M":
            continue
        k = species.index(tok)
        nu[k] = nu.get(k, 0) + 1
    return nu


def _einstein_cp(T, base, thetas, scale):
    """cp/R of the synthetic heat-capacity model: base + sum of Einstein terms."""
    T = np.asarray(T, dtype=np.float64)
    cp = np.full_like(T, base)
    for th in thetas:
        x = th / T
        ex = np.exp(-x)
        cp = cp + scale * x * x * ex / (1.0 - ex) ** 2
    return cp


def _fit_nasa(cp_fn, hf, s0):
    """NASA-7 low/high tables for one species, C1-continuous in cp at T_MID.

    cp/R is fitted by a quartic on each range (least squares on a dense grid).  The
    high-range quartic is written as a Taylor expansion about T_MID whose first two
    terms are the low fit's value and slope there, so cp and dcp/dT are continuous.
    The enthalpy and entropy constants (a6, a7) anchor h(298.15) = hf and
    s(298.15) = s0 on the low range and make h and s continuous at T_MID.
    """
    sc = 1000.0  # fit in t = T/1000 for conditioning
    t_lo = np.linspace(T_LO, T_MID, 161) / sc
    c_lo = np.polynomial.polynomial.polyfit(t_lo, cp_fn(t_lo * sc), 4)
    tm = T_MID / sc
    v = np.polynomial.polynomial.polyval(tm, c_lo)
    s = np.polynomial.polynomial.polyval(tm, np.polynomial.polynomial.polyder(c_lo))
    t_hi = np.linspace(T_MID, T_HI, 301) / sc
    u = t_hi - tm
    rhs = cp_fn(t_hi * sc) - v - s * u
    d, *_ = np.linalg.lstsq(np.stack([u ** 2, u ** 3, u ** 4], axis=1), rhs, rcond=None)
    taylor = np.array([v, s, d[0], d[1], d[2]])
    # expand sum_i taylor_i (t - tm)^i into powers of t
    c_hi = np.zeros(5)
    for i, ti in enumerate(taylor):
        c_hi[: i + 1] += ti * np.polynomial.polynomial.polypow([-tm, 1.0], i)
    a_lo = np.array([c_lo[i] / sc ** i for i in range(5)])
    a_hi = np.array([c_hi[i] / sc ** i for i in range(5)])

    def h_poly(a, T):  # h/R without the a6 constant
        return a[0] * T + a[1] * T ** 2 / 2 + a[2] * T ** 3 / 3 + a[3] * T ** 4 / 4 + a[4] * T ** 5 / 5

    def s_poly(a, T):  # s/R without the a7 constant
        return a[0] * np.log(T) + a[1] * T + a[2] * T ** 2 / 2 + a[3] * T ** 3 / 3 + a[4] * T ** 4 / 4

    R = 8.31446261815324
    a6_lo = hf / R - h_poly(a_lo, T_REF)
    a7_lo = s0 / R - s_poly(a_lo, T_REF)
    a6_hi = h_poly(a_lo, T_MID) + a6_lo - h_poly(a_hi, T_MID)
    a7_hi = s_poly(a_lo, T_MID) + a7_lo - s_poly(a_hi, T_MID)
    return np.concatenate([a_lo, [a6_lo, a7_lo]]), np.concatenate([a_hi, [a6_hi, a7_hi]])


def build(seed: int = 0) -> dict:
    """The seeded synthetic 9-species / 21-reaction H2-O2-N2 mechanism.

    Returns a dict with
      species [S] names, elements [E] names,
      W [S] molar masses (kg/mol), ncomp [S, E] element counts (int),
      nasa_lo, nasa_hi [S, 7] NASA-7 tables, T_lo, T_mid, T_hi [S] (K),
      nu_f, nu_r [R, S] reactant / product stoichiometric coefficients (int),
      rtype [R] (0 elementary, 1 third body, 2 fall-off),
      A, b, Ea [R] (high-pressure limit for fall-off; SI),
      A0, b0, Ea0 [R] low-pressure limit (fall-off only, else 0),
      troe [R, 4] (alpha, T***, T*, T**), troe_n [R] (0 Lindemann, 3 or 4),
      eff [R, S] third-body efficiencies (1 where unused),
      reversible [R] (int), duplicate [R] (int), equations [R] strings.
    """
    species = [sp + (0.0,) for sp in _SPECIES]
    return _build(species, list(_REACTIONS), seed, f"synthetic-h2o2-9sp21r-seed{seed}", {}, set())


def build13(seed: int = 0) -> dict:
    """The seeded synthetic 13-species / 27-reaction mechanism: the paper's mechanism
    size (13 species, 27 reactions; Sec. 5.2.3), built like ``build`` with argon,
    helium, CO and CO2 as colliders and six more reactions (_REACTIONS13_EXTRA).  Same
    dict layout as ``build``; species order SPECIES13."""
    species = [sp + (0.0,) for sp in _SPECIES] + list(_SPECIES13_EXTRA)
    return _build(species, list(_REACTIONS) + list(_REACTIONS13_EXTRA), seed,
                  f"synthetic-h2o2-13sp27r-seed{seed}", _COLLIDERS13, _SEPARATE13)


def _build(species_tab, reactions, seed, name, colliders, separate) -> dict:
    """Draw a mechanism's coefficients (module docstring).  colliders: third-body
    efficiencies of the extra species in every +M reaction (0 for Ar, He in the
    reactions listed in `separate`, whose Ar / He channels are their own reactions)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    names = tuple(sp[0] for sp in species_tab)
    S, Rn = len(species_tab), len(reactions)
    W = np.array([sum(n * ATOMIC_MASS[el] for n, el in zip(comp, ELEMENTS)) + other
                  for _, comp, _, _, _, _, other in species_tab])
    ncomp = np.array([comp for _, comp, *_ in species_tab], dtype=np.int32)

    nasa_lo = np.zeros((S, 7))
    nasa_hi = np.zeros((S, 7))
    for k, (nm, _, hf, s0, base, thetas, other) in enumerate(species_tab):
        th = tuple(t * rng.uniform(0.95, 1.05) for t in thetas)
        scale = rng.uniform(0.97, 1.0)
        noble = nm in ("AR", "HE")
        lin = rng.uniform(0.0, 0.05) if not thetas and not noble else 0.0  # electronic term for atoms

        def cp_fn(T, base=base, th=th, scale=scale, lin=lin):
            return _einstein_cp(T, base, th, scale) + lin * (T / 1000.0)

        nasa_lo[k], nasa_hi[k] = _fit_nasa(cp_fn, hf, s0)

    nu_f = np.zeros((Rn, S), dtype=np.int32)
    nu_r = np.zeros((Rn, S), dtype=np.int32)
    rtype = np.zeros(Rn, dtype=np.int32)
    A = np.zeros(Rn); b = np.zeros(Rn); Ea = np.zeros(Rn)
    A0 = np.zeros(Rn); b0 = np.zeros(Rn); Ea0 = np.zeros(Rn)
    troe = np.zeros((Rn, 4)); troe_n = np.zeros(Rn, dtype=np.int32)
    eff = np.ones((Rn, S))
    dup = np.zeros(Rn, dtype=np.int32)

    def draw(centre):
        lgA, bc, ea_kj = centre
        lgA = lgA + rng.uniform(-0.2, 0.2)
        bb = bc if float(bc).is_integer() else bc + rng.uniform(-0.1, 0.1)
        ea = 0.0 if ea_kj == 0.0 else ea_kj * 1e3 * rng.uniform(0.95, 1.05)
        return 10.0 ** lgA, bb, ea

    for j, (eq, typ, centre, centre0, effs, is_dup) in enumerate(reactions):
        lhs, rhs = eq.split("=")
        for k, n in _parse_side(lhs, names).items():
            nu_f[j, k] = n
        for k, n in _parse_side(rhs, names).items():
            nu_r[j, k] = n
        order = int(nu_f[j].sum())
        rtype[j] = {"elem": 0, "tb": 1, "troe": 2}[typ]
        a_cgs, b[j], Ea[j] = draw(centre)
        # cm^3 -> m^3: A_SI = A_cgs * (1e-6)^(order - 1); a third body adds one order
        A[j] = a_cgs * 1e-6 ** (order - 1 + (1 if typ == "tb" else 0))
        if typ == "troe":
            a0_cgs, b0[j], Ea0[j] = draw(centre0)
            A0[j] = a0_cgs * 1e-6 ** order
            troe_n[j] = _TROE_NPARAM[eq]
            troe[j, 0] = rng.uniform(0.4, 0.8)
            troe[j, 1] = rng.uniform(50.0, 300.0)
            troe[j, 2] = rng.uniform(1000.0, 5000.0)
            troe[j, 3] = rng.uniform(3000.0, 8000.0) if troe_n[j] == 4 else 0.0
        if effs and "*" in effs:
            eff[j, :] = effs["*"]
        if typ != "elem" and not (effs and "*" in effs):
            for nm, val in colliders.items():
                eff[j, names.index(nm)] = 0.0 if (eq in separate and nm in ("AR", "HE")) else val
        if effs:
            for nm, val in effs.items():
                if nm == "*":
                    continue
                eff[j, names.index(nm)] = val if "*" in effs else val * rng.uniform(0.9, 1.1)
        dup[j] = int(is_dup)

    return {
        "name": name,
        "species": list(names), "elements": list(ELEMENTS),
        "W": W, "ncomp": ncomp,
        "nasa_lo": nasa_lo, "nasa_hi": nasa_hi,
        "T_lo": np.full(S, T_LO), "T_mid": np.full(S, T_MID), "T_hi": np.full(S, T_HI),
        "nu_f": nu_f, "nu_r": nu_r, "rtype": rtype,
        "A": A, "b": b, "Ea": Ea, "A0": A0, "b0": b0, "Ea0": Ea0,
        "troe": troe, "troe_n": troe_n, "eff": eff,
        "reversible": np.ones(Rn, dtype=np.int32), "duplicate": dup,
        "equations": [r[0] for r in reactions],
    }


def custom(species, W, ncomp, nasa_lo, nasa_hi, reactions, T_mid=1000.0) -> dict:
    """A small hand-specified mechanism in the same dict layout as ``build``.

    ``reactions`` is a list of dicts with keys nu_f, nu_r (dict species index -> int),
    type ("elem", "tb", "troe"), A, b, Ea and, where they apply, A0, b0, Ea0,
    troe (tuple of 0, 3 or 4 numbers), eff (dict index -> value), reversible.
    Used for test mechanisms with closed-form behaviour (isomerisation, pure
    third-body recombination, single-species thermo).
    """
    S = len(species)
    Rn = len(reactions)
    m = {
        "name": "custom", "species": list(species), "elements": list(ELEMENTS),
        "W": np.asarray(W, dtype=np.float64), "ncomp": np.asarray(ncomp, dtype=np.int32),
        "nasa_lo": np.asarray(nasa_lo, dtype=np.float64), "nasa_hi": np.asarray(nasa_hi, dtype=np.float64),
        "T_lo": np.full(S, T_LO), "T_mid": np.full(S, T_mid), "T_hi": np.full(S, T_HI),
        "nu_f": np.zeros((Rn, S), dtype=np.int32), "nu_r": np.zeros((Rn, S), dtype=np.int32),
        "rtype": np.zeros(Rn, dtype=np.int32),
        "A": np.zeros(Rn), "b": np.zeros(Rn), "Ea": np.zeros(Rn),
        "A0": np.zeros(Rn), "b0": np.zeros(Rn), "Ea0": np.zeros(Rn),
        "troe": np.zeros((Rn, 4)), "troe_n": np.zeros(Rn, dtype=np.int32),
        "eff": np.ones((Rn, S)), "reversible": np.ones(Rn, dtype=np.int32),
        "duplicate": np.zeros(Rn, dtype=np.int32), "equations": [f"R{j}" for j in range(Rn)],
    }
    for j, r in enumerate(reactions):
        for k, n in r["nu_f"].items():
            m["nu_f"][j, k] = n
        for k, n in r["nu_r"].items():
            m["nu_r"][j, k] = n
        m["rtype"][j] = {"elem": 0, "tb": 1, "troe": 2}[r.get("type", "elem")]
        m["A"][j], m["b"][j], m["Ea"][j] = r["A"], r.get("b", 0.0), r.get("Ea", 0.0)
        m["A0"][j], m["b0"][j], m["Ea0"][j] = r.get("A0", 0.0), r.get("b0", 0.0), r.get("Ea0", 0.0)
        tr = tuple(r.get("troe", ()))
        m["troe_n"][j] = len(tr)
        m["troe"][j, : len(tr)] = tr
        for k, v in r.get("eff", {}).items():
            m["eff"][j, k] = v
        m["reversible"][j] = int(r.get("reversible", True))
    return m
