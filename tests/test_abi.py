"""Host-side checks of the C ABI (no GPU needed).

* libchem.so builds, loads and exports every entry point include/chem.h declares;
* the ctypes structures have the sizes and field offsets of the C header (compiled
  with gcc here);
* chem_setup's validation: wrong structure -> UNSUPPORTED, unbalanced reaction or
  discontinuous NASA-7 tables -> INVALID, and a valid mechanism without a device ->
  CUDA error (no CPU fallback).
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from chem_inputs import mechanism as M
from paper_2506_02602_gb300 import build as B
from paper_2506_02602_gb300 import chem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "chem.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return chem.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chem_[A-Za-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 7
    out = subprocess.run(["nm", "-D", "--defined-only", chem.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (chem_[A-Za-z_0-9]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_every_structure_library_exports_every_symbol(lib):
    """One library per compiled mechanism structure; each exports the whole ABI (the
    13-species one answers the surrogate calls with CHEM_ERR_UNSUPPORTED)."""
    names = declared_functions()
    for n_sp, path in chem.LIB_PATHS.items():
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                             check=True).stdout
        exported = set(re.findall(r"\bT (chem_[A-Za-z_0-9]+)", out))
        assert not [n for n in names if n not in exported], (n_sp, path)
    L13 = chem.load(13)
    assert L13.chem_surrogate_param_count() == 0
    assert L13.chem_surrogate_save(None, b"x") == chem.ERR_UNSUPPORTED


def test_generated_structure_headers_are_current():
    """csrc/mech_*.cuh are what gen_mech.py writes for the mechanism descriptions."""
    import importlib.util
    gen = os.path.join(ROOT, "paper_2506_02602_gb300", "csrc", "gen_mech.py")
    spec = importlib.util.spec_from_file_location("gen_mech", gen)
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    for tag, fn in (("h2o2_9", M.build), ("h2o2_13", M.build13)):
        with open(os.path.join(ROOT, "paper_2506_02602_gb300", "csrc", f"mech_{tag}.cuh")) as f:
            assert f.read() == g.header(tag, fn(0)), tag


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "chem.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(chem_mechanism), sizeof(chem_options), sizeof(chem_state),
         sizeof(chem_stats));
  printf("%zu %zu %zu %zu\n", offsetof(chem_mechanism, eff), offsetof(chem_mechanism, reversible),
         offsetof(chem_state, d_nsteps), offsetof(chem_stats, status_count));
  printf("%zu %zu %zu %zu\n", sizeof(chem_batch), sizeof(chem_batch_options),
         offsetof(chem_batch, d_box_nsub), offsetof(chem_batch_options, d_cost_hint));
  printf("%zu %zu %zu %zu\n", sizeof(chem_pairs), sizeof(chem_train_cfg), sizeof(chem_surrogate_gate),
         offsetof(chem_train_cfg, seed));
  printf("%zu %zu %zu\n", sizeof(chem_tune_result), offsetof(chem_tune_result, ms),
         offsetof(chem_tune_result, ctas_per_sm));
  return 0;
}''')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    a, b, c, d, t = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:5]
    assert [int(x) for x in a.split()] == [C.sizeof(chem.Mechanism), C.sizeof(chem.Options),
                                          C.sizeof(chem.State), C.sizeof(chem.Stats)]
    assert [int(x) for x in b.split()] == [chem.Mechanism.eff.offset, chem.Mechanism.reversible.offset,
                                          chem.State.d_nsteps.offset, chem.Stats.status_count.offset]
    assert [int(x) for x in c.split()] == [C.sizeof(chem.Batch), C.sizeof(chem.BatchOptions),
                                          chem.Batch.d_box_nsub.offset, chem.BatchOptions.d_cost_hint.offset]
    assert [int(x) for x in d.split()] == [C.sizeof(chem.Pairs), C.sizeof(chem.TrainCfg), C.sizeof(chem.Gate),
                                          chem.TrainCfg.seed.offset]
    assert [int(x) for x in t.split()] == [C.sizeof(chem.TuneResult), chem.TuneResult.ms.offset,
                                          chem.TuneResult.ctas_per_sm.offset]


def _setup_rc(lib, mech, variant=0, scheme=0):
    m = chem.make_mechanism(mech)
    opt = chem.Options()
    opt.variant = variant
    opt.scheme = scheme
    h = C.c_void_p()
    rc = lib.chem_setup(C.byref(m), C.byref(opt), C.byref(h))
    msg = lib.chem_last_error(None).decode()
    if rc == 0:
        lib.chem_teardown(h)
    return rc, msg


def test_setup_rejects_other_structure(lib):
    m = M.build(0)
    m["nu_r"] = m["nu_r"].copy()
    m["nu_f"] = m["nu_f"].copy()
    # swap the products of two reactions: still balanced, but not the compiled structure
    m["nu_r"][[9, 10]] = m["nu_r"][[10, 9]]
    rc, msg = _setup_rc(lib, m)
    assert rc == chem.ERR_UNSUPPORTED and "stoichiometry" in msg
    small = M.custom(["X"], [0.028], [[0, 0, 2]], np.ones((1, 7)), np.ones((1, 7)), [])
    rc, msg = _setup_rc(lib, small)
    assert rc == chem.ERR_UNSUPPORTED


def test_setup_rejects_unbalanced_reaction(lib):
    m = M.build(0)
    m["nu_r"] = m["nu_r"].copy()
    m["nu_r"][0, M.SPECIES.index("OH")] = 0
    m["nu_r"][0, M.SPECIES.index("H")] = 1  # H + O2 -> O + H: loses an oxygen
    rc, msg = _setup_rc(lib, m)
    assert rc == chem.ERR_INVALID and "balance" in msg


def test_setup_rejects_discontinuous_thermo(lib):
    m = M.build(0)
    m["nasa_hi"] = m["nasa_hi"].copy()
    m["nasa_hi"][2, 5] += 50.0
    rc, msg = _setup_rc(lib, m)
    assert rc == chem.ERR_INVALID and "discontinuous" in msg


def test_setup_rejects_bad_options(lib):
    rc, msg = _setup_rc(lib, M.build(0), variant=7)
    assert rc == chem.ERR_INVALID
    rc, msg = _setup_rc(lib, M.build(0), scheme=3)
    assert rc == chem.ERR_INVALID and "scheme" in msg


def test_fma_probe_validates_its_arguments(lib):
    """chem_diag_fma_peak rejects an unknown pipe, empty grids, partial warps and a
    missing sink before launching anything."""
    for args in ((2, 1, 32, 1), (0, 0, 32, 1), (0, 1, 48, 1), (1, 1, 2048, 1), (0, 1, 32, 0)):
        assert lib.chem_diag_fma_peak(*args, C.c_void_p(8), None) == chem.ERR_INVALID, args
    assert lib.chem_diag_fma_peak(0, 1, 32, 1, None, None) == chem.ERR_INVALID


def test_ln_inv_kc_diagnostic_rejects_a_missing_context(lib):
    """chem_diag_ln_inv_kc needs a context (its mechanism tables) and refuses NULL
    before launching anything."""
    assert lib.chem_diag_ln_inv_kc(None, 0, 4, C.c_void_p(8), C.c_void_p(8), None) == chem.ERR_INVALID


def test_setup_matches_structure_to_library(lib):
    """The 13-species mechanism is refused by the 9-species library (and the other way
    round) before any device is touched."""
    rc, msg = _setup_rc(lib, M.build13(0))
    assert rc == chem.ERR_UNSUPPORTED and "13" in msg
    rc, msg = _setup_rc(chem.load(13), M.build(0))
    assert rc == chem.ERR_UNSUPPORTED


def test_valid_mechanism_needs_a_device(lib):
    import torch
    for L, mech in ((lib, M.build(0)), (chem.load(13), M.build13(0))):
        rc, msg = _setup_rc(L, mech)
        if torch.cuda.is_available():
            assert rc == chem.OK
        else:
            assert rc == chem.ERR_CUDA and "CUDA device" in msg


def test_diag_math_validates_its_arguments(lib):
    """chem_diag_math's operations 0-14 (the kernels' exp / log, the refined reciprocals,
    the integer-pipe conversions, the hi/lo split, the network's GELU and GELU' and their
    library-erff forms) are accepted and an empty call does nothing; anything else is
    rejected before any device work."""
    for op in range(15):
        assert lib.chem_diag_math(op, 0, None, None, None) == chem.OK, op
    for op in (-1, 15, 99):
        assert lib.chem_diag_math(op, 0, None, None, None) == chem.ERR_INVALID, op
    assert lib.chem_diag_math(0, -1, None, None, None) == chem.ERR_INVALID
    assert lib.chem_diag_math(4, 8, None, None, None) == chem.ERR_INVALID
