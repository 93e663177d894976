"""The roofline's credited work follows the compiled mechanism structure.

roofline.py credits flops per reaction from its (reactant count, product count, type,
Troe parameter count).  These checks hold its built-in 9-species table and the structure
it derives from a mechanism description to the generated compiled headers
(csrc/mech_h2o2_*.cuh), and pin the per-step figures the benchmark reports, so that a
change to the kernels' formulation or to a mechanism cannot leave the credited work
silently stale.
"""
import os
import re

from chem_inputs import mechanism as M
from paper_2506_02602_gb300 import roofline

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2506_02602_gb300", "csrc")
_TYPES = {"ELEM": 0, "THIRD_BODY": 1, "FALLOFF": 2}


def _compiled(header):
    """(species count, [(n_reactants, n_products, type, troe_n)]) of a generated header."""
    with open(os.path.join(CSRC, header)) as f:
        txt = f.read()
    nsp = int(re.search(r"constexpr int NSP = (\d+);", txt).group(1))
    rx = []
    for r0, r1, p0, p1, ty, tn in re.findall(
            r"\{(\w+), (\w+), (\w+), (\w+), (ELEM|THIRD_BODY|FALLOFF), (\d+)\}", txt):
        rx.append(((r0 != "NONE") + (r1 != "NONE"), (p0 != "NONE") + (p1 != "NONE"), _TYPES[ty], int(tn)))
    return nsp, rx


def test_builtin_table_is_the_compiled_9_species_structure():
    nsp, rx = _compiled("mech_h2o2_9.cuh")
    assert nsp == roofline.NSP and rx == roofline._RX


def test_structure_from_a_mechanism_matches_its_compiled_header():
    for mech, header in ((M.build(0), "mech_h2o2_9.cuh"), (M.build13(0), "mech_h2o2_13.cuh")):
        assert roofline._structure(mech) == _compiled(header)


def test_credited_work_per_unit():
    """The figures quoted with the benchmark's roofline: per attempted step of the
    two-register scheme (fp64 and the mixed kernel's fp64 part), of the comparators, and
    per cell for the final temperature solve."""
    m9, m13 = M.build(0), M.build13(0)
    assert roofline.step_flops(m9) == 8224
    assert roofline.step_flops(m9, scheme=1) == 8304
    assert roofline.step_flops(m9, scheme=2) == 9991
    assert roofline.step_flops(m13) == 11246
    assert roofline.step_flops_mixed_fp64(m9) == 1809
    assert roofline.cell_flops(m9) == 157 and roofline.cell_flops(m13) == 205
    # one launch: attempted steps x per-step work + cells x per-cell work
    assert roofline.launch_flops(10, 3, m9) == 10 * 8224 + 3 * 157
