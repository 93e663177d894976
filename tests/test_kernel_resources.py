"""Compile-time resources of the integration kernels (ptxas reports of the in-tree build),
on the CPU: the register caps the launch shapes rely on for their residency."""
import pytest

from paper_2506_02602_gb300 import build


@pytest.fixture(scope="module")
def res():
    build.build()
    return {"9": build.kernel_resources("k_lsrk"),
            "13": build.kernel_resources("k_lsrk", build.LIBS["h2o2_13"]["build"])}


def _regs(rs, prefix):
    hits = [r for r in rs if r["kernel"].startswith(prefix)]
    assert hits, prefix
    return hits[0]["registers"]


def test_mixed_two_register_kernel_runs_32_warps_per_sm(res):
    # k_lsrk<MIXED, 64, 16, LSRK> and <MIXED, 32, 32, LSRK>: 64 registers (32 warps per SM)
    for lib in ("9", "13"):
        assert _regs(res[lib], "_ZN4chem6k_lsrkILi1ELi64ELi16ELi0E") <= 64
        assert _regs(res[lib], "_ZN4chem6k_lsrkILi1ELi32ELi32ELi0E") <= 64


def test_fp64_kernel_keeps_its_12_warp_budget(res):
    # k_lsrk<FP64, 128, 3, LSRK>: at most 170 registers (12 warps per SM); the 9-species
    # structure fits without spills
    assert _regs(res["9"], "_ZN4chem6k_lsrkILi0ELi128ELi3ELi0E") <= 170
    r = [x for x in res["9"] if x["kernel"].startswith("_ZN4chem6k_lsrkILi0ELi128ELi3ELi0E")][0]
    assert r["spill_stores"] == 0 and r["spill_loads"] == 0


def test_persistent_mixed_shape_4_is_the_32_warp_one(res):
    rs = build.kernel_resources("k_lsrk_persistent")
    assert _regs(rs, "_ZN4chem17k_lsrk_persistentILi1ELi64ELi16E") <= 64
