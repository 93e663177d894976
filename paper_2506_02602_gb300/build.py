"""In-tree build of the libraries for sm_103a (GB300).

Each CUDA translation unit under csrc/ compiles in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo); the objects link into
paper_2506_02602_gb300/libchem.so (the 9-species mechanism structure) and
libchem_h2o2_13.so (the 13-species one), the same sources compiled once per
structure.  ptxas resource reports (registers, spills) land in
_build/<unit>.ptxas.txt (and _build/h2o2_13/).  The build is skipped when every library
is newer than every source and header.
"""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libchem.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
         "-I", os.path.join(ROOT, "include")]

# One library per compiled mechanism structure (csrc/mech_*.cuh): the 9-species /
# 21-reaction mechanism with the learned surrogate, and the 13-species / 27-reaction one
# (the paper's mechanism size) whose surrogate entry points are stubs.
_SURROGATE = ("mlp.cu", "mlp_fused.cu", "mlp_tc.cu", "mlp_gemm_tc.cu", "surrogate.cu", "surrogate_kernels.cu")
LIBS = {
    "h2o2_9": {"lib": LIB, "defines": [], "skip": ("surrogate_stub.cu",), "build": BUILD},
    "h2o2_13": {"lib": os.path.join(PKG, "libchem_h2o2_13.so"), "defines": ["-DCHEM_MECH_H2O2_13"],
                "skip": _SURROGATE, "build": os.path.join(BUILD, "h2o2_13")},
}


def _inputs():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + [os.path.join(ROOT, "include", "chem.h")])


def up_to_date() -> bool:
    for spec in LIBS.values():
        if not os.path.exists(spec["lib"]):
            return False
        t = os.path.getmtime(spec["lib"])
        if not all(os.path.getmtime(f) <= t for f in _inputs()):
            return False
    return True


def _compile(job) -> str:
    src, defines, bdir = job
    name = os.path.splitext(os.path.basename(src))[0]
    obj = os.path.join(bdir, name + ".o")
    log = os.path.join(bdir, name + ".ptxas.txt")
    r = subprocess.run([NVCC, *ARCH, *FLAGS, *defines, "-c", src, "-o", obj], capture_output=True, text=True)
    with open(log, "w") as f:
        f.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src} {' '.join(defines)}:\n{r.stderr[-4000:]}")
    return obj


def build(force: bool = False) -> str:
    """Compile and link every library of LIBS (all translation units of all libraries in
    one parallel pool); returns the path of the 9-species libchem.so."""
    if not force and up_to_date():
        return LIB
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    jobs, per_lib = [], {}
    for tag, spec in LIBS.items():
        os.makedirs(spec["build"], exist_ok=True)
        mine = [s for s in srcs if os.path.basename(s) not in spec["skip"]]
        per_lib[tag] = (len(jobs), len(mine))
        jobs += [(s, spec["defines"], spec["build"]) for s in mine]
    # the heaviest units first so the pool's tail is short
    order = sorted(range(len(jobs)), key=lambda i: -os.path.getsize(jobs[i][0]))
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4, len(jobs))) as ex:
        done = dict(zip(order, ex.map(_compile, [jobs[i] for i in order])))
    for tag, spec in LIBS.items():
        first, count = per_lib[tag]
        objs = [done[i] for i in range(first, first + count)]
        tmp = spec["lib"] + f".tmp{os.getpid()}"
        r = subprocess.run([NVCC, *ARCH, "-shared", *objs, "-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {spec['lib']} failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, spec["lib"])
    return LIB


def ptxas_report() -> str:
    """Concatenated ptxas register/spill lines of the last build."""
    out = []
    for f in sorted(glob.glob(os.path.join(BUILD, "*.ptxas.txt"))):
        with open(f) as fh:
            lines = [ln.strip() for ln in fh if "registers" in ln or "spill" in ln or "Function properties" in ln]
        out.append(os.path.basename(f) + ":\n  " + "\n  ".join(lines))
    return "\n".join(out)


def kernel_resources(pattern: str = "", build_dir: str | None = None) -> list:
    """Registers, stack frame and spill bytes per compiled kernel of the last build (from
    ptxas -v), for kernels whose mangled name contains `pattern` (build_dir: a library's
    object folder, LIBS[...]["build"]; the 9-species one by default)."""
    import re
    out = []
    for f in sorted(glob.glob(os.path.join(build_dir or BUILD, "*.ptxas.txt"))):
        with open(f) as fh:
            txt = fh.read()
        for blk in re.split(r"Compiling entry function '", txt)[1:]:
            name = blk.split("'")[0]
            if pattern not in name:
                continue
            st = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", blk)
            rg = re.search(r"Used (\d+) registers", blk)
            if st and rg:
                out.append({"kernel": name, "registers": int(rg.group(1)), "stack": int(st.group(1)),
                            "spill_stores": int(st.group(2)), "spill_loads": int(st.group(3))})
    return out


if __name__ == "__main__":
    print(build(force=True))
    print(ptxas_report())
