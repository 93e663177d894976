"""In-tree build of libchem.so for sm_103a (GB300).

Each CUDA translation unit under csrc/ compiles in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo); the objects link into
paper_2506_02602_gb300/libchem.so.  ptxas resource reports (registers, spills) land in
_build/<unit>.ptxas.txt.  The build is skipped when the library is newer than every
source and header.
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


def _inputs():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + [os.path.join(ROOT, "include", "chem.h")])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(src: str) -> str:
    name = os.path.splitext(os.path.basename(src))[0]
    obj = os.path.join(BUILD, name + ".o")
    log = os.path.join(BUILD, name + ".ptxas.txt")
    r = subprocess.run([NVCC, *ARCH, *FLAGS, "-c", src, "-o", obj], capture_output=True, text=True)
    with open(log, "w") as f:
        f.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr[-4000:]}")
    return obj


def build(force: bool = False) -> str:
    """Compile and link libchem.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(_compile, srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([NVCC, *ARCH, "-shared", *objs, "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB


def ptxas_report() -> str:
    """Concatenated ptxas register/spill lines of the last build."""
    out = []
    for f in sorted(glob.glob(os.path.join(BUILD, "*.ptxas.txt"))):
        with open(f) as fh:
            lines = [ln.strip() for ln in fh if "registers" in ln or "spill" in ln or "Function properties" in ln]
        out.append(os.path.basename(f) + ":\n  " + "\n  ".join(lines))
    return "\n".join(out)


def kernel_resources(pattern: str = "") -> list:
    """Registers, stack frame and spill bytes per compiled kernel of the last build (from
    ptxas -v), for kernels whose mangled name contains `pattern`."""
    import re
    out = []
    for f in sorted(glob.glob(os.path.join(BUILD, "*.ptxas.txt"))):
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
