"""Build libtcm.so (the CUDA library behind include/tcm.h) in-tree with nvcc.

Only sm_103a code is generated.  Floating-point flags keep Eq. 3 bit-exact:
no FMA contraction (-fmad=false), no flush-to-zero, IEEE division and square
root.  The runtime and kernels compile once per supported brick shape (with
their entry points renamed per shape), plus the dispatcher of the public C
ABI; all translation units compile in parallel and link into one shared
library with the CUDA runtime linked statically.

With TCM_CHECKED=1 in the environment the same sources build the checked
library, libtcm_checked.so (compiled with -DTCM_CHECKED: every box, brick,
free-stack, list and claim index is bounds-checked on the device, an index
out of range sets an error bit that the next status read turns into
TCM_EDEVICE, and the access is skipped), which the binding then loads.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB_NORMAL = os.path.join(HERE, "libtcm.so")
LIB_CHECKED = os.path.join(HERE, "libtcm_checked.so")


def checked() -> bool:
    """Whether this process builds and loads the bounds-checked library."""
    return os.environ.get("TCM_CHECKED", "") == "1"


LIB = LIB_CHECKED if checked() else LIB_NORMAL
UNITS = ["tcm_kernels.cu", "tcm_api.cu", "tcm_noalloc.cu"]
DISPATCH = "tcm_dispatch.cpp"
DEPS = UNITS + ["tcm_internal.cuh", DISPATCH]
# One build of the runtime and kernels per brick shape and CTA blocking
# (bx, by, bz, warps per CTA of the step kernel, name); tcm_dispatch.cpp
# routes the public entry points to them.  8 warps per CTA is the default of
# every shape; the 8x8x8 shape also has 4- and 16-warp builds for the
# autotuner.
SHAPES = [(4, 4, 4, 8, "b444"), (8, 8, 8, 8, "b888"), (16, 8, 8, 8, "b1688"),
          (8, 8, 8, 4, "b888w4"), (8, 8, 8, 12, "b888w12")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-ftz=false", "-prec-div=true",
         "-prec-sqrt=true", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I", os.path.join(ROOT, "include")]


def public_names():
    """Entry points declared in include/tcm.h (renamed per shape build)."""
    import re
    src = open(os.path.join(ROOT, "include", "tcm.h")).read()
    return sorted(set(re.findall(r"\b(tcm_[a-z_]+)\s*\(", src)))


def shape_defines(bx, by, bz, warps, name):
    d = [f"-DTCM_BX={bx}", f"-DTCM_BY={by}", f"-DTCM_BZ={bz}", f"-DTCM_P1_WARPS={warps}", f"-Dtcm=tcm_{name}",
         f"-Dtcm_sim=tcm_{name}_sim", f"-Dtcm_batch=tcm_{name}_batch",
         f"-Dtcm_internal_view=tcm_{name}_internal_view"]
    d += [f"-D{f}=tcm_{name}_{f[4:]}" for f in public_names()]
    return d


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(ROOT, "include", "tcm.h"),
                                                    os.path.abspath(__file__)]
    return any(os.path.getmtime(s) > t for s in srcs)


def _compile(unit: str, extra, tag: str = "") -> str:
    if checked():
        extra = list(extra) + ["-DTCM_CHECKED"]
        tag += "_checked"
    obj = os.path.join(BUILD, unit.replace(".cu", "").replace(".cpp", "") + tag + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {unit}{tag}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile libtcm.so if any source is newer than it; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    jobs = [(u, extra + shape_defines(*sh), "_" + sh[4]) for sh in SHAPES for u in UNITS]
    jobs.append((DISPATCH, [], ""))
    with cf.ThreadPoolExecutor(min(len(jobs), max(4, os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda j: _compile(*j), jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
