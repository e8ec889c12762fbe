"""Build libmt.so (the C-ABI library) in-tree for sm_103a with nvcc.

Each translation unit under csrc/ compiles in its own nvcc process (in
parallel), then they link into paper_2603_28907_gb300/libmt.so with the CUDA
runtime linked statically.  ``python -m paper_2603_28907_gb300.build`` runs it;
``--checked`` builds libmt_checked.so instead, with MT_BOUNDS_CHECK (every cell
and voxel index the kernels form is verified; one out of range latches the
device status word, see mt_sync).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libmt.so")
BUILD = os.path.join(HERE, "_build")
OUT_CHECKED = os.path.join(HERE, "libmt_checked.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmt.so")


def _flags(verbose_ptxas: bool) -> list:
    # host code: no fused multiply-add contraction, so that it rounds alike
    # on x86 and Arm hosts
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr", "-Xcompiler", "-fvisibility=hidden"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return ARCH + f


def _sources() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list:
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def up_to_date(out: str = OUT) -> bool:
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None,
          checked: bool = False) -> str:
    out, bdir = (OUT_CHECKED, BUILD_CHECKED) if checked else (OUT, BUILD)
    if not force and up_to_date(out):
        return out
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    srcs = _sources()
    extra = ["-DMT_BOUNDS_CHECK"] if checked else []

    def one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, "-c", src, "-o", obj] + _flags(verbose_ptxas) + extra
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        res = list(ex.map(one, srcs))
    if verbose_ptxas:
        for _, log in res:
            sys.stderr.write(log)
    objs = [o for o, _ in res]
    tmp = out + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, checked="--checked" in sys.argv))
