"""Compile-time resources of the hot kernels (ptxas -v, sm_103a, no GPU):
every instantiation of the ray kernel and of the adjoint compiles without
register spills, and the ray kernel of the FP32 modes fits its CTA of
MT_DX_THREADS threads in the registers an SM has (65 536)."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import tempfile

import pytest

from paper_2603_28907_gb300 import build as B

CSRC = os.path.join(os.path.dirname(B.OUT), "csrc")
UNITS = ["march_f32.cu", "march_f32c.cu", "march_bf16.cu", "march_f64.cu", "adjoint.cu"]


def _ptxas_report(unit, tmp):
    cmd = [B.nvcc(), "-c", os.path.join(CSRC, unit), "-o", os.path.join(tmp, unit + ".o")] + B._flags(True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = {}
    for block in r.stderr.split("Compiling entry function '")[1:]:
        name = block.split("'", 1)[0]
        regs = [int(x) for x in re.findall(r"Used (\d+) registers", block)]
        spills = [int(x) for x in re.findall(r"(\d+) bytes spill (?:stores|loads)", block)]
        out[name] = (max(regs) if regs else 0, max(spills) if spills else 0)
    return out


@pytest.fixture(scope="module")
def reports():
    try:
        B.nvcc()
    except Exception:
        pytest.skip("nvcc not available")
    tmp = tempfile.mkdtemp(prefix="mt_ptxas_")
    try:
        with cf.ThreadPoolExecutor(len(UNITS)) as ex:
            res = dict(zip(UNITS, ex.map(lambda u: _ptxas_report(u, tmp), UNITS)))
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return res


def test_hot_kernels_do_not_spill(reports):
    n = 0
    for unit, rep in reports.items():
        for name, (regs, spill) in rep.items():
            if "k_march" in name or "k_adjoint" in name:
                assert spill == 0, (unit, name, regs, spill)
                n += 1
    assert n >= 10


def _march_threads():
    """The FP32 march's CTA size, as march.cuh defines it."""
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2603_28907_gb300", "csrc", "march.cuh")).read()
    return int(re.search(r"#define MT_DX_THREADS (\d+)", src).group(1))


def test_fp32_ray_kernel_fits_its_cta(reports):
    """Registers per thread times the CTA's threads fit the SM's 65 536
    registers (allocated in units of 8 per thread), so the launch succeeds."""
    threads = _march_threads()
    limit = (65536 // threads) // 8 * 8
    n = 0
    for unit in ("march_f32.cu", "march_f32c.cu"):
        for name, (regs, _) in reports[unit].items():
            if "k_march" in name:
                assert 0 < regs <= limit, (unit, name, regs, threads)
                n += 1
    assert n >= 2
