"""The bounds-checked build (MT_BOUNDS_CHECK, libmt_checked.so): every cell
and voxel index the kernels form from the ray table is verified and one out
of range would latch bit 4 of the device status word.  On the edge cases
(odd grids, downward-looking pixels, a grid marched one surface at a time and
one whose records live in HBM, every
precision, the gradient, the linearised model, capped NUTS) the checked
library must report a clean status word and give exactly the normal
library's results."""
import json
import os
import subprocess
import sys

import pytest

from paper_2603_28907_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(checked):
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    env["MT_CHECKED"] = "1" if checked else "0"
    r = subprocess.run([sys.executable, "-m", "tests.checked_cases"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_is_clean_and_identical():
    build.build(checked=True)
    chk, ref = _run(True), _run(False)
    assert chk["lib"].endswith("libmt_checked.so") and ref["lib"].endswith("libmt.so")
    for name, rec in chk.items():
        if name == "lib":
            continue
        assert rec["clean"], (name, rec.get("error"))
        assert rec == ref[name], (name, rec, ref[name])
