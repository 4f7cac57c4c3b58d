"""The step kernel's index checks over many models and modes (the stand-in for a memory checker).

libmsim_check.so is the library built with MSIM_BOUNDS_CHECK: every index through the step
kernel's views of its per-environment workspace regions and of the model image's tables is
compared with the extent of its region or table, and an index outside it is recorded (and
replaced by 0, so the run itself stays in bounds).  tests/bounds_child.py runs the tiny model,
the whole body (eval, steps, geometry labels, body positions, 1 and 4 warps per environment,
learned geometry checked and unchecked), the wrapped body with cylinders and spheres, the free
root, compliant tendons, the model at every size limit and a mixed launch of three skeletons,
once with the checking library and once with the normal one, each in a process of its own.
No index may be out of range, and the checking build must compute what the normal one does.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(lib, out):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_child.py"), lib, out],
                       capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_no_index_out_of_range_and_same_results(tmp_path):
    from paper_2603_29332_b300 import build as B
    check_lib = B.build_check()
    checked = _child(check_lib, str(tmp_path / "check.npz"))
    normal = _child(B.build(), str(tmp_path / "normal.npz"))
    assert checked["checking"] and not normal["checking"]
    print("\nbounds records [hits, first site (line), index, extent]:", checked["records"])
    assert len(checked["records"]) == 7
    for name, rec in checked["records"].items():
        assert rec[0] == 0, (name, rec)
    a, b = np.load(tmp_path / "check.npz"), np.load(tmp_path / "normal.npz")
    assert sorted(a.files) == sorted(b.files)
    worst = 0.0
    for k in a.files:
        if k.endswith("_status"):
            assert np.array_equal(a[k], b[k]), k
            continue
        assert np.all(np.isfinite(a[k])), k
        scale = max(1.0, float(np.abs(b[k]).max()))
        diff = float(np.abs(a[k] - b[k]).max()) / scale
        worst = max(worst, diff)
        assert diff <= 1e-4, (k, diff)
    print("largest difference between the checking and the normal build: %.2e (relative)" % worst)
