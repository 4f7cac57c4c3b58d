"""The C-ABI library builds, loads without a GPU and exports every entry point include/*.h declares."""
import os
import re

from paper_2603_29332_b300 import build as B
from paper_2603_29332_b300 import msim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names.update(re.findall(r"MSIM_API\s+[\w\s\*]+?\b(msim_\w+)\s*\(", src))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = msim.load_library(path)
    names = declared_entry_points()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(msim.EXPORTS) == names
    assert lib.msim_version() >= 1


def test_create_without_device_fails_cleanly():
    """No GPU here: create must fail with an error code, not crash or fall back to the CPU."""
    import ctypes as C
    import torch
    if torch.cuda.is_available():
        return
    from paper_2603_29332_b300 import modelgen as mg
    lib = msim.load_library()
    d, keep = msim.model_desc(mg.config_model("c0_tiny"))
    arr = (msim.ModelDesc * 1)(d)
    epm = (C.c_int32 * 1)(4)
    args = msim.CreateArgs(1, arr, epm, 0, 1e-3, 0, 0)
    h = C.c_void_p()
    st = lib.msim_create(C.byref(args), C.byref(h))
    assert st in (2, 3) and not h.value
    assert len(lib.msim_last_error(None)) > 0


def test_model_validation_errors_are_reported_without_a_device():
    """Validation happens before any CUDA call: a broken model is MSIM_ERR_MODEL on any host."""
    import ctypes as C
    import numpy as np
    from paper_2603_29332_b300 import modelgen as mg
    lib = msim.load_library()
    m = mg.config_model("c0_tiny")
    bad = dict(m.__dict__)
    cases = []
    mm = mg.Model(**bad); mm.body_parent = m.body_parent.copy(); mm.body_parent[3] = 5
    cases.append((mm, "body_parent"))
    mm = mg.Model(**bad); mm.dof_axis = m.dof_axis * 2.0
    cases.append((mm, "unit"))
    mm = mg.Model(**bad); mm.point_body = m.point_body.copy()
    # insertion on a body outside the origin's subtree: put the last point of muscle 0 on body 0
    mm.point_body[m.muscle_point_start[1] - 1] = 0 if m.point_body[0] != 0 else 1
    cases.append((mm, "descendant"))
    for model, word in cases:
        d, keep = msim.model_desc(model)
        arr = (msim.ModelDesc * 1)(d)
        epm = (C.c_int32 * 1)(4)
        args = msim.CreateArgs(1, arr, epm, 0, 1e-3, 0, 0)
        h = C.c_void_p()
        st = lib.msim_create(C.byref(args), C.byref(h))
        assert st == 4, (word, st)
        assert word in lib.msim_last_error(None).decode()
