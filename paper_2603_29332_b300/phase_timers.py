"""Per-phase cycle breakdown of the step kernel (profiling build).

``python -m paper_2603_29332_b300.phase_timers`` compiles the library with MSIM_PHASE_TIMERS into
``libmsim_timers.so`` beside the normal build (each environment group's lane 0 adds its
``clock64`` deltas per phase), steps the whole-body model and prints the cycles per
environment-substep of each phase as one JSON line (``--learned``: the learned-geometry substep).  The counts are wall cycles of one
environment group, so they include the issue slots it shares with the other resident groups;
their ratios show where a substep's time goes.  The timers add work: time the normal build.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import subprocess

from . import build as B

LIB = os.path.join(B.HERE, "libmsim_timers.so")
# slots of msim_debug_phase_cycles (the PHASE_MARK / SUB_MARK indices of step_kernels.cu)
NAMES = ["kinematics", "subtree", "crba", "muscles", "contact", "limits", "factor_solve", "-",
         "muscles.geometry", "muscles.hill", "muscles.scatter", "factor.pivot", "factor.scale", "factor.eliminate",
         "factor.x_solve", "kinematics.recursion"]


def build_timers():
    """Compile the profiling build unless the one on disk matches the sources."""
    stamp = LIB + ".sha256"
    dig = B._digest() + "-timers"
    if os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read().strip() == dig:
        return LIB
    cmd = ["nvcc"] + B.ARCH + B.FLAGS + ["-DMSIM_PHASE_TIMERS", "-I", os.path.join(B.ROOT, "include"), "-o", LIB] + \
          [os.path.join(B.CSRC, s) for s in B.SOURCES] + ["-lcudart"]
    subprocess.check_call(cmd)
    with open(stamp, "w") as f:
        f.write(dig + "\n")
    return LIB


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--model", default="c1_whole")
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--substeps", type=int, default=10)
    ap.add_argument("--calls", type=int, default=10)
    ap.add_argument("--shape", type=int, nargs=3, default=(7, 0, 2), metavar=("EPB", "STAGE", "WPE"))
    ap.add_argument("--learned", action="store_true",
                    help="learned-geometry substeps (a briefly trained network, checks off; one substep per call)")
    args = ap.parse_args()
    build_timers()
    from . import modelgen as mg, msim
    lib = msim.load_library(LIB)
    lib.msim_debug_phase_cycles.argtypes = [C.c_void_p, C.POINTER(C.c_ulonglong), C.c_int32]
    import torch
    model = mg.config_model(args.model)
    E, sub = args.envs, (1 if args.learned else args.substeps)
    sim = msim.Sim(model, E, dt=1e-3)
    sim.set_launch(0, *args.shape)
    if args.learned:
        sim.train_surrogate(8192, 1, batch=4096, lr=3e-3)
        sim.set_geometry_mode(1)
        sim.surrogate_set_check(0.0, 1e-3)
    q0, qd0, a0 = mg.initial_state(model, E, seed=1)
    exc = mg.smooth_excitations(model, E, args.calls + 3, seed=1, dt=1e-3 * sub)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    for t in range(3):
        sim.step(sim.pad_m(exc[t]), sub)
    buf = (C.c_ulonglong * 16)()
    lib.msim_debug_phase_cycles(sim.h, buf, 1)   # reset
    for t in range(args.calls):
        sim.step(sim.pad_m(exc[3 + t]), sub)
    torch.cuda.synchronize()
    lib.msim_debug_phase_cycles(sim.h, buf, 0)
    per = E * sub * args.calls
    out = {n: round(buf[i] / per) for i, n in enumerate(NAMES) if n != "-"}
    out["total"] = sum(out[n] for n in NAMES[:7])
    print(json.dumps({"model": args.model, "geometry": "learned" if args.learned else "exact", "envs": E,
                      "substeps_per_call": sub, "calls": args.calls,
                      "launch": dict(zip(("envs_per_block", "stage_points", "warps_per_env"), args.shape)),
                      "cycles_per_env_substep": out}))


if __name__ == "__main__":
    main()
