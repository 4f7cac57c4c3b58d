"""Child process of tests/test_gpu_bounds.py: runs one library (argv[1]) over the models and modes
of the step kernel, writes the final states to argv[2] (npz) and prints one JSON line with the
bounds record of every case (a checking library) or nothing to record (the normal one).

Cases: the tiny model (eval, 20 substeps); the whole body (eval, 15 substeps, geometry labels,
body positions, launches of 1 and 4 warps per environment, learned-geometry substeps with every
environment checked and with none); the wrapped body with cylinders and spheres; the free root;
compliant tendons; the model at every size limit; three skeletons in one mixed launch.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

from paper_2603_29332_b300 import modelgen as mg  # noqa: E402
from paper_2603_29332_b300 import msim  # noqa: E402
from tests.test_gpu_limits import max_model  # noqa: E402

lib = msim.load_library(sys.argv[1])
checking = hasattr(lib, "msim_debug_bounds")
if checking:
    import ctypes
    lib.msim_debug_bounds.argtypes = [ctypes.c_void_p]
    lib.msim_debug_bounds.restype = ctypes.c_int
records, states = {}, {}


def record(name):
    if checking:
        rec = np.zeros(4, np.uint32)
        assert lib.msim_debug_bounds(rec.ctypes.data) == 0
        records[name] = [int(x) for x in rec]


def rand(model, E, seed):
    rng = np.random.default_rng(seed)
    q = rng.uniform(-0.3, 0.3, (E, model.n_dofs)).astype(np.float32)
    lo, hi = model.dof_limit[:, 0], model.dof_limit[:, 1]
    on = lo < hi
    q[:, on] = np.clip(q[:, on], lo[on], hi[on])
    if model.free_root:
        q[:, :6] = 0.0
    qd = rng.normal(0, 0.5, (E, model.n_dofs)).astype(np.float32)
    act = rng.uniform(0, 1, (E, model.n_muscles)).astype(np.float32)
    exc = rng.uniform(0, 1, (E, model.n_muscles)).astype(np.float32)
    return q, qd, act, exc


def run(name, model, E, n_sub, seed, extra=None):
    sim = msim.Sim(model, E, dt=1e-3, seed=3)
    q, qd, act, exc = rand(model, E, seed)
    sim.reset(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act))
    ev = sim.eval(sim.pad_n(q), sim.pad_n(qd), sim.pad_m(act), sim.pad_m(exc))
    states[name + "_eval_qdd"] = ev["qdd"][:, : model.n_dofs].cpu().numpy()
    for _ in range(n_sub // 5):
        sim.step(sim.pad_m(exc), 5)
    if extra:
        extra(sim, q, exc)
    st = sim.state()
    states[name + "_q"] = st["q"][:, : model.n_dofs].cpu().numpy()
    states[name + "_status"] = st["status"].cpu().numpy()
    record(name)
    sim.close()


def whole_extra(sim, q, exc):
    model = sim.models[0]
    qp = sim.pad_n(q)
    states["c1_geometry"] = sim.geometry(qp).cpu().numpy()
    states["c1_bodies"] = sim.body_positions(qp).cpu().numpy()
    for wpe in (1, 4):
        sim.set_launch(0, warps_per_env=wpe)
        sim.step(sim.pad_m(exc), 2)
    sim.set_launch(0)
    sim.train_surrogate(8192, 1, batch=4096, lr=3e-3)
    sim.set_geometry_mode(1)
    for frac in (1.0, 0.0):
        sim.surrogate_set_check(frac, 1e-3)
        sim.step(sim.pad_m(exc), 2)
    sim.set_geometry_mode(0)
    assert model.n_muscles == 700


run("c0_tiny", mg.config_model("c0_tiny"), 64, 20, 1)
run("c1_whole", mg.config_model("c1_whole"), 300, 15, 2, whole_extra)
run("c1_wrap_mix", mg.config_model("c1_wrap_mix"), 100, 10, 3)
run("c1_float", mg.config_model("c1_float"), 100, 10, 4)
base = mg.config_model("c1_whole")
probe = msim.Sim(base, 8, dt=1e-3)
L0 = probe.geometry(probe.pad_n(np.zeros((1, base.n_dofs), np.float32)))[0, : base.n_muscles].cpu().numpy()
probe.close()
run("c1_tendon", mg.with_tendons(base, L0), 100, 10, 5)
run("limits", max_model(), 4, 5, 6)
models = [mg.config_model("c2_upper"), mg.config_model("c2_lower"), mg.config_model("c1_whole")]
mix = msim.Sim(models, [90, 90, 120], dt=5e-4)
mix.set_mixed_launch(True)
rows = [rand(mm, e, 7 + i) for i, (mm, e) in enumerate(zip(models, (90, 90, 120)))]
mix.reset(torch.cat([mix.pad_n(r[0]) for r in rows]), torch.cat([mix.pad_n(r[1]) for r in rows]),
          torch.cat([mix.pad_m(r[2]) for r in rows]))
mix.step(torch.cat([mix.pad_m(r[3]) for r in rows]), 10)
states["mixed_q"] = mix.state()["q"].cpu().numpy()
record("mixed")
torch.cuda.synchronize()
np.savez(sys.argv[2], **states)
print(json.dumps({"checking": checking, "records": records}))
