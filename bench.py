"""Benchmark of the batched muscle-driven forward-dynamics step (one JSON line on stdout).

Default workload: the whole-body synthetic model (60 bodies, 90 hinge DoFs, 700 Hill muscles,
8 foot contact spheres), 4096 environments; one bench step = one msim_step call of 10 substeps
of dt = 1 ms (the paper's 10 simulation substeps per control step), smooth random excitations.
Metric: env-steps/s = environments x substeps / device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank steps its own 4096 environments (weak scaling, no data-path
collective); the max over ranks of the timed region is used.  `--impl reference` times the
FP64 CPU oracle on the host cores instead (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_29332_b300 import flops as FL  # noqa: E402
from paper_2603_29332_b300 import modelgen as mg  # noqa: E402

METRIC = "env-steps/s, 700-muscle body x4096 envs: exact vs surrogate at stated error"
UNIT = "env-steps/s"
MODEL = "c1_whole"
DT = 1e-3


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp32_peak_tflops(sm_mhz, n_sm=148):
    """FP32 FMA peak: SMs x 128 lanes x 2 FLOP x clock."""
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_traffic(envs):
    """DRAM bytes per step launch from the committed ncu summary, or None if the kernel sources
    changed since those counters were taken."""
    try:
        from paper_2603_29332_b300 import build
        d = json.load(open(os.path.join(ROOT, "profiles", "k_step_traffic.json")))
        if d.get("source_digest") != build._digest():
            return None
        return d["dram_bytes_per_env_per_launch"] * envs
    except Exception:
        return None


def cpu_baseline(model, envs=512, substeps=20):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the workload."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as ora
    om = ora.OracleModel(model)
    q0, qd0, a0 = mg.initial_state(model, envs, seed=1)
    exc = mg.smooth_excitations(model, envs, 1, seed=1)[0]
    t0 = time.perf_counter()
    ora.step(om, DT, q0, qd0, a0, exc, substeps)
    dt = time.perf_counter() - t0
    return {"value": envs * substeps / dt, "unit": UNIT, "cores": ora.max_threads(), "kind": "oracle",
            "sample": "%d envs x %d substeps of the whole-body model, FP64, OpenMP over envs, %.1f s" %
                      (envs, substeps, dt)}


def run_reference(args, rank):
    if rank != 0:
        return None
    model = mg.config_model(MODEL)
    from oracle import oracle as ora
    om = ora.OracleModel(model)
    envs, sub = args.ref_envs, args.substeps
    q0, qd0, a0 = mg.initial_state(model, envs, seed=1)
    excs = mg.smooth_excitations(model, envs, args.steps + args.warmup, seed=1, dt=DT * sub)
    q, qd, act = q0, qd0, a0
    for t in range(args.warmup):
        q, qd, act, *_ = ora.step(om, DT, q, qd, act, excs[t], sub)
    t0 = time.perf_counter()
    for t in range(args.steps):
        q, qd, act, *_ = ora.step(om, DT, q, qd, act, excs[args.warmup + t], sub)
    el = time.perf_counter() - t0
    value = envs * sub * args.steps / el
    cores = ora.max_threads()
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d envs x %d substeps per step (bounded sample of %d envs)" %
                                       (envs, sub, args.envs)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _config(args):
    return {"workload": "whole-body synthetic model (60 bodies, 90 hinge DoF, 700 Hill muscles, 8 contact "
                        "spheres), %d envs, %d substeps x dt %.0e s per step, smooth excitations, exact geometry"
                        % (args.envs, args.substeps, DT),
            "envs_per_gpu": args.envs, "substeps_per_step": args.substeps, "dt": DT, "geometry": "exact",
            "l2": "flushed (256 MB write) between timed steps; excitation inputs cycle over 32 distinct buffers"}


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2603_29332_b300 import msim
    torch.cuda.set_device(local_rank)
    model = mg.config_model(MODEL)
    E, sub = args.envs, args.substeps
    sim = msim.Sim([model], [E], dt=DT, device=local_rank)
    q0, qd0, a0 = mg.initial_state(model, E, seed=1 + rank)
    n_buf = 32
    excs_h = mg.smooth_excitations(model, E, n_buf, seed=1 + rank, dt=DT * sub)
    excs = [sim.pad_m(excs_h[t]) for t in range(n_buf)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    stream = torch.cuda.current_stream()
    for t in range(args.warmup):
        sim.step(excs[t % n_buf], sub)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for t in range(args.steps):
            flush.fill_(float(t))                       # evict L2 between timed steps
            starts[t].record(stream)
            sim.step(excs[(args.warmup + t) % n_buf], sub)
            ends[t].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(ms))
    if world > 1:
        tt = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    st, flags = sim.status()
    # end-to-end through the C ABI with host buffers: H2D excitations, step, D2H q and qd
    k_e2e = min(args.steps, 20)
    pinned = [torch.from_numpy(np.ascontiguousarray(np.pad(excs_h[t], ((0, 0), (0, sim.pitch_m - model.n_muscles)))))
              .pin_memory() for t in range(min(k_e2e, n_buf))]
    q_out = torch.empty((E, sim.pitch_n), dtype=torch.float32).pin_memory()
    qd_out = torch.empty((E, sim.pitch_n), dtype=torch.float32).pin_memory()
    sim.step_host(pinned[0], sub, q_out, qd_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for t in range(k_e2e):
        sim.step_host(pinned[t % len(pinned)], sub, q_out, qd_out)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * E * sub * k_e2e / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": E * sim.pitch_m * 4, "d2h_bytes_per_step": 2 * E * sim.pitch_n * 4}
    if rank != 0:
        return None
    value = world * E * sub * args.steps / (total_ms * 1e-3)
    fl = FL.flops_per_env_substep(model)["total"]
    launch_ms = total_ms / args.steps
    achieved = fl * E * sub / (launch_ms * 1e-3) / 1e12
    clocks = clk.summary()
    peak_max = fp32_peak_tflops(2032.0)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_max, "unit": "TFLOP/s", "frac": achieved / peak_max,
            "traffic": measured_traffic(E), "traffic_unit": "bytes per launch (ncu dram read + write)",
            "kernel": "k_step (one launch per bench step)",
            "flops_per_env_substep": fl,
            "peak_note": "FP32 FMA peak 148 SMs x 128 lanes x 2 x 2032 MHz (no FP32 figure in MEASURED_PEAKS.json)"}
    if clocks:
        roof["frac_at_sampled_clock"] = achieved / fp32_peak_tflops(clocks["sm_mhz"])
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": launch_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(args),
           "roofline": roof, "e2e": e2e, "gpu_launches": args.steps, "clocks": clocks,
           "status_flags": flags,
           "precision_note": "FP32 throughout except the mass-matrix entries and their L^T L factorisation, "
                             "which use float-float pairs on the FP32 pipes"}
    if args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(model)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--substeps", type=int, default=10)
    ap.add_argument("--ref-envs", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        out = run_gpu(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
