"""Benchmark of the batched muscle-driven forward-dynamics step (one JSON line on stdout).

Default workload: the whole-body synthetic model (60 bodies, 90 hinge DoFs, 700 Hill muscles,
8 foot contact spheres), 4096 environments; one bench step = one msim_step call of 10 substeps
of dt = 1 ms (the paper's 10 simulation substeps per control step), smooth random excitations.
Metric: env-steps/s = environments x substeps / device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank steps its own 4096 environments (weak scaling, no data-path
collective); the max over ranks of the timed region is used.  `--impl reference` times the
FP64 CPU oracle on the host cores instead (rank 0 only).

Beside the exact path, the default run (rank 0, N = 1) trains the learned-geometry surrogate
(2M configurations, 50 epochs) and times the same rollout with it ("surrogate" in the line).
Two more workloads print their own line:
  --workload c2_mixed   three skeletons in one handle (8192 envs, 10 x 0.5 ms substeps per call,
                        captured in a CUDA graph): per-model launches vs the autotuned mixed launch;
  --workload c4_policy  16384 whole-body envs with a policy MLP in the loop (one inference per
                        2 substeps, CUDA graphs), exact vs learned geometry;
  --workload c3_mlp     the surrogate network's forward pass alone (tensor-core GEMMs);
  --workload c3_width   the learned geometry's accuracy and cost against the network width.
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


def max_over_ranks(value, world, device="cpu"):
    """The largest value over the ranks (a timed region's duration); the value itself on one rank.
    Environments are independent, so this is the only collective of a multi-GPU run."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(envs_per_rank, substeps, steps, world, seconds):
    """Whole-job env-steps/s: every rank steps its own environments (weak scaling)."""
    return world * envs_per_rank * substeps * steps / seconds


def measured_traffic(envs, workload):
    """(DRAM bytes per step launch, kernel) of a workload from the committed ncu summaries, or
    (None, None) if it has none or the kernel sources changed since those counters were taken.
    The capture ran 2 substeps; the figure is scaled by environments only (a workload whose
    state is read and written every substep, the tendon strains, moves a little more at 10)."""
    try:
        from paper_2603_29332_b300 import build
        d = json.load(open(os.path.join(ROOT, "profiles", "k_step_traffic.json")))
        w = d["workloads"].get(workload)
        if w is None or d.get("source_digest") != build.step_digest():
            return None, None
        return w["dram_bytes_per_env_per_launch"] * envs, w["kernel"]
    except Exception:
        return None, None


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
    out = {"value": envs * substeps / dt, "unit": UNIT, "cores": ora.max_threads(), "kind": "oracle",
           "sample": "%d envs x %d substeps of the whole-body model, FP64, OpenMP over envs, %.1f s" %
                     (envs, substeps, dt)}
    # the tiny model on all cores, then one core (bounded samples)
    tiny = mg.config_model("c0_tiny")
    ot = ora.OracleModel(tiny)
    qt, qdt, at = mg.initial_state(tiny, 64, seed=0)
    ut = mg.uniform_excitations(tiny, 64, 1, seed=0)[0]
    t0 = time.perf_counter()
    ora.step(ot, DT, qt, qdt, at, ut, 100, n_threads=ora.max_threads())
    d2 = time.perf_counter() - t0
    out["c0_tiny"] = {"value": 64 * 100 / d2, "cores": ora.max_threads(),
                      "sample": "64 envs x 100 substeps of the 14-DoF model, %.2f s" % d2}
    e1, s1 = 16, 20
    t0 = time.perf_counter()
    ora.step(om, DT, q0[:e1], qd0[:e1], a0[:e1], exc[:e1], s1, n_threads=1)
    d1 = time.perf_counter() - t0
    out["one_core"] = {"value": e1 * s1 / d1, "cores": 1, "sample": "%d envs x %d substeps, %.1f s" % (e1, s1, d1)}
    return out


def bench_model(name, rest_lengths=None):
    """The workload's model.  c1_tendon: the whole body with compliant tendons on every muscle
    whose slack length (its length at q = 0 less l_opt) is at least 0.6 l_opt; the rest lengths
    come from the caller (the library's device geometry on the GPU arm, the oracle on the CPU
    arm)."""
    if name != "c1_tendon":
        return mg.config_model(name)
    return mg.with_tendons(mg.config_model(MODEL), rest_lengths, seed=1)


def _device_rest_lengths(device):
    import torch
    from paper_2603_29332_b300 import msim
    base = mg.config_model(MODEL)
    sim = msim.Sim([base], [1], dt=DT, device=device)
    L0 = sim.geometry(torch.zeros((1, sim.pitch_n), device=sim.device))[0, :base.n_muscles].double().cpu().numpy()
    sim.close()
    return L0


def run_reference(args, rank):
    if rank != 0:
        return None
    from oracle import oracle as ora
    model = bench_model(args.model, ora.OracleModel(mg.config_model(MODEL)).L0 if args.model == "c1_tendon" else None)
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
            "config": _config(args, model),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d envs x %d substeps per step (bounded sample of %d envs)" %
                                       (envs, sub, args.envs)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _config(args, model):
    wrap = {"c1_wrap": ", 188 of them wrapping a cylinder",
            "c1_wrap_mix": ", 188 of them wrapping a cylinder (92) or a sphere (96)",
            "c1_tendon": ", %d of them with compliant tendons" % int((model.muscle_tendon_strain > 0).sum())
            }.get(args.model, "")
    dofs = "a free root (6 DoF) and 89 hinge DoF" if args.model == "c1_float" else "90 hinge DoF"
    return {"workload": "whole-body synthetic model (60 bodies, %s, 700 Hill muscles%s, 8 contact "
                        "spheres), %d envs, %d substeps x dt %.0e s per step, smooth excitations, exact geometry"
                        % (dofs, wrap, args.envs, args.substeps, DT),
            "envs_per_gpu": args.envs, "substeps_per_step": args.substeps, "dt": DT, "geometry": "exact",
            "l2": "flushed (256 MB write) between timed steps; excitation inputs cycle over 32 distinct buffers"}


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2603_29332_b300 import msim
    torch.cuda.set_device(local_rank)
    model = bench_model(args.model, _device_rest_lengths(local_rank) if args.model == "c1_tendon" else None)
    E, sub = args.envs, args.substeps
    sim = msim.Sim([model], [E], dt=DT, device=local_rank)
    q0, qd0, a0 = mg.initial_state(model, E, seed=1 + rank)
    n_buf = 32
    excs_h = mg.smooth_excitations(model, E, n_buf, seed=1 + rank, dt=DT * sub)
    excs = [sim.pad_m(excs_h[t]) for t in range(n_buf)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    tune = sim.autotune(None, n_sub=sub) if args.autotune else None   # launch shape (state restored)
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
    total_ms = max_over_ranks(sum(ms), world, "cuda")
    st, flags = sim.status()
    # end-to-end through the C ABI with host buffers: H2D excitations, step, D2H q and qd
    k_e2e = min(args.steps, 20)
    pinned = [torch.from_numpy(np.ascontiguousarray(np.pad(excs_h[t], ((0, 0), (0, sim.pitch_m - model.n_muscles)))))
              .pin_memory() for t in range(min(k_e2e, n_buf))]
    q_out = torch.empty((E, sim.pitch_n), dtype=torch.float32).pin_memory()
    qd_out = torch.empty((E, sim.pitch_n), dtype=torch.float32).pin_memory()
    sim.step_host(pinned[0], sub, q_out, qd_out)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for t in range(k_e2e):
        sim.step_host(pinned[t % len(pinned)], sub, q_out, qd_out)
    sync_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    # pipelined: every step still uploads its excitations and downloads q and qd, on the handle's
    # copy streams, overlapping the neighbouring steps
    sim.step_host_async(pinned[0], sub, q_out, qd_out)
    sim.host_wait()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for t in range(k_e2e):
        sim.step_host_async(pinned[t % len(pinned)], sub, q_out, qd_out)
    sim.host_wait()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e = {"value": job_rate(E, sub, k_e2e, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": E * sim.pitch_m * 4, "d2h_bytes_per_step": 2 * E * sim.pitch_n * 4,
           "api": "msim_step_host_async x %d, then msim_host_wait (pinned host buffers)" % k_e2e,
           "synchronous": {"value": job_rate(E, sub, k_e2e, world, sync_s), "api": "msim_step_host"}}
    if rank != 0:
        return None
    value = job_rate(E, sub, args.steps, world, total_ms * 1e-3)
    fl = FL.flops_per_env_substep(model)["total"]
    launch_ms = total_ms / args.steps
    achieved = fl * E * sub / (launch_ms * 1e-3) / 1e12
    clocks = clk.summary()
    peak_max = fp32_peak_tflops(2032.0)
    tr, tr_kernel = measured_traffic(E, args.model)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_max, "unit": "TFLOP/s", "frac": achieved / peak_max,
            "traffic": tr, "traffic_unit": "bytes per launch (ncu dram read + write)",
            "kernel": (tr_kernel or "k_step") + " (one launch per bench step)",
            "flops_per_env_substep": fl,
            "peak_note": "FP32 FMA peak 148 SMs x 128 lanes x 2 x 2032 MHz (no FP32 figure in MEASURED_PEAKS.json)"}
    if clocks:
        roof["frac_at_sampled_clock"] = achieved / fp32_peak_tflops(clocks["sm_mhz"])
    try:   # our own FMA microbenchmark on this GPU, beside the derived figure
        pk_meas = msim.measure_fp32_peak(local_rank)
        roof["peak_fma_microbenchmark"] = pk_meas
        roof["frac_of_fma_microbenchmark"] = achieved / pk_meas
    except Exception:
        pass
    # algorithmic HBM bytes per launch: read exc, act, q, qd; write act, force, v_m, q, qd, q_dd;
    # compliant tendons: read and write their strains
    alg = 4 * E * (5 * model.n_muscles + 5 * model.n_dofs) + 8 * E * int((model.muscle_tendon_strain > 0).sum())
    pk_hbm = _peaks().get("hbm_gbs", 6400.0)
    roof["hbm_algorithmic"] = {"bytes_per_launch": alg, "achieved_gbs": alg / (launch_ms * 1e-3) / 1e9,
                               "peak_gbs": pk_hbm, "frac": alg / (launch_ms * 1e-3) / 1e9 / pk_hbm,
                               "peak_note": "hbm_gbs of measured"}
    if tr:
        roof["hbm"] = {"achieved_gbs": tr / (launch_ms * 1e-3) / 1e9, "peak_gbs": _peaks().get("hbm_gbs", 6400.0),
                       "frac": tr / (launch_ms * 1e-3) / 1e9 / _peaks().get("hbm_gbs", 6400.0),
                       "peak_note": "hbm_gbs of measured"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": launch_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(args, model),
           "roofline": roof, "e2e": e2e, "gpu_launches": args.steps, "clocks": clocks,
           "launch_shape": {"warps_per_env": sim.dims.warps_per_env[0], "envs_per_block": sim.dims.envs_per_block[0],
                            "points_in_smem": sim.dims.points_in_smem[0],
                            "autotuned": tune is not None},
           "status_flags": flags,
           "precision_note": "FP32 throughout except the mass-matrix entries and their L^T L factorisation, "
                             "which use float-float pairs on the FP32 pipes"}
    if args.surrogate and world == 1:
        # the network that meets the stated error (1 mm), then the configured 512-wide one
        out["surrogate"] = run_surrogate(args, sim, model, excs, flush, value, args.surr_hidden)
        if args.surr_hidden != 512:
            out["surrogate_configured_width"] = run_surrogate(args, sim, model, excs, flush, value, 512)
    if args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(model)
    return out


def _mlp_flops(sizes):
    return sum(2 * a * b for a, b in zip(sizes[:-1], sizes[1:]))


def run_surrogate(args, sim, model, excs, flush, exact_value, hidden=512):
    """Same rollout with the learned geometry: train, then time K steps twice, as configured (1 %
    checks, fallback per environment) and with the checks off (every environment inside the box
    on the network: the learned path's own throughput).

    Reports the network's accuracy on fresh configurations of the training box (per entry and
    per environment, the check's measure), the fractions of environment-substeps that used the
    network / fell outside the box / were flagged / were checked, the q drift of each learned
    rollout from the exact rollout of the same initial state and excitations, and the network's
    forward pass alone against the tensor-core peak."""
    import torch
    E, sub = args.envs, args.substeps
    n_buf = len(excs)
    sim.surrogate_set_width(hidden)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.train_surrogate(args.surr_samples, args.surr_epochs, batch=4096, lr=args.surr_lr)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # accuracy on fresh configurations in the training box
    lo, hi = model.dof_limit[:, 0].astype(np.float64), model.dof_limit[:, 1].astype(np.float64)
    c, hw = 0.5 * (lo + hi), 0.5 * (hi - lo) * 1.05
    rng = np.random.default_rng(99)
    qs = (c + hw * rng.uniform(-1, 1, (4096, model.n_dofs))).astype(np.float32)
    qg = torch.zeros((4096, sim.pitch_n), device="cuda")
    qg[:, : model.n_dofs] = torch.from_numpy(qs).cuda()
    err = (sim.surrogate_predict(qg) - sim.geometry(qg)).abs()
    m = model.n_muscles
    eR = err[:, m:].flatten()[::5].float()
    eL = err[:, :m].flatten().float()
    env_err = torch.maximum(err[:, m:].pow(2).mean(1).sqrt(), err[:, :m].pow(2).mean(1).sqrt())
    q0, qd0, a0 = mg.initial_state(model, E, seed=1)

    def rollout(mode, check_frac):
        sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
        sim.set_geometry_mode(mode)
        if mode == 1:
            sim.surrogate_set_check(check_frac, 1e-3)
        for t in range(args.warmup):
            sim.step(excs[t % n_buf], sub)
        torch.cuda.synchronize()
        sim.surrogate_stats(reset=True)
        stream = torch.cuda.current_stream()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for t in range(args.steps):
            flush.fill_(float(t))
            starts[t].record(stream)
            sim.step(excs[(args.warmup + t) % n_buf], sub)
            ends[t].record(stream)
        torch.cuda.synchronize()
        ms = float(sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)))
        st = sim.surrogate_stats()
        _, flags = sim.status()
        state = sim.state()
        sim.surrogate_set_check(0.01, 1e-3)
        return ms, st, flags, state["q"][:, : model.n_dofs].clone(), int((state["status"] & 1).count_nonzero())

    _, _, _, q_exact, _ = rollout(0, 0.0)
    runs = {}
    for name, frac in (("checked", 0.01), ("unchecked", 0.0)):
        ms, st, flags, q_l, nonfinite = rollout(1, frac)
        n = max(st["env_substeps"], 1)
        value = E * sub * args.steps / (ms * 1e-3)
        dq = (q_l - q_exact).abs().max(1).values
        runs[name] = {"value": value, "ms_per_step": ms / args.steps, "vs_exact": value / exact_value,
                      "check_fraction": frac, "fraction_learned": st["learned"] / n,
                      "fraction_out_of_box": st["out_of_box"] / n, "fraction_flagged": st["flagged"] / n,
                      "fraction_checked": st["checked"] / n, "checks": st["checked"],
                      "checks_failed": st["check_failed"],
                      "checks_failed_fraction": st["check_failed"] / max(st["checked"], 1),
                      "max_check_error_m": st["max_check_error"], "flagged_envs_at_end": st["flagged_envs"],
                      "q_vs_exact_rollout_rad": {"median": float(dq.median()), "max": float(dq.max()),
                                                 "after_substeps": (args.warmup + args.steps) * sub},
                      "envs_non_finite": nonfinite, "status_flags": flags}
    # q_dd of one learned substep against the exact geometry's (which matches the FP64 oracle
    # within 1e-4) at the same states: the end of the last rollout
    n = model.n_dofs
    s0 = sim.state()
    exc_n = excs[(args.warmup + args.steps) % n_buf]
    sim.set_geometry_mode(0)
    qdd_ex = sim.eval(s0["q"], s0["qd"], s0["act"], exc_n)["qdd"][:, :n].double()
    sim.reset(s0["q"], s0["qd"], s0["act"])
    sim.set_geometry_mode(1)
    sim.surrogate_set_check(0.0, 1e-3)
    sim.surrogate_stats(reset=True)
    sim.step(exc_n, 1)
    qdd_l = sim.state()["qdd"][:, :n].double()
    learned_here = sim.surrogate_stats()["learned"] / E
    sim.surrogate_set_check(0.01, 1e-3)
    rel = (qdd_l - qdd_ex).norm(dim=1) / qdd_ex.norm(dim=1).clamp_min(1e-3)
    qdd_err = {"median": float(rel.median()), "p90": float(rel.quantile(0.9)), "max": float(rel.max()),
               "fraction_on_network": learned_here,
               "definition": "|q_dd learned - q_dd exact| / max(|q_dd exact|, 1e-3) per env, one substep from "
                             "the rollout's final states; the exact path matches the FP64 oracle within 1e-4"}
    sim.set_geometry_mode(0)
    # the network alone at this batch, for its tensor-pipe fraction (timed alone: burst peak)
    net = sim.surrogate_network()
    X = torch.zeros((E, net.in_pitch), dtype=torch.bfloat16, device="cuda")
    Y = torch.empty((E, net.out_pitch), device="cuda")
    for _ in range(3):
        net.forward(X, Y)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(20):
        net.forward(X, Y)
    e1.record(stream)
    torch.cuda.synchronize()
    mlp_ms = e0.elapsed_time(e1) / 20
    mlp_tf = _mlp_flops([model.n_dofs, net.hidden, net.hidden, net.d_out]) * E / (mlp_ms * 1e-3) / 1e12
    pk = _peaks().get("bf16_tflops") or 1800.0
    q = lambda x, p: float(x.quantile(p))
    ck = runs["checked"]
    out = {"value": ck["value"], "unit": UNIT, "ms_per_step": ck["ms_per_step"], "vs_exact": ck["vs_exact"],
           "label": ("learned geometry" if ck["fraction_learned"] >= 0.5 else
                     "mostly exact geometry (fallback) plus the network (fraction_learned below 0.5)"),
           "hidden": hidden, "train_s": train_s, "train_samples": args.surr_samples,
           "train_epochs": args.surr_epochs, "train_loss_normalised_mse": sim.surrogate_stats()["train_loss"],
           "moment_arm_abs_err_m": {"median": q(eR, 0.5), "p99": q(eR, 0.99), "p999": q(eR, 0.999),
                                    "max": float(err[:, m:].max())},
           "length_abs_err_m": {"median": q(eL[::3], 0.5), "p99": q(eL[::3], 0.99), "max": float(err[:, :m].max())},
           "env_check_error_m": {"median": q(env_err, 0.5), "p99": q(env_err, 0.99),
                                 "fraction_within_tol": float((env_err <= 1e-3).float().mean()),
                                 "definition": "max(rms of the env's moment-arm errors, rms of its length errors)"},
           "rollouts": runs, "qdd_rel_err_vs_exact": qdd_err,
           "mlp_forward": {"ms": mlp_ms, "tflops": mlp_tf, "peak_tflops": pk, "frac": mlp_tf / pk,
                           "peak_note": "bf16_tflops (burst) of measured: the forward is timed alone"},
           "network": "90 -> %d -> %d -> %d, SiLU, BF16, joint-block connectivity" % (net.hidden, net.hidden,
                                                                                    net.d_out),
           "box": "joint limits widened by 5 % of each range",
           "check": "1 % of envs per substep; fallback when the env's check error exceeds 1 mm"}
    return out


def run_substep(args):
    """The learned-geometry substep against the exact one, per substep (for launch lists): the
    whole body, a briefly trained network (8192 configurations, 1 epoch: its accuracy is not the
    point), the exact step of 2 substeps, then K learned substeps with the checks off."""
    import torch
    from paper_2603_29332_b300 import msim
    model = mg.config_model(MODEL)
    E = args.envs
    sim = msim.Sim(model, E, dt=DT, seed=3)
    sim.surrogate_set_width(args.surr_hidden)
    sim.train_surrogate(8192, 1, batch=4096, lr=args.surr_lr)
    q0, qd0, a0 = mg.initial_state(model, E, seed=1)
    exc = sim.pad_m(mg.smooth_excitations(model, E, 1, seed=1, dt=DT * 10)[0])
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    cur = torch.cuda.current_stream()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(cur)
    sim.step(exc, 2)
    e1.record(cur)
    sim.set_geometry_mode(1)
    sim.surrogate_set_check(0.0, 1e-3)
    for _ in range(args.steps):
        sim.step(exc, 1)
    e2.record(cur)
    torch.cuda.synchronize()
    sim.set_geometry_mode(0)
    exact_us, learned_us = e0.elapsed_time(e1) * 1e3 / 2, e1.elapsed_time(e2) * 1e3 / args.steps
    return {"metric": "us per substep, learned geometry (width %d, checks off) vs exact, whole body x %d envs"
                      % (args.surr_hidden, E), "value": learned_us, "unit": "us per substep",
            "exact_us_per_substep": exact_us, "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
            "data": "synthetic"}


def run_mlp(args):
    """The surrogate network's forward pass alone (90 -> 512 -> 512 -> m + nnz, random init) at
    the whole-body batch: the tensor-core kernels of the learned geometry, for profiling."""
    import torch
    from paper_2603_29332_b300 import msim
    model = mg.config_model(MODEL)
    sim = msim.Sim(model, 8, dt=DT)
    E = args.envs
    net = msim.MLP(model.n_dofs, 512, model.n_muscles + sim.dims.nnz[0], max_batch=E, seed=3)
    X = net.pad_input(np.random.default_rng(3).uniform(-1, 1, (E, model.n_dofs)))
    Y = torch.empty((E, net.out_pitch), device="cuda")
    for _ in range(args.warmup):
        net.forward(X, Y)
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for _ in range(args.steps):
        net.forward(X, Y)
    e1.record(cur)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    fl = _mlp_flops([model.n_dofs, 512, 512, net.d_out]) * E
    pk = _peaks().get("bf16_tflops") or 1800.0
    return {"metric": "MLP forward TFLOP/s (surrogate network, batch %d)" % E, "value": fl / (ms * 1e-3) / 1e12,
            "unit": "TFLOP/s", "ms_per_step": ms, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "roofline": {"bound": "tensor", "achieved": fl / (ms * 1e-3) / 1e12, "peak": pk,
                         "unit": "TFLOP/s", "frac": fl / (ms * 1e-3) / 1e12 / pk,
                         "peak_note": "bf16_tflops (burst) of measured"}}


def run_width(args):
    """Learned geometry against the hidden width (2M samples, 50 epochs each, training box =
    limits + 5 %, joint-block connectivity): accuracy on fresh configurations of the box, network
    cost, and the whole-body rollout with the learned geometry (checked as configured, and with
    the checks off) beside the exact rollout."""
    import torch
    from paper_2603_29332_b300 import msim
    model = mg.config_model(MODEL)
    E, sub = args.envs, args.substeps
    sim = msim.Sim(model, E, dt=DT, seed=3)
    n_buf = 32
    excs = [sim.pad_m(x) for x in mg.smooth_excitations(model, E, n_buf, seed=1, dt=DT * sub)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    q0, qd0, a0 = mg.initial_state(model, E, seed=1)
    sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
    for t in range(args.warmup):
        sim.step(excs[t % n_buf], sub)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(args.steps):
        sim.step(excs[(args.warmup + t) % n_buf], sub)
    e1.record()
    torch.cuda.synchronize()
    exact_value = E * sub * args.steps / (e0.elapsed_time(e1) * 1e-3)
    rows = [run_surrogate(args, sim, model, excs, flush, exact_value, hidden) for hidden in args.widths]
    return {"metric": "learned geometry vs hidden width (whole body, %d samples x %d epochs, %d envs)"
                      % (args.surr_samples, args.surr_epochs, E),
            "value": rows[0]["moment_arm_abs_err_m"]["p99"], "unit": "m (p99 moment-arm error, first width)",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "exact_value": exact_value,
            "widths": rows}


def run_mixed(args):
    """Three skeletons in one handle: per-model launches vs the autotuned mixed launch (graphs)."""
    import torch
    from paper_2603_29332_b300 import msim
    names = ("c2_upper", "c2_lower", "c1_whole")
    counts = (2458, 2458, 3276)
    dt, sub = 5e-4, 10
    models = [mg.config_model(nm) for nm in names]
    sim = msim.Sim(models, list(counts), dt=dt)
    qs, qds, acts, ex = [], [], [], []
    for i, (mdl, E) in enumerate(zip(models, counts)):
        q, qd, a = mg.initial_state(mdl, E, seed=2 + i)
        qs.append(sim._pad(q, sim.pitch_n)); qds.append(sim._pad(qd, sim.pitch_n)); acts.append(sim._pad(a, sim.pitch_m))
        ex.append(sim._pad(mg.smooth_excitations(mdl, E, 1, seed=2 + i)[0], sim.pitch_m))
    q0, qd0, a0, exc = torch.cat(qs), torch.cat(qds), torch.cat(acts), torch.cat(ex)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()

    def timed(label):
        sim.reset(q0, qd0, a0)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            sim.step(exc, sub)
        torch.cuda.synchronize()
        sim.reset(q0, qd0, a0)
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        cur = torch.cuda.current_stream()
        for t in range(args.steps):
            flush.fill_(float(t))
            starts[t].record(cur)
            g.replay()
            ends[t].record(cur)
        torch.cuda.synchronize()
        ms = float(sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))) / args.steps
        return sum(counts) * sub / (ms * 1e-3), ms

    base_value, base_ms = timed("per-model default")
    if args.autotune:
        tune = sim.autotune(None, n_sub=sub)
    else:   # the shape the autotuner picks for this batch on a B300 (for short profiling runs)
        tune = {"mixed_warps_per_env": 2, "mixed_slots": 8, "mixed_stage_points_mask": 0x700, "candidates": 0}
    sim.set_mixed_launch(False)
    permodel_value, permodel_ms = timed("per-model tuned")
    sim.set_mixed_launch(True, tune["mixed_warps_per_env"], tune["mixed_slots"], tune["mixed_stage_points_mask"])
    with ClockSampler(0) as clk:
        mixed_value, mixed_ms = timed("mixed tuned")
    st, flags = sim.status()
    return {"metric": "env-steps/s, mixed batch of 3 skeletons x 8192 envs, one persistent launch",
            "value": mixed_value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": mixed_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "2458 upper-body (30 DoF, 250 muscles) + 2458 lower-limb (40 DoF, 300 muscles, "
                                   "contact) + 3276 whole-body envs; 10 substeps x 0.5 ms per CUDA-graph replay",
                       "l2": "flushed (256 MB write) between timed replays"},
            "per_model_launches": {"default_shapes": base_value, "tuned_shapes": permodel_value,
                                   "tuned_ms_per_step": permodel_ms},
            "mixed_vs_per_model_tuned": mixed_value / permodel_value, "autotune": tune,
            "clocks": clk.summary(), "status_flags": flags}


def run_policy(args):
    """16384 whole-body envs with a policy MLP in the loop, exact vs learned geometry (graphs)."""
    import torch
    from paper_2603_29332_b300 import msim
    model = mg.config_model(MODEL)
    E, per_act, acts_per_graph = args.policy_envs, 2, 50
    sim = msim.Sim(model, E, dt=DT, seed=4)
    pol = msim.MLP(2182, 1024, model.n_muscles, out_sigmoid=True, max_batch=E, seed=4)
    sim.policy_attach(pol)
    q0, qd0, a0 = mg.initial_state(model, E, seed=4)
    stream = torch.cuda.Stream()
    res = {}
    flow = None
    for mode in ("exact", "exact_flow", "learned"):
        if mode == "exact_flow":
            # flow refinement of the action: 20 Euler steps of a 2883 -> 1024 -> 1024 -> 700 network
            flow = msim.MLP(2182 + model.n_muscles + 1, 1024, model.n_muscles, max_batch=E, seed=5)
            sim.flow_attach(flow, n_steps=20, dt=0.05, sigma=0.05)
        if mode == "learned":
            sim.flow_attach(None)
            sim.train_surrogate(args.surr_samples, args.surr_epochs, batch=4096, lr=args.surr_lr)
            sim.set_geometry_mode(1)
        sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            sim.policy_step(per_act, acts_per_graph)
        torch.cuda.synchronize()
        sim.reset(sim.pad_n(q0), sim.pad_n(qd0), sim.pad_m(a0))
        g.replay()
        torch.cuda.synchronize()
        replays = max(1, args.policy_steps // (per_act * acts_per_graph))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream()
        e0.record(cur)
        for _ in range(replays):
            g.replay()
        e1.record(cur)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        steps = replays * per_act * acts_per_graph
        est = sim.state()["status"]
        res[mode] = {"value": E * steps / (ms * 1e-3), "ms_per_substep": ms / steps, "steps": steps,
                     "status": sim.status(), "envs_non_finite": int((est & 1).count_nonzero()),
                     "envs_not_spd": int((est & 2).count_nonzero())}
        if mode == "learned":
            res[mode]["surrogate_stats"] = sim.surrogate_stats()
    return {"metric": "env-steps/s, closed loop with policy MLP, whole body x %d envs" % E,
            "value": res["exact"]["value"], "unit": UNIT, "n_gpus": 1, "steps": res["exact"]["steps"],
            "warmup": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
            "data": "synthetic, random-init policy",
            "config": {"workload": "whole body, %d envs, policy 2182 -> 1024 -> 1024 -> 700 sigmoid every 2 "
                                   "substeps of 1 ms, %d acts per CUDA graph" % (E, acts_per_graph)},
            "exact": res["exact"], "learned_geometry": res["learned"],
            "learned_vs_exact": res["learned"]["value"] / res["exact"]["value"],
            "exact_with_flow_refinement": res["exact_flow"],
            "flow_note": "initial sampler + 20 Euler steps (dt 0.05) of a 3-layer 1024 flow network per control step"}


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
    ap.add_argument("--no-surrogate", dest="surrogate", action="store_false")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--surr-samples", type=int, default=2097152)
    ap.add_argument("--surr-epochs", type=int, default=50)
    ap.add_argument("--widths", type=int, nargs="+", default=[512, 1024, 2048])
    ap.add_argument("--surr-lr", type=float, default=6e-3)
    ap.add_argument("--surr-hidden", type=int, default=2048)
    ap.add_argument("--workload", default="c1_exact", choices=["c1_exact", "c2_mixed", "c4_policy", "c3_mlp", "c3_width", "c3_substep"])
    ap.add_argument("--model", default=MODEL, choices=[MODEL, "c1_wrap", "c1_wrap_mix", "c1_float", "c1_tendon"],
                    help="model of the c1_exact workload (c1_wrap: a quarter of the muscles wrap a cylinder; "
                         "c1_float: a free root; c1_tendon: compliant tendons)")
    ap.add_argument("--policy-envs", type=int, default=16384)
    ap.add_argument("--policy-steps", type=int, default=2000)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
    elif args.workload == "c2_mixed":
        out = run_mixed(args)
    elif args.workload == "c4_policy":
        out = run_policy(args)
    elif args.workload == "c3_mlp":
        out = run_mlp(args)
    elif args.workload == "c3_substep":
        out = run_substep(args)
    elif args.workload == "c3_width":
        out = run_width(args)
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
