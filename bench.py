#!/usr/bin/env python
"""Throughput of the MPS time step (particle-steps/s) on the 3D dam break.

Workload: 0.40 x 0.60 x 0.30 m water column in a 1.6 x 0.6 x 0.6 m open-top tank,
l0 = 0.0075 m, 2 wall + 2 dummy layers to full height: 169,600 fluid + 270,432 wall/dummy
= 440,032 particles; re_n = 2.1 l0, re_lap = 4 l0, dt = 5e-5 s, PPE by CG to a relative
FP64 residual of 1e-8, started from the quadratic extrapolation of the last three steps'
solutions (--cg-x0 3; the mixed step with the other starts, zero included, is reported
under "other_x0").  Synthetic seeded lattice with 1e-4 l0 jitter.

The headline `value` is the mixed-precision path (FP32 pair terms and inner CG, FP64 number
density, dot products and refinement); the plain FP64 path is timed on the same scene and
reported under "fp64", the equation-of-state pressure (Eq. 16) instead of the PPE under
"eos", and the mixed path with candidate lists kept for up to 4 steps
under "kept_lists" (exact neighbour sets either way); the two-phase 3D dam break (Sec. 3.2.1,
l0 = 0.004 m, 1,125,000 fluid particles) under "two_phase"; 256 independent 2D dam breaks
stepped together in one context under "ensemble"; the reverse step (vector-Jacobian
product, FP64) against the forward step on the 3D sloshing tank (85,564 particles) under
"adjoint".  `e2e` repeats the mixed measurement through the C ABI with host
buffers: every step uploads positions, velocities and kinds from pinned memory and reads
back positions, velocities and pressure (a written state starts its solve from zero).

--impl reference times the FP64 CPU oracle on the host cores on the same workload (one
oracle step per bench step).

Multi-GPU: a single scene does not shard (replicas only): each rank runs an independent
replica and `value` sums the particle-steps of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "particle-steps/s (3D ~200k dam break) FP64 vs mixed at PPE resid 1e-8; % HBM peak"
UNIT = "particle-steps/s"
# the PPE's initial guess (cg_x0); the stop rule is the same FP64 residual either way
X0_NAMES = {0: "zero", 1: "previous step's solution (before the clamp)",
            2: "linear extrapolation of the last 2 solutions",
            3: "quadratic extrapolation of the last 3 solutions",
            4: "cubic extrapolation of the last 4 solutions"}
WORKLOAD = "3D dam break, 0.40x0.60x0.30 m column in 1.6x0.6x0.6 m tank, l0=0.0075 m"

# Whole-step algorithmic bytes per particle (matrix-free minimum: every array read or
# written once per stage, neighbour re-reads served on chip): bucket 182, predict 97 (FP64)
# or 113 (mixed), density/flags/RHS 42, clamp + gradient 146; the PPE 113 per FP64 CG
# iteration, or 57 per FP32 inner iteration plus 65 per FP64 residual (mixed).
STEP_BYTES_FIXED = {0: 182.0 + 97.0 + 42.0 + 146.0, 1: 182.0 + 113.0 + 42.0 + 146.0}

# Method-level arithmetic of one pair evaluation (what the method computes per pair, in FP32
# flops, a fused multiply-add counting 2): the squared distance from the three coordinate
# differences (3 + 1 + 2 x 2 = 8), the weight w = re/r - 1 of Eq. 4 from the reciprocal
# square root (1 for the root, 1 multiply, 1 subtract = 3), and for a PPE coefficient
# c_ij = K w with its add into the diagonal (2): 13; for a number-density term its add into
# n* (1): 12.  A candidate distance test of the gather is the squared distance and one
# compare (9).  These are the units of the ALU roofline; the float-float arithmetic the
# mixed build actually issues per coefficient is far larger and reported beside it.
METHOD_FLOPS_PPE_PAIR = 13.0
METHOD_FLOPS_PND_PAIR = 12.0
METHOD_FLOPS_TEST = 9.0
# FP32 instructions the mixed build issues per unit (float-float terms): 8 per candidate-list
# entry classified at r*, 133 per PPE coefficient, 62 more per number-density term
ISSUED_FLOPS_LIST_TEST, ISSUED_FLOPS_PPE_PAIR, ISSUED_FLOPS_PND_PAIR = 8.0, 133.0, 62.0
# Stored-coefficient bytes of the build kernel (what the design must move): per PPE
# coefficient its column, FP32 value and float-float low part written (12 B); per candidate-
# list entry its slot read (4 B); per particle r* (hi and lo float4: 32 B) read and n*,
# flag, diagonal (FP64 and FP32), right-hand side and the two list counts written (37 B).
BUILD_BYTES_PER_COEF, BUILD_BYTES_PER_LIST_ENTRY, BUILD_BYTES_PER_PARTICLE = 12.0, 4.0, 69.0
# DRAM bytes (read + write) per PPE coefficient of one launch, from the ncu captures in
# profiles/kernels_dam_break_3d_227k_mixed.md (227,136-particle case, 25.19 M coefficients,
# rows grouped 8 entries per row, cell skin 0.05, 256-thread build): FP32 SpMV 208.7 + 3.8
# MB, build 163.4 + 290.1 MB, float-float residual 316.3 + 4.3 MB; the gather per
# candidate-list entry (31.09 M): 6.2 + 77.5 MB.  The rows and lists scale with the
# coefficients and entries.
SPMV_TRAFFIC_PER_COEF = (208.70e6 + 3.84e6) / 25.19e6
BUILD_TRAFFIC_PER_COEF = (163.36e6 + 290.07e6) / 25.19e6
RESID_TRAFFIC_PER_COEF = (316.26e6 + 4.28e6) / 25.19e6
GATHER_TRAFFIC_PER_ENTRY = (6.20e6 + 77.45e6) / 31.086e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200, help="timed steps (the workload runs 200)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed steps of the FP64 comparison (default: --steps)")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--cpu-sample-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--l0", type=float, default=0.0075, help="particle spacing (testing only)")
    ap.add_argument("--only", choices=["mixed", "fp64", "ensemble", "adjoint"], default=None,
                    help="time one precision only and print its stage profile (profiling runs)")
    ap.add_argument("--list-every", type=int, default=0,
                    help="with --only: keep candidate lists for up to this many steps")
    ap.add_argument("--kept-steps", type=int, default=None,
                    help="timed steps of the kept-list comparison (default: --steps)")
    ap.add_argument("--two-phase-steps", type=int, default=20,
                    help="timed steps of each two-phase path (0: skip)")
    ap.add_argument("--two-phase-l0", type=float, default=0.004)
    ap.add_argument("--ensemble-steps", type=int, default=20,
                    help="timed steps of the batched ensemble (0: skip)")
    ap.add_argument("--ensemble-scenes", type=int, default=256)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (the mixed runs are autotuned first)")
    ap.add_argument("--no-step-graph", action="store_true",
                    help="launch kernel by kernel instead of one CUDA graph per step "
                         "(profiling: identical results; the bucket build stays a graph)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel one by one, the bucket build included (profiling: "
                         "identical results; ncu does not see the kernels of graphs with "
                         "conditional nodes)")
    ap.add_argument("--build-block", type=int, default=0, choices=[0, 64, 128, 256],
                    help="row build block without the autotuner (profiling; 0: the default)")
    ap.add_argument("--cell-skin", type=float, default=0.1,
                    help="cell skin s at creation (the autotuner may choose another)")
    ap.add_argument("--ppe-host-loop", action="store_true",
                    help="drive the mixed PPE solve from the host (profiling: identical results)")
    ap.add_argument("--cg-x0", type=int, default=3, choices=[0, 1, 2, 3, 4],
                    help="PPE initial guess: 0 zero, 1 the previous step's solution, 2 / 3 / 4 "
                         "its linear / quadratic / cubic extrapolation (default 3); the full run "
                         "also "
                         "times the mixed step with each of the others")
    ap.add_argument("--stiff-steps", type=int, default=10,
                    help="timed steps of the stiff PPE (alpha_c = 0) comparison (0: skip)")
    ap.add_argument("--rollout-steps", type=int, default=200,
                    help="steps of the timed differentiable sloshing rollout (0: skip)")
    ap.add_argument("--adjoint-steps", type=int, default=20,
                    help="forward and reverse steps timed on the 3D sloshing tank (0: skip)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ replicas over ranks
# One rank per GPU runs an independent replica of the workload (a single scene does not
# shard without a halo exchange per CG iteration); the only collectives are the barriers
# around the timed region and the maximum of the ranks' times.
def rank_barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def rank_max(x: float, world: int, device=None) -> float:
    """Largest value of x over the ranks (the slowest rank's time)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank * steps / (ms_max * 1e-3)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}",
                                       f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_rate(sc, steps: int, threads: int | None = None):
    import oracle
    oracle.build()
    if threads:
        oracle.set_threads(threads)
    used = oracle.get_threads()
    prm = oracle.params_for(sc, dt=5e-5)
    st = oracle.State.from_scene(sc)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.step(prm, st)
    dt = time.perf_counter() - t0
    return sc.n * steps / dt, used, dt


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    sc = scenes.dam_break_3d(seed=args.seed, l0=args.l0)
    threads = os.cpu_count()
    import oracle
    oracle.build()
    oracle.set_threads(threads)
    prm = oracle.params_for(sc, dt=5e-5)
    st = oracle.State.from_scene(sc)
    for _ in range(args.warmup):
        oracle.step(prm, st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(prm, st)
    dt = time.perf_counter() - t0
    value = sc.n * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles": sc.n, "fluid": sc.n_fluid, "dt": 5e-5,
                   "cg_tol": 1e-8, "l2": "GPU: 512 MiB written before every timed step"},
        "ppe_x0": X0_NAMES[0], "precision": "fp64",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                         "kind": "oracle",
                         "sample": f"{args.steps} oracle steps of the full workload after {args.warmup} warm-up steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU
def run_gb300(args):
    import torch

    from paper_2105_01677_gb300 import mps
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    # one rank per node compiles (the objects and the library are written in-tree); the
    # others wait at the barrier and then only load what it built
    if local == 0:
        __graft_entry__.build()
    rank_barrier(world)
    if local != 0:
        import paper_2105_01677_gb300 as pkg
        pkg.lib()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # before any CUDA work: the oracle on the host cores, bounded sample
        sc_cpu = scenes.dam_break_3d(seed=args.seed, l0=args.l0)
        v, cores, secs = cpu_oracle_rate(sc_cpu, args.cpu_sample_steps, os.cpu_count())
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample_steps} FP64 oracle steps of the full 440,032-particle "
                         f"workload ({secs:.1f} s)"}

    sc = scenes.dam_break_3d(seed=args.seed + rank, l0=args.l0)
    n = sc.n
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    # measured FMA rates of this GPU (the denominators of the ALU rooflines)
    alu_peaks = {name: mps.mps_measure_peak(which, device=local, repeats=5,
                                            stream=stream.cuda_stream)[0]
                 for name, which in (("ffma_tflops", mps.PEAK_FFMA),
                                     ("ffma2_tflops", mps.PEAK_FFMA2),
                                     ("dfma_tflops", mps.PEAK_DFMA))}
    fp32_peak = max(alu_peaks["ffma_tflops"], alu_peaks["ffma2_tflops"])
    # --ppe-host-loop: the mixed PPE solve driven from the host instead of one CUDA graph
    # (identical results; ncu cannot profile the kernels of a graph with conditional nodes)
    common = dict(dt=5e-5, cg_tol=1e-8, ppe_host_loop=1 if args.ppe_host_loop else 0,
                  cg_x0=args.cg_x0, build_block=args.build_block, cell_skin=args.cell_skin,
                  step_graph=2 if args.no_graphs else (0 if args.no_step_graph else 1))

    def timed_steps(sim, k, profile=False, profile_steps=20):
        """CUDA-event time of k steps with the stage timers off (a step then runs as one CUDA
        graph where the path allows it).  With `profile`, a further short pass with the stage
        timers on (launch by launch: the same kernels) gives the per-stage times; `launches`
        and `graph_steps` are those of the timed pass."""
        mps.mps_set_profiling(sim.h, False)          # also resets the launch counter
        total = 0.0
        s_ev = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        e_ev = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        iters = []
        graph_steps = 0
        for i in range(k):
            flush.zero_()
            s_ev[i].record(stream)
            rc, rep = sim.step(1)
            e_ev[i].record(stream)
            graph_steps += rep["step_graph"]
            iters.append((rep["cg_iters"], rep["cg_outer"], rep["cg_resid"], rep["cand_tests"],
                          rep["pairs_ppe"], rep["pairs_pnd"], rep["list_tests"]))
        torch.cuda.synchronize(dev)
        for i in range(k):
            total += s_ev[i].elapsed_time(e_ev[i])
        prof = {"launches": mps.mps_get_profile(sim.h)["launches"], "graph_steps": graph_steps}
        if profile:
            mps.mps_set_profiling(sim.h, True)
            kp = min(k, profile_steps)
            for i in range(kp):
                flush.zero_()
                sim.step(1)
            torch.cuda.synchronize(dev)
            pp = mps.mps_get_profile(sim.h)
            prof["stage_ms"], prof["stage_calls"] = pp["stage_ms"], pp["stage_calls"]
            prof["profiled_steps"] = kp
            prof["stage_ms_per_step"] = {s_: pp["stage_ms"][s_] / kp for s_ in pp["stage_ms"]}
            mps.mps_set_profiling(sim.h, False)
        return total, iters, prof

    def barrier():
        rank_barrier(world)
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        return rank_max(x, world, dev)

    def adjoint_bench(ka):
        # ---- reverse step (vector-Jacobian product) on the 3D sloshing tank, FP64: forward
        # steps under the tank-frame forcing, then reverse steps from the reached state (each
        # repeats its forward step, solves the adjoint PPE and copies the cotangents in and out)
        sc5 = scenes.sloshing_3d(seed=args.seed + rank)
        dt5 = 5e-5
        sim5 = mps.Simulation(sc5, torch_alloc=True, use_torch_stream=True, precision=0,
                              dt=dt5, cg_tol=1e-8, step_graph=common["step_graph"])
        force = lambda t: (float(scenes.sloshing_forcing(t * dt5)), 0.0, -9.81)
        for t in range(args.warmup):
            sim5.set_gravity(force(t))
            sim5.step(1)
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(2 * ka)]
        for i in range(ka):
            sim5.set_gravity(force(args.warmup + i))
            flush.zero_()
            ev[i][0].record(stream)
            sim5.step(1)
            ev[i][1].record(stream)
        rng5 = np.random.default_rng(args.seed)
        ga = rng5.standard_normal((sc5.n, 3))
        gb_ = rng5.standard_normal((sc5.n, 3))
        # reverse steps with the cotangents in device memory (CUDA tensors), then with host
        # buffers (copies in and out inside the timed call)
        ga_d, gb_d = torch.from_numpy(ga).to(dev), torch.from_numpy(gb_).to(dev)
        ro_d, uo_d = torch.empty_like(ga_d), torch.empty_like(gb_d)
        evh = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(ka)]
        its5 = []
        for i in range(ka):
            flush.zero_()
            ev[ka + i][0].record(stream)
            _, _, vrep = sim5.step_vjp_device(ga_d, gb_d, ro_d, uo_d)
            ev[ka + i][1].record(stream)
            its5.append(vrep["cg_iters"])
        for i in range(ka):
            flush.zero_()
            evh[i][0].record(stream)
            sim5.step_vjp(ga, gb_)
            evh[i][1].record(stream)
        torch.cuda.synchronize(dev)
        ms_f = sum(ev[i][0].elapsed_time(ev[i][1]) for i in range(ka))
        ms_r = sum(ev[ka + i][0].elapsed_time(ev[ka + i][1]) for i in range(ka))
        ms_rh = sum(evh[i][0].elapsed_time(evh[i][1]) for i in range(ka))
        barrier()
        ms_f, ms_r, ms_rh = max_over_ranks(ms_f), max_over_ranks(ms_r), max_over_ranks(ms_rh)
        sim5.close()
        # the differentiable rollout: args.rollout_steps steps from rest with a checkpoint every
        # 20, then d(kinetic energy)/d(nu, u0) through torch.autograd (the backward recomputes
        # each segment from its checkpoint and runs the reverse steps); wall clock on the host
        # around each pass with the device synchronised, CUDA tensors throughout
        roll = None
        if args.rollout_steps > 0:
            from paper_2105_01677_gb300 import autograd
            TR = args.rollout_steps
            simr = mps.Simulation(sc5, torch_alloc=True, use_torch_stream=True, precision=0,
                                  dt=dt5, cg_tol=1e-8)
            fr = torch.tensor([force(t) for t in range(TR)], dtype=torch.float64)
            x0 = torch.tensor(sc5.pos, dtype=torch.float64, device=dev)
            times = []
            for rep_i in range(2):   # the first pass captures the graphs: the second is timed
                u0 = torch.zeros((sc5.n, 3), dtype=torch.float64, device=dev, requires_grad=True)
                nu = torch.tensor(1e-6, dtype=torch.float64, requires_grad=True)
                barrier()
                t0 = time.perf_counter()
                xT, uT = autograd.rollout(simr, x0, u0, fr, checkpoint_every=20, nu=nu)
                ke = autograd.kinetic_energy(uT, sc5.types)
                torch.cuda.synchronize(dev)
                t1 = time.perf_counter()
                ke.backward()
                torch.cuda.synchronize(dev)
                t2 = time.perf_counter()
                times.append((t1 - t0, t2 - t1))
            simr.close()
            tf_, tb_ = max_over_ranks(times[-1][0]), max_over_ranks(times[-1][1])
            roll = {"steps": TR, "checkpoint_every": 20, "loss": "final kinetic energy",
                    "wrt": ["nu", "u0"], "precision": "fp64", "cg_tol": 1e-8,
                    "forward_s": tf_, "backward_s": tb_,
                    "value": world * sc5.n * TR / (tf_ + tb_), "unit": UNIT,
                    "timing": "host wall clock with the device synchronised (second pass)"}
        adjoint = {"workload": "3D sloshing tank 0.5 x 0.3 x 0.3 m half full, l0 0.008 m, "
                               "forcing 0.02 m at 1.2 Hz as a tank-frame body force, dt 5e-5 s",
                   "particles": sc5.n, "fluid": sc5.n_fluid, "precision": "fp64",
                   "forward": {"value": world * sc5.n * ka / (ms_f * 1e-3), "unit": UNIT,
                               "ms_per_step": ms_f / ka, "steps": ka},
                   "reverse": {"value": world * sc5.n * ka / (ms_r * 1e-3), "unit": UNIT,
                               "ms_per_step": ms_r / ka, "steps": ka,
                               "adjoint_cg_iters_mean": float(np.mean(its5)),
                               "cotangents": "device memory (mps_step_vjp_device)",
                               "includes": "the repeated forward step and the adjoint solve"},
                   "reverse_host": {"value": world * sc5.n * ka / (ms_rh * 1e-3), "unit": UNIT,
                                    "ms_per_step": ms_rh / ka, "steps": ka,
                                    "h2d_bytes_per_step": int(2 * sc5.n * 3 * 8),
                                    "d2h_bytes_per_step": int(2 * sc5.n * 3 * 8 + 24),
                                    "cotangents": "pageable host buffers (mps_step_vjp)"},
                   "reverse_over_forward": ms_r / ms_f,
                   "rollout": roll}
        return adjoint


    if args.only == "ensemble":
        E = scenes.ensemble_2d(count=args.ensemble_scenes, seed=args.seed + rank)
        ens = mps.Ensemble(E, torch_alloc=True, use_torch_stream=True, precision=1, dt=1e-4,
                           cg_tol=1e-8, cg_x0=args.cg_x0)
        ens.step(2)
        tuning = ens.autotune(3)
        ens.step(args.warmup)
        barrier()
        ms, its, prof = timed_steps(ens, args.steps, profile=True)
        res = ens.residuals()
        ens.close()
        if rank == 0:
            print(json.dumps({"only": "ensemble", "particles": sum(sc.n for sc in E),
                              "ms_per_step": ms / args.steps, "tuning": tuning,
                              "value": sum(sc.n for sc in E) * args.steps / (ms * 1e-3),
                              "cg": [x[:3] for x in its], "worst_resid": float(res.max()),
                              "profile": prof}), flush=True)
        return
    if args.only == "adjoint":
        res = adjoint_bench(args.steps)
        if rank == 0:
            print(json.dumps({"only": "adjoint", **res}), flush=True)
        return
    if args.only:
        prec = 1 if args.only == "mixed" else 0
        simo = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, precision=prec,
                              list_every=args.list_every, **common)
        simo.step(2)
        tuning = None if args.no_autotune else simo.autotune(3)
        simo.step(args.warmup)
        barrier()
        ms, its, prof = timed_steps(simo, args.steps, profile=True)
        # the PPE's SpMV (and the float-float residual) timed alone, outside the graph
        kern = {}
        for name, which in (("spmv32", mps.KERNEL_SPMV32), ("resid_ff", mps.KERNEL_RESID_FF),
                            ("spmv64", mps.KERNEL_SPMV64)):
            if (which == mps.KERNEL_SPMV64) == (prec == 0):
                kms, kby = mps.mps_time_kernel(simo.h, which, 5)
                kern[name] = {"ms_per_launch": kms, "bytes_per_launch": kby,
                              "gbs": kby / (kms * 1e-3) / 1e9}
        simo.close()
        if rank == 0:
            print(json.dumps({"only": args.only, "particles": n, "ms_per_step": ms / args.steps,
                              "tuning": tuning,
                              "value": n * args.steps / (ms * 1e-3), "cg": its, "profile": prof,
                              "kernels": kern}), flush=True)
        return

    # ---- mixed (headline): the library's autotuner picks the launch shapes and the inner
    # CG's form on the state after two steps (the choice is reported under "tuning")
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, precision=1, **common)
    sim.step(2)
    tuning = None if args.no_autotune else sim.autotune(3)
    sim.step(args.warmup)
    clocks = ClockSampler(local)
    barrier()
    ms_mixed, it_mixed, prof = timed_steps(sim, args.steps, profile=True)
    barrier()
    clk = clocks.stop()
    ms_mixed = max_over_ranks(ms_mixed)
    # The dominant kernel of the step is the FP32 SpMV of the inner CG (the launch list's
    # largest share).  The solve launches it inside the graph's conditional loops, where CUDA
    # events cannot bracket single launches, so it is timed alone right after the timed
    # region, on the system of the last timed step, with CUDA events on the library's stream
    # (coefficients 441 MB, larger than L2); likewise the float-float outer residual.
    spmv_ms, spmv_bytes = mps.mps_time_kernel(sim.h, mps.KERNEL_SPMV32, 20)
    resid_ms, resid_bytes = mps.mps_time_kernel(sim.h, mps.KERNEL_RESID_FF, 10)
    sim.close()

    # ---- the same mixed step with the other PPE initial guess
    # the same mixed step with the other PPE initial guesses
    x0_runs = {}
    for x0 in (v for v in sorted(X0_NAMES) if v != args.cg_x0):
        simz = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, precision=1,
                              **{**common, "cg_x0": x0})
        simz.step(args.warmup)
        barrier()
        ms_z, it_z, _ = timed_steps(simz, args.steps)
        barrier()
        ms_z = max_over_ranks(ms_z)
        simz.close()
        x0_runs[x0] = {"cg_x0": x0, "ppe_x0": X0_NAMES[x0],
                       "value": world * n * args.steps / (ms_z * 1e-3), "unit": UNIT,
                       "ms_per_step": ms_z / args.steps, "steps": args.steps,
                       "cg_inner_iters_mean": float(np.mean([x[0] for x in it_z])),
                       "cg_outer_mean": float(np.mean([x[1] for x in it_z]))}

    # ---- plain FP64 on the same scene
    k64 = args.fp64_steps or args.steps
    sim64 = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, precision=0, **common)
    sim64.step(args.warmup)
    barrier()
    ms_64, it_64, prof64 = timed_steps(sim64, k64, profile=True)
    barrier()
    ms_64 = max_over_ranks(ms_64)
    sim64.close()

    # ---- the equation-of-state pressure (Eq. 16, c0 = 20 m/s, gamma = 7) instead of the
    # PPE, same scene, mixed and FP64
    eos = {"c0": 20.0, "gamma": 7.0}
    for name, prec in (("mixed", 1), ("fp64", 0)):
        simw = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, precision=prec,
                              pressure_mode=1, c0=20.0, gamma=7.0, **common)
        simw.step(args.warmup)
        barrier()
        ms_w, _, prof_w = timed_steps(simw, args.steps, profile=True)
        barrier()
        ms_w = max_over_ranks(ms_w)
        simw.close()
        eos[name] = {"value": world * n * args.steps / (ms_w * 1e-3), "unit": UNIT,
                     "ms_per_step": ms_w / args.steps, "steps": args.steps,
                     "stage_ms_per_step": prof_w["stage_ms_per_step"]}

    # ---- mixed with candidate lists kept for up to 4 steps (the paper's fast mode refreshes
    # its neighbour lists every 4 steps; here the sets stay exact)
    kk = args.kept_steps or args.steps
    simk = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, precision=1, list_every=4,
                          **common)
    simk.step(args.warmup)
    barrier()
    ms_k, it_k, profk = timed_steps(simk, kk, profile=True)
    barrier()
    ms_k = max_over_ranks(ms_k)
    simk.close()

    # ---- the stiff PPE: the same scene with Eq. 13 alone (alpha_c = 0, no diagonal term
    # from the PPE listing), so that CG needs ~10x the iterations; mixed and FP64 to the same
    # true FP64 residual 1e-8, same initial guess
    stiff = None
    if args.stiff_steps > 0:
        ks = args.stiff_steps
        stiff = {"alpha_c": 0.0, "steps": ks}
        for name, prec in (("mixed", 1), ("fp64", 0)):
            sims = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, precision=prec,
                                  alpha_c=0.0, **common)
            sims.step(args.warmup)
            barrier()
            ms_s, it_s, prof_s = timed_steps(sims, ks)
            barrier()
            ms_s = max_over_ranks(ms_s)
            sims.close()
            stiff[name] = {"value": world * n * ks / (ms_s * 1e-3), "ms_per_step": ms_s / ks,
                           "cg_iters_mean": float(np.mean([x[0] for x in it_s])),
                           "cg_outer_mean": float(np.mean([x[1] for x in it_s])),
                           "resid_max": float(max(x[2] for x in it_s))}
        stiff["mixed_over_fp64"] = stiff["mixed"]["value"] / stiff["fp64"]["value"]

    # ---- two-phase 3D dam break (light fluid over water in the same column geometry):
    # equation-of-state and PPE paths, mixed precision
    two_phase = None
    if args.two_phase_steps > 0:
        sc2 = scenes.dam_break_3d(seed=args.seed + rank, l0=args.two_phase_l0)
        rho_i, nu_i = scenes.two_phase(sc2, rho=(1000.0, 800.0), nu=(1e-6, 5e-6))
        two_phase = {"workload": f"3D two-phase dam break, l0={args.two_phase_l0} m, densities "
                                 "1000/800 kg/m^3, nu 1e-6/5e-6 m^2/s (lower / upper half of the "
                                 "column)", "particles": sc2.n, "fluid": sc2.n_fluid}
        for name, mode in (("eos", 1), ("ppe", 0)):
            k2 = args.two_phase_steps
            sim2 = mps.Simulation(sc2, torch_alloc=True, use_torch_stream=True, precision=1,
                                  pressure_mode=mode, c0=20.0, rho_i=rho_i, nu_i=nu_i, **common)
            sim2.step(args.warmup)
            barrier()
            ms2, it2, prof2 = timed_steps(sim2, k2, profile=True)
            barrier()
            ms2 = max_over_ranks(ms2)
            sim2.close()
            two_phase[name] = {"value": world * sc2.n * k2 / (ms2 * 1e-3), "unit": UNIT,
                               "ms_per_step": ms2 / k2, "steps": k2,
                               "stage_ms_per_step": prof2["stage_ms_per_step"]}
            if mode == 0:
                two_phase[name]["cg_iters_mean"] = float(np.mean([x[0] for x in it2]))
        del sc2, rho_i, nu_i

    # ---- batched ensemble: independent 2D dam breaks of seeded sizes in one context, mixed
    ensemble = None
    if args.ensemble_steps > 0:
        E = scenes.ensemble_2d(count=args.ensemble_scenes, seed=args.seed + rank)
        ne = sum(sc.n for sc in E)
        ens = mps.Ensemble(E, torch_alloc=True, use_torch_stream=True, precision=1, dt=1e-4,
                           cg_tol=1e-8, cg_x0=args.cg_x0)
        ens.step(2)   # the tuner's cell side needs the motion of a step
        tuning_e = ens.autotune(3)
        ens.step(args.warmup)
        barrier()
        ke = args.ensemble_steps
        ms_e, it_e, prof_e = timed_steps(ens, ke, profile=True)
        barrier()
        ms_e = max_over_ranks(ms_e)
        res = ens.residuals()
        ens.close()
        ensemble = {"workload": f"{len(E)} independent 2D dam breaks, 500-20,000 fluid particles, "
                                "column aspect 0.5-2, l0 0.005-0.01 m, dt 1e-4 s",
                    "scenes": len(E), "particles": ne, "fluid": int(sum(sc.n_fluid for sc in E)),
                    "ppe_x0": X0_NAMES[args.cg_x0],
                    "value": world * ne * ke / (ms_e * 1e-3), "unit": UNIT,
                    "ms_per_step": ms_e / ke, "steps": ke, "tuning": tuning_e,
                    "cg_iters_mean": float(np.mean([x[0] for x in it_e])),
                    "worst_scene_resid": float(res.max()),
                    "launches_per_step": prof_e["launches"] / max(ke, 1),
                    "graph_launches_per_step": prof_e["graph_steps"] / max(ke, 1),
                    "host_syncs_per_step": 1 if prof_e["graph_steps"] == ke else None,
                    "stage_ms_per_step": prof_e["stage_ms_per_step"],
                    "stage_timing": "a further pass launched kernel by kernel with the stage "
                                    "timers on (the same kernels)"}
        del E

    adjoint = adjoint_bench(args.adjoint_steps) if args.adjoint_steps > 0 else None

    # ---- end to end through the C ABI with host buffers (mixed)
    ke = args.e2e_steps or args.steps
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    h_pos = pin((n, 3), torch.float64)
    h_vel = pin((n, 3), torch.float64)
    h_typ = pin((n,), torch.int8)
    h_p = pin((n,), torch.float64)
    h_pos[:] = sc.pos
    h_vel[:] = sc.vel
    h_typ[:] = sc.types
    sime = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, precision=1, **common)
    for _ in range(args.warmup):
        sime.write(h_pos, h_vel, h_typ)
        sime.step(1)
        sime.read(pos=h_pos, vel=h_vel, p=h_p, want=("pos", "vel", "p"))
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        sime.write(h_pos, h_vel, h_typ)
        sime.step(1)
        sime.read(pos=h_pos, vel=h_vel, p=h_p, want=("pos", "vel", "p"))
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    sime.close()
    h2d = h_pos.nbytes + h_vel.nbytes + h_typ.nbytes
    d2h = h_pos.nbytes + h_vel.nbytes + h_p.nbytes

    if rank != 0:
        return

    # ---- rooflines (live CUDA-event times on the library's stream)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    hbm_src = ("MEASURED_PEAKS.json hbm_gbs, burst copy (measured)" if "hbm_gbs" in peaks
               else "fallback 6.8 TB/s")
    alu_src = "mps_measure_peak on this GPU before the run (measured)"
    st_ms = prof["stage_ms"]
    st_calls = prof["stage_calls"]
    per_call = {k: (st_ms[k] / st_calls[k] if st_calls[k] else 0.0) for k in st_ms}
    mean = lambda idx: float(np.mean([x[idx] for x in it_mixed]))
    inner, outer = mean(0), mean(1)
    tests, ppe_pairs, pnd_pairs, list_tests = mean(3), mean(4), mean(5), mean(6)
    resid_launches = outer + (1 if args.cg_x0 else 0)
    step_ms = ms_mixed / args.steps

    def bound(kernel, ms, launches, flops=None, nbytes=None, **extra):
        """Roofline of one kernel: the method's flops against the measured FP32 FMA rate
        and its algorithmic bytes against the measured HBM copy rate; the bound is the roof
        the kernel is closer to (the larger fraction)."""
        r = {"kernel": kernel}
        fr = {}
        if flops is not None:
            a = flops / (ms * 1e-3) / 1e12
            fr["alu"] = {"achieved": a, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": a / fp32_peak, "peak_source": alu_src}
        if nbytes is not None:
            a = nbytes / (ms * 1e-3) / 1e9
            fr["hbm"] = {"achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                         "peak_source": hbm_src}
        b = max(fr, key=lambda k: fr[k]["frac"])
        r.update({"bound": b, **fr[b]})
        r["other_bound"] = {k: v for k, v in fr.items() if k != b} or None
        r.update({"ms_per_launch": ms, "launches_per_step": launches,
                  "ms_per_step": ms * launches, "share_of_step": ms * launches / step_ms})
        r.update(extra)
        return r

    build_flops = METHOD_FLOPS_PPE_PAIR * ppe_pairs + METHOD_FLOPS_PND_PAIR * pnd_pairs
    build_bytes = (BUILD_BYTES_PER_COEF * ppe_pairs + BUILD_BYTES_PER_LIST_ENTRY * list_tests +
                   BUILD_BYTES_PER_PARTICLE * n)
    roof_build = bound(
        "k_build<mixed> (number density, flags, PPE rows)", per_call["build"], 1.0,
        flops=build_flops, nbytes=build_bytes,
        traffic=BUILD_TRAFFIC_PER_COEF * ppe_pairs if BUILD_TRAFFIC_PER_COEF else None,
        work={"pairs_ppe": ppe_pairs, "pairs_pnd": pnd_pairs, "list_entries": list_tests,
              "pair_evals": ppe_pairs + pnd_pairs,
              "pair_evals_per_s": (ppe_pairs + pnd_pairs) / (per_call["build"] * 1e-3),
              "flops_per_pair": {"ppe": METHOD_FLOPS_PPE_PAIR, "pnd": METHOD_FLOPS_PND_PAIR},
              "bytes": {"per_coef": BUILD_BYTES_PER_COEF,
                        "per_list_entry": BUILD_BYTES_PER_LIST_ENTRY,
                        "per_particle": BUILD_BYTES_PER_PARTICLE},
              "issued_ff_tflops": (ISSUED_FLOPS_PPE_PAIR * ppe_pairs + ISSUED_FLOPS_PND_PAIR *
                                   pnd_pairs + ISSUED_FLOPS_LIST_TEST * list_tests)
                                  / (per_call["build"] * 1e-3) / 1e12})
    roof_gather = bound("k_gather<VerletOp> (candidate lists)", per_call["gather"], 1.0,
                        flops=METHOD_FLOPS_TEST * tests, nbytes=4.0 * list_tests + 48.0 * n,
                        traffic=GATHER_TRAFFIC_PER_ENTRY * list_tests,
                        work={"cand_tests": tests, "list_entries": list_tests,
                              "flops_per_test": METHOD_FLOPS_TEST,
                              "bytes": "4 per list entry written, 48 per particle read"})
    roof_spmv = bound("k_spmv32_t (FP32 SpMV of the inner CG)", spmv_ms, inner,
                      nbytes=spmv_bytes,
                      traffic=SPMV_TRAFFIC_PER_COEF * ppe_pairs if SPMV_TRAFFIC_PER_COEF else None,
                      bytes_per_launch=spmv_bytes,
                      timing="timed alone after the timed region (CUDA events, 20 launches)")
    roof_resid = bound("k_resid_ff_t (float-float FP64 residual)", resid_ms, resid_launches,
                       nbytes=resid_bytes, traffic=RESID_TRAFFIC_PER_COEF * ppe_pairs,
                       bytes_per_launch=resid_bytes,
                       timing="timed alone after the timed region (CUDA events, 10 launches)")
    rooflines = sorted([roof_build, roof_spmv, roof_gather, roof_resid],
                       key=lambda r: -r["ms_per_step"])
    roofline = dict(rooflines[0])
    roofline["dominant"] = "largest device time per step among the step's kernels"
    # whole-step bytes under both models of the survey: matrix-free minimum, and the stored
    # coefficients this design streams (build writes them, every SpMV and residual reads them)
    mf_bytes = n * (STEP_BYTES_FIXED[1] + 57.0 * inner + 65.0 * (outer + 1))
    stored_bytes = (n * (182.0 + 113.0 + 146.0 + 48.0) + 4.0 * list_tests + build_bytes +
                    inner * (spmv_bytes + 36.0 * n) + resid_launches * (resid_bytes + 40.0 * n))
    step_gbs = lambda b: b / (step_ms * 1e-3) / 1e9
    step_hbm = {"matrix_free": {"bytes_per_step": mf_bytes, "achieved_gbs": step_gbs(mf_bytes),
                                "frac": step_gbs(mf_bytes) / hbm,
                                "model": "483 B per particle + 57 per FP32 inner iteration + "
                                         "65 per FP64 residual"},
                "stored_coefficients": {"bytes_per_step": stored_bytes,
                                        "achieved_gbs": step_gbs(stored_bytes),
                                        "frac": step_gbs(stored_bytes) / hbm,
                                        "model": "per-particle state traffic of every stage, "
                                                 "candidate lists written and read, PPE rows "
                                                 "written, each SpMV / residual launch's "
                                                 "algorithmic bytes"},
                "peak_gbs": hbm, "peak_source": hbm_src}

    value = replica_rate(n, args.steps, world, ms_mixed)
    value64 = replica_rate(n, k64, world, ms_64)
    # key order: the contract's keys first, the detail in the middle, and the two arms of the
    # metric (mixed against FP64, on the regularised and on the stiff PPE) at the very end
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64 mixed", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles": n, "fluid": sc.n_fluid, "dt": 5e-5,
                   "cg_tol": 1e-8, "l2": "GPU: 512 MiB written before every timed step"},
        "ppe_x0": X0_NAMES[args.cg_x0], "precision": "mixed", "parallelism": f"replicas{world}",
        "fluid_particle_steps_per_s": world * sc.n_fluid * args.steps / (ms_mixed * 1e-3),
        "tuning": tuning,
        "gpu_launches": int(prof["launches"]),
        "graph_launches_per_step": prof["graph_steps"] / args.steps,
        "stage_timing": "stage times from a further pass launched kernel by kernel with the "
                        "stage timers on (the same kernels); the timed pass runs each step as "
                        "one CUDA graph",
        "e2e": {"value": world * n * ke / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "ppe_x0": X0_NAMES[args.cg_x0],
                "note": "every step writes the state read after the previous one (the "
                        "context's own, bit for bit: the write changes nothing) and reads "
                        "positions, velocities and pressure back"},
        "cpu_baseline": cpu,
        "clocks": clk,
        "alu_peaks": alu_peaks,
        "other_x0": [x0_runs[k] for k in sorted(x0_runs)],
        "two_phase": two_phase,
        "ensemble": ensemble,
        "adjoint": adjoint,
        "eos": eos,
        "kept_lists": {"list_every": 4, "value": world * n * kk / (ms_k * 1e-3), "unit": UNIT,
                       "ms_per_step": ms_k / kk, "steps": kk,
                       "gathers_per_step": profk["stage_calls"]["gather"] / profk["profiled_steps"],
                       "stage_ms_per_step": profk["stage_ms_per_step"]},
        "fp64_stage_ms_per_step": prof64["stage_ms_per_step"],
        "stage_ms_per_step": {k: per_call[k] for k in per_call},
        "rooflines": rooflines[1:],
        "step_hbm": step_hbm,
        "roofline": roofline,
        "stiff_ppe": stiff,
        "cg": {"inner_iters_mean": inner, "outer_mean": outer,
               "resid_max": float(max(x[2] for x in it_mixed))},
        "fp64": {"value": value64, "unit": UNIT, "ms_per_step": ms_64 / k64, "steps": k64,
                 "cg_iters_mean": float(np.mean([x[0] for x in it_64])),
                 "resid_max": float(max(x[2] for x in it_64))},
        "mixed_over_fp64": value / value64,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
