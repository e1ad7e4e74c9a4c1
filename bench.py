"""Benchmark of the adjoint-LBM sensitivity solve (primal + adjoint MLUPS).

One bench step is one full unsteady sensitivity solve of the D3Q19 MRT
mixer (256x128x128 nodes, two D3Q7 passive scalars, velocity inlet and
pressure outlet, tau = 0.6, theta ~ U[0,1] on the 128x96x96 design region,
J = outlet scalar variance averaged over the last 500 steps): 10000 primal
steps, then 10000 adjoint steps with level-1 checkpoints every 500 steps
and recomputation of the states in between, accumulating dJ/dtheta in FP64.

value = nodes * (primal steps + adjoint steps) / seconds / 1e6 (recomputed
primal steps are work, not credit), timed with CUDA events around whole
solves; the per-kernel split (GB/s, roofline fraction) comes from one more
solve with events around every launch.  Inputs (550 MB of populations per
state) are larger than L2, so no flush is needed between steps.

At N = 1 the same JSON line also carries the other workloads of the problem
statement, measured on the same GPU after the headline: ``exchanger3d``
(the 512x256x256 heat exchanger with FP32, BF16 and FP16 storage: solve
MLUPS, kernel GB/s and dJ/dtheta against the FP32 path), ``serving``
(Poisson-arriving requests at 1, 10 and 100 per second, 100 each, served
with continuous batching against one-at-a-time FIFO service) and
``batch64`` (64 instances through the batched autograd Function against
one at a time); ``--no-extras`` leaves them out.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With torchrun (N > 1) every rank solves its own independent replica (the
path does not shard in this build: replicas only) and rank 0 prints the
aggregate.

Other workloads (--workload): exchanger3d (512x256x256 BGK + D3Q7, heat
flux), batch64 (64 instances through the batched autograd Function), serve
(continuous batching of Poisson-arriving requests), oneshot (the one-shot
optimisation of Sec. 3.3 on the exchanger), meshes (primal and adjoint
kernel rates on the paper's 400K / 3M / 12M scaling meshes), paper (the
paper's empty mixer and exchanger channels against its printed values) and
mma (MMA design iterations of Sec. 3.3 on the exchanger).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1501_04741_gb300 import inputs  # noqa: E402

METRIC = "primal+adjoint MLUPS & % HBM roofline"
UNIT = "MLUPS"

# algorithmic bytes per node update (FP32 populations, 33 densities):
#   primal : read 33 x 4 + write 33 x 4 + theta 4 + flag 1
#   adjoint: read lambda 33 x 4 + read f 33 x 4 + write lambda 33 x 4
#            + theta 4 + flag 1 + FP64 gradient read + write 16
def bytes_per_node(M: int, storage: int, kind: str) -> int:
    if kind == "primal":
        return M * storage * 2 + 5
    return M * 4 * 2 + M * storage + 21


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# the ncu capture of the 256x128x64 profile case, scaled by the node count to
# the 256x128x128 lattice (traffic grows with the nodes); valid for the FP32
# mixer kernels as captured: the forms without objective terms (primal
# OBJ = 0, adjoint SRC = 0), which run 95 % of the steps.
TRAFFIC_MIXER_FP32 = {"primal": 1.0288e9, "adjoint": 1.6775e9}


def workload(args) -> inputs.Problem:
    P = inputs.exchanger3d() if args.workload == "exchanger3d" else inputs.mixer3d()
    if args.nsteps:
        P = P.replace(nsteps=args.nsteps, obj_window=min(P.obj_window, args.nsteps))
    if args.precision != "fp32":
        P = P.replace(precision=args.precision)
    if args.kernel != "auto":
        P = P.replace(kernel=args.kernel)
    return P


def aggregate_ranks(ms_local: float, updates_per_step: float, steps: int, world: int,
                    device: str = "cuda"):
    """Whole-job figure of a replicas run: the slowest rank's time bounds the
    job, and every rank processed ``updates_per_step`` node updates per step
    (weak scaling).  Returns (max ms over ranks, MLUPS of all ranks)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * updates_per_step * steps / (ms_max / 1e3) / 1e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = self.rows
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        smax = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# the oracle, timed on the host cores (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
ORACLE_SAMPLE_DIMS = (96, 48, 48)
ORACLE_SAMPLE_STEPS = 6
ORACLE_SAMPLE_DIMS_1T = (48, 24, 24)
ORACLE_SAMPLE_STEPS_1T = 4
ORACLE_REPEATS = 5


def oracle_sample(P: inputs.Problem, dims=ORACLE_SAMPLE_DIMS, steps=ORACLE_SAMPLE_STEPS):
    """Time the FP64 oracle on a bounded sample of the workload: the same
    physics on a sub-lattice (96x48x48 by default), `steps` primal then
    `steps` adjoint steps."""
    import torch
    from oracle.solver import Oracle
    Ps = inputs.scaled(P, dims, nsteps=steps, obj_window=min(P.obj_window, steps))
    o = Oracle(Ps, inputs.theta_uniform(Ps, 0))
    t0 = time.perf_counter()
    _, traj = o.primal()
    o.adjoint(traj)
    dt = time.perf_counter() - t0
    updates = o.n * steps * 2
    sample = (f"{Ps.lattice} {Ps.collision} + {Ps.nscalars} scalars on "
              f"{'x'.join(map(str, dims))}, {steps} primal + {steps} adjoint steps (FP64 oracle)")
    return updates / dt / 1e6, dt, torch.get_num_threads(), sample


def cpu_baseline_record(P: inputs.Problem, args) -> dict:
    """The oracle on the host cores, timed in a fresh process (as the
    reference arm is: the process that drove the GPU times the host code
    slower), see cpu_baseline_local."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-only",
           "--workload", args.workload, "--precision", args.precision]
    if args.nsteps:
        cmd += ["--nsteps", str(args.nsteps)]
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    for line in out.stdout.splitlines():
        if line.startswith("{"):
            rec = json.loads(line)
            rec["process"] = "fresh host process, no CUDA context"
            return rec
    raise RuntimeError(f"cpu baseline process failed: {out.stderr[-2000:]}")


def cpu_baseline_local(P: inputs.Problem) -> dict:
    """The oracle on the host cores: all threads torch uses (the reference
    arm's sample and statistic: median of ORACLE_REPEATS runs after one
    warm-up), and one thread on a smaller sample."""
    import torch
    oracle_sample(P)
    runs = [oracle_sample(P) for _ in range(ORACLE_REPEATS)]
    value = float(np.median([r[0] for r in runs]))
    threads = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        oracle_sample(P, ORACLE_SAMPLE_DIMS_1T, ORACLE_SAMPLE_STEPS_1T)
        one = [oracle_sample(P, ORACLE_SAMPLE_DIMS_1T, ORACLE_SAMPLE_STEPS_1T)
               for _ in range(ORACLE_REPEATS)]
    finally:
        torch.set_num_threads(threads)
    return {"value": value, "unit": UNIT, "cores": threads, "host_cpus": os.cpu_count(),
            "kind": "oracle", "sample": runs[0][3],
            "statistic": f"median of {ORACLE_REPEATS} runs after 1 warm-up",
            "seconds_per_run": float(np.median([r[1] for r in runs])),
            "single_thread": {"value": float(np.median([r[0] for r in one])), "unit": UNIT,
                              "cores": 1, "sample": one[0][3],
                              "statistic": f"median of {ORACLE_REPEATS} runs after 1 warm-up"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    P = workload(args)
    for _ in range(args.warmup):
        oracle_sample(P)
    t_all = time.perf_counter()
    runs = [oracle_sample(P) for _ in range(args.steps)]
    wall = time.perf_counter() - t_all
    value = float(np.median([r[0] for r in runs]))
    cores, sample = runs[0][2], runs[0][3]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(P, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "host_cpus": os.cpu_count(), "kind": "oracle", "sample": sample,
                         "statistic": "median over the timed steps (one sample each)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(P, args):
    return {"workload": args.workload, "lattice": P.lattice, "collision": P.collision,
            "dims": list(P.dims), "nscalars": P.nscalars, "tau": P.tau,
            "primal_steps": P.nsteps, "adjoint_steps": P.nsteps, "ckpt_every": P.ckpt_every,
            "objective": P.objective, "obj_window": P.obj_window, "precision": P.precision,
            "kernel": P.kernel,
            "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{args.gpus}"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1501_04741_gb300.albm import Solver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    P = workload(args)
    theta = inputs.theta_grf(P, rank) if args.workload == "exchanger3d" else \
        inputs.theta_uniform(P, rank)
    stream = torch.cuda.Stream()
    th_dev = torch.from_numpy(theta.reshape(-1)).cuda()
    s = Solver(P, th_dev, stream=stream, mem_budget=args.mem_budget)
    N = s.N
    M = s.M
    storage = {"fp32": 4, "bf16": 2, "fp16": 2}[P.precision]

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    # warm-up (allocates the state pool too)
    for _ in range(args.warmup):
        s.run()
    barrier()
    # the timed region: whole solves, no per-launch instrumentation
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            s.run()
        ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    J = s.objective()
    recompute = s.recompute_steps()
    updates_per_step = N * P.nsteps * 2
    ms_max, value = aggregate_ranks(ms, updates_per_step, args.steps, world)

    # kernel split: one more solve with CUDA events around every launch (the
    # schedule of a solve after the warm-up is the same every time)
    s.profile(True)
    s.run()
    prof = s.profile_read()
    s.profile(False)
    n_p, ms_p = prof["primal"]
    n_r, ms_r = prof["recompute"]
    n_a, ms_a = prof["adjoint"]
    peak, peak_kind = _peaks()
    bp = bytes_per_node(M, storage, "primal")
    ba = bytes_per_node(M, storage, "adjoint")
    prim_ms = (ms_p + ms_r) / max(n_p + n_r, 1)
    adj_ms = ms_a / max(n_a, 1)
    prim_gbs = bp * N / (prim_ms / 1e3) / 1e9
    adj_gbs = ba * N / (adj_ms / 1e3) / 1e9
    share_adj = ms_a / max(ms_p + ms_r + ms_a, 1e-9)
    dom = "adjoint" if share_adj >= 0.5 else "primal"
    ach = adj_gbs if dom == "adjoint" else prim_gbs

    # end to end through the C ABI with host buffers (pinned), copies inside
    th_host = torch.from_numpy(theta.reshape(-1)).pin_memory()
    g_host = torch.empty(N, dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        s.set_theta(th_host.numpy())
        s.run()
        s.gradient(g_host.numpy())
        s.objective()
    barrier()
    dt = time.perf_counter() - t0
    e2e = {"value": world * updates_per_step * max(1, args.e2e_steps) / dt / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": int(N * 4), "d2h_bytes_per_step": int(N * 8 + 16 * (P.nsteps + 1))}
    s.close()
    launches_per_solve = prof["launches"]
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if P.precision == "fp32" else f"f32 ({P.precision} storage)",
            "data": "synthetic", "config": _config(P, args),
            "roofline": {"bound": "hbm", "kernel": f"{dom}_kernel", "achieved": ach,
                         "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "peak_source": peak_kind,
                         "traffic": (TRAFFIC_MIXER_FP32[dom] if (args.workload == "mixer3d" and
                                                                 P.precision == "fp32" and
                                                                 P.kernel == "auto" and
                                                                 not args.nsteps) else None),
                         "algorithmic_bytes": (bp if dom == "primal" else ba) * N},
            "kernels": {
                "timing": "one solve after the timed region, CUDA events around every launch",
                "primal": {"launches": n_p + n_r, "avg_ms": prim_ms, "GB_s": prim_gbs,
                           "frac": prim_gbs / peak, "bytes_per_node": bp,
                           "MLUPS": N / (prim_ms / 1e3) / 1e6},
                "adjoint": {"launches": n_a, "avg_ms": adj_ms, "GB_s": adj_gbs,
                            "frac": adj_gbs / peak, "bytes_per_node": ba,
                            "MLUPS": N / (adj_ms / 1e3) / 1e6},
                "share_adjoint": share_adj, "recompute_steps_per_solve": recompute},
            "J": J,
            "e2e": e2e,
            "gpu_launches": int(launches_per_solve * args.steps),
            "clocks": clk,
            "cpu_baseline": None,
        }
        if world == 1 and not args.no_extras and args.workload == "mixer3d" and not args.nsteps:
            # the other workloads of the problem statement, on the same GPU
            line["exchanger3d"] = exchanger_precisions(args)
            line["serving"] = serve_sweep(args)
            line["batch64"] = batch64_record(args)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_record(P, args)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def exchanger_precisions(args) -> dict:
    """The full 512x256x256 exchanger (1000 + 1000 steps) with FP32, BF16 and
    FP16 population storage on one theta: solve MLUPS (one warm-up solve,
    one timed solve without instrumentation), the kernels' GB/s from one
    instrumented solve, and J and dJ/dtheta against the FP32 path."""
    import torch
    from paper_1501_04741_gb300.albm import Solver
    P0 = inputs.exchanger3d()
    th = torch.from_numpy(inputs.theta_grf(P0, 0).reshape(-1)).cuda()
    stream = torch.cuda.Stream()
    peak, _ = _peaks()
    rows, ref = {}, None
    for prec in ("fp32", "bf16", "fp16"):
        P = P0.replace(precision=prec)
        storage = 4 if prec == "fp32" else 2
        with Solver(P, th, stream=stream) as s:
            s.run()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.run()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            J = s.objective()
            g = s.gradient().clone()
            s.profile(True)
            s.run()
            prof = s.profile_read()
            s.profile(False)
            N, M = s.N, s.M
        (n_p, ms_p), (n_r, ms_r), (n_a, ms_a) = prof["primal"], prof["recompute"], prof["adjoint"]
        pm = (ms_p + ms_r) / max(n_p + n_r, 1)
        am = ms_a / max(n_a, 1)
        bp, ba = bytes_per_node(M, storage, "primal"), bytes_per_node(M, storage, "adjoint")
        row = {"MLUPS": 2.0 * N * P.nsteps / (ms / 1e3) / 1e6, "solve_ms": ms, "J": J,
               "primal": {"avg_ms": pm, "bytes_per_node": bp, "GB_s": bp * N / pm / 1e6,
                          "frac": bp * N / pm / 1e6 / peak},
               "adjoint": {"avg_ms": am, "bytes_per_node": ba, "GB_s": ba * N / am / 1e6,
                           "frac": ba * N / am / 1e6 / peak}}
        if ref is None:
            ref = (J, g)
        else:
            row["J_rel_err_vs_fp32"] = abs(J - ref[0]) / abs(ref[0])
            row["dJdtheta_rel_err_vs_fp32"] = float((g - ref[1]).abs().max() / ref[1].abs().max())
        rows[prec] = row
        del g
    return {"dims": list(P0.dims), "steps": P0.nsteps, "objective": P0.objective,
            "theta": "Gaussian random field (sigma 4) on the middle 3/7", "rows": rows}


def fifo_finish_times(arrivals, service):
    """Finish times of one server taking requests first come first served:
    each starts at the later of its arrival and the previous finish."""
    done, fin = [], 0.0
    for a, sv in zip(arrivals, service):
        fin = max(a, fin) + sv
        done.append(fin)
    return done


def serve_sweep(args) -> dict:
    """Config 5 served with continuous batching at several arrival rates,
    against one-at-a-time plain FP32 FIFO service of the same requests.

    The same seeded requests serve every rate (arrival times scale as 1 /
    rate).  The one-at-a-time baseline solves each request alone once and
    times it (handle creation, solve, J and dJ/dtheta to the host); its FIFO
    latencies at each rate follow from those service times and the arrival
    times (start = max(arrival, previous finish)), which is what a real-time
    one-at-a-time server would see, without waiting out the idle gaps."""
    import torch
    from paper_1501_04741_gb300.albm import Solver
    from paper_1501_04741_gb300.serve import Request, Server
    rates = [float(r) for r in args.serve_rates.split(",")]
    count = args.serve_count
    spec1 = inputs.serving_requests(count, rate=1.0, seed=0, node_range=(1e4, args.max_nodes))
    # one-at-a-time service times (plain FP32 handles, one after the other)
    stream = torch.cuda.Stream()
    svc, J_alone, g_alone = [], [], []
    for _, P, th in spec1:
        t0 = time.perf_counter()
        with Solver(P, th, stream=stream) as s:
            s.run()
            J_alone.append(s.objective())
            g_alone.append(s.gradient().cpu().numpy())
        svc.append(time.perf_counter() - t0)
    updates = float(sum(2.0 * P.n_nodes * P.nsteps for _, P, _ in spec1))
    rows = []
    for rate in rates:
        arrivals = [t / rate for t, _, _ in spec1]
        done = fifo_finish_times(arrivals, svc)
        lat_seq = [d - a for d, a in zip(done, arrivals)]
        reqs = [Request(i, a, P, th) for i, (a, (_, P, th)) in enumerate(zip(arrivals, spec1))]
        srv = Server(steps_per_tick=args.tick, keep_gradients=True)
        st = srv.run(reqs)
        torch.cuda.synchronize()
        ok = all(r.error is None for r in reqs)
        same = ok and all(r.J == j and np.array_equal(r.grad, g)
                          for r, j, g in zip(reqs, J_alone, g_alone))
        for r in reqs:
            r.grad = None
        rows.append({"rate_per_s": rate, "requests": len(reqs),
                     "served": {"p50_s": st.p50, "p99_s": st.p99, "MLUPS": st.mlups,
                                "makespan_s": st.makespan, "max_resident": st.max_resident},
                     "one_at_a_time": {"p50_s": float(np.percentile(lat_seq, 50)),
                                       "p99_s": float(np.percentile(lat_seq, 99)),
                                       "MLUPS": updates / max(done[-1], 1e-9) / 1e6,
                                       "makespan_s": done[-1]},
                     "results_identical_to_alone": bool(same)})
    return {"requests_per_rate": count, "node_range": [1e4, args.max_nodes],
            "steps_range": [500, 5000], "lattices": "D2Q9 / D3Q19 channels at 50/50",
            "service_s_total": float(sum(svc)), "rows": rows}


def batch64_record(args) -> dict:
    """Config 4: 64 seeded D2Q9 / D3Q19 instances (sizes log-uniform,
    1000-5000 steps) through the batched torch.autograd.Function, against
    the same instances one at a time through the single-instance Function."""
    import torch
    from paper_1501_04741_gb300.albm import Solver
    from paper_1501_04741_gb300.autograd import albm_objective, albm_objectives
    batch = inputs.batch_instances(args.count or 64, seed=0, size_scale=args.size_scale)
    free, _ = torch.cuda.mem_get_info()
    sizes = [P.n_nodes * (9 if P.lattice == "D2Q9" else 19) * 4 for P, _ in batch]
    budget = 0.6 * free
    stream = torch.cuda.Stream()
    solvers, thetas = [], []
    for (P, th), sz in zip(batch, sizes):
        t = torch.from_numpy(th.reshape(-1)).cuda().requires_grad_(True)
        thetas.append(t)
        solvers.append(Solver(P, t.detach(), stream=stream,
                              mem_budget=max(8 * sz, budget * sz / sum(sizes))))
    updates = sum(2.0 * P.n_nodes * P.nsteps for P, _ in batch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Js = albm_objectives(thetas, solvers)
    Js.sum().backward()
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    g_batch = [t.grad.clone() for t in thetas]
    for t in thetas:
        t.grad = None
    t0 = time.perf_counter()
    for t, s in zip(thetas, solvers):
        albm_objective(t, s).backward()
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    finite = all(bool(torch.isfinite(t.grad).all()) for t in thetas)
    same = all(torch.equal(a, t.grad) for a, t in zip(g_batch, thetas))
    for s in solvers:
        s.close()
    return {"instances": len(batch), "nodes_total": sum(P.n_nodes for P, _ in batch),
            "d2q9": sum(P.lattice == "D2Q9" for P, _ in batch), "size_scale": args.size_scale,
            "batched_MLUPS": updates / t_batch / 1e6, "batched_s": t_batch,
            "one_at_a_time_MLUPS": updates / t_seq / 1e6, "one_at_a_time_s": t_seq,
            "gradients_identical": bool(same), "gradients_finite": finite}


def run_batch64(args):
    rec = batch64_record(args)
    print(json.dumps({"metric": "batched autograd primal+adjoint MLUPS", "workload": "batch64",
                      "value": rec["batched_MLUPS"], "unit": UNIT, "higher_is_better": True,
                      **rec}), flush=True)
    return 0


def run_serve(args):
    rec = serve_sweep(args)
    print(json.dumps({"metric": "served p50/p99 vs one-at-a-time FP32", "workload": "serve",
                      **rec}), flush=True)
    return 0


def run_precision(args):
    rec = exchanger_precisions(args)
    print(json.dumps({"metric": "exchanger solve MLUPS and dJ/dtheta error by storage",
                      "workload": "precision", **rec}), flush=True)
    return 0


def run_oneshot(args):
    """One-shot optimisation (Sec. 3.3) on the full 512x256x256 exchanger:
    per iteration one primal step, one ALBS step at the current state and the
    design update, all on the device; node updates counted as 2 per node and
    iteration (primal + adjoint), as in the headline metric."""
    import torch
    from paper_1501_04741_gb300.albm import Solver
    P = inputs.exchanger3d()
    if args.precision != "fp32":
        P = P.replace(precision=args.precision)
    theta = inputs.theta_grf(P, 0)
    mask = inputs.design_mask(P).reshape(-1).astype(np.uint8)
    iters = args.oneshot_iters
    zeta, pen = 1.0, 1e-4
    stream = torch.cuda.Stream()
    s = Solver(P, torch.from_numpy(theta.reshape(-1)).cuda(), stream=stream)
    N = s.N
    s.set_design(mask)
    s.oneshot_reset()
    for _ in range(args.warmup):
        s.oneshot_step(iters, zeta, pen, True)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    s.profile(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            s.oneshot_step(iters, zeta, pen, True)
        ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    prof = s.profile_read()
    s.profile(False)
    clk = clocks.stop()
    J, Pv = s.oneshot_eval()
    peak, peak_kind = _peaks()
    storage = {"fp32": 4, "bf16": 2, "fp16": 2}[P.precision]
    bp = bytes_per_node(s.M, storage, "primal")
    # one-shot adjoint: lambda in/out and f as in the unsteady step, theta and
    # flag read, design mask read, theta written, gradient estimate written
    ba = s.M * 4 * 2 + s.M * storage + 4 + 1 + 1 + 4 + 8
    (n_p, ms_p), (n_a, ms_a) = prof["primal"], prof["adjoint"]
    prim_ms, adj_ms = ms_p / max(n_p, 1), ms_a / max(n_a, 1)
    adj_gbs = ba * N / (adj_ms / 1e3) / 1e9
    updates = 2.0 * N * iters * args.steps
    # end to end: host theta and mask in, iterations, J, P and theta out
    th_host = torch.from_numpy(theta.reshape(-1)).pin_memory()
    th_out = torch.empty(N, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_theta(th_host.numpy())
    s.set_design(mask)
    s.oneshot_reset()
    s.oneshot_step(iters, zeta, pen, True)
    s.oneshot_eval()
    s.theta(th_out)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    print(json.dumps({
        "metric": "one-shot optimisation primal+adjoint MLUPS", "workload": "oneshot",
        "value": updates / (ms / 1e3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "dtype": "f32" if P.precision == "fp32" else f"f32 ({P.precision} storage)",
        "data": "synthetic",
        "config": {"workload": "oneshot", "lattice": P.lattice, "collision": P.collision,
                   "dims": list(P.dims), "nscalars": P.nscalars, "objective": P.objective,
                   "iterations_per_step": iters, "zeta": zeta, "penalty": pen,
                   "design_nodes": int(mask.sum()), "l2": "inputs larger than L2 (no flush)"},
        "iterations_per_s": iters * args.steps / (ms / 1e3),
        "roofline": {"bound": "hbm", "kernel": "adjoint_kernel", "achieved": adj_gbs,
                     "peak": peak, "unit": "GB/s", "frac": adj_gbs / peak,
                     "peak_source": peak_kind, "traffic": None,
                     "algorithmic_bytes": ba * N},
        "kernels": {"primal": {"launches": n_p, "avg_ms": prim_ms,
                               "GB_s": bp * N / (prim_ms / 1e3) / 1e9},
                    "adjoint": {"launches": n_a, "avg_ms": adj_ms, "GB_s": adj_gbs},
                    "other_per_iteration_ms": (ms - ms_p - ms_a) / (iters * args.steps)},
        "J": J, "P": Pv,
        "e2e": {"value": 2.0 * N * iters / dt / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": int(N * 4 + N), "d2h_bytes_per_step": int(N * 4 + 16)},
        "gpu_launches": int(prof["launches"]), "clocks": clk}), flush=True)
    return 0


# the paper's scaling meshes (Sec. 4.3): D3Q19 MRT fluid + one D3Q7 scalar,
# with its one-GPU (Tesla M2090) primal / adjoint MLUPS for context
MESHES = [("400K", (160, 50, 50), 289, 104), ("3M", (320, 100, 100), 298, 109),
          ("12M", (320, 200, 200), None, None)]


def run_meshes(args):
    """Primal and adjoint kernel MLUPS on the paper's three scaling meshes
    (heat-exchanger physics with the MRT fluid collision of Sec. 4), and the
    adjoint / primal time ratio the paper reports as about 2.65."""
    import torch
    from paper_1501_04741_gb300.albm import Solver
    nsteps = args.nsteps or 200
    rows = []
    for name, dims, p_mlups, a_mlups in MESHES:
        P = inputs.scaled(inputs.exchanger3d(), dims, nsteps=nsteps).replace(collision="MRT")
        th = torch.from_numpy(inputs.theta_grf(P, 0).reshape(-1)).cuda()
        with Solver(P, th, stream=torch.cuda.Stream()) as s:
            for _ in range(args.warmup):
                s.run()
            s.profile(True)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                s.run()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            prof = s.profile_read()
            s.profile(False)
            N = s.N
        (n_p, ms_p), (n_r, ms_r), (n_a, ms_a) = prof["primal"], prof["recompute"], prof["adjoint"]
        prim = N / ((ms_p + ms_r) / max(n_p + n_r, 1) / 1e3) / 1e6
        adj = N / (ms_a / max(n_a, 1) / 1e3) / 1e6
        rows.append({"mesh": name, "dims": list(dims), "nodes": N, "dof": N * 26,
                     "primal_MLUPS": prim, "adjoint_MLUPS": adj, "adjoint_over_primal_time": prim / adj,
                     "solve_MLUPS": 2.0 * N * nsteps * args.steps / wall / 1e6,
                     "paper_m2090_primal_MLUPS": p_mlups, "paper_m2090_adjoint_MLUPS": a_mlups})
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"metric": "primal and adjoint MLUPS on the paper's scaling meshes",
                      "workload": "meshes", "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "primal_steps": nsteps, "dtype": "f32",
                      "data": "synthetic", "rows": rows}), flush=True)
    return 0


def run_paper(args):
    """The paper's empty mixer and exchanger channels (Tab. tab:cases) for the
    iterations Tab. tab:results lists: J and outlet statistics against the
    printed Empty rows, and the primal MLUPS of the run."""
    import torch
    from paper_1501_04741_gb300.albm import Solver
    from tests.test_gpu_paper_tables import _golden, outlet_stats
    rows = []
    gold = _golden()
    for case, P in (("mixer", inputs.paper_mixer_empty()), ("exchanger", inputs.paper_exchanger_empty())):
        th = torch.zeros(P.n_nodes, dtype=torch.float32, device="cuda")
        with Solver(P, th) as s:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.primal_step(P.nsteps)
            J = s.objective()
            dt = time.perf_counter() - t0
            um, us, Tm, Ts = outlet_stats(s, P)
        ref = gold[case]
        rows.append({"case": case, "dims": list(P.dims), "steps": P.nsteps, "objective": P.objective,
                     "J": J, "J_paper": ref["J"], "u_mean": um, "u_sd": us, "u_paper": ref["u"],
                     "T_mean": Tm, "T_sd": Ts, "T_paper": ref["T"],
                     "primal_MLUPS": P.n_nodes * P.nsteps / dt / 1e6})
        print(json.dumps(rows[-1]), flush=True)
    # the fin study of Sec. 4.2 on the exchanger (row "Fins")
    from tests.test_gpu_paper_tables import _golden_fins, run_fins
    P = inputs.paper_exchanger_empty()
    fins = []
    for n, w in inputs.fin_sweep(P):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, (um, us, Tm, Ts) = run_fins(P, n, w)
        dt = time.perf_counter() - t0
        fins.append({"fins": n, "width": w, "J": J, "u_mean": um, "u_sd": us, "T_mean": Tm,
                     "T_sd": Ts, "primal_MLUPS": P.n_nodes * P.nsteps / dt / 1e6})
    best = max(fins, key=lambda r: r["J"])
    fref = _golden_fins()
    print(json.dumps({"metric": "paper empty channels and fin study vs Tab. tab:results",
                      "workload": "paper", "unit": UNIT, "n_gpus": 1, "dtype": "f32",
                      "data": "synthetic", "rows": rows, "fins": fins,
                      "fins_best": best, "fins_paper": fref}), flush=True)
    return 0


def run_mma(args):
    """MMA design iterations (Sec. 3.3) on the full exchanger: per iteration
    the 1000 + 1000-step unsteady solve and one MMA update of theta."""
    import torch
    from paper_1501_04741_gb300.albm import Solver
    P = inputs.exchanger3d()
    theta = inputs.theta_grf(P, 0)
    mask = inputs.design_mask(P).reshape(-1).astype(np.uint8)
    iters = max(1, args.steps)
    stream = torch.cuda.Stream()
    s = Solver(P, torch.from_numpy(theta.reshape(-1)).cuda(), stream=stream)
    N = s.N
    s.set_design(mask)
    s.mma_reset()
    for _ in range(args.warmup):
        s.run()
        s.mma_update(True, 0.2)
    torch.cuda.synchronize()
    hist = []
    t0 = time.perf_counter()
    t_upd = 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(iters):
        s.run()
        hist.append(s.objective())            # synchronises
        e0.record(stream)
        s.mma_update(True, 0.2)               # the update kernel (and the reset's small memsets)
        e1.record(stream)
        e1.synchronize()
        t_upd += e0.elapsed_time(e1) / 1e3
    wall = time.perf_counter() - t0
    s.close()
    # per design node: theta, x^{k-1}, L, U read and written, x^{k-2} written,
    # the FP64 gradient read; the design mask is read for every node
    upd_bytes = int(mask.sum()) * (4 * 2 * 4 + 4 + 8) + N
    print(json.dumps({
        "metric": "MMA design iterations, primal+adjoint MLUPS", "workload": "mma",
        "value": 2.0 * N * P.nsteps * iters / wall / 1e6, "unit": UNIT, "n_gpus": 1,
        "steps": iters, "warmup": args.warmup, "ms_per_step": 1e3 * wall / iters,
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "mma", "lattice": P.lattice, "collision": P.collision,
                   "dims": list(P.dims), "objective": P.objective, "steps_per_solve": P.nsteps,
                   "move": 0.2, "design_nodes": int(mask.sum())},
        "J_per_iteration": hist,
        "update_ms": 1e3 * t_upd / iters,
        "update_GB_s": upd_bytes / (t_upd / iters) / 1e9}), flush=True)
    return 0


def run_profile_case(args):
    """A few launches of each kernel on a lattice that still exceeds L2."""
    import torch
    from paper_1501_04741_gb300.albm import Solver
    # 6 steps with a 2-step objective window: primal launches 1-4 and
    # adjoint launches 3-6 are the no-objective kernels that dominate a long
    # horizon, the others carry the objective terms
    base = inputs.exchanger3d() if args.workload == "exchanger3d" else inputs.mixer3d()
    P = inputs.scaled(base, (256, 128, 64), nsteps=6, obj_window=2, ckpt_every=1,
                      precision=args.precision, kernel=args.kernel)
    th = torch.from_numpy(inputs.theta_uniform(P, 0).reshape(-1)).cuda()
    with Solver(P, th) as s:
        s.primal_step(P.nsteps)
        s.adjoint_step(P.nsteps)
        J = s.objective()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": f"{args.workload} 256x128x64", "precision": args.precision,
                      "J": J}))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nsteps", type=int, default=0, help="override the 10000-step horizon")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--mem-budget", type=float, default=0.0)
    ap.add_argument("--kernel", default="auto", choices=["auto", "plain", "tiles", "async"],
                    help="step kernels: tile-staged when nx allows (auto), per node, or staged")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="mixer3d",
                    choices=["mixer3d", "exchanger3d", "batch64", "serve", "oneshot", "meshes",
                             "paper", "mma", "precision"])
    ap.add_argument("--count", type=int, default=0, help="batch64: instances (default 64)")
    ap.add_argument("--size-scale", type=float, default=1.0, help="batch64: linear size factor")
    ap.add_argument("--serve-rates", default="1,10,100", help="serve: arrival rates per second")
    ap.add_argument("--serve-count", type=int, default=100, help="serve: requests per rate")
    ap.add_argument("--max-nodes", type=float, default=1e6, help="serve: largest request")
    ap.add_argument("--no-extras", action="store_true",
                    help="mixer3d: skip the exchanger precision, serving and batch64 records")
    ap.add_argument("--tick", type=int, default=200, help="serve: most steps per request per tick")
    ap.add_argument("--oneshot-iters", type=int, default=200,
                    help="oneshot: one-shot iterations per timed step")
    ap.add_argument("--profile-case", action="store_true",
                    help="run the small ncu case instead: the mixer3d (or, with --workload "
                         "exchanger3d, the exchanger) physics on 256x128x64, 6 primal + 6 "
                         "adjoint steps, objective over the last 2 (277 MB per FP32 mixer "
                         "state, > L2)")
    ap.add_argument("--cpu-baseline-only", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args(argv)
    if args.cpu_baseline_only:
        print(json.dumps(cpu_baseline_local(workload(args))), flush=True)
        return 0
    if args.profile_case:
        return run_profile_case(args)
    if args.workload == "batch64":
        return run_batch64(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "oneshot":
        return run_oneshot(args)
    if args.workload == "meshes":
        return run_meshes(args)
    if args.workload == "paper":
        return run_paper(args)
    if args.workload == "mma":
        return run_mma(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
