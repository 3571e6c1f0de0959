"""Benchmark of the adaptive-parareal hot path on GB300.

Default workload (--config c2): Kolmogorov flow b = (sin 4y, 0, 0), eps = 0.01, 64^3
periodic grid, T = 10, N = 64 subintervals of 157 fine implicit-Euler steps
(dt = 9.952e-4), 32 snapshots per window, POD rank <= 16, seeded smooth forcing |k| <= 4
(synthetic inputs, see pr_inputs).  --config c3 / c4 select the 128^3 ABC and the 256^3
perturbed-Kolmogorov workloads.

A step is one parareal iteration over all subintervals: the fine sweep (one persistent
launch), level-1 and level-2 POD with Galerkin matrices, the sequential augmented coarse
sweep and the convergence check.  value = fine grid-point-steps propagated per second of
whole-iteration time (GDOF-steps/s), in the precision of --precision (default: the FP32
Krylov mode).  Beside it, on rank 0 (--extras 1): the same iteration in FP64
(fp64_iteration), the wall time of pr_solve to rel. L2 <= 1e-6 against the sequential
fine solution in both modes (solve_fp32, solve_fp64; the plain FP64 GPU parareal is the
comparison the mixed-precision mode is measured against), the sequential fine solution
on the GPU in both precisions (the cost_seq form), and the FP64 CPU oracle on real
subinterval blocks, single-threaded and on all host cores (cpu_baseline).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64] [--config c2]
    python bench.py --impl reference      # the FP64 CPU oracle on bounded samples
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "parareal wall time at rel L2<=1e-6; fine GDOF-steps/s vs HBM roof; p50/p99 lat"
UNIT = "GDOF-steps/s"
FINE_SRC = os.path.join(ROOT, "paper_2601_10981_gb300", "csrc", "fine_kernel.cuh")


CONFIGS = {
    "c2": ("kolmogorov4_64_eps0.01_N64",
           "Kolmogorov sin(4y), eps=0.01, 64^3, T=10, N=64 subintervals x 157 fine steps, "
           "32 snapshots/window, POD rank<=16, seeded forcing |k|<=4"),
    "c3": ("abc128_eps0.005_N256",
           "ABC (1,1,1), eps=0.005, 128^3 (2,097,152 points, the paper's DOF count), T=50, "
           "N=256 subintervals x 391 fine steps, 64 snapshots/window, POD rank<=32"),
    "c4": ("kolmogorov8_256_pert_eps0.002_N128",
           "Kolmogorov sin(8y) + seeded divergence-free perturbation 0.05, eps=0.002, 256^3, T=20, "
           "N=128 subintervals x 625 fine steps, 16 snapshots/window, POD rank<=8"),
}


# context options per workload: the 128^3 and 256^3 workloads stream each iteration in
# waves of subintervals (the form whose workspace fits one GPU)
# (128^3: 38 subintervals x 8 CTAs fill all 304 co-resident CTA slots of the fine kernel,
# 6.12 s an iteration against 6.33 s with waves of 32 x 9 CTAs)
CONFIG_OPTS = {"c2": {}, "c3": {"wave": 38}, "c4": {"wave": 8}}


def workload(config: str = "c2", subintervals: int = 0):
    """The named workload; `subintervals` > 0 keeps DeltaT (and so the fine steps per
    subinterval) and shortens the horizon, for small profiling captures."""
    import dataclasses
    import pr_inputs as pi
    w = pi.WORKLOADS[CONFIGS[config][0]]
    if subintervals > 0 and subintervals != w.n_sub:
        w = dataclasses.replace(w, name=f"{w.name}_first{subintervals}", n_sub=subintervals,
                                T=w.T * subintervals / w.n_sub)
    return w


def config_dict(w, precision, config: str = "c2"):
    return {
        "workload": f"{w.name}: {CONFIGS[config][1]}",
        "precision": "fp32-delta fine, fp64 state/reduced" if precision == "fp32" else "fp64",
        "step": f"one parareal iteration k=1 over all {w.n_sub} subintervals: fine sweep + level-1/2 "
                "POD + Galerkin + sequential coarse sweep + convergence check",
        "l2": "no flush; working set (snapshots, bases, states) of several GB >> 129 MB L2",
    }


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def fine_src_hash() -> str:
    with open(FINE_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def recorded_traffic(precision: str):
    """DRAM bytes per fine-sweep launch from the committed ncu summary, if it was taken on
    the current fine-kernel source."""
    p = os.path.join(ROOT, "profiles", "fine_sweep_kol64_traffic.txt")
    if not os.path.exists(p):
        return None
    h = fine_src_hash()
    for line in open(p):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == "traffic" and parts[1] == precision and parts[3] == h:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(x: float, dist, device) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- CPU oracle
# The oracle legs run the FP64 numpy oracle on real blocks of the workload: iteration 0 once
# (untimed), then, per sample, the fine propagator with snapshots and the level-1 POD of a
# block of consecutive subintervals (one process per subinterval, all host cores), the
# level-2 POD of each subinterval's real neighbours and the sequential augmented coarse
# updates of the block, i.e. one parareal iteration restricted to the block.

def _oracle_threads_env():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def _oracle_fine_pod(args):
    """Worker: the fine propagator with snapshots over the first `steps` fine steps of
    subinterval n_idx, then POD_Mode of that window (level 1)."""
    wname, n_idx, u_start, steps = args
    import oracle as O
    w = _workload_by_name(wname)
    prm = O.derive_params(w)
    op = O.make_operator(w)
    t = time.perf_counter()
    F, W = O.fine_propagate(op, u_start, prm.T0 + n_idx * prm.DeltaT, steps, prm.dt, prm.dM,
                            steps // prm.dM + 1, tol=prm.lin_tol)
    t_f = time.perf_counter() - t
    t = time.perf_counter()
    R1, m1, _ = O.pod_mode(W, prm.gamma2, prm.m_cap, prm.tau)
    return n_idx, F, R1, m1, t_f, time.perf_counter() - t


def _workload_by_name(name):
    import pr_inputs as pi
    return pi.WORKLOADS[name]


class OracleBlocks:
    """Iteration 1 of the oracle restricted to blocks of B consecutive subintervals, each
    propagated over the first 1/frac of its window (a bounded sample)."""

    def __init__(self, w, frac: int = 4):
        import oracle as O
        self.O, self.w = O, w
        self.prm = O.derive_params(w)
        self.op = O.make_operator(w)
        self.steps = max(2 * self.prm.dM, self.prm.S // frac)
        t = time.perf_counter()
        self.U0, self.V0, _ = O.iteration0(w, self.prm, self.op)
        self.t_setup = time.perf_counter() - t

    def step(self, b0: int, B: int, pool=None):
        import numpy as np
        O, prm = self.O, self.prm
        N = prm.N
        idx = [(b0 + i) % N for i in range(B)]
        t0 = time.perf_counter()
        tasks = [(self.w.name, n, self.U0[n], self.steps) for n in idx]
        res = pool.map(_oracle_fine_pod, tasks) if pool is not None else list(map(_oracle_fine_pod, tasks))
        t_par = time.perf_counter() - t0
        F = {r[0]: r[1] for r in res}
        R1 = {r[0]: r[2] for r in res}
        # level-2 POD of eq. (W^k_n) at k = 1 from the block's real neighbours (the missing
        # previous-iteration block is V0, reading R8), then the sequential coarse updates
        t = time.perf_counter()
        shape = self.U0[0].shape
        U = F[idx[0]]
        for j in range(1, B):
            n, left = idx[j], idx[j - 1]
            R2, _, _ = O.pod_mode(np.concatenate([R1[left], R1[n], self.V0], axis=1), prm.gamma3,
                                  prm.m_cap, prm.tau)
            V, _ = O.augment(R2, U, prm.aug_tol)
            t_n = prm.T0 + n * prm.DeltaT
            g_new, _ = O.coarse_propagate(self.op, V, U, t_n, prm.Lc, prm.dT)
            g_old, _ = O.coarse_propagate(self.op, V, self.U0[n], t_n, prm.Lc, prm.dT)
            U = (g_new + F[n].reshape(-1) - g_old).reshape(shape)
        t_seq = time.perf_counter() - t
        wall = time.perf_counter() - t0
        dofs = B * self.steps * self.w.Ng
        return {"wall_s": wall, "value": dofs / wall / 1e9, "subintervals": B,
                "fine_steps_each": self.steps, "t_parallel_s": t_par, "t_sequential_s": t_seq,
                "t_fine_mean_s": sum(r[4] for r in res) / B, "t_pod1_mean_s": sum(r[5] for r in res) / B}


def oracle_pool(workers: int):
    """Process pool for the oracle (spawn: safe after CUDA initialisation)."""
    import multiprocessing as mp
    _oracle_threads_env()
    return mp.get_context("spawn").Pool(workers)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_measure(w):
    """The oracle on real blocks of the workload: single-threaded (two consecutive
    subintervals, one process) and on all host cores (one subinterval per core)."""
    _oracle_threads_env()
    cores = host_cores()
    t = time.time()
    ob = OracleBlocks(w)
    one = ob.step(0, 2, None)
    with oracle_pool(cores) as pool:
        allc = ob.step(2, min(cores, ob.prm.N), pool)
    return {"value": allc["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{w.name}: FP64 numpy oracle, iteration 1 restricted to {allc['subintervals']} "
                       f"consecutive subintervals, each over the first {ob.steps} of its "
                       f"{ob.prm.S} fine steps (fine propagator with snapshots + level-1 POD one "
                       f"process per subinterval on {cores} cores, then level-2 POD of the real "
                       f"neighbours and the sequential augmented coarse updates); value = "
                       f"grid-point-steps of the sample / its wall time; iteration 0 computed "
                       f"first, untimed ({ob.t_setup:.1f} s); whole leg {time.time() - t:.1f} s"),
            "all_cores": allc,
            "single_thread": dict(one, cores=1,
                                  sample="the same on 2 consecutive subintervals in one process")}


def _oracle_steps_worker(args):
    """Worker: `steps` fine steps of the oracle from a seeded state (timing only)."""
    wname, steps, seed = args
    import numpy as np
    import oracle as O
    import pr_inputs as pi
    w = _workload_by_name(wname)
    prm = O.derive_params(w)
    op = O.make_operator(w)
    u = pi.initial_state(w.n, seed=seed)
    t = time.perf_counter()
    O.fine_propagate(op, u, prm.T0, steps, prm.dt, tol=prm.lin_tol)
    return time.perf_counter() - t


def cpu_baseline_extrapolated(w, steps: int = 2):
    """The oracle on the 128^3 / 256^3 workloads, whose iteration 0 alone takes the oracle
    many minutes: measured per-fine-step time (one process per core, all cores at once),
    one level-1 POD of a window of the workload's size and one augmented coarse update,
    extrapolated to one iteration over all subintervals.  Labelled as an extrapolation."""
    import numpy as np
    import oracle as O
    import pr_inputs as pi
    _oracle_threads_env()
    cores = host_cores()
    t0 = time.time()
    prm = O.derive_params(w)
    op = O.make_operator(w)
    with oracle_pool(cores) as pool:
        t_par = time.perf_counter()
        per = pool.map(_oracle_steps_worker, [(w.name, steps, 10 + c) for c in range(cores)])
        t_par = time.perf_counter() - t_par
    t_step_core = statistics.median(per) / steps          # one fine step on one busy core
    # a window of the workload's snapshot count: seeded smooth fields (their POD has the
    # workload's sizes; the cost does not depend on the values)
    rng = np.random.default_rng(0)
    base = [pi.initial_state(w.n, seed=20 + j).reshape(-1) for j in range(4)]
    Wm = np.stack([base[j % 4] * (1.0 + 0.01 * j) + 1e-3 * rng.standard_normal(w.Ng)
                   for j in range(prm.n_s)], axis=1)
    t = time.perf_counter()
    R1, m1, _ = O.pod_mode(Wm, prm.gamma2, prm.m_cap, prm.tau)
    t_pod = time.perf_counter() - t
    del Wm
    u = pi.initial_state(w.n, seed=1).reshape(-1)
    t = time.perf_counter()
    V, _ = O.augment(R1, u, prm.aug_tol)
    O.coarse_propagate(op, V, u, prm.T0, prm.Lc, prm.dT)
    O.coarse_propagate(op, V, u, prm.T0, prm.Lc, prm.dT)
    t_coarse = time.perf_counter() - t
    # one iteration: N subintervals x S steps spread over the cores, then per subinterval a
    # level-1 and a level-2 POD (taken as two level-1 costs; parallel over the cores) and
    # the sequential coarse updates
    t_iter = (prm.N * prm.S * t_step_core / cores + 2 * prm.N * t_pod / cores + (prm.N - 1) * t_coarse)
    dofs = prm.N * prm.S * w.Ng
    return {"value": dofs / t_iter / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{w.name}: EXTRAPOLATED from measured FP64 numpy oracle times: {steps} fine "
                       f"steps in each of {cores} processes at once ({t_step_core:.2f} s a step and "
                       f"core), one level-1 POD of a {prm.n_s}-column window ({t_pod:.1f} s, m = {m1}), "
                       f"one augmented coarse update ({t_coarse:.1f} s); one iteration = N S steps over "
                       f"{cores} cores + 2 N PODs over {cores} cores + (N - 1) sequential updates = "
                       f"{t_iter:.0f} s; whole leg {time.time() - t0:.0f} s"),
            "extrapolated": True}


def oracle_c1_solve():
    """The oracle end to end on the 16^3 ABC workload: sequential fine reference, then
    Algorithm 2 to rel. L2 <= 1e-6 against it (single thread)."""
    _oracle_threads_env()
    import oracle as O
    import pr_inputs as pi
    w = pi.ABC_16
    prm = O.derive_params(w)
    t = time.perf_counter()
    ref = O.sequential_fine(w, prm)
    t_ref = time.perf_counter() - t
    t = time.perf_counter()
    h = O.parareal(w, prm, k_max=w.n_sub, tol=1e-6, reference=ref, record=False)
    t_sol = time.perf_counter() - t
    return {"workload": w.name, "tol": 1e-6, "iterations": h["k"],
            "max_err": max(h["err"][-1]), "wall_s": t_sol, "sequential_fine_s": t_ref,
            "cores": 1}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    _oracle_threads_env()
    w = workload(args.config)
    if args.config != "c2":
        # the oracle's iteration 0 alone takes many minutes at 128^3 / 256^3: one
        # extrapolated measurement stands for the run (see its sample text)
        cb = cpu_baseline_extrapolated(w)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config_dict(w, "fp64", args.config), "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0
    cores = host_cores()
    c1 = oracle_c1_solve()
    ob = OracleBlocks(w)
    B = min(cores, ob.prm.N)
    times = []
    with oracle_pool(cores) as pool:
        for i in range(args.warmup + args.steps):
            d = ob.step((i * B) % ob.prm.N, B, pool)
            if i >= args.warmup:
                times.append(d)
    val = statistics.median(x["value"] for x in times)
    ms = statistics.median(x["wall_s"] for x in times) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, "fp64"),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": (f"each step: iteration 1 of the FP64 numpy oracle restricted to "
                                        f"{B} consecutive subintervals of {w.name}, each over the first "
                                        f"{ob.steps} of its {ob.prm.S} fine steps (fine propagator with "
                                        f"snapshots + level-1 POD one process per subinterval, level-2 "
                                        f"POD of the real neighbours, sequential coarse updates); value "
                                        f"= grid-point-steps of the sample / its wall time; blocks "
                                        f"rotate over the {ob.prm.N} subintervals; iteration 0 untimed "
                                        f"({ob.t_setup:.1f} s)")},
            "oracle_c1_solve": c1,
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def fine_bytes_per_dof_step(w_bytes: int, lin_iters: float, dM: int, has_f: bool, has_pert: bool = False) -> float:
    """Algorithmic DRAM bytes of the fused fine sweep per grid point and fine step:
    setup reads the state (8 B: FP64, or the hi + lo float pair of the FP32 mode) and
    delta (w), writes the state (8 B), r and rhat (2w), reads f (w); each BiCGStab
    iteration streams 17 words (phase 1: r, p', v', rhat in, p, v out; phase 2: r, v in,
    t out; phase 3: delta, p, r, v, t, rhat in, delta, r out); one FP64 snapshot value
    every dM steps.  A stored velocity perturbation adds its three words at every stencil
    march: the setup's and two per BiCGStab iteration."""
    pert = 3 * w_bytes * (1 + 2 * lin_iters) if has_pert else 0.0
    return 16 + 3 * w_bytes + (w_bytes if has_f else 0) + lin_iters * 17 * w_bytes + 8 / dM + pert


def serving_sample(n_req: int, rate: float, t_scale: float, seed: int = 5):
    """The first n_req requests of the mixed Poisson request stream (grids 32^3..128^3, ABC
    or Kolmogorov flows, eps log-uniform in [0.002, 0.05], N in {16, 32, 64}; see
    pr_inputs.serving_stream) with their horizons T scaled by t_scale, so that the whole
    sample is served in about a minute."""
    import dataclasses
    import pr_inputs as pi
    reqs = pi.serving_stream(n_req, rate, seed)
    for r in reqs:
        r["workload"] = dataclasses.replace(r["workload"], T=r["workload"].T * t_scale)
    return reqs


def run_serving(bd, n_req: int, rate: float, t_scale: float, tol: float = 1e-6):
    """Serve the sample in real time: requests are submitted at their arrival times, the
    server steps whenever it holds work; latency = finish - arrival."""
    import math
    import numpy as np
    reqs = serving_sample(n_req, rate, t_scale)
    srv = bd.Server()
    ids, arrival, finish, work = {}, {}, {}, {}
    nxt = 0
    t0 = time.perf_counter()
    active = pending = 0
    while len(finish) < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt]["arrival"] <= now:
            w = reqs[nxt]["workload"]
            ids[nxt] = srv.submit(w, w.u0(), None, tol=tol, precision=bd.PR_FP32)
            arrival[nxt] = reqs[nxt]["arrival"]
            nxt += 1
        if active == 0 and pending == 0 and nxt < len(reqs) and len(ids) == len(finish):
            time.sleep(max(0.0, reqs[nxt]["arrival"] - (time.perf_counter() - t0)))
            continue
        active, pending = srv.step()
        now = time.perf_counter() - t0
        for i, rid in ids.items():
            if i in finish:
                continue
            st, k, _ = srv.query(rid)
            if st in (bd.PR_REQ_DONE, bd.PR_REQ_FAILED):
                finish[i] = now
                w = reqs[i]["workload"]
                S = math.ceil(w.T / w.n_sub / w.dt - 1e-9)
                # iteration 0 (one subinterval) + iterations 1..k over N-k+1 subintervals
                work[i] = (S + sum(w.n_sub - kk + 1 for kk in range(1, k + 1)) * S) * w.n ** 3 \
                    if st == bd.PR_REQ_DONE else 0
                if st == bd.PR_REQ_FAILED:
                    work[i] = -1
    makespan = max(finish.values())
    failed = sum(1 for v in work.values() if v < 0)
    lat = np.array([finish[i] - arrival[i] for i in finish])
    srv.close()
    sizes = sorted({r["workload"].n for r in reqs})
    return {
        "requests": len(reqs), "failed": failed, "rate_per_s": rate,
        "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
        "throughput_req_per_s": len(reqs) / makespan,
        "gdof_steps_per_s": sum(v for v in work.values() if v > 0) / makespan / 1e9,
        "makespan_s": makespan, "grids": sizes, "tol_increment": tol, "precision": "fp32",
        "sample": f"first {len(reqs)} requests of the seeded Poisson stream (rate {rate}/s), "
                  f"horizons T x {t_scale}",
    }


def _timed_iterations(s, st, steps, warmup, torch, barrier=None, wave=False):
    """Repeat iteration 1 from the same iterate `steps` times after `warmup` untimed
    repetitions; CUDA events on the context stream around the whole loop and around each
    fine sweep.  Returns (total ms, mean fine-kernel ms per iteration, launches).  In wave
    mode the fine-sweep phase holds the whole streamed iteration, so the fine-kernel time
    is the library's own event pairs around each wave's fine launch (pr_get_fine_ms), read
    after each step (one host synchronisation per iteration of several seconds)."""
    from paper_2601_10981_gb300 import binding as bd

    def one_step(ev_f0=None, ev_f1=None):
        s.rewind()
        if ev_f0 is not None:
            ev_f0.record(st)
        s.fine_sweep(1)
        if ev_f1 is not None:
            ev_f1.record(st)
        s.pod_update(1)
        s.coarse_sweep(1)
        return s.check(1)

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wave_fine = []
    l0 = bd.launch_count()
    if barrier is not None:
        barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for i in range(steps):
        one_step(*fe[i])
        if wave:
            wave_fine.append(s.fine_ms()[0])
    e1.record(st)
    torch.cuda.synchronize()
    if barrier is not None:
        barrier()
    launches = bd.launch_count() - l0
    if wave:
        fine_ms = statistics.mean(wave_fine)
    else:
        fine_ms = statistics.mean(a.elapsed_time(b) for a, b in fe)
    return e0.elapsed_time(e1), fine_ms, launches


def _solve_leg(bd, w, prec, torch, tol=1e-6, k_max=0):
    """Wall time of pr_solve to rel. L2 <= tol against the GPU's FP64 sequential fine
    solution (eq. (error)), with the sequential fine solution itself timed (the cost_seq
    form of Sec. 3.3) in FP64 and in the context's precision."""
    s = bd.Parareal.from_workload(w, precision=prec)
    s.set_initial(w.u0(), w.f())
    out = {}
    if prec == bd.PR_FP32:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.compute_reference(False)
        torch.cuda.synchronize()
        out["sequential_fine_fp32_s"] = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.compute_reference(True)
    torch.cuda.synchronize()
    out["sequential_fine_fp64_s"] = time.perf_counter() - t0
    rep = s.solve(tol, k_max=k_max)
    out.update({"tol": tol, "converged": bool(rep["converged"]), "iterations": rep["k"],
                "wall_s": rep["t_total"], "max_err": rep["max_err"], "t_fine": rep["t_fine"],
                "t_pod": rep["t_pod"], "t_coarse": rep["t_coarse"], "t_iter0": rep["t_iter0"],
                "lin_iters_mean": rep["lin_iters_mean"], "m1_max": rep["m1_max"],
                "m2_max": rep["m2_max"]})
    s.close()
    return out


def _large_leg(bd, config, torch, steps=2):
    """One parareal iteration of a large workload (wave mode), repeated `steps` times after
    one warm-up: time per iteration, the fine kernel's time and its fraction of the HBM
    roof (algorithmic bytes)."""
    try:
        w = workload(config)
        s = bd.Parareal.from_workload(w, precision=bd.PR_FP32, **CONFIG_OPTS[config])
        s.set_initial(w.u0(), w.f())
        t0 = time.perf_counter()
        s.iteration0()
        torch.cuda.synchronize()
        t_it0 = time.perf_counter() - t0
        s.iterate(1)
        tot, _ = s.lin_stats()
        lin_mean = float(tot.sum()) / (w.n_sub * s.S)
        t_ms, fine_ms, launches = _timed_iterations(s, s.stream, steps, 1, torch, wave=True)
        dofs = w.n_sub * s.S * w.Ng
        bpd = fine_bytes_per_dof_step(4, lin_mean, s.dM, w.f_seed is not None, w.flow.pert_seed > 0)
        peak, _ = measured_peaks()
        ws_gib = s.workspace_bytes() / 2**30
        s.close()
        del s
        torch.cuda.empty_cache()
        ms = t_ms / steps
        return {"workload": f"{w.name}: {CONFIGS[config][1]}", "precision": "fp32",
                "form": f"wave mode: each iteration streamed in waves of {CONFIG_OPTS[config]['wave']} subintervals",
                "ms_per_iteration": ms, "value": dofs / (ms * 1e-3) / 1e9, "unit": UNIT,
                "fine_kernel_ms_per_iteration": fine_ms,
                "fine_roofline_frac": bpd * dofs / (fine_ms * 1e-3) / 1e9 / peak if peak else None,
                "iteration0_s": t_it0, "steps": steps, "lin_iters_per_step": lin_mean,
                "workspace_gib": ws_gib, "launches_per_iteration": launches / steps,
                "fine_bytes_per_dof_step": bpd, "peak_gbs": peak}
    except Exception as e:   # report, do not hide the headline
        torch.cuda.empty_cache()
        return {"error": f"{type(e).__name__}: {e}"[:400]}


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2601_10981_gb300 import binding as bd
    w = workload(args.config, args.subintervals)
    prec = bd.PR_FP32 if args.precision == "fp32" else bd.PR_FP64
    copts = dict(CONFIG_OPTS[args.config])
    copts["gram_mode"] = {"auto": bd.PR_GRAM_AUTO, "df": bd.PR_GRAM_DF, "tensor": bd.PR_GRAM_TENSOR}[args.gram_mode]
    s = bd.Parareal.from_workload(w, precision=prec, **copts)
    st = s.stream
    s.set_initial(w.u0(), w.f())
    l_setup = bd.launch_count()
    s.iteration0()
    if args.mode == "fine":
        # profiling mode: iteration 1 repeated warmup + steps times, no timing; the launch
        # counts let an ncu capture skip to one chosen iteration (-s, -c)
        l_it0 = bd.launch_count()
        per = []
        for _ in range(args.warmup + args.steps):
            l0 = bd.launch_count()
            s.fine_sweep(1)
            s.pod_update(1)
            s.coarse_sweep(1)
            s.check(1)
            s.rewind()
            per.append(bd.launch_count() - l0)
        torch.cuda.synchronize()
        print(json.dumps({"mode": "fine", "workload": w.name, "launches": bd.launch_count(),
                          "launches_before_iterations": l_it0, "launches_setup": l_setup,
                          "launches_per_iteration": per}))
        return 0
    s.iterate(1)                      # first iteration: the state every timed step repeats
    dofs_per_step = w.n_sub * s.S * w.Ng

    def barrier():
        if dist is not None:
            dist.barrier()

    s.rewind()
    s.iterate(1)
    tot, mx = s.lin_stats()
    lin_mean = float(tot.sum()) / (w.n_sub * s.S)
    sampler = ClockSampler(local)
    sampler.start()
    t_ms, fine_ms, launches = _timed_iterations(s, st, args.steps, args.warmup, torch, barrier,
                                                wave=bool(copts.get("wave")))
    clocks = sampler.stop()
    t_max = reduce_max(t_ms, dist, "cuda")
    ms_per_step = t_max / args.steps
    value = ws * dofs_per_step / (ms_per_step * 1e-3) / 1e9

    # end to end through the C ABI: pinned host U^0 in, host U^1 out, every step
    U0 = torch.empty((w.n_sub + 1, w.Ng), dtype=torch.float64, pin_memory=True).numpy()
    Uout = torch.empty((w.n_sub + 1, w.Ng), dtype=torch.float64, pin_memory=True).numpy()
    s.rewind()
    U0[:] = s.interfaces().reshape(w.n_sub + 1, -1)
    s.iterate(1)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.rewind()
        s.set_interfaces(U0, 0)
        s.iterate(1)
        s.interfaces(out=Uout)   # device -> pinned host, no staging copy
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ms = reduce_max(e2e_ms, dist, "cuda")
    e2e_val = ws * dofs_per_step / (e2e_ms * 1e-3) / 1e9

    wb = 4 if args.precision == "fp32" else 8
    bpd = fine_bytes_per_dof_step(wb, lin_mean, s.dM, w.f_seed is not None, w.flow.pert_seed > 0)
    achieved = bpd * dofs_per_step / (fine_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = recorded_traffic(args.precision) if args.config == "c2" and not args.subintervals else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": config_dict(w, args.precision, args.config),
        "e2e": {"value": e2e_val, "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(U0.nbytes), "d2h_bytes_per_step": int(Uout.nbytes)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None, "traffic": traffic,
                     "traffic_source": ("DRAM bytes of one full-size fine launch from a committed "
                                        "ncu capture (profiles/fine_sweep_kol64_traffic.txt) of "
                                        "the same fine-kernel source; not measured in this run")
                                       if traffic is not None else None,
                     "kernel": "fine_kernel (persistent BiCGStab fine sweep)" + (
                         f", {copts['wave']} subintervals a launch (wave mode), time summed over the waves"
                         if copts.get("wave") else ""),
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                                    if peak_kind == "measured" else peak_kind,
                     "bytes_per_dof_step": bpd, "lin_iters_per_step": lin_mean,
                     "fine_ms_per_launch": fine_ms},
        "clocks": clocks,
    }
    s.close()
    del s
    if copts.get("wave"):
        line["config"]["form"] = (f"wave mode: each iteration streamed in waves of {copts['wave']} "
                                  f"subintervals (fine sweep, level-1/2 POD, Galerkin, coarse sweep)")
    if rank == 0 and args.extras and args.config == "c2":
        if args.large:
            line["c3_iteration"] = _large_leg(bd, "c3", torch)
        # the same iteration in the paper's arithmetic (FP64 everywhere)
        if args.precision == "fp32":
            s64 = bd.Parareal.from_workload(w, precision=bd.PR_FP64)
            s64.set_initial(w.u0(), w.f())
            s64.iteration0()
            s64.iterate(1)
            k64 = max(1, min(3, args.steps))
            t64, f64, _ = _timed_iterations(s64, s64.stream, k64, 1, torch)
            line["fp64_iteration"] = {"ms_per_step": t64 / k64,
                                      "value": dofs_per_step / (t64 / k64 * 1e-3) / 1e9,
                                      "unit": UNIT, "fine_ms_per_launch": f64, "steps": k64}
            s64.close()
            del s64
        if args.solve:
            line["solve_fp32"] = _solve_leg(bd, w, bd.PR_FP32, torch, 1e-6, args.solve_kmax)
            line["solve_fp64"] = _solve_leg(bd, w, bd.PR_FP64, torch, 1e-6, args.solve_kmax)
            line["solve"] = dict(line["solve_fp32"] if args.precision == "fp32" else line["solve_fp64"])
    if rank == 0 and args.serve_requests > 0:
        line["serving"] = run_serving(bd, args.serve_requests, args.serve_rate, args.serve_tscale)
    if rank == 0 and not args.no_cpu:
        try:
            line["cpu_baseline"] = (cpu_baseline_measure(w) if args.config == "c2"
                                    else cpu_baseline_extrapolated(w))
        except Exception as e:  # report, do not hide the GPU number
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": host_cores(),
                                    "kind": "oracle", "sample": f"failed: {e}"[:300]}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--config", default="c2", choices=sorted(CONFIGS),
                    help="c2: 64^3 Kolmogorov (default); c3: 128^3 ABC; c4: 256^3 perturbed Kolmogorov")
    ap.add_argument("--extras", type=int, default=1,
                    help="also time the FP64 iteration and the solves (rank 0)")
    ap.add_argument("--gram-mode", default="auto", choices=["auto", "df", "tensor"],
                    help="FP32 mode's symmetric POD Grams: auto, double-float, or tensor cores (pr_opts.gram_mode)")
    ap.add_argument("--large", type=int, default=1,
                    help="with --config c2 and extras: also time one iteration of the 128^3 workload")
    ap.add_argument("--solve", type=int, default=1, help="also time full solves to 1e-6")
    ap.add_argument("--solve-kmax", type=int, default=0, help="0: N (finite termination)")
    ap.add_argument("--serve-requests", type=int, default=16,
                    help="requests of the mixed serving stream to serve (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=5.0)
    ap.add_argument("--serve-tscale", type=float, default=0.1)
    ap.add_argument("--subintervals", type=int, default=0,
                    help="profiling: first N subintervals of the workload (same per-subinterval size)")
    ap.add_argument("--mode", default="bench", choices=["bench", "fine"],
                    help="fine: run iterations without timing or JSON (for ncu captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
