"""Benchmark of the adaptive-parareal hot path on GB300.

Workload: Kolmogorov flow b = (sin 4y, 0, 0), eps = 0.01, 64^3 periodic grid, T = 10,
N = 64 subintervals of 157 fine implicit-Euler steps (dt = 9.952e-4), 32 snapshots per
window, POD rank <= 16, seeded smooth forcing |k| <= 4 (synthetic inputs, see pr_inputs).

A step is one parareal iteration over all 64 subintervals: the fine sweep (one persistent
launch), level-1 and level-2 POD with Galerkin matrices, the sequential augmented coarse
sweep and the convergence check.  value = fine grid-point-steps propagated per second of
whole-iteration time (GDOF-steps/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
    python bench.py --impl reference      # the FP64 CPU oracle on a bounded sample
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


def workload(subintervals: int = 0):
    """The 64^3 Kolmogorov workload; `subintervals` > 0 keeps DeltaT (and so the 157 fine
    steps per subinterval) and shortens the horizon, for small profiling captures."""
    import dataclasses
    import pr_inputs as pi
    w = pi.KOL_64
    if subintervals > 0 and subintervals != w.n_sub:
        w = dataclasses.replace(w, name=f"{w.name}_first{subintervals}", n_sub=subintervals,
                                T=w.T * subintervals / w.n_sub)
    return w


def config_dict(w, precision):
    return {
        "workload": f"{w.name}: Kolmogorov sin(4y), eps=0.01, 64^3, T=10, N=64 subintervals x 157 "
                    f"fine steps, 32 snapshots/window, POD rank<=16, seeded forcing |k|<=4",
        "precision": "fp32-delta fine, fp64 state/reduced" if precision == "fp32" else "fp64",
        "step": "one parareal iteration k=1 over all 64 subintervals: fine sweep + level-1/2 POD "
                "+ Galerkin + sequential coarse sweep + convergence check",
        "l2": "no flush; working set ~9 GB (snapshots, bases, states) >> 129 MB L2",
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
CPU_SAMPLE_CODE = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle as O
import pr_inputs as pi
w = pi.KOL_64
prm = O.derive_params(w)
op = O.make_operator(w)
u = w.u0()
fine_steps = int(sys.argv[2])
t = time.perf_counter()
_, W = O.fine_propagate(op, u, prm.T0, fine_steps, prm.dt, 1, fine_steps + 1, tol=prm.lin_tol)
t_step = (time.perf_counter() - t) / fine_steps
Wfull = np.concatenate([W] * ((prm.n_s + W.shape[1] - 1) // W.shape[1]), axis=1)[:, :prm.n_s]
Wfull = Wfull + 1e-3 * np.random.default_rng(0).standard_normal(Wfull.shape)
t = time.perf_counter()
R1, m1, _ = O.pod_mode(Wfull, prm.gamma2, prm.m_cap, prm.tau)
t_pod1 = time.perf_counter() - t
t = time.perf_counter()
R2, m2, _ = O.pod_mode(np.concatenate([R1, R1[:, ::-1], R1 * 0.5 + 1e-3], axis=1), prm.gamma3, prm.m_cap, prm.tau)
t_pod2 = time.perf_counter() - t
t = time.perf_counter()
V, _ = O.augment(R2, u)
a, _ = O.coarse_propagate(op, V, u, prm.T0, prm.Lc, prm.dT)
b, _ = O.coarse_propagate(op, V, u, prm.T0, prm.Lc, prm.dT)
t_coarse = time.perf_counter() - t
t_iter = prm.N * (prm.S * t_step + t_pod1 + t_pod2 + t_coarse)
dofs = prm.N * prm.S * w.Ng
print(json.dumps(dict(t_step=t_step, t_pod1=t_pod1, t_pod2=t_pod2, t_coarse=t_coarse,
                      t_iter=t_iter, value=dofs / t_iter / 1e9, fine_steps=fine_steps)))
"""


def cpu_oracle_sample(fine_steps: int = 4):
    """Time the FP64 oracle, single-threaded, on a bounded sample of the workload and scale
    it to one parareal iteration over all 64 subintervals."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    t0 = time.time()
    r = subprocess.run([sys.executable, "-c", CPU_SAMPLE_CODE, ROOT, str(fine_steps)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    d["wall"] = time.time() - t0
    return d


def cpu_baseline_obj(d):
    return {"value": d["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"64^3 FP64 numpy oracle, 1 thread: {d['fine_steps']} fine implicit-Euler "
                       f"steps (BiCGStab) + one level-1 POD (32 snapshots) + one level-2 POD + one "
                       f"augmented coarse update, scaled to one iteration over 64 subintervals x "
                       f"157 steps (measured {d['wall']:.1f} s)")}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    w = workload()
    times = []
    for i in range(args.warmup + args.steps):
        d = cpu_oracle_sample(2)
        if i >= args.warmup:
            times.append(d)
    val = statistics.median(x["value"] for x in times)
    ms = statistics.median(x["t_iter"] for x in times) * 1e3
    cb = cpu_baseline_obj(times[0])
    cb["value"] = val
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, "fp64"),
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def fine_bytes_per_dof_step(w_bytes: int, lin_iters: float, dM: int, has_f: bool) -> float:
    """Algorithmic DRAM bytes of the fused fine sweep per grid point and fine step:
    setup reads the state (8 B: FP64, or the hi + lo float pair of the FP32 mode) and
    delta (w), writes the state (8 B), r and rhat (2w), reads f (w); each BiCGStab
    iteration streams 17 words (phase 1: r, p', v', rhat in, p, v out; phase 2: r, v in,
    t out; phase 3: delta, p, r, v, t, rhat in, delta, r out); one FP64 snapshot value
    every dM steps."""
    return 16 + 3 * w_bytes + (w_bytes if has_f else 0) + lin_iters * 17 * w_bytes + 8 / dM


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
    w = workload(args.subintervals)
    prec = bd.PR_FP32 if args.precision == "fp32" else bd.PR_FP64
    s = bd.Parareal.from_workload(w, precision=prec)
    st = s.stream
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    if args.mode == "fine":
        # profiling mode: fine sweeps of iteration 1 only, no JSON line
        for _ in range(args.warmup + args.steps):
            s.fine_sweep(1)
            s.pod_update(1)
            s.coarse_sweep(1)
            s.check(1)
            s.rewind()
        torch.cuda.synchronize()
        print(json.dumps({"mode": "fine", "workload": w.name, "launches": bd.launch_count()}))
        return 0
    s.iterate(1)                      # first iteration: the state every timed step repeats
    dofs_per_step = w.n_sub * s.S * w.Ng

    def barrier():
        if dist is not None:
            dist.barrier()

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

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    tot, mx = s.lin_stats()
    lin_mean = float(tot.sum()) / (w.n_sub * s.S)
    sampler = ClockSampler(local)
    sampler.start()
    fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = bd.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0.record(st)
    for i in range(args.steps):
        one_step(*fe[i])
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    launches = bd.launch_count() - l0
    clocks = sampler.stop()
    t_ms = e0.elapsed_time(e1)
    fine_ms = statistics.mean(a.elapsed_time(b) for a, b in fe)
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
    bpd = fine_bytes_per_dof_step(wb, lin_mean, s.dM, True)
    achieved = bpd * dofs_per_step / (fine_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = recorded_traffic(args.precision)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": config_dict(w, args.precision),
        "e2e": {"value": e2e_val, "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(U0.nbytes), "d2h_bytes_per_step": int(Uout.nbytes)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None, "traffic": traffic,
                     "kernel": "fine_kernel (persistent BiCGStab fine sweep)",
                     "peak_source": peak_kind,
                     "bytes_per_dof_step": bpd, "lin_iters_per_step": lin_mean,
                     "fine_ms_per_launch": fine_ms},
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu:
        try:
            line["cpu_baseline"] = cpu_baseline_obj(cpu_oracle_sample(4))
        except Exception as e:  # report, do not hide the GPU number
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {e}"[:300]}
    if rank == 0 and args.solve:
        # wall time to rel. L2 <= 1e-6 against the sequential fine solution (eq. (error)),
        # the sequential fine solution itself timed as the plain GPU fine-only form
        s2 = bd.Parareal.from_workload(w, precision=prec)
        s2.set_initial(w.u0(), w.f())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2.compute_reference(True)
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        rep = s2.solve(1e-6, k_max=args.solve_kmax)
        line["solve"] = {"tol": 1e-6, "converged": bool(rep["converged"]), "iterations": rep["k"],
                         "wall_s": rep["t_total"], "max_err": rep["max_err"],
                         "t_fine": rep["t_fine"], "t_pod": rep["t_pod"],
                         "t_coarse": rep["t_coarse"], "t_iter0": rep["t_iter0"],
                         "sequential_fine_fp64_s": t_seq}
        s2.close()
    if rank == 0 and args.serve_requests > 0:
        s.close()
        line["serving"] = run_serving(bd, args.serve_requests, args.serve_rate, args.serve_tscale)
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
    ap.add_argument("--solve", type=int, default=1, help="also time a full solve to 1e-6")
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
