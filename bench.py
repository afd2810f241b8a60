"""Benchmark of the STFAS/ADMM hot path on GB300.

A step is one ADMM iteration of Alg. 3 on the 2D letters workload (128^2 cells,
40 steps, fp32 state, one blurred disc/bar keyframe at t = T, metric with 6
Gaussian levels, r = 1e-3): the AO fixed point (2 warm-started
backward/projection/blend/forward passes), a fixed number of STFAS V-cycles,
the KKT metric and the multiplier update -- every row of the hot path.  The
metric is STFAS spacetime cells/s: fine cells x timesteps x V-cycles per step /
step time (the AO and KKT time counts against it).

Two more legs follow on rank 0 at N = 1 (skip with --no-solve / --serve 0):
* time to solution: stc_solve on the same workload from scratch, with the
  seconds until the relative KKT residual first reached 1e-4 (if it did within
  the iteration cap) and the paper's own stop (Alg. 3's density test);
* serving: the first --serve requests of the seeded Poisson stream
  (workloads.config_serving: n in {32..128}, N in [16, 48], 1-3 keyframes,
  4 requests/s) replayed in real time into stc_server with a 64 GB budget;
  p50/p99 time to solution (submit to result) and problems/hour.

--workload 3d runs the same step on the 3D workload instead (64^3 cells, 60
steps, two seeded ellipsoid-union keyframes at t = 30 and 60, metric with 5
levels); its time-to-solution leg solves that problem, and it has no serving leg.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference];
N > 1 under torchrun runs one independent replica per GPU (the method has no
data-path collective) and reports the summed throughput over the max time.
"""
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
sys.path.insert(0, ROOT)

N_CELLS, N_STEPS, VCYCLES = 128, 40, 4
WORKLOAD = ("2D smoke control, 128^2 cells, 40 timesteps, dt=1/40, fp32 state with fp64 reductions and "
            "fp64 coarsest level; Gaussian ball (sigma 0.08) at (0.5,0.25) to a seeded (2002) blurred "
            "(1.5 cells) mass-matched union of 3-5 discs/bars at t=T; r=1e-3, K=1, C_i with 6 Gaussian "
            "levels; one ADMM iteration per step = AO(2) + %d V(2,2)-cycles + KKT metric + lambda update"
            % VCYCLES)
WORKLOAD_3D = ("3D smoke control, 64^3 cells, 60 timesteps, dt=1/60, fp32 state with fp64 reductions and "
               "fp64 coarsest level; Gaussian ball (sigma 0.1) at (0.5,0.2,0.5); keyframes at t=30 and t=60, "
               "each a seeded (3003) union of 2-4 ellipsoids (semi-axes 0.05-0.2) blurred by 1 cell and "
               "mass-matched; r=1e-3, K=1, C_i with 5 Gaussian levels; one ADMM iteration per step = AO(2) + "
               "%d V(2,2)-cycles + KKT metric + lambda update" % VCYCLES)
ORACLE_STEPS = 2  # timesteps of the bounded oracle sample (same grid, same per-step work)
# dram__bytes_read.sum + dram__bytes_write.sum of one finest-level SCGS colour launch
# of this workload (ncu --set full, profiles/scgs_colour_finest_letters_128x40.md);
# to be re-measured whenever scgs_colour_kernel changes
SCGS_FINEST_DRAM_BYTES = 23257856 + 768


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# oracle sample (CPU): one ADMM iteration of the same grid on ORACLE_STEPS steps
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import sys, time, json
sys.path.insert(0, %r)
import numpy as np
from oracle import kkt, admm, stfas
from paper_1608_01102_gb300 import workloads
Ns, V = %d, %d
cfg = workloads.config_letters(128, 40)
star = cfg["keyframes"][40][0]
P = kkt.Problem(128, 128, Ns, 1.0 / 40, cfg["rho0"], r=1e-3, K=1.0, keyframes={Ns: (star, 1.0)},
                metric_levels=6)
v = np.zeros((Ns + 1, P.grid.F)); lam = np.zeros((Ns, P.grid.F)); x = kkt.zero_state(P)
t = time.perf_counter()
vs, rhos, _ = admm.ao(P, v, lam)
z = vs - lam / P.K
for c in range(V):
    stfas.stfas_cycle(P, x, z)
kkt.kkt_norm(P, x["v"])
el = time.perf_counter() - t
print(json.dumps({"seconds": el, "cells": 128 * 128 * Ns * V}))
"""


def oracle_sample():
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET % (ROOT, ORACLE_STEPS, VCYCLES)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["cells"] / d["seconds"], d["seconds"]


def cpu_baseline_obj(value):
    return {"value": value, "unit": "cells/s", "cores": 1, "kind": "oracle",
            "sample": "fp64 numpy oracle, one ADMM iteration (AO(2) + %d V-cycles + KKT metric) of the same "
                      "128^2 workload restricted to %d timesteps (per-timestep work of the V-cycle is the "
                      "same; the paper's cost is linear in N), single thread" % (VCYCLES, ORACLE_STEPS)}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.lines = []
        self.idx = str(gpu_index)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.idx, "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    vals = []
    secs = []
    for i in range(args.warmup + args.steps):
        v, s = oracle_sample()
        if i >= args.warmup:
            vals.append(v)
            secs.append(s)
    value = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": "STFAS spacetime cells/s", "value": value, "unit": "cells/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(secs) / len(secs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + "; oracle sample restricted to %d timesteps" % ORACLE_STEPS},
            "cpu_baseline": cpu_baseline_obj(value),
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_spec(name, workloads):
    """(cfg, n, nz, N, metric levels, description) of a bench workload."""
    if name == "3d":
        return workloads.config_3d(64, 60), 64, 64, 60, 5, WORKLOAD_3D
    return workloads.config_letters(N_CELLS, N_STEPS), N_CELLS, 0, N_STEPS, 6, WORKLOAD


def run_native(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1608_01102_gb300 import stc, workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # oracle baseline first, in a separate process, before heavy GPU work
    cpu = None
    d3 = args.workload == "3d"
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not d3:
        cpu = oracle_sample()[0]

    cfg, n, nz, N, levels, desc = workload_spec(args.workload, workloads)
    keys = cfg["keyframes"]
    prm = stc.default_params(n, n, N, precision=0, r=1e-3, K=1.0, metric_levels=levels, nz=nz)
    stream = torch.cuda.Stream(device=dev)
    G = stc.Problem(prm, cfg["rho0"], stream=stream.cuda_stream)
    G.set_keyframes(keys)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    warm = [False]

    def step():
        G.ao(2, warm=warm[0])      # Alg. 3 continues the AO fixed point after its first iteration
        warm[0] = True
        G.vcycle(VCYCLES)
        G.kkt_residual()
        G.admm_update()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    G.set_kernel_timing(True)
    n0 = G.launch_count()
    sampler = ClockSampler(local_rank)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches = G.launch_count() - n0
    k_ms, k_n = G.kernel_timing()
    G.set_kernel_timing(False)
    cells = n * n * (nz or 1) * N * VCYCLES
    ms, value = aggregate(sum(times) / len(times), cells, world, dev)

    # end to end through the public API with host buffers: keyframes up, forces down
    h2d = sum(a.nbytes for a, _ in keys.values())
    d2h = N * G.field_shape("U")[1] * 8
    e2e_times = []
    for _ in range(max(2, args.steps // 2)):
        t0 = time.perf_counter()
        G.set_keyframes(keys)
        step()
        u = G.forces()
        e2e_times.append(time.perf_counter() - t0)
    assert u.shape[0] == N
    e2e = {"value": world * cells / (sum(e2e_times) / len(e2e_times)), "unit": "cells/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # roofline of the dominant kernel: the finest-level SCGS colour sweep.  Per
    # timestep it reads v (F) and the residual rows at the colour's faces and
    # cells, and reads and writes the colour's unknowns: a colour holds 1/2^d of
    # the cells and (in 2D) half, (in 3D) a quarter of the faces of each direction
    F = G.field_shape("V")[1]
    C = G.field_shape("RHO")[1]
    if d3:
        bytes_per_launch = 4.0 * N * (2.5 * F + 0.75 * C)
    else:
        bytes_per_launch = 4.0 * N * (4 * F + 1.5 * C)
    peak, kind = _peaks()
    achieved = bytes_per_launch / (k_ms / k_n * 1e-3) / 1e9 if k_n else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "traffic": None if d3 else SCGS_FINEST_DRAM_BYTES,
            "kernel": ("scgs3_colour_kernel<float> (finest level)" if d3
                       else "scgs_colour_kernel<float> (finest level)"), "peak_kind": kind,
            "launches_timed": k_n, "avg_launch_us": 1e3 * k_ms / k_n if k_n else None,
            "algorithmic_bytes_per_launch": bytes_per_launch}
    if rank != 0:
        return
    line = {"metric": "STFAS spacetime cells/s", "value": value, "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "vcycles_per_step": VCYCLES,
                       "l2": "256 MiB buffer written between timed steps (outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof, "e2e": e2e, "gpu_launches": int(launches * world), "clocks": clocks}
    if cpu is not None:
        line["cpu_baseline"] = cpu_baseline_obj(cpu)
    G.close()
    if world == 1 and not args.no_solve:
        line["time_to_solution"] = solve_leg(stc, cfg, n, nz, N, levels, args.solve_max_admm)
    if world == 1 and args.serve > 0 and not d3:
        line["served"] = serve_leg(stc, workloads, args.serve, args.serve_max_admm)
    print(json.dumps(line), flush=True)


def aggregate(ms, cells, world, device):
    """Whole-job figures over `world` independent replicas: the step time is the
    slowest rank's (max over ranks), the throughput all ranks' cells per step
    over it.  Returns (ms, cells/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * cells / (ms * 1e-3)


def solve_leg(stc, cfg, n, nz, N, levels, max_admm):
    """stc_solve from scratch on the bench workload (fp32 policy)."""
    # eps_admm = 0 switches Alg. 3's density test off: the solve runs to the KKT tolerance or the cap
    prm = stc.default_params(n, n, N, precision=0, r=1e-3, K=1.0, metric_levels=levels, eps_admm=0.0, nz=nz)
    with stc.Problem(prm, cfg["rho0"]) as G:
        G.set_keyframes(cfg["keyframes"])
        t0 = time.perf_counter()
        rep = G.solve(tol=1e-4, max_admm=max_admm)
        wall = time.perf_counter() - t0
    return {"workload": "same as config.workload, solved from v = 0", "tol_kkt_rel": 1e-4,
            "max_admm": max_admm, "seconds": wall, "admm_iters": rep["admm_iters"],
            "vcycles": rep["vcycles"], "rejected_vcycles": rep["rejected_vcycles"],
            "kkt_rel": rep["kkt_rel"], "seconds_to_1e-4": rep["seconds_to_1e4"] if rep["seconds_to_1e4"] >= 0
            else None, "drho_last": rep["drho"],
            "paper_stop": {"rule": "Alg. 3: max_i ||rho_i - rho_i^last||_inf < max|rho_0|/100",
                           "admm_iters": rep["density_stop_iter"] or None,
                           "seconds": rep["seconds_to_density_stop"] if rep["seconds_to_density_stop"] >= 0
                           else None},
            "stopped_by": "kkt" if rep["kkt_rel"] <= 1e-4 else "iteration cap"}


def serve_leg(stc, workloads, count, max_admm, budget=64 << 30, workers=8, ao_trials=1):
    """Replay the first `count` requests of the seeded stream in real time.
    The requests try AO blend factors one at a time (ao_trials = 1): the
    concurrent solves already share the GPU, and speculative trials would
    compete with them."""
    reqs = workloads.config_serving(count)
    with stc.Server(budget, workers=workers) as S:
        t0 = time.perf_counter()
        tickets = []
        for r in reqs:
            delay = r["arrival"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            n, N = r["nx"], r["N"]
            prm = stc.default_params(n, n, N, precision=0, r=r["r"], K=1.0,
                                     metric_levels=max(0, int(np.floor(np.log2(n / 2)))), ao_trials=ao_trials)
            tickets.append(S.submit(prm, r["rho0"], r["keyframes"], tol=1e-4, max_admm=max_admm))
        infos = [S.wait(t) for t in tickets]
        peak = S.stats()["peak_bytes"]
    lat = [i["t_done"] - i["t_submit"] for i in infos if i["state"] == "done"]
    span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
    kk = [i["report"]["kkt_rel"] for i in infos if i["state"] == "done"]
    return {"requests": count, "completed": len(lat), "failed": sum(i["state"] == "failed" for i in infos),
            "p50_s": float(np.percentile(lat, 50)) if lat else None,
            "p99_s": float(np.percentile(lat, 99)) if lat else None,
            "problems_per_hour": 3600.0 * len(lat) / span if span > 0 else None,
            "reached_kkt_1e-4": sum(k <= 1e-4 for k in kk), "kkt_rel_median": float(np.median(kk)) if kk else None,
            "admm_iters_median": float(np.median([i["report"]["admm_iters"] for i in infos])),
            "budget_bytes": budget, "peak_bytes": peak, "workers": workers, "max_admm": max_admm,
            "stream": "workloads.config_serving(seed 4004): Poisson 4/s, n in {32,48,64,96,128}, N in [16,48], "
                      "1-3 disc/bar keyframes, fp32 policy, stop at KKT 1e-4 or Alg. 3's density test"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--solve-max-admm", type=int, default=100)
    ap.add_argument("--serve", type=int, default=24, help="serving requests to replay (0: skip)")
    ap.add_argument("--serve-max-admm", type=int, default=50)
    ap.add_argument("--workload", default="letters", choices=["letters", "3d"],
                    help="letters: the 2D 128^2 x 40 workload (default); 3d: 64^3 x 60")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_native(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
