"""Benchmark of the STFAS/ADMM hot path on GB300.

A step is one ADMM iteration of Alg. 3 on the 2D letters workload (128^2 cells,
40 steps, fp32 state, one blurred disc/bar keyframe at t = T, metric with 6
Gaussian levels, r = 1e-3): the AO fixed point (2 forward/backward/projection
passes), a fixed number of STFAS V-cycles, the KKT metric and the multiplier
update -- every row of the hot path.  The metric is STFAS spacetime cells/s:
fine cells x timesteps x V-cycles per step / step time (the AO and KKT time
counts against it).

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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS, N_STEPS, VCYCLES = 128, 40, 4
WORKLOAD = ("2D smoke control, 128^2 cells, 40 timesteps, dt=1/40, fp32 state with fp64 reductions and "
            "fp64 coarsest level; Gaussian ball (sigma 0.08) at (0.5,0.25) to a seeded (2002) blurred "
            "(1.5 cells) mass-matched union of 3-5 discs/bars at t=T; r=1e-3, K=1, C_i with 6 Gaussian "
            "levels; one ADMM iteration per step = AO(2) + %d V(2,2)-cycles + KKT metric + lambda update"
            % VCYCLES)
ORACLE_STEPS = 2  # timesteps of the bounded oracle sample (same grid, same per-step work)


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


def run_native(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1608_01102_gb300 import stc, workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    # oracle baseline first, in a separate process, before heavy GPU work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample()[0]

    cfg = workloads.config_letters(N_CELLS, N_STEPS)
    star = cfg["keyframes"][N_STEPS][0]
    prm = stc.default_params(N_CELLS, N_CELLS, N_STEPS, precision=0, r=1e-3, K=1.0, metric_levels=6)
    stream = torch.cuda.Stream(device=dev)
    G = stc.Problem(prm, cfg["rho0"], stream=stream.cuda_stream)
    G.set_keyframes({N_STEPS: (star, 1.0)})
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def step():
        G.ao(2)
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
    ms = sum(times) / len(times)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    cells = N_CELLS * N_CELLS * N_STEPS * VCYCLES
    value = world * cells / (ms * 1e-3)

    # end to end through the public API with host buffers: keyframe up, forces down
    h2d = star.nbytes
    d2h = N_STEPS * G.field_shape("U")[1] * 8
    e2e_times = []
    for _ in range(max(2, args.steps // 2)):
        t0 = time.perf_counter()
        G.set_keyframes({N_STEPS: (star, 1.0)})
        step()
        u = G.forces()
        e2e_times.append(time.perf_counter() - t0)
    assert u.shape[0] == N_STEPS
    e2e = {"value": world * cells / (sum(e2e_times) / len(e2e_times)), "unit": "cells/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # roofline of the dominant kernel: the finest-level SCGS colour sweep
    F = G.field_shape("V")[1]
    C = G.field_shape("RHO")[1]
    bytes_per_launch = 4.0 * N_STEPS * (4 * F + 1.5 * C)
    peak, kind = _peaks()
    achieved = bytes_per_launch / (k_ms / k_n * 1e-3) / 1e9 if k_n else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": None,
            "kernel": "scgs_colour_kernel<float> (finest level)", "peak_kind": kind,
            "launches_timed": k_n, "avg_launch_us": 1e3 * k_ms / k_n if k_n else None,
            "algorithmic_bytes_per_launch": bytes_per_launch}
    if rank != 0:
        return
    line = {"metric": "STFAS spacetime cells/s", "value": value, "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "vcycles_per_step": VCYCLES,
                       "l2": "256 MiB buffer written between timed steps (outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof, "e2e": e2e, "gpu_launches": int(launches * world), "clocks": clocks}
    if cpu is not None:
        line["cpu_baseline"] = cpu_baseline_obj(cpu)
    print(json.dumps(line), flush=True)
    G.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
