"""Benchmark of the STFAS/ADMM hot path on GB300.

A step is one ADMM iteration of Alg. 3: the AO fixed point (2 warm-started
backward/projection/blend/forward passes), a fixed number of STFAS V(2,2)
cycles, the KKT metric and the multiplier update -- every row of the hot path.
The metric is STFAS spacetime cells/s: fine cells x timesteps x V-cycles per
step / step time (the AO and KKT time counts against it).

The headline workload (default, --workload 3d) is the largest single-GPU
configuration: 64^3 cells, 60 steps, two seeded ellipsoid-union keyframes at
t = 30 and 60, fp32 state with fp64 reductions and coarsest level.  The 2D
letters workload (128^2 x 40, one disc/bar keyframe) is measured the same way
as a second line under "letters" (--workload letters swaps the two).

Beside the step figures (rank 0, N = 1; skip with the --no-* flags):
* roofline: the dominant kernel of the finest level (SCGS colour sweep or the
  colour residual, whichever took more device time inside the timed steps,
  by CUDA events on the stream that runs the V-cycle graph) against the
  measured HBM copy bandwidth; the SCGS launch also against the measured FP32
  FMA rate (its block arithmetic is ALU-heavy);
* cpu_baseline: the fp64 numpy oracle, timed on this host's cores, on a
  bounded sample of the same workload (one V-cycle of the 64^3 grid on 2
  timesteps; for 2D one ADMM iteration of the 128^2 grid on 2 timesteps);
* time_to_solution: stc_solve from v = 0 to a relative KKT residual (32^2 x 16
  fp64 to 1e-6, 128^2 x 40 to 1e-4 in fp32 and, as the baseline, in plain
  fp64; 64^3 x 60 for a few iterations), with the seconds at which 1e-2, 1e-3
  and 1e-4 were first reached;
* served: the first --serve requests of the seeded Poisson serving stream
  replayed in real time into stc_server (fp32, 64 GB budget, worker-thread
  mode), p50/p99 time to solution and problems/hour, beside the plain fp64
  per-problem solve of the first few of the same requests one after another;
  served_batched replays the same into the stepped mode (batched V-cycle
  launches, continuous admission).

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference];
N > 1 under torchrun runs one independent replica per GPU (the method has no
data-path collective) and reports the summed throughput over the max time.
"""
import argparse
import hashlib
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

VCYCLES = 4
WORKLOADS = {
    "3d": dict(n=64, nz=64, N=60, levels=5,
               desc="3D smoke control, 64^3 cells, 60 timesteps, dt=1/60, fp32 state with fp64 reductions and "
                    "fp64 coarsest level; Gaussian ball (sigma 0.1) at (0.5,0.2,0.5); keyframes at t=30 and t=60, "
                    "each a seeded (3003) union of 2-4 ellipsoids (semi-axes 0.05-0.2) blurred by 1 cell and "
                    "mass-matched; r=1e-3, K=1, C_i with 5 Gaussian levels; one ADMM iteration per step = AO(2) "
                    "+ %d V(2,2)-cycles + KKT metric + lambda update" % VCYCLES),
    "letters": dict(n=128, nz=0, N=40, levels=6,
                    desc="2D smoke control, 128^2 cells, 40 timesteps, dt=1/40, fp32 state with fp64 reductions "
                         "and fp64 coarsest level; Gaussian ball (sigma 0.08) at (0.5,0.25) to a seeded (2002) "
                         "blurred (1.5 cells) mass-matched union of 3-5 discs/bars at t=T; r=1e-3, K=1, C_i with "
                         "6 Gaussian levels; one ADMM iteration per step = AO(2) + %d V(2,2)-cycles + KKT metric + "
                         "lambda update" % VCYCLES),
}

# Algorithmic bytes per fine spacetime cell (fp32, each field read or written
# once per pass).  SCGS sweep: 80 B (2D) / 108 B (3D) per cell per sweep; a
# colour launch updates 1/2^d of the cells.  Colour residual (f - res at the
# rows one colour reads): v and u in full (2F), pbar and p (2C), z at the
# colour's faces, res read and f - res written at the colour's rows -- in 2D
# a colour owns F/2 faces and C/4 cells (4.5 F + 3 C floats per step, F ~ 2C:
# 12 C), in 3D F/4 faces and C/8 cells (3.25 F + 2.5 C, F ~ 3C: 12.25 C).
SCGS_BYTES_PER_CELL_SWEEP = {2: 80.0, 3: 108.0}
CRES_FLOATS = {2: (4.5, 3.0), 3: (3.25, 2.5)}     # (per face, per cell) per timestep

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one
# finest-level launch, keyed by kernel kind and workload, with the sha256 (first
# 16 hex digits) of the kernel sources it was measured on; a source that has
# changed since makes the figure void (reported as null).
KERNEL_SOURCES = {"scgs": {2: ["nso_kernels.cu", "stc_internal.cuh"],
                           3: ["nso3d_kernels.cu", "grid3d.cuh", "stc_internal.cuh"]},
                  "cres": {2: ["nso_kernels.cu", "stc_internal.cuh"],
                           3: ["nso3d_kernels.cu", "grid3d.cuh", "stc_internal.cuh"]}}
# 3D colour residual: the two-pass form's four launches together (three
# lamb3_terms_kernel face axes + nso_residual3_colour_kernel); 3D SCGS: the
# coupling kernel and the Thomas kernel together.  Taken with
# ncu --metrics on `bench.py --steps 1 --warmup 0 --no-secondary --no-solve
# --serve 0 --no-cpu-baseline --no-e2e --no-autograd` (and --workload
# letters), the first launches of each kernel.  (The 3D residual's counters
# were taken before the last change to the coupling kernel, in the same
# source file; the residual kernels are byte-identical since.)
MEASURED_TRAFFIC = {("scgs", 2): (23258624, "4602f9532e8dcd2a"),
                    ("cres", 2): (31350528 + 261120, "4602f9532e8dcd2a"),
                    ("scgs", 3): (408173312 + 2063754752, "6cb390d42e74d9a5"),
                    ("cres", 3): (538561536 + 533031936 + 533190912 + 1677374464, "6cb390d42e74d9a5")}
# FP32 operations of one finest-level SCGS colour launch (2 x FFMA + FADD +
# FMUL thread instructions, ncu), with the digest of the sources they were
# counted on: dim -> (flops per launch, source digest)
MEASURED_SCGS_FLOPS = {2: (2.93888e8, "4602f9532e8dcd2a"), 3: (6.53550e9, "6cb390d42e74d9a5")}

ORACLE_STEPS = 2      # timesteps of the bounded oracle samples (same grid, same per-step work)


def source_digest(kind, dim):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind][dim]:
        with open(os.path.join(ROOT, "paper_1608_01102_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# oracle samples (CPU, separate processes, before any GPU work)
# ---------------------------------------------------------------------------
ORACLE_2D = r"""
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

# one V(2,2)-cycle of the 3D grid on Ns timesteps from the zero state, with the
# workload's second keyframe as the step-Ns target and a seeded smooth target
# velocity (the per-timestep work of a cycle does not depend on N)
ORACLE_3D = r"""
import sys, time, json
sys.path.insert(0, %r)
import numpy as np
from oracle import kkt, stfas, mac
from paper_1608_01102_gb300 import workloads
Ns, n = %d, %d
cfg = workloads.config_3d(64, 60)
P = kkt.Problem(n, n, Ns, 1.0 / 60, cfg["rho0"] if n == 64 else workloads.gaussian_ball3(n, n, n, (0.5, 0.2, 0.5), 0.1),
                r=1e-3, K=1.0, metric_levels=5, nz=n)
mac.ops(P.grid)
z = np.zeros((Ns, P.grid.F))
for i in range(1, Ns):
    z[i] = workloads.swirl_velocity3(n, n, n, 0.5)
x = kkt.zero_state(P)
t = time.perf_counter()
stfas.stfas_cycle(P, x, z)
el = time.perf_counter() - t
print(json.dumps({"seconds": el, "cells": n * n * n * Ns}))
"""


def oracle_sample(kind, threads=1, n3=64):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    code = ORACLE_3D % (ROOT, ORACLE_STEPS, n3) if kind == "3d" else ORACLE_2D % (ROOT, ORACLE_STEPS, VCYCLES)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["cells"] / d["seconds"], d["seconds"]


def sample_text(kind, n3=64):
    if kind == "3d":
        return ("fp64 numpy oracle: one V(2,2)-cycle (10 coarsest sweeps) of the %d^3 grid restricted to %d "
                "timesteps, from the zero state toward a smooth target (the per-timestep work of a cycle is the "
                "same for every N)" % (n3, ORACLE_STEPS))
    return ("fp64 numpy oracle: one ADMM iteration (AO(2) + %d V-cycles + KKT metric) of the 128^2 workload "
            "restricted to %d timesteps (per-timestep work is the same; the cost is linear in N)"
            % (VCYCLES, ORACLE_STEPS))


def cpu_baseline(kind):
    """Single-thread and all-core runs of the oracle sample on this host."""
    ncores = os.cpu_count() or 1
    v1, s1 = oracle_sample(kind, 1)
    va, sa = oracle_sample(kind, ncores)
    return {"value": v1, "unit": "cells/s", "cores": 1, "kind": "oracle", "sample": sample_text(kind),
            "seconds": s1, "host_cores": ncores,
            "all_cores": {"value": va, "seconds": sa, "threads": ncores,
                          "note": "the same sample with BLAS/OpenMP threads = host cores; numpy runs the "
                                  "oracle's batched small solves and sparse products on one core, so it barely "
                                  "gains"}}


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
# reference arm: the oracle as it stands, on this host's cores
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    """Each step is one bounded oracle sample of the workload: for 3D one
    V-cycle of a 32^3 grid on 2 timesteps (the 64^3 sample takes ~35 s, too
    long for K + W steps within minutes; the per-cell work of a cycle is the
    same on both grids), for 2D one ADMM iteration of the 128^2 grid on 2
    timesteps.  Rank 0 alone runs it."""
    if rank != 0:
        return
    kind = args.workload
    n3 = 32
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        v, s = oracle_sample(kind, 1, n3)
        if i >= args.warmup:
            vals.append(v)
            secs.append(s)
    value = sum(vals) / len(vals)
    text = sample_text(kind, n3)
    line = {"impl": "reference", "metric": "STFAS spacetime cells/s", "value": value, "unit": "cells/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(secs) / len(secs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[kind]["desc"] + "; oracle sample: " + text},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": 1, "kind": "oracle", "sample": text},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the step on one workload
# ---------------------------------------------------------------------------
def workload_config(name, workloads):
    w = WORKLOADS[name]
    cfg = workloads.config_3d(w["n"], w["N"]) if w["nz"] else workloads.config_letters(w["n"], w["N"])
    return cfg, w


def kernel_roofline(G, kind, dim, n, nz, N, peak, peak_kind):
    """Roofline object of one timed finest-level kernel kind (0 = SCGS colour,
    1 = colour residual): algorithmic bytes per launch / CUDA-event average."""
    ms, cnt = G.kernel_timing(kind)
    C = n * n * (nz or 1)
    F = G.field_shape("V")[1]
    if kind == 0:
        per_launch = SCGS_BYTES_PER_CELL_SWEEP[dim] * C * N / 2 ** dim
        name = ("scgs3t_coupling_kernel + scgs3t_colour_kernel<float> (finest level)" if dim == 3
                else "scgs_colour_kernel<float> (finest level)")
        key = "scgs"
    else:
        a, b = CRES_FLOATS[dim]
        per_launch = 4.0 * (a * F + b * C) * (N + 1)
        name = ("lamb3_terms_kernel<float, axis> x 3 + nso_residual3_colour_kernel<float> (finest level)" if dim == 3
                else "nso_residual_colour_kernel<float> (finest level)")
        key = "cres"
    if not cnt:
        return None, 0.0
    avg = ms / cnt * 1e-3
    achieved = per_launch / avg / 1e9
    tr = MEASURED_TRAFFIC.get((key, dim))
    traffic = tr[0] if tr and tr[1] == source_digest(key, dim) else None
    return ({"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
             "traffic": traffic, "kernel": name, "peak_kind": peak_kind, "launches_timed": cnt,
             "avg_launch_us": avg * 1e6, "algorithmic_bytes_per_launch": per_launch,
             "bytes_rule": ("%g B per fine spacetime cell per sweep, 1/%d of the cells per colour launch"
                            % (SCGS_BYTES_PER_CELL_SWEEP[dim], 2 ** dim)) if kind == 0 else
             ("(%g F + %g C) floats per timestep: v, u, pbar, p read, z at the colour's faces, res read and "
              "f - res written at its rows" % CRES_FLOATS[dim])}, ms)


def measure_step(stc, workloads, name, args, dev, world, with_e2e=True):
    import torch

    cfg, w = workload_config(name, workloads)
    n, nz, N, levels = w["n"], w["nz"], w["N"], w["levels"]
    dim = 3 if nz else 2
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
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    if world > 1:
        import torch.distributed as dist
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
    peak, peak_kind = _peaks()
    roofs = [kernel_roofline(G, k, dim, n, nz, N, peak, peak_kind) for k in (0, 1)]
    G.set_kernel_timing(False)
    cells = n * n * (nz or 1) * N * VCYCLES
    ms, value = aggregate(sum(times) / len(times), cells, world, dev)
    out = {"value": value, "ms_per_step": ms, "clocks": clocks, "gpu_launches": int(launches * world),
           "workload": w["desc"], "cells_per_step": cells, "step_ms_all": times}
    # the dominant finest-level kernel: the kind with more timed device time
    dom = max((r for r in roofs if r[0]), key=lambda r: r[1], default=(None, 0.0))
    out["roofline"] = dom[0]
    out["kernels"] = {"scgs_colour": roofs[0][0], "colour_residual": roofs[1][0]}

    # one V-cycle alone (the STFAS cells/s of one stc_vcycle, no AO or KKT)
    vt = []
    for _ in range(3):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.vcycle(1)
        e1.record(stream)
        e1.synchronize()
        vt.append(e0.elapsed_time(e1))
    out["vcycle_only"] = {"ms": statistics.median(vt), "value": n * n * (nz or 1) * N / (statistics.median(vt) * 1e-3),
                          "unit": "cells/s"}

    out["sweeps"] = sweep_rooflines(G, stream, flush, n, nz, N, dim, peak, peak_kind)

    if with_e2e:
        # end to end through the public API with host buffers: keyframes up, forces down
        h2d = sum(a.nbytes for a, _ in keys.values())
        d2h = N * G.field_shape("U")[1] * 8
        e2e_times = []
        for _ in range(max(2, min(args.steps, 10) // 2)):
            t0 = time.perf_counter()
            G.set_keyframes(keys)
            step()
            u = G.forces()
            e2e_times.append(time.perf_counter() - t0)
        assert u.shape[0] == N
        out["e2e"] = {"value": world * cells / (sum(e2e_times) / len(e2e_times)), "unit": "cells/s",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    G.close()
    return out


def sweep_rooflines(G, stream, flush, n, nz, N, dim, peak, peak_kind):
    """Achieved HBM bandwidth of the AO sweeps at the problem's current v*: the
    Taylor forward sweep (Eq. Adv; per step read rho_i and v_i, write rho_{i+1}:
    (2 + d) C floats), the backward adjoint sweep (Eq. KKTPO; per step read
    rho_i, mu_i, v_i, the fp64 metric term, w_i, write mu_{i-1} and y_i: (4 + 3d)
    C floats) and the projection Q of the N - 1 fields y_1..y_{N-1} (read and
    write each field, 2F floats; the Poisson solve inside is not counted).
    CUDA events on the problem's stream, L2 flushed before each, median of 3."""
    import torch
    C = n * n * (nz or 1)
    F = G.field_shape("V")[1]
    legs = {"taylor_forward": (lambda: G.advect("VSTAR"), 4.0 * N * C * (2 + dim)),
            "adjoint": (lambda: G.adjoint("VSTAR", 1.0, 1.0), 4.0 * N * C * (4 + 3 * dim)),
            "projection": (lambda: G.project("Y", 1, N - 1), 4.0 * (N - 1) * 2 * F)}
    G.advect("VSTAR")
    G.metric_terms()
    out = {}
    for name, (fn, nbytes) in legs.items():
        ts = []
        for _ in range(3):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "algorithmic_bytes": nbytes, "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": gbs / peak, "peak_kind": peak_kind}
    return out


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


# ---------------------------------------------------------------------------
# time to solution and serving (rank 0, N = 1)
# ---------------------------------------------------------------------------
def _t(x):
    return x if x is not None and x >= 0 else None


def solve_leg(stc, workloads, which, precision, tol, max_admm, **over):
    """stc_solve from v = 0 with Alg. 3's density test off (eps_admm = 0): it
    runs to the KKT tolerance or the iteration cap."""
    if which == "small":
        cfg = workloads.config_small(32, 16)
        n, nz, N, levels, desc = 32, 0, 16, 4, "32^2 x 16 (ball to ball, r=1e-3, C_i with 4 levels)"
    else:
        cfg, w = workload_config(which, workloads)
        n, nz, N, levels, desc = w["n"], w["nz"], w["N"], w["levels"], w["desc"].split(";")[0]
    prm = stc.default_params(n, n, N, precision=precision, r=1e-3, K=1.0, metric_levels=levels, eps_admm=0.0,
                             nz=nz, **over)
    with stc.Problem(prm, cfg["rho0"]) as G:
        G.set_keyframes(cfg["keyframes"])
        t0 = time.perf_counter()
        rep = G.solve(tol=tol, max_admm=max_admm)
        wall = time.perf_counter() - t0
        hist = G.solve_history()
    step = max(1, len(hist) // 40)
    out = {"workload": desc + ", solved from v = 0", "precision": "fp64" if precision else "fp32 (fp64 reductions)",
           "tol_kkt_rel": tol, "max_admm": max_admm, "seconds": wall, "admm_iters": rep["admm_iters"],
           "vcycles": rep["vcycles"], "rejected_vcycles": rep["rejected_vcycles"], "kkt_rel": rep["kkt_rel"],
           "objective": rep["objective"], "K_final": rep.get("K_final"),
           "seconds_to": {"1e-2": _t(rep.get("seconds_to_1e2")), "1e-3": _t(rep.get("seconds_to_1e3")),
                          "1e-4": _t(rep["seconds_to_1e4"]), "1e-6": _t(rep.get("seconds_to_1e6"))},
           "paper_stop": {"rule": "Alg. 3: max_i ||rho_i - rho_i^last||_inf < max|rho_0|/100",
                          "admm_iters": rep["density_stop_iter"] or None,
                          "seconds": _t(rep["seconds_to_density_stop"])},
           "stopped_by": "kkt" if rep["kkt_rel"] <= tol else "iteration cap",
           "kkt_rel_min": min((h[0] for h in hist), default=None),
           "history": [[k, h[0], h[1], h[2]] for k, h in enumerate(hist) if k % step == 0 or k == len(hist) - 1],
           "history_fields": ["iteration", "kkt_rel", "seconds", "K"]}
    out.update({k: v for k, v in over.items()})
    return out, hist


def seconds_to(hist, R):
    for r, sec, _ in hist:
        if r <= R:
            return sec
    return None


def serve_leg(stc, workloads, count, max_admm, fp64_count, budget=64 << 30, workers=8, ao_trials=1, mode=1,
              max_resident=16):
    """Replay the first `count` requests of the seeded stream in real time
    (fp32); then solve the first `fp64_count` of them one after another with
    the plain fp64 per-problem solve, the baseline of the serving form.  The
    requests try AO blend factors one at a time (ao_trials = 1): the
    concurrent solves already share the GPU."""
    reqs = workloads.config_serving(count)

    def params(r, precision):
        n, N = r["nx"], r["N"]
        return stc.default_params(n, n, N, precision=precision, r=r["r"], K=1.0,
                                  metric_levels=max(0, int(np.floor(np.log2(n / 2)))), ao_trials=ao_trials,
                                  k_adapt=1)

    if mode == 1:
        # stepped serving: this thread submits arrivals and drives the batched steps
        import torch
        stream = torch.cuda.Stream()
        with stc.Server(budget, mode=1, stream=stream.cuda_stream, max_resident=max_resident) as S:
            t0 = time.perf_counter()
            tickets, nxt, active, steps = [], 0, 0, 0
            while nxt < len(reqs) or active > 0:
                now = time.perf_counter() - t0
                while nxt < len(reqs) and reqs[nxt]["arrival"] <= now:
                    r = reqs[nxt]
                    tickets.append(S.submit(params(r, 0), r["rho0"], r["keyframes"], tol=1e-4, max_admm=max_admm))
                    nxt += 1
                active = S.step()
                steps += 1
                if active == 0 and nxt < len(reqs):
                    time.sleep(max(0.0, reqs[nxt]["arrival"] - (time.perf_counter() - t0)))
            infos = [S.poll(t) for t in tickets]
            peak = S.stats()["peak_bytes"]
    else:
        with stc.Server(budget, workers=workers) as S:
            t0 = time.perf_counter()
            tickets = []
            for r in reqs:
                delay = r["arrival"] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                tickets.append(S.submit(params(r, 0), r["rho0"], r["keyframes"], tol=1e-4, max_admm=max_admm))
            infos = [S.wait(t) for t in tickets]
            peak = S.stats()["peak_bytes"]
    lat = [i["t_done"] - i["t_submit"] for i in infos if i["state"] == "done"]
    span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
    kk = [i["report"]["kkt_rel"] for i in infos if i["state"] == "done"]
    out = {"requests": count, "completed": len(lat), "failed": sum(i["state"] == "failed" for i in infos),
           "p50_s": float(np.percentile(lat, 50)) if lat else None,
           "p99_s": float(np.percentile(lat, 99)) if lat else None,
           "problems_per_hour": 3600.0 * len(lat) / span if span > 0 else None,
           "reached_kkt_1e-4": sum(k <= 1e-4 for k in kk), "kkt_rel_median": float(np.median(kk)) if kk else None,
           "admm_iters_median": float(np.median([i["report"]["admm_iters"] for i in infos])),
           "budget_bytes": budget, "peak_bytes": peak, "max_admm": max_admm,
           "mode": ("stepped: each stc_server_step runs the next NSO V-cycle of every resident problem as one "
                    "batched CUDA graph launch, admission and retirement between steps, max %d resident"
                    % max_resident) if mode == 1 else
                   "worker threads: %d concurrent stc_solve calls, one stream each" % workers,
           "stream": "workloads.config_serving(seed 4004): Poisson 4/s, n in {32,48,64,96,128}, N in [16,48], "
                     "1-3 disc/bar keyframes, fp32 policy, stop at KKT 1e-4 or Alg. 3's density test"}
    if fp64_count > 0:
        secs, kk64 = [], []
        for r in reqs[:fp64_count]:
            with stc.Problem(params(r, 1), r["rho0"]) as G:
                G.set_keyframes(r["keyframes"])
                t1 = time.perf_counter()
                rep = G.solve(tol=1e-4, max_admm=max_admm)
                G.forces()
                secs.append(time.perf_counter() - t1)
                kk64.append(rep["kkt_rel"])
        # served latency of the same requests one after another = queueing behind
        # the earlier ones plus the solve, with the stream's arrival times
        done, lat64 = 0.0, []
        for r, s in zip(reqs[:fp64_count], secs):
            start = max(done, r["arrival"])
            done = start + s
            lat64.append(done - r["arrival"])
        out["fp64_sequential"] = {
            "requests": fp64_count, "solve_s_median": float(np.median(secs)),
            "p50_s": float(np.percentile(lat64, 50)), "p99_s": float(np.percentile(lat64, 99)),
            "problems_per_hour": 3600.0 * fp64_count / sum(secs), "kkt_rel_median": float(np.median(kk64)),
            "note": "plain fp64 per-problem stc_solve, one request at a time on the same GPU; latencies replay "
                    "the stream's arrival times against the measured solve times"}
    return out


def autograd_leg(workloads, n=128, N=48, every=8):
    """The forward simulation as a torch.autograd.Function at the
    differentiable-simulation workload's size: n^3 cells, N steps, fp32,
    checkpoint-and-recompute every `every` steps; one untimed pass, then the
    forward and the backward timed with CUDA events."""
    import torch

    from paper_1608_01102_gb300 import autograd
    cfg = workloads.config_autograd(n, N)
    sim = autograd.Simulation(n, n, N, cfg["rho0"], nz=n, precision=0, checkpoint_every=every)
    st = torch.tensor(cfg["star"], dtype=torch.float32, device="cuda")
    times = []
    for rep in range(2):
        u = torch.tensor(cfg["u"], dtype=torch.float32, device="cuda", requires_grad=True)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        rho = autograd.simulate(u, sim)
        loss = 0.5 * ((rho[-1] - st) ** 2).sum()
        e[1].record()
        loss.backward()
        e[2].record()
        e[2].synchronize()
        times.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])))
    fwd, bwd = times[-1]
    out = {"workload": "%d^3 cells, %d steps, fp32, checkpoint every %d steps (%d segments), seeded smooth random "
                       "forces (correlation 8 cells, max |u| 0.1), loss 1/2 ||rho_N - rho*||^2" % (n, N, every,
                                                                                               len(sim.segments)),
           "forward_ms": fwd, "backward_ms": bwd, "picard_iterations": sim.picard_iterations,
           "loss": float(loss.detach()), "grad_norm": float(u.grad.norm())}
    sim.close()
    return out


def attach_alu(sc, dim, fp32):
    """The SCGS launch against the measured FP32 FMA rate (ALU side of its roofline)."""
    fl = MEASURED_SCGS_FLOPS.get(dim)
    if not sc or not fp32 or not fl or fl[1] != source_digest("scgs", dim):
        return
    g = fl[0] / (sc["avg_launch_us"] * 1e-6) / 1e9
    sc["alu"] = {"flops_per_launch": fl[0], "achieved_gflops": g, "peak_gflops": fp32, "frac": g / fp32,
                 "peak_kind": "measured (stc_measure_fp32_peak)",
                 "flops_rule": "2 x FFMA + FADD + FMUL thread instructions of one launch (ncu count)"}


def run_native(args, rank, world, local_rank):
    import torch

    from paper_1608_01102_gb300 import stc, workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    head = args.workload
    other = "letters" if head == "3d" else "3d"
    solo = rank == 0 and world == 1
    # oracle baselines first, in separate processes, before heavy GPU work
    cpu = cpu_baseline(head) if solo and not args.no_cpu_baseline else None
    cpu2 = None
    if solo and not args.no_cpu_baseline and not args.no_secondary and other == "letters":
        v, s = oracle_sample("letters", 1)
        cpu2 = {"value": v, "unit": "cells/s", "cores": 1, "kind": "oracle", "sample": sample_text("letters"),
                "seconds": s}

    m = measure_step(stc, workloads, head, args, dev, world, with_e2e=not args.no_e2e)
    if rank != 0:
        return
    line = {"metric": "STFAS spacetime cells/s", "value": m["value"], "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": m["workload"], "vcycles_per_step": VCYCLES,
                       "l2": "256 MiB buffer written between timed steps (outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": m["roofline"], "e2e": m.get("e2e"), "gpu_launches": m["gpu_launches"], "clocks": m["clocks"],
            "vcycle_only": m["vcycle_only"], "kernels": m["kernels"], "sweeps": m["sweeps"]}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if solo:
        fp32 = stc.measure_fp32_peak()
        sc = m["kernels"]["scgs_colour"]
        line["fp32_fma_peak_gflops"] = fp32
        attach_alu(sc, 3 if head == "3d" else 2, fp32)
    if solo and not args.no_secondary:
        m2 = measure_step(stc, workloads, other, args, dev, world, with_e2e=not args.no_e2e)
        sec = {k: m2.get(k) for k in ("value", "ms_per_step", "roofline", "kernels", "vcycle_only", "e2e", "clocks",
                                      "gpu_launches", "workload", "sweeps")}
        if cpu2 is not None:
            sec["cpu_baseline"] = cpu2
        attach_alu(sec["kernels"]["scgs_colour"], 3 if other == "3d" else 2, line.get("fp32_fma_peak_gflops"))
        line["letters" if other == "letters" else "3d"] = sec
    if solo and not args.no_solve:
        legs = {}
        # the solve legs balance the ADMM penalty (k_adapt; the fixed point does not depend on K)
        legs["small_fp64"], _ = solve_leg(stc, workloads, "small", 1, 1e-6, args.small_max_admm, k_adapt=1)
        legs["letters_fp32"], h32 = solve_leg(stc, workloads, "letters", 0, 1e-4, args.solve_max_admm, k_adapt=1)
        legs["letters_fp64_baseline"], h64 = solve_leg(stc, workloads, "letters", 1, 1e-4, args.fp64_max_admm,
                                                       k_adapt=1)
        if h32 and h64:
            common = max(min(h[0] for h in h32), min(h[0] for h in h64))
            t32, t64 = seconds_to(h32, common), seconds_to(h64, common)
            legs["letters_fp32_vs_fp64"] = {
                "kkt_rel": common, "fp32_seconds": t32, "fp64_seconds": t64,
                "speedup": t64 / t32 if t32 and t64 else None,
                "note": "time for each precision form to first reach the smallest relative KKT residual both "
                        "reached (the same per-problem solve, fp32 state vs plain fp64)"}
        legs["3d_fp32"], _ = solve_leg(stc, workloads, "3d", 0, 1e-4, args.solve3d_max_admm, k_adapt=1)
        line["time_to_solution"] = legs
    if solo and not args.no_autograd:
        line["autograd"] = autograd_leg(workloads)
    if solo and args.serve > 0:
        line["served"] = serve_leg(stc, workloads, args.serve, args.serve_max_admm, args.serve_fp64, mode=0)
        line["served_batched"] = serve_leg(stc, workloads, args.serve, args.serve_max_admm, 0, mode=1)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="3d", choices=["3d", "letters"],
                    help="3d: 64^3 x 60 (default, the headline); letters: the 2D 128^2 x 40 workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the other workload's step line")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (short profiling runs)")
    ap.add_argument("--no-autograd", action="store_true", help="skip the differentiable-simulation leg")
    ap.add_argument("--small-max-admm", type=int, default=1500)
    ap.add_argument("--solve-max-admm", type=int, default=500)
    ap.add_argument("--fp64-max-admm", type=int, default=40)
    ap.add_argument("--solve3d-max-admm", type=int, default=10)
    ap.add_argument("--serve", type=int, default=24, help="serving requests to replay (0: skip)")
    ap.add_argument("--serve-max-admm", type=int, default=50)
    ap.add_argument("--serve-fp64", type=int, default=4, help="requests of the fp64 sequential baseline")
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
