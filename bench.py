"""Benchmark: AMG-PCG time to 1e-10 relative residual on the 3D Poisson
workload (ellipsoid, semi-axes 0.7/0.5/0.4, seeded rotation, 256^3 nodes on
[-1,1]^3, u = exp(x) sin(y+z)).

One step = one pcg_solve from x = 0 to ||r||/||b|| <= 1e-10 with the AMG
hierarchy built beforehand; the metric is DOF/s = N_C / time-to-tolerance
(N_C = computational points).  Build and setup times are reported beside it.
L2 (129 MB) is flushed between timed steps by a 512 MB write outside the
timed events.  Under torchrun every rank solves its own copy (replicas; no
collective on the data path) and rank 0 prints one JSON line.

--impl reference runs the FP64 CPU oracle (plain numpy / scipy) on a bounded
sample of the same workload on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "AMG-PCG DOF/s and time to 1e-10 rel. residual; stencil HBM GB/s vs peak"
UNIT = "DOF/s"
RTOL = 1e-10
N_FULL = 256
# level-0 Chebyshev step of the FP32 V-cycle: reads x, b, d and writes x_out, d
# (4 bytes each) per computational point
CHEB_BYTES_PER_DOF = 20
ROOFLINE_KERNEL = "k_g_cheb_step<3, float, float>"
CPU_SAMPLE_N = 112


def workload_config(n=N_FULL):
    return {"workload": f"3D Poisson AMG-PCG, ellipsoid (0.7,0.5,0.4) seeded rotation, {n}^3 nodes on [-1,1]^3, "
                        f"u=exp(x)sin(y+z), rtol {RTOL:g}",
            "n": n, "rtol": RTOL,
            "vcycle": "FP32 storage and arithmetic, Chebyshev-2, smoothed aggregation; outer flexible PCG in FP64",
            "l2": "flushed between timed steps (512 MB write outside the timed events)"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_fingerprint():
    h = hashlib.sha256()
    for f in ("amg_vcycle.cu", "stencil.cuh", "tiles.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2204_06083_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """Per-launch DRAM bytes of the roofline kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "cheb_step_3d_256_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("fingerprint") != kernel_fingerprint():
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- oracle leg
def cpu_oracle_sample(n=CPU_SAMPLE_N):
    """Times the oracle's AMG-PCG solve on the same workload at n^3 nodes in a
    fresh single-threaded process; returns its JSON record."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
import eb_inputs as ei
from oracle import amg, eb, solvers
g, ls = ei.ellipsoid_k3({n}, 0)
t0 = time.perf_counter(); s = eb.build(g, ls); t1 = time.perf_counter()
pts = ei.grid_points(g)
b = eb.rhs(s, ei.f_k3(*pts), ei.u_k3(*[s.cut_xg[:, a] for a in range(3)]))
t2 = time.perf_counter(); H = amg.setup(s.A); t3 = time.perf_counter()
x, st = solvers.pcg(s.A, b, M=lambda r: amg.vcycle(H, r), rtol={RTOL})
t4 = time.perf_counter()
print(json.dumps(dict(n={n}, num_cp=s.num_cp, build_s=t1 - t0, setup_s=t3 - t2, solve_s=t4 - t3,
                      iterations=st.iterations, rel=st.true_rel_residual)))
"""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    times = []
    rec = None
    for i in range(args.warmup + args.steps):
        rec = cpu_oracle_sample()
        if i >= args.warmup:
            times.append(rec["solve_s"])
    t = sum(times) / len(times)
    value = rec["num_cp"] / t
    sample = (f"oracle AMG-PCG solve to {RTOL:g} on the same ellipsoid at {CPU_SAMPLE_N}^3 nodes "
              f"(N_C={rec['num_cp']}, {rec['iterations']} iterations); DOF/s of that solve")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(CPU_SAMPLE_N),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- GPU leg
def run_gpu(args):
    import numpy as np
    import torch

    import eb_inputs as ei
    import paper_2204_06083_gb300 as eb
    from paper_2204_06083_gb300 import build as ebuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        ebuild.build()
    if dist is not None:
        dist.barrier()
    ebuild.build()
    dev = torch.device("cuda", torch.cuda.current_device())

    grid, ls = ei.ellipsoid_k3(N_FULL, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = eb.EB(grid, ls)
    torch.cuda.synchronize()
    build_ms = 1000.0 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    solver = eb.AMG(h, 0.0, vcycle_prec=eb.EB_F32)
    setup_ms = 1000.0 * (time.perf_counter() - t0)
    solver64 = eb.AMG(h, 0.0)
    nc = h.info.num_cp
    pts = ei.grid_points(grid)
    f = torch.tensor(ei.f_k3(*pts), device=dev)
    _, _, _, xg = h.cuts()
    xg = xg.cpu().numpy()
    ug = torch.tensor(ei.u_k3(xg[:, 0], xg[:, 1], xg[:, 2]), device=dev)
    b = h.rhs(f, ug)
    x = torch.zeros_like(b)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(profile):
        x.zero_()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, st = solver.solve(b, x=x, rtol=RTOL, maxit=500, profile=profile)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), st

    for _ in range(args.warmup):
        step(False)
    clocks = ClockSampler(torch.cuda.current_device())
    ms, iters, prof_ms, prof_n, launches = [], [], 0.0, 0, 0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with clocks:
        for _ in range(args.steps):
            t, st = step(True)
            ms.append(t)
            iters.append(st.iterations)
            prof_ms += st.prof_kernel_ms
            prof_n += st.prof_launches
            launches += st.launches
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    tot = torch.tensor([sum(ms)], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    ms_per_step = float(tot.item()) / args.steps
    value = world * nc / (ms_per_step / 1000.0)

    # the plain FP64 AMG-PCG on the same input, for comparison
    f64_ms, f64_it = [], 0
    for i in range(args.warmup + args.steps):
        x.zero_()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, st64 = solver64.solve(b, x=x, rtol=RTOL, maxit=500)
        e1.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            f64_ms.append(e0.elapsed_time(e1))
            f64_it = st64.iterations

    # end to end through the C ABI: pinned host b -> device, solve, x -> pinned host
    hb = b.cpu().pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    db = torch.empty_like(b)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        db.copy_(hb, non_blocking=True)
        x.zero_()
        solver.solve(db, x=x, rtol=RTOL, maxit=500)
        hx.copy_(x, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_t = torch.tensor([sum(e2e_ms) / len(e2e_ms)], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = world * nc / (float(e2e_t.item()) / 1000.0)
    # solution check against the manufactured solution (second order)
    xs = hx.numpy().reshape(-1)
    nodes, _ = h.cp_data()
    nodes = nodes.cpu().numpy()
    ue = ei.u_k3(*pts).reshape(-1)[nodes]
    err_linf = float(np.abs(xs[nodes] - ue).max())

    peak, peak_kind = peaks()
    avg_launch_s = (prof_ms / prof_n) / 1000.0 if prof_n else float("nan")
    achieved = CHEB_BYTES_PER_DOF * nc / avg_launch_s / 1e9 if prof_n else None
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rec = cpu_oracle_sample()
        cpu = {"value": rec["num_cp"] / rec["solve_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle AMG-PCG solve to {RTOL:g} of the same ellipsoid at {CPU_SAMPLE_N}^3 nodes "
                         f"(N_C={rec['num_cp']}, {rec['iterations']} its, {rec['solve_s']:.1f} s), one thread"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 outer, f32 V-cycle", "data": "synthetic",
            "config": workload_config(),
            "fp64_vcycle": {"time_to_tol_ms": sum(f64_ms) / len(f64_ms), "iterations": f64_it,
                            "dof_per_s": nc / (sum(f64_ms) / len(f64_ms) / 1000.0)},
            "num_cp": nc, "iterations": iters[-1], "time_to_tol_ms": ms_per_step,
            "build_ms": build_ms, "setup_ms": setup_ms, "amg_levels": solver.rows,
            "max_err_vs_exact": err_linf,
            "roofline": {"bound": "hbm", "kernel": ROOFLINE_KERNEL, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": recorded_traffic(),
                         "algorithmic_bytes_per_launch": CHEB_BYTES_PER_DOF * nc,
                         "avg_launch_us": avg_launch_s * 1e6, "launches_timed": prof_n},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": hb.numel() * 8,
                    "d2h_bytes_per_step": hx.numel() * 8},
            "gpu_launches": launches, "clocks": clocks.summary(), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
