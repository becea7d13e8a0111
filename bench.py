"""Benchmarks of the embedded-boundary hot path on one GB300, one JSON line per run.

--workload (default poisson3d):

poisson3d  3D Poisson AMG-PCG: ellipsoid with semi-axes 0.7/0.5/0.4 and a seeded
           rotation, 256^3 nodes on [-1,1]^3, u = exp(x) sin(y+z).  One step =
           one pcg_solve from x = 0 to ||r||/||b|| <= 1e-10 (FP32 V-cycle,
           flexible PCG with its vectors in double-float, the exit test on the
           FP64 true residual); the FP64 outer iteration, the plain FP64
           V-cycle and the BF16-storage V-cycle are timed beside it.
poisson2d  2D Poisson, plain FP64 AMG-PCG: circle R = 0.5 at (0.02, 0.01),
           128^2 nodes, u = sin(2x) cos(3y), rtol 1e-10.
wave       Leapfrog wave equation on the star r = 0.5 + 0.1 sin(5 phi), 4096^2
           nodes, dt = 0.9 of the periodic CFL limit, 10,000 steps from a
           seeded Gaussian pulse; one step = the whole 10,000-step run in FP32
           (one wave_step call: cached CUDA graphs of one launch per time
           step), FP64 timed beside it.
batched    64 seeded stars on grids from 128^2 to 1024^2, backward-Euler heat
           with dt = h, 50 steps of all 64 geometries per bench step (one
           batch_heat_step per time step, forcing and boundary data frozen at
           t = 0; the per-geometry PCG in double-float); the FP64 outer
           iteration and the same time step solved geometry by geometry with
           the plain FP64 AMG-PCG are timed beside it.
conv       The learned stage's network alone: one forward pass (6 layers, the four
           32 -> 32 layers on tcgen05) over a 2048^2 image of seeded inputs.
learned    The learned preconditioner stage: trained (outside the timed
           region) on 20,000 solver-generated pairs at 512^2 on random stars,
           then one step = one flexible PCG solve with V-cycle + stage to
           1e-10 on a random star at 2048^2 (u = sin(2x) cos(3y)); the plain
           FP64 AMG-PCG is timed beside it.

Before timing, the tile shape of the grid kernels is chosen by the library's
autotuner (V-cycle or apply timed for each candidate shape; the winner and
the timings are in the line).  L2 (129 MB) is flushed between timed steps by
a 512 MB write outside the timed events.  Under torchrun every rank runs its own copy (replicas; no
collective on the data path) and rank 0 prints the line.

--impl reference runs the FP64 CPU oracle (plain numpy / scipy) of the same
workload on a bounded sample on the host cores instead.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "AMG-PCG DOF/s and time to 1e-10 rel. residual; stencil HBM GB/s vs peak"
RTOL = 1e-10
N_FULL = 256
# level-0 Chebyshev step: reads x, b, d and writes x_out, d per computational point
CHEB_BYTES_PER_DOF = {"f32": 20, "f64": 40}
# leapfrog step per computational point: reads u^n, u^{n-1}, the node code, writes u^{n+1}
LEAPFROG_BYTES_PER_DOF = {"f32": 13, "f64": 25}
# one 32 -> 32 convolution of the learned stage per pixel: 2 x 9 x 32 x 32 FLOP
CONV_FLOP_PER_PX = 18432
# and its bytes per pixel: 32 BF16 channels read and 32 written
CONV_BYTES_PER_PX = 128
# the whole network per pixel: 2 x 9 x (2 x 32 + 4 x 32 x 32 + 32 x 1) FLOP, of
# which the four 32 -> 32 layers (on the tensor cores) are 4 x 18432
NET_FLOP_PER_PX = 75456
NET_TENSOR_FLOP_PER_PX = 4 * CONV_FLOP_PER_PX
# and its bytes when all six layers run in one kernel: the two input channels
# (float) read, the output (float) written
NET_BYTES_PER_PX = 12
ALONE_LAUNCHES = 20
L2_CLEAR_BYTES = 512 << 20
ALONE_NOTE = ("amg_time_kernel: back-to-back launches of the kernel on the solver's own level data in one CUDA "
              "graph, CUDA events around the graph; each launch preceded by a read of a 512 MB buffer that leaves "
              "none of the kernel's data (and no dirty line) in L2 (its own time, measured the same way, "
              "subtracted), so the kernel reads its data from DRAM")
PROF_NOTE = ("CUDA events around every launch of the kernel in as many solves (batched: one bench step) run right "
             "after the timed ones on the same input; those use the captured iteration with a host check, since "
             "the timed device-side loop cannot bracket single launches")
WORKLOADS = ("poisson3d", "poisson2d", "wave", "batched", "learned", "conv", "heat_cn", "wave_theta", "helmholtz",
             "qoi", "rs_w", "mixed")


def pk_hbm():
    return peaks()[0]["hbm_gbs"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_fingerprint(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2204_06083_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """Per-launch DRAM bytes (read + write) of a roofline kernel from the
    committed ncu summaries, if they were taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "kernel_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d or d.get("fingerprint") != kernel_fingerprint(d["files"]):
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw nvidia-smi samples (the summary goes into the JSON line);
        # EB_CLOCKS_DIR keeps them somewhere other than the temporary directory
        folder = os.environ.get("EB_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.q = q
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
            # a timed region shorter than nvidia-smi's start-up leaves no sample:
            # take one right at its end (the clocks have not left the load state)
            self.at_end = False
            if not any(len(line.split(",")) >= 9 for line in open(self.path)):
                try:
                    out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.q}",
                                          "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                         timeout=20).stdout
                    with open(self.path, "a") as f:
                        f.write(out)
                    self.at_end = True
                except (OSError, subprocess.TimeoutExpired):
                    pass

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
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
               "reasons": sorted(reasons), "samples": len(sm)}
        if getattr(self, "at_end", False):
            out["sampled"] = "once, right after the timed region (shorter than nvidia-smi's sampling start-up)"
        return out


# ---------------------------------------------------------------- workloads
def config_of(w, small=None):
    if w == "poisson3d":
        n = small or N_FULL
        return {"workload": f"3D Poisson AMG-PCG, ellipsoid (0.7,0.5,0.4) seeded rotation, {n}^3 nodes on [-1,1]^3, "
                            f"u=exp(x)sin(y+z), rtol {RTOL:g}", "n": n, "rtol": RTOL,
                "vcycle": "FP32 storage and arithmetic, Chebyshev-2, smoothed aggregation; outer flexible PCG with "
                          "double-float vectors (pcg_opts.outer_prec = EB_DF64), FP64 scalars and exit test",
                "l2": "flushed between timed steps (512 MB write outside the timed events)"}
    if w == "poisson2d":
        return {"workload": f"2D Poisson plain FP64 AMG-PCG, circle R=0.5 at (0.02,0.01), 128^2 nodes on [-1,1]^2, "
                            f"u=sin(2x)cos(3y), rtol {RTOL:g}", "n": 128, "rtol": RTOL,
                "l2": "flushed between timed steps (512 MB write outside the timed events)"}
    if w == "wave":
        n = small or 4096
        return {"workload": f"2D leapfrog wave, star r=0.5+0.1 sin(5 phi), {n}^2 nodes on [-1,1]^2, "
                            f"dt=0.9 h/sqrt(2), 10000 steps, seeded Gaussian pulse", "n": n, "steps_per_run": 10000,
                "precision": "FP32 fields (FP64 timed beside)",
                "l2": "fields (2 x 67 MB FP32) and the 512 MB flush between runs"}
    if w == "batched":
        return {"workload": "batched backward-Euler heat, 64 seeded stars r=0.5+sum a_k sin(k phi+p_k), k=2..6, "
                            "grids 128^2..1024^2, dt=h, 50 steps of all geometries per bench step, "
                            "forcing and boundary data of u=exp(-t) sin(2x) cos(3y) frozen at t=0",
                "geometries": 64, "time_steps": 50, "rtol": RTOL,
                "vcycle": "FP32 V-cycle on the block-diagonal hierarchy, per-geometry flexible PCG with double-float "
                          "vectors (batch_set_outer_prec EB_DF64), FP64 scalars and exit test",
                "l2": "batch vectors exceed L2 (26M nodes x 8 B)"}
    if w == "conv":
        return {"workload": "learned-stage network forward, one 2048^2 image, He-initialised weights (seed 8), "
                            "seeded normal residual channel, mask of the random star (seed 999)",
                "n": 2048, "network": "6 x conv3x3, 32 channels, BF16 activations, FP32 accumulation",
                "l2": "activations 268 MB per layer exceed L2; 512 MB flush between steps"}
    if w == "learned":
        return {"workload": "flexible PCG with V-cycle + learned CNN stage, random star at 2048^2, "
                            f"u=sin(2x)cos(3y), rtol {RTOL:g}; network trained on 20000 solver pairs at 512^2 "
                            "(2500 random stars x 8)", "n": 2048, "train_n": 512, "train_pairs": 20000,
                "network": "6 x conv3x3, 32 channels, BF16 activations, FP32 accumulation",
                "l2": "flushed between timed steps (512 MB write outside the timed events)"}
    if w in PAPER_WORKLOADS:
        return dict(PAPER_WORKLOADS[w]["config"], l2="flushed between timed steps (512 MB write outside the timed "
                                                      "events)")
    raise ValueError(w)


# The paper's other experiments on the GPU path (one workload each; Sec. 2.2-3.6)
PAPER_WORKLOADS = {
    "heat_cn": {"config": {"workload": "Crank-Nicolson heat (Sec. 3.4): disk r < 0.5 in [-1,1]^2, beta = 0.25 - r^2, "
                                       "u = exp(-t)(r^2 - 0.25), dt = h, 2048^2 nodes, 50 steps per bench step, "
                                       "warm-started AMG-PCG (FP32 V-cycle, double-float outer iteration) to 1e-10",
                           "n": 2048, "steps": 50}},
    "wave_theta": {"config": {"workload": "implicit theta = 1/12 wave scheme (Sec. 3.5, Table 1): Bessel J_7 mode on "
                                          "the unit disk in [-1.1,1.1]^2, 1602^2 nodes, dt = 0.85 h, 100 steps per "
                                          "bench step, AMG-PCG (FP32 V-cycle, double-float outer iteration) to 1e-10 "
                                          "per step", "n": 1602,
                              "steps": 100}},
    "helmholtz": {"config": {"workload": "Helmholtz omega = 50 (Sec. 3.3.2): star r = 0.5 + 0.2 sin 5 theta, "
                                         "802^2 nodes, 1000 x unit-integral hat source, MINRES preconditioned by the "
                                         "Laplacian's V-cycle to 1e-10", "n": 802}},
    "qoi": {"config": {"workload": "QOI sweep (Sec. 3.6): 64 rotated ellipses (semi-axes 4, 2) on 502^2 grids of "
                                   "[-5,5]^2, Lap u = 3, one batched steady AMG-PCG solve (FP32 V-cycle, double-float "
                                   "outer iteration) to 1e-10 and the 64 rectangle integrals per bench step", "n": 502,
                                   "geometries": 64}},
    "rs_w": {"config": {"workload": "classical (Ruge-Stueben) AMG with W-cycle (Sec. 3): star r = 0.5 + 0.1 sin 5 phi, "
                                    "2048^2 nodes, u = sin(2x)cos(3y), PCG to 1e-10 from x = 0", "n": 2048}},
    "mixed": {"config": {"workload": "mixed line-by-line / RBF closure (Sec. 2.2-2.3): star r = 0.5 + 0.2 sin 5 phi, "
                                     "4096^2 nodes, build with the RBF cuts then AMG-PCG (FP32 V-cycle, double-float "
                                     "outer iteration) to 1e-10 of u = sin(2x)cos(3y)", "n": 4096}},
}


UNITS = {"heat_cn": "DOF-steps/s", "wave_theta": "DOF-steps/s", "helmholtz": "DOF/s", "qoi": "DOF/s",
         "rs_w": "DOF/s", "mixed": "DOF/s",
         "poisson3d": "DOF/s", "poisson2d": "DOF/s", "wave": "DOF-steps/s", "batched": "DOF/s",
         "learned": "DOF/s", "conv": "pixels/s"}


# ------------------------------------------------------------------ oracle
def _oracle_run(code, timeout=900):
    r = subprocess.run([sys.executable, "-c", f"import sys; sys.path.insert(0, {ROOT!r})\n" + code],
                       capture_output=True, text=True, env=_oracle_env(), timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_cpu():
    """Core count and CPU model of the host the oracle runs on."""
    fields = {}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ":" in ln:
                k, v = ln.split(":", 1)
                fields.setdefault(k.strip(), v.strip())
    except Exception:
        pass
    model = fields.get("Model name") or fields.get("Vendor ID")
    import platform
    return {"nproc": os.cpu_count(), "model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


# The oracle on the full default workload: build, AMG setup (not timed), then
# `reps` solves from x = 0, each timed.  READY / stdin: the all-cores run starts
# every process's timed solves together.
POISSON3D_ORACLE = """
import json, sys, time
import eb_inputs as ei
from oracle import amg, eb, solvers
g, ls = ei.ellipsoid_k3({n}, 0)
s = eb.build(g, ls)
pts = ei.grid_points(g)
b = eb.rhs(s, ei.f_k3(*pts), ei.u_k3(*[s.cut_xg[:, a] for a in range(3)]))
H = amg.setup(s.A)
if {wait}:
    print("READY", flush=True)
    sys.stdin.readline()
secs = []
for _ in range({reps}):
    t0 = time.perf_counter()
    x, st = solvers.pcg(s.A, b, M=lambda r: amg.vcycle(H, r), rtol={rtol})
    secs.append(time.perf_counter() - t0)
print(json.dumps(dict(dof=s.num_cp, secs=secs, sec=sum(secs) / len(secs), iterations=st.iterations)))
"""


def _oracle_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def oracle_poisson3d(reps, n=N_FULL):
    return _oracle_run(POISSON3D_ORACLE.format(n=n, wait=False, reps=reps, rtol=RTOL), timeout=1800)


def oracle_poisson3d_all_cores(n=N_FULL, max_procs=16):
    """One single-threaded oracle process per host core (at most max_procs),
    each solving the full workload once, all timed solves started together
    after every process has built its system and hierarchy: the host's
    aggregate oracle throughput.  Returns (DOF/s, processes, record)."""
    procs_n = max(1, min(os.cpu_count() or 1, max_procs))
    code = f"import sys; sys.path.insert(0, {ROOT!r})\n" + POISSON3D_ORACLE.format(n=n, wait=True, reps=1, rtol=RTOL)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=_oracle_env()) for _ in range(procs_n)]
    try:
        for p in procs:
            line = p.stdout.readline()
            if line.strip() != "READY":
                raise RuntimeError("oracle process failed: " + p.stderr.read()[-2000:])
        for p in procs:
            p.stdin.write("go\n")
            p.stdin.flush()
        recs = []
        for p in procs:
            out, err = p.communicate(timeout=1800)
            if p.returncode != 0:
                raise RuntimeError("oracle process failed: " + err[-2000:])
            recs.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    wall = max(r["sec"] for r in recs)
    return sum(r["dof"] for r in recs) / wall, procs_n, {"dof": recs[0]["dof"], "wall_s": wall,
                                                         "iterations": recs[0]["iterations"]}


def cpu_oracle_sample(w):
    """Times the oracle on a bounded sample of workload w in a fresh
    single-threaded process; returns (value, unit-consistent sample text, record)."""
    if w == "poisson3d":
        rec = oracle_poisson3d(1)
        return rec["dof"] / rec["sec"], (f"oracle AMG-PCG solve to {RTOL:g} of the full workload ({N_FULL}^3 nodes, "
                                         f"N_C={rec['dof']}, {rec['iterations']} its, {rec['sec']:.1f} s; "
                                         f"build and AMG setup not timed)"), rec
    if w == "poisson2d":
        rec = _oracle_run(f"""
import json, time
import eb_inputs as ei
from oracle import amg, eb, solvers
g, ls = ei.circle_k1(128)
s = eb.build(g, ls)
X, Y = ei.grid_points(g)
b = eb.rhs(s, ei.f_k1(X, Y), ei.u_k1(s.cut_xg[:, 0], s.cut_xg[:, 1]))
H = amg.setup(s.A)
t0 = time.perf_counter()
reps = 0
while time.perf_counter() - t0 < 10.0:
    x, st = solvers.pcg(s.A, b, M=lambda r: amg.vcycle(H, r), rtol={RTOL})
    reps += 1
t1 = time.perf_counter()
print(json.dumps(dict(dof=s.num_cp, sec=(t1 - t0) / reps, iterations=st.iterations, reps=reps)))
""")
        return rec["dof"] / rec["sec"], (f"oracle AMG-PCG solve of the full 128^2 workload (N_C={rec['dof']}, "
                                         f"{rec['iterations']} its), mean of {rec['reps']} solves"), rec
    if w == "wave":
        rec = _oracle_run("""
import json, math, time
import eb_inputs as ei
from oracle import eb, solvers
g = ei.box_grid(2, 1024)
ls = ei.star(ei.STAR_CENTER, 0.5, [5], [0.1], [0.0])
s = eb.build(g, ls)
X, Y = ei.grid_points(g)
c, w = ei.pulse_params(0)
u0 = s.from_grid(ei.pulse(X, Y, c, w))
dt = 0.9 * g.h / math.sqrt(2.0)
u1 = u0 - 0.5 * dt * dt * (s.A @ u0)
t0 = time.perf_counter()
solvers.leapfrog(s.A, u0, u1, dt, 4000)
t1 = time.perf_counter()
print(json.dumps(dict(dof=s.num_cp, steps=4000, sec=t1 - t0)))
""")
        return rec["dof"] * rec["steps"] / rec["sec"], (
            f"oracle leapfrog (scipy CSR matvec) on the same star at 1024^2 nodes, 4000 steps "
            f"(N_C={rec['dof']}, {rec['sec']:.1f} s)"), rec
    if w == "batched":
        rec = _oracle_run(f"""
import json, time
import numpy as np
import scipy.sparse as sp
import eb_inputs as ei
from oracle import amg, eb, solvers
cfg = ei.star_batch(64, 0)
pick = list(range(12))
dof, sec, its = 0, 0.0, []
for i in pick:
    nb, ls = cfg[i]
    g = ei.box_grid(2, nb)
    s = eb.build(g, ls)
    dt = g.h
    M0 = (s.A + (1.0 / dt) * sp.identity(s.num_cp, format="csr")).tocsr()
    H = amg.setup(M0)
    X, Y = ei.grid_points(g)
    u = s.from_grid(ei.u_heat(X, Y, 0.0))
    b = eb.rhs(s, -ei.f_heat(X, Y, 0.0), ei.u_heat(s.cut_xg[:, 0], s.cut_xg[:, 1], 0.0))
    t0 = time.perf_counter()
    u, st = solvers.pcg(M0, u / dt + b, x0=u, M=lambda r: amg.vcycle(H, r), rtol={RTOL})
    sec += time.perf_counter() - t0
    dof += s.num_cp
    its.append(st.iterations)
print(json.dumps(dict(dof=dof, sec=sec, iterations=its, sizes=[cfg[i][0] for i in pick])))
""")
        return rec["dof"] / rec["sec"], (
            f"oracle backward-Euler step (AMG-PCG, warm start) of batch geometries 0-11 (n={rec['sizes']}, "
            f"N_C={rec['dof']}, iterations {rec['iterations']}, {rec['sec']:.1f} s)"), rec
    if w == "learned":
        rec = _oracle_run(f"""
import json, time
import numpy as np
import eb_inputs as ei
from oracle import amg, cnn, eb
g = ei.box_grid(2, 128)
s = eb.build(g, ei.random_star(999))
X, Y = ei.grid_points(g)
b = eb.rhs(s, ei.f_k1(X, Y), ei.u_k1(s.cut_xg[:, 0], s.cut_xg[:, 1]))
H = amg.setup(s.A)
theta = cnn.init_params(8) * 0.1
t0 = time.perf_counter()
x, it = cnn.fpcg(s.A, b, lambda r: cnn.stage(s, s.A, H, theta, r), rtol={RTOL})
t1 = time.perf_counter()
print(json.dumps(dict(dof=s.num_cp, sec=t1 - t0, iterations=it)))
""")
        return rec["dof"] / rec["sec"], (
            f"oracle flexible PCG with V-cycle + FP64 CNN stage (untrained weights) on a random star at 128^2 "
            f"(N_C={rec['dof']}, {rec['iterations']} its, {rec['sec']:.1f} s)"), rec
    if w in PAPER_WORKLOADS:
        code = PAPER_ORACLE[w]
        rec = _oracle_run(code.replace("RTOL", repr(RTOL)), timeout=1800)
        return rec["units"] / rec["sec"], rec["sample"], rec
    if w == "conv":
        rec = _oracle_run("""
import json, time
import numpy as np
from oracle import cnn
theta = cnn.init_params(8)
rng = np.random.default_rng(0)
s_hat = rng.standard_normal((256, 256))
m = np.ones((256, 256))
t0 = time.perf_counter()
cnn.forward(theta, s_hat, m)
t1 = time.perf_counter()
print(json.dumps(dict(px=256 * 256, sec=t1 - t0)))
""")
        return rec["px"] / rec["sec"], (f"oracle FP64 network forward (numpy einsum) on a 256^2 image "
                                        f"({rec['sec']:.1f} s)"), rec
    raise ValueError(w)


# oracle samples of the paper workloads: fresh single-threaded processes;
# "units" in the workload's unit (DOF or DOF-steps), "sec" the timed part
PAPER_ORACLE = {
    "heat_cn": """
import json, time
import numpy as np, scipy.sparse as sp
import eb_inputs as ei
from oracle import amg, eb, solvers
g, ls = ei.heat_disk(512)
s = eb.build(g, ls, beta=ei.beta_half_points(g, ei.beta_heat_disk))
X, Y = ei.grid_points(g)
dt, th = g.h, 0.5
lhs = (sp.identity(s.num_cp, format="csr") / dt + th * s.A).tocsr()
H = amg.setup(lhs)
b = lambda t: eb.rhs(s, -ei.f_heat_disk(X, Y, t), np.zeros(s.cut_cp.size))
u = s.from_grid(ei.u_heat_disk(X, Y, 0.0))
t0 = time.perf_counter()
for k in range(10):
    u, st = solvers.theta_heat_step(s.A, u, dt, th, b((k + 1) * dt), b(k * dt), M=lambda r: amg.vcycle(H, r), rtol=RTOL)
sec = time.perf_counter() - t0
print(json.dumps(dict(units=10 * s.num_cp, sec=sec, sample="oracle Crank-Nicolson steps of the same disk problem at 512^2 (10 steps, AMG-PCG, N_C=%d)" % s.num_cp)))
""",
    "wave_theta": """
import json, math, time
import numpy as np
import eb_inputs as ei
from oracle import eb, solvers
g, ls = ei.disk_bessel(402)
s = eb.build(g, ls)
X, Y = ei.grid_points(g)
xs, ys = X.reshape(-1)[s.cp_nodes], Y.reshape(-1)[s.cp_nodes]
dt = 0.85 * g.h
t0 = time.perf_counter()
solvers.theta_wave(s.A, ei.bessel_mode(xs, ys, -dt), ei.bessel_mode(xs, ys, 0.0), dt, 1.0 / 12.0, 50)
sec = time.perf_counter() - t0
print(json.dumps(dict(units=50 * s.num_cp, sec=sec, sample="oracle theta = 1/12 steps (sparse LU, factorised inside the timed part) of the Bessel disk at 402^2 (50 steps, N_C=%d)" % s.num_cp)))
""",
    "helmholtz": """
import json, time
import numpy as np, scipy.sparse as sp
import eb_inputs as ei
from oracle import amg, eb, solvers
g, ls = ei.helmholtz_star(402)
s = eb.build(g, ls)
K = (s.A - ei.HELMHOLTZ_OMEGA ** 2 * sp.identity(s.num_cp, format="csr")).tocsr()
b = eb.rhs(s, ei.hat_source(g), np.zeros(s.cut_cp.size))
H = amg.setup(s.A)
t0 = time.perf_counter()
x, st = solvers.minres(K, b, M=lambda r: amg.vcycle(H, r), rtol=RTOL, maxit=20000)
sec = time.perf_counter() - t0
print(json.dumps(dict(units=s.num_cp, sec=sec, sample="oracle MINRES (V-cycle preconditioned) of the same Helmholtz star at 402^2 (N_C=%d, %d its)" % (s.num_cp, st.iterations))))
""",
    "qoi": """
import json, math, time
import numpy as np, scipy.sparse.linalg as spla
import eb_inputs as ei
from oracle import eb
units, sec = 0, 0.0
for t in np.linspace(0.0, math.pi, 4, endpoint=False):
    g, ls = ei.qoi_rotated(t)
    s = eb.build(g, ls)
    b = eb.rhs(s, np.full(g.shape(), ei.QOI_F), np.zeros(s.cut_cp.size))
    t0 = time.perf_counter()
    x = spla.spsolve(s.A.tocsc(), b)
    q = float(s.to_grid(x).reshape(-1) @ ei.qoi_rect_weights(g).reshape(-1))
    sec += time.perf_counter() - t0
    units += s.num_cp
print(json.dumps(dict(units=units, sec=sec, sample="oracle direct solves and QOIs of 4 of the rotated ellipses at 502^2 (N_C total %d)" % units)))
""",
    "rs_w": """
import json, time
import numpy as np
import eb_inputs as ei
from oracle import amg, eb, solvers
g, ls = ei.star_wave(512)
s = eb.build(g, ls)
X, Y = ei.grid_points(g)
b = eb.rhs(s, ei.f_k1(X, Y), ei.u_k1(s.cut_xg[:, 0], s.cut_xg[:, 1]))
H = amg.setup(s.A, "rs")
t0 = time.perf_counter()
x, st = solvers.pcg(s.A, b, M=lambda r: amg.vcycle(H, r, gamma=2), rtol=RTOL)
sec = time.perf_counter() - t0
print(json.dumps(dict(units=s.num_cp, sec=sec, sample="oracle RS + W-cycle PCG of the same star at 512^2 (N_C=%d, %d its)" % (s.num_cp, st.iterations))))
""",
    "mixed": """
import json, time
import numpy as np
import eb_inputs as ei
from oracle import amg, eb, solvers
g, ls = ei.helmholtz_star(512)
s = eb.build(g, ls, closure="mixed")
X, Y = ei.grid_points(g)
p = s.sample_points()
b = eb.rhs(s, ei.f_k1(X, Y), ei.u_k1(p[:, 0], p[:, 1]))
H = amg.setup(s.A)
t0 = time.perf_counter()
x, st = solvers.pcg(s.A, b, M=lambda r: amg.vcycle(H, r), rtol=RTOL)
sec = time.perf_counter() - t0
print(json.dumps(dict(units=s.num_cp, sec=sec, sample="oracle AMG-PCG solve of the same mixed-closure star at 512^2 (N_C=%d, %d RBF cuts)" % (s.num_cp, s.rbf_cut.size))))
""",
}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = args.workload
    vals, secs, rec, sample = [], [], None, ""
    if w == "poisson3d":
        # the full workload: one build and AMG setup, then warm-up and timed solves
        rec = oracle_poisson3d(args.warmup + args.steps)
        secs = rec["secs"][args.warmup:]
        vals = [rec["dof"] / t for t in secs]
        sample = (f"oracle AMG-PCG solves to {RTOL:g} of the full workload ({N_FULL}^3 nodes, N_C={rec['dof']}, "
                  f"{rec['iterations']} its each); one step = one solve; build and AMG setup not timed")
    else:
        for i in range(args.warmup + args.steps):
            v, sample, rec = cpu_oracle_sample(w)
            if i >= args.warmup:
                vals.append(v)
                secs.append(rec["sec"])
    value = statistics.mean(vals)
    unit = UNITS[w]
    small = {"wave": 1024}.get(w)
    cfg = config_of(w, small)
    cfg["same_config"] = small is None and w in ("poisson3d", "poisson2d")
    cfg["l2"] = "not applicable: the oracle runs on the host cores"
    if w == "poisson3d":
        cfg["vcycle"] = ("FP64 oracle: Chebyshev-2 smoothed-aggregation V-cycle (numpy / scipy), plain FP64 PCG; "
                         "the same hierarchy specification as the GPU path")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample,
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- GPU leg
class Ctx:
    """One rank of the run: rank and world size from the torchrun environment,
    NCCL between the ranks' GPUs (replicas: only the barrier and the max over
    ranks of the timings cross ranks).  cpu=True: gloo on host tensors and no
    GPU, for testing the multi-rank logic."""

    def __init__(self, cpu=False):
        import torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if cpu:
            if self.world > 1:
                import torch.distributed as dist
                dist.init_process_group("gloo")
                self.dist = dist
            self.dev = torch.device("cpu")
            self.flush_buf = None
            return
        if self.world > 1:
            import torch.distributed as dist
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
            self.dist = dist
        else:
            torch.cuda.set_device(0)
        from paper_2204_06083_gb300 import build as ebuild
        if self.rank == 0:
            ebuild.build()
        self.barrier()
        ebuild.build()
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.flush_buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=self.dev)

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def flush(self):
        self.flush_buf.fill_(1.0)

    def max_over_ranks(self, v):
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64, device=self.dev)
        if self.dist is not None:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def tune_tiles(fn):
    """Runs one of the library's tile autotuners (through its JSON cache);
    returns (shape in use, {shape: microseconds} when it timed)."""
    shape, res = fn()
    tune = None if res is None else {f"{a}x{b}x{c}": round(u, 2) for (a, b, c), u in zip(res.shapes, res.us)}
    return list(shape), tune


def profiled(ctx, args, solve):
    """The dominant kernel's launches timed with CUDA events in args.steps
    solves run right after the timed ones (same input, L2 flushed before each):
    the timed solves loop on the device (conditional graph node), where single
    launches cannot be bracketed by events, so these solves use the captured
    iteration with a host check per iteration; kernel durations do not depend
    on the loop.  Returns (summed ms, launches)."""
    import torch
    ms, n = 0.0, 0
    for _ in range(args.steps):
        ctx.flush()
        torch.cuda.synchronize()
        st = solve()
        ms += st.prof_kernel_ms
        n += st.prof_launches
    return ms, n


def timed(fn):
    """Runs fn between CUDA events on torch's current stream; returns (ms, result)."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    r = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), r


def loop(ctx, args, step, clocks_index):
    """warm-up, then exactly args.steps timed steps between barriers; returns
    (list of per-step results, max-over-ranks mean ms, clock summary)."""
    import torch
    for _ in range(args.warmup):
        ctx.flush()
        timed(step)
    res, ms = [], []
    ctx.barrier()
    torch.cuda.synchronize()
    with ClockSampler(clocks_index) as clk:
        for _ in range(args.steps):
            ctx.flush()
            torch.cuda.nvtx.range_push("timed")
            t, r = timed(step)
            torch.cuda.nvtx.range_pop()
            ms.append(t)
            res.append(r)
    torch.cuda.synchronize()
    ctx.barrier()
    return res, ctx.max_over_ranks(sum(ms) / len(ms)), clk.summary()


def gpu_poisson(ctx, args, dim):
    from paper_2204_06083_gb300 import autotune
    import numpy as np
    import torch
    import eb_inputs as ei
    import paper_2204_06083_gb300 as eb
    dev = ctx.dev
    if dim == 3:
        grid, ls = ei.ellipsoid_k3(N_FULL, 0)
    else:
        grid, ls = ei.circle_k1(128)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = eb.EB(grid, ls)
    torch.cuda.synchronize()
    build_ms = 1000.0 * (time.perf_counter() - t0)
    prec = eb.EB_F32 if dim == 3 else eb.EB_F64
    t0 = time.perf_counter()
    solver = eb.AMG(h, 0.0, vcycle_prec=prec)
    setup_ms = 1000.0 * (time.perf_counter() - t0)
    solver64 = eb.AMG(h, 0.0) if dim == 3 else solver
    tile, tune = tune_tiles(lambda: autotune.tune_amg(solver, reps=10))
    # the CSR row groups, cached like the tile shape: a later run on this GPU and
    # problem (e.g. under a profiler, which distorts timings) reuses the choice
    epl, epl_us = autotune.tune_csr(solver, reps=10)
    if solver64 is not solver:
        autotune.tune_csr(solver64, reps=5)
    nc = h.info.num_cp
    pts = ei.grid_points(grid)
    _, _, _, xg = h.cuts()
    xg = xg.cpu().numpy()
    if dim == 3:
        f = torch.tensor(ei.f_k3(*pts), device=dev)
        ug = torch.tensor(ei.u_k3(xg[:, 0], xg[:, 1], xg[:, 2]), device=dev)
        uex = ei.u_k3(*pts)
    else:
        f = torch.tensor(ei.f_k1(*pts), device=dev)
        ug = torch.tensor(ei.u_k1(xg[:, 0], xg[:, 1]), device=dev)
        uex = ei.u_k1(*pts)
    b = h.rhs(f, ug)
    x = torch.zeros_like(b)

    loop_kind = 2 if args.host_loop else 1
    # 3D (FP32 V-cycle): the outer iteration in double-float (pcg_opts.outer_prec);
    # the FP64 outer iteration is timed beside it
    outer = eb.EB_DF64 if dim == 3 else eb.EB_F64

    def step():
        x.zero_()
        return solver.solve(b, x=x, rtol=RTOL, maxit=500, use_graph=loop_kind, outer=outer)[1]

    sts, ms_per_step, clocks = loop(ctx, args, step, torch.cuda.current_device())
    launches = sum(s.launches for s in sts) // len(sts)

    def prof(mode, o=outer):
        return profiled(ctx, args, lambda: solver.solve(b, x=x.zero_(), rtol=RTOL, maxit=500, profile=mode,
                                                        outer=o)[1])
    prof_ms, prof_n = prof(1)
    l1_ms, l1_n = prof(3) if solver.num_levels > 2 else (0.0, 0)
    xp_ms, xp_n = prof(4)
    up_ms, up_n = prof(5)
    value = ctx.world * nc / (ms_per_step / 1000.0)
    extra = {}
    if dim == 3:
        o64 = []
        for i in range(args.warmup + args.steps):
            x.zero_()
            ctx.flush()
            t, sto = timed(lambda: solver.solve(b, x=x, rtol=RTOL, maxit=500)[1])
            if i >= args.warmup:
                o64.append(t)
        xp64_ms, xp64_n = prof(4, eb.EB_F64)
        up64_ms, up64_n = prof(5, eb.EB_F64)
        extra["fp64_outer"] = {"time_to_tol_ms": statistics.mean(o64), "iterations": sto.iterations,
                               "true_rel_residual": sto.true_rel_residual,
                               "dof_per_s": nc / (statistics.mean(o64) / 1000.0),
                               "kernel_time_ms_per_solve": {"pcg_p_update_apply": xp64_ms / max(args.steps, 1),
                                                            "pcg_xr_update": up64_ms / max(args.steps, 1)}}
        f64 = []
        for i in range(args.warmup + args.steps):
            x.zero_()
            ctx.flush()
            t, st64 = timed(lambda: solver64.solve(b, x=x, rtol=RTOL, maxit=500)[1])
            if i >= args.warmup:
                f64.append(t)
        extra["fp64_vcycle"] = {"time_to_tol_ms": statistics.mean(f64), "iterations": st64.iterations,
                                "dof_per_s": nc / (statistics.mean(f64) / 1000.0)}
        solver16 = eb.AMG(h, 0.0, vcycle_prec=eb.EB_BF16)
        autotune.tune_csr(solver16, reps=5)
        b16 = []
        for i in range(args.warmup + args.steps):
            x.zero_()
            ctx.flush()
            t, st16 = timed(lambda: solver16.solve(b, x=x, rtol=RTOL, maxit=500)[1])
            if i >= args.warmup:
                b16.append(t)
        extra["bf16_vcycle"] = {"time_to_tol_ms": statistics.mean(b16), "iterations": st16.iterations,
                                "dof_per_s": nc / (statistics.mean(b16) / 1000.0)}
        solver16.close()
    # end to end through the C ABI: pinned host b -> device, solve, x -> pinned host
    hb = b.cpu().pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    db = torch.empty_like(b)
    e2e = []

    def e2e_step():
        db.copy_(hb, non_blocking=True)
        x.zero_()
        solver.solve(db, x=x, rtol=RTOL, maxit=500, outer=outer)
        hx.copy_(x, non_blocking=True)

    for i in range(args.warmup + args.steps):
        ctx.flush()
        torch.cuda.synchronize()
        t, _ = timed(e2e_step)
        if i >= args.warmup:
            e2e.append(t)
    e2e_value = ctx.world * nc / (ctx.max_over_ranks(statistics.mean(e2e)) / 1000.0)
    nodes, _ = h.cp_data()
    nodes = nodes.cpu().numpy()
    err = float(np.abs(hx.numpy().reshape(-1)[nodes] - uex.reshape(-1)[nodes]).max())
    pk, kind = peaks()
    # Each roofline kernel is also timed on its own: back-to-back launches in
    # one graph, events around the graph (no per-launch event), with an
    # L2-clearing read before each launch (DRAM-cold: the HBM roof applies)
    # and without (warm).  The per-launch event pairs of the in-solve timing add
    # about 4.5 us to each launch (13.6 us back to back against 18.3 us
    # bracketed, measured on the level-1 step), which the alone figure avoids.
    alone = {}
    for lev in ((0, 1) if solver.num_levels > 2 else (0,)):
        alone[lev] = {"cold_us": solver.time_smoother_step(lev, ALONE_LAUNCHES, L2_CLEAR_BYTES),
                      "warm_us": solver.time_smoother_step(lev, 4 * ALONE_LAUNCHES, 0)}
    avg_s = (prof_ms / prof_n) / 1000.0 if prof_n else float("nan")
    vb = CHEB_BYTES_PER_DOF["f32" if dim == 3 else "f64"]

    def size_matched(nbytes, us):
        # a plain streaming copy of the same bytes in the same harness: what a
        # single DRAM-cold launch of this size achieves at best
        cu = eb.time_copy_us(nbytes, ALONE_LAUNCHES, L2_CLEAR_BYTES)
        return {"copy_us": cu, "copy_GBs": nbytes / (cu * 1e-6) / 1e9, "frac_of_copy": cu / us,
                "note": "eb_time_copy: 16-byte streaming copy moving the kernel's algorithmic bytes, timed like "
                        "amg_time_kernel (graph, L2 cleared before each launch)"}
    alg0 = vb * nc
    cold0 = alone[0]["cold_us"] * 1e-6
    stencil = {"bound": "hbm",
               "kernel": f"k_g_cheb_step<{dim}, {'float, float' if dim == 3 else 'double, double'}>",
               "achieved": alg0 / cold0 / 1e9, "peak": pk["hbm_gbs"], "peak_kind": kind + " (burst: kernel timed alone)",
               "unit": "GB/s", "frac": alg0 / cold0 / 1e9 / pk["hbm_gbs"],
               "traffic": recorded_traffic("k_g_cheb_step<3, float, float>") if dim == 3 else None,
               "algorithmic_bytes_per_launch": alg0, "avg_launch_us": alone[0]["cold_us"],
               "timing": ALONE_NOTE, "warm_l2_us": alone[0]["warm_us"],
               "warm_l2_frac": alg0 / (alone[0]["warm_us"] * 1e-6) / 1e9 / pk["hbm_gbs"],
               "in_solve_event_us": avg_s * 1e6 if prof_n else None, "in_solve_launches_timed": prof_n,
               "in_solve_timing": PROF_NOTE, "size_matched_copy": size_matched(alg0, alone[0]["cold_us"])}
    roof = stencil
    if 1 in alone:
        # level-1 Chebyshev step: values + column indices per nonzero, and per row the row
        # pointer, x gathered once, b, D^-1, d read and written, x written (word size 4 or 8)
        w = 4 if dim == 3 else 8
        n1, nnz1 = solver.rows[1], solver.nnz[1]
        l1_bytes = nnz1 * (w + 4) + n1 * (4 + 6 * w)
        cold1 = alone[1]["cold_us"] * 1e-6
        level1 = {"bound": "hbm", "kernel": f"k_c_cheb_step<G, {'float' if dim == 3 else 'double'}> (level 1, CSR)",
                  "achieved": l1_bytes / cold1 / 1e9, "peak": pk["hbm_gbs"],
                  "peak_kind": kind + " (burst: kernel timed alone)", "unit": "GB/s",
                  "frac": l1_bytes / cold1 / 1e9 / pk["hbm_gbs"],
                  "traffic": recorded_traffic("k_c_cheb_step<G, float> level 1") if dim == 3 else None,
                  "algorithmic_bytes_per_launch": l1_bytes, "avg_launch_us": alone[1]["cold_us"],
                  "rows": n1, "nnz": nnz1, "timing": ALONE_NOTE, "warm_l2_us": alone[1]["warm_us"],
                  "warm_l2_frac": l1_bytes / (alone[1]["warm_us"] * 1e-6) / 1e9 / pk["hbm_gbs"],
                  "in_solve_event_us": (l1_ms / l1_n) * 1000.0 if l1_n else None, "in_solve_launches_timed": l1_n,
                  "in_solve_timing": PROF_NOTE, "size_matched_copy": size_matched(l1_bytes, alone[1]["cold_us"])}
    # The PCG's kernels.  DF outer iteration (3D): both are memory passes,
    # against HBM -- k_xpby_apply_df: per DOF z read (FP32), p and q read and
    # written (DF, 8 B each), the code byte: 37 B; k_update_first_df: r, q, p,
    # x read and x, r written (DF), z read, the level-0 right-hand side,
    # iterate and direction written (FP32), the code byte: 65 B.  FP64 outer
    # iteration: k_xpby_apply against the measured FP64 FMA peak (per DOF the
    # 7-point sum, 5 adds, and D x - sum, one FMA, then p = z + beta p, q = B z
    # + beta q and the p.q partial, three FMAs: 13 FLOP), k_update_first against
    # HBM (69 B with FP32 V-cycle vectors, 81 B with FP64).
    fp64_tflops = eb.fp64_peak_tflops(reps=20)
    share = {"level0_smoother": prof_ms, "level1_smoother": l1_ms, "pcg_p_update_apply": xp_ms,
             "pcg_xr_update": up_ms}
    xp_flop = (13 if dim == 3 else 11) * nc

    def fp64_apply_roof(ms, n):
        sec = (ms / n) / 1000.0 if n else float("nan")
        return {"bound": "alu", "kernel": f"k_xpby_apply<{dim}, false, true> (p update + next operator apply, FP64)",
                "achieved": xp_flop / sec / 1e12, "peak": fp64_tflops,
                "peak_kind": "measured FP64 FMA throughput (eb_fp64_peak, this run)", "unit": "TFLOP/s",
                "frac": xp_flop / sec / 1e12 / fp64_tflops, "traffic": None,
                "algorithmic_flop_per_launch": xp_flop, "algorithmic_bytes_per_launch": 41 * nc,
                "hbm_frac": 41 * nc / sec / 1e9 / pk_hbm(), "avg_launch_us": sec * 1e6, "launches_timed": n,
                "timing": PROF_NOTE + "; each bracketed launch carries the event pair's few microseconds"}

    def hbm_roof(kernel, nbytes, ms, n):
        sec = (ms / n) / 1000.0 if n else float("nan")
        return {"bound": "hbm", "kernel": kernel, "achieved": nbytes / sec / 1e9, "peak": pk_hbm(),
                "peak_kind": "measured HBM copy (burst)", "unit": "GB/s", "frac": nbytes / sec / 1e9 / pk_hbm(),
                "traffic": None, "algorithmic_bytes_per_launch": nbytes, "avg_launch_us": sec * 1e6,
                "launches_timed": n,
                "timing": PROF_NOTE + "; each bracketed launch carries the event pair's few microseconds"}
    if outer == eb.EB_DF64:
        pcg_apply = hbm_roof(f"k_xpby_apply_df<{dim}, false, true> (p update + next operator apply, double-float)",
                             37 * nc, xp_ms, xp_n)
        pcg_apply["traffic"] = recorded_traffic("k_xpby_apply_df<3>")
        pcg_update = hbm_roof(f"k_update_first_df<{dim}, float> (x/r update in double-float + first level-0 "
                              "smoothing step)", 65 * nc, up_ms, up_n)
        pcg_update["traffic"] = recorded_traffic("k_update_first_df<3, float>")
        extra["fp64_outer"]["p_update_apply_roofline"] = fp64_apply_roof(xp64_ms, xp64_n)
        extra["fp64_outer"]["xr_update_roofline"] = hbm_roof(
            f"k_update_first<{dim}, float> (x/r update + first level-0 smoothing step, FP64)", 69 * nc,
            up64_ms, up64_n)
    else:
        pcg_apply = fp64_apply_roof(xp_ms, xp_n)
        up_bytes = (69 if dim == 3 else 81) * nc
        pcg_update = hbm_roof(f"k_update_first<{dim}, {'float' if dim == 3 else 'double'}> "
                              "(x/r update + first level-0 smoothing step)", up_bytes, up_ms, up_n)
    if 1 in alone:
        by_kernel = {"level0_smoother": stencil, "level1_smoother": level1, "pcg_p_update_apply": pcg_apply,
                     "pcg_xr_update": pcg_update}
        # the line's roofline is the kernel with the largest share of the solve
        roof = by_kernel[max(share, key=share.get)]
    line = {"value": value, "ms_per_step": ms_per_step,
            "dtype": ("df64 outer (double-float: FP32 pairs, ~48-bit; exit test on the FP64 true residual), "
                      "f32 V-cycle") if dim == 3 else "f64",
            "true_rel_residual": sts[-1].true_rel_residual,
            "num_cp": nc, "iterations": sts[-1].iterations, "time_to_tol_ms": ms_per_step,
            "build_ms": build_ms, "setup_ms": setup_ms, "amg_levels": solver.rows, "max_err_vs_exact": err,
            "tile": tile, "autotune_us_per_vcycle": tune,
            "csr_entries_per_lane": epl, "csr_tune_us_per_vcycle": ({str(k): round(v, 2) for k, v in epl_us.items()} if epl_us else None),
            "roofline": roof, "stencil_roofline": stencil,
            "kernel_time_ms_per_solve": {k: v / max(args.steps, 1) for k, v in share.items()},
            "pcg_rooflines": {"p_update_apply": pcg_apply, "xr_update": pcg_update},
            "fp64_peak_tflops": fp64_tflops,
            "e2e": {"value": e2e_value, "unit": "DOF/s", "h2d_bytes_per_step": hb.numel() * 8,
                    "d2h_bytes_per_step": hx.numel() * 8},
            "gpu_launches": launches, "clocks": clocks}
    line.update(extra)
    if dim == 3:
        line["stencil_subrecords"] = stencil_subrecords(ctx, args, h)
    return line


SUB_WAVE_STEPS = 320


def stencil_subrecords(ctx, args, h3):
    """The metric's stencil GB/s beside the solve: eb_apply on the solve's own
    256^3 grid (FP64 and FP32) and the leapfrog step of the 4096^2 star wave
    workload (FP32 and FP64, 320 steps = 10 graph chunks per timed call), each
    against the measured HBM peak (the FP64 apply against the measured FP64
    peak, which bounds it).  Algorithmic bytes per DOF: apply 16 (FP64) / 8
    (FP32): x read, y written; leapfrog 25 / 13: u^n, u^{n-1} read, u^{n+1}
    written, the code byte."""
    from paper_2204_06083_gb300 import autotune
    import torch
    import eb_inputs as ei
    import paper_2204_06083_gb300 as eb
    hbm = pk_hbm()
    out = {}
    nc = h3.info.num_cp
    rng = torch.Generator(device=ctx.dev).manual_seed(5)
    fp64_tflops = eb.fp64_peak_tflops(reps=20)
    dim = len(h3.shape())
    # FP64 instructions per CP of the apply: the 2 dim - 1 adds of the
    # neighbour sum, D x - sum (one FMA), then core / h^2 + sigma x (a multiply
    # and an FMA); the FP64 FMA peak (an FMA counted as 2 FLOP) issues half as
    # many instructions
    f64_instr = (2 * dim - 1 + 3) * nc
    for name, dtype, bpd in (("apply_256cubed_f64", torch.float64, 16), ("apply_256cubed_f32", torch.float32, 8)):
        xin = torch.randn(h3.shape(), generator=rng, device=ctx.dev, dtype=torch.float64).to(dtype)
        y = torch.zeros_like(xin)
        for _ in range(3):
            h3.apply(xin, out=y)
        cold_us = h3.time_apply_us(xin, y, launches=20, clear_bytes=L2_CLEAR_BYTES)
        warm_us = h3.time_apply_us(xin, y, launches=50)
        copy_us = eb.time_copy_us(bpd * nc, launches=20, clear_bytes=L2_CLEAR_BYTES)
        gbs = bpd * nc / (cold_us * 1e-6) / 1e9
        rec = {"bound": "hbm", "kernel": f"k_apply<{'double' if dtype == torch.float64 else 'float'}, {dim}> "
                                         "(eb_apply, matrix free, one CP pair per thread)",
               "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
               "algorithmic_bytes_per_launch": bpd * nc, "avg_launch_us": cold_us,
               "timing": "eb_time_apply: 20 back-to-back launches in one CUDA graph, CUDA events around the "
                         "graph, each launch after a 512 MB read that leaves none of its data in L2 (the "
                         "read's own time subtracted)",
               "warm_us": warm_us, "warm_frac": bpd * nc / (warm_us * 1e-6) / 1e9 / hbm,
               "size_matched_copy": {"copy_us": copy_us, "frac_of_copy": copy_us / cold_us}}
        if dtype == torch.float64:
            # the FP64 pipe, not HBM, bounds the FP64 apply on this part
            instr_rate = fp64_tflops / 2.0 * 1e12
            rec.update({"bound": "alu", "unit": "TFLOP/s", "peak": fp64_tflops,
                        "achieved": 2.0 * f64_instr / (cold_us * 1e-6) / 1e12,
                        "frac": f64_instr / (cold_us * 1e-6) / instr_rate,
                        "peak_kind": "measured FP64 FMA throughput (eb_fp64_peak, this run)",
                        "algorithmic_fp64_instructions_per_launch": f64_instr,
                        "achieved_note": "FP64 instructions per second x 2 (the peak's FLOP per FMA)",
                        "hbm_GBs": gbs, "hbm_frac": gbs / hbm,
                        "alu_bound_us": f64_instr / instr_rate * 1e6,
                        "warm_alu_frac": f64_instr / (warm_us * 1e-6) / instr_rate})
            del rec["warm_frac"]
        out[name] = rec
        del xin, y
    grid, ls = ei.star_wave(4096)
    hw = eb.EB(grid, ls)
    ncw = hw.info.num_cp
    tile, _ = tune_tiles(lambda: autotune.tune_eb(hw, eb.EB_F32, reps=5, op=eb.EB_TUNE_LEAPFROG))
    X, Y = ei.grid_points(grid)
    c, w = ei.pulse_params(0)
    dt = 0.9 * grid.h / math.sqrt(2.0)
    u0 = torch.tensor(ei.pulse(X, Y, c, w), device=ctx.dev)
    u1 = u0 - 0.5 * dt * dt * hw.apply(u0)
    for name, dtype, bpd in (("leapfrog_4096sq_f32", torch.float32, 13), ("leapfrog_4096sq_f64", torch.float64, 25)):
        a0, b0 = u0.to(dtype), u1.to(dtype)
        a, bb = torch.empty_like(a0), torch.empty_like(b0)
        ts = []
        for i in range(3 + args.steps):
            a.copy_(a0)
            bb.copy_(b0)
            ctx.flush()
            torch.cuda.synchronize()
            t, _ = timed(lambda: hw.wave_step(a, bb, dt, SUB_WAVE_STEPS))
            if i >= 3:
                ts.append(t)
        step_s = statistics.mean(ts) / 1000.0 / SUB_WAVE_STEPS
        out[name] = {"bound": "hbm", "kernel": f"k_leapfrog<{'float' if dtype == torch.float32 else 'double'}, 2> "
                                               "(one launch per step, 32-step CUDA-graph chunks)",
                     "achieved": bpd * ncw / step_s / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": bpd * ncw / step_s / 1e9 / hbm, "algorithmic_bytes_per_launch": bpd * ncw,
                     "avg_launch_us": step_s * 1e6, "num_cp": ncw, "tile": tile,
                     "timing": f"CUDA events around a {SUB_WAVE_STEPS}-step wave_step call (L2 flushed before it); "
                               "per-step time = call time / steps; the two fields of the active tiles fit in L2, so "
                               "the figure can exceed what DRAM alone would allow"}
        del a, bb, a0, b0
    hw.close()
    return out


def gpu_wave(ctx, args):
    from paper_2204_06083_gb300 import autotune
    import torch
    import eb_inputs as ei
    import paper_2204_06083_gb300 as eb
    nsteps = 10000
    grid, ls = ei.star_wave(4096)
    h = eb.EB(grid, ls)
    nc = h.info.num_cp
    tile, tune = tune_tiles(lambda: autotune.tune_eb(h, eb.EB_F32, reps=5, op=eb.EB_TUNE_LEAPFROG))
    X, Y = ei.grid_points(grid)
    c, w = ei.pulse_params(0)
    dt = 0.9 * grid.h / math.sqrt(2.0)
    u0 = torch.tensor(ei.pulse(X, Y, c, w), device=ctx.dev)
    u1 = u0 - 0.5 * dt * dt * h.apply(u0)
    fields = {}
    for dt_name, dtype in (("f32", torch.float32), ("f64", torch.float64)):
        fields[dt_name] = (u0.to(dtype), u1.to(dtype))
    a = torch.empty_like(fields["f32"][0])
    bfield = torch.empty_like(fields["f32"][0])

    def step():
        a.copy_(fields["f32"][0])
        bfield.copy_(fields["f32"][1])
        return timed(lambda: h.wave_step(a, bfield, dt, nsteps))[0]

    kern_ms, ms_per_step, clocks = loop(ctx, args, step, torch.cuda.current_device())
    value = ctx.world * nc * nsteps / (ms_per_step / 1000.0)
    a64 = torch.empty_like(fields["f64"][0])
    b64 = torch.empty_like(fields["f64"][0])
    f64 = []
    for i in range(1 + args.steps):
        a64.copy_(fields["f64"][0])
        b64.copy_(fields["f64"][1])
        ctx.flush()
        t, _ = timed(lambda: h.wave_step(a64, b64, dt, nsteps))
        if i >= 1:
            f64.append(t)
    diff = float((bfield.double() - b64).abs().max().item() / b64.abs().max().item())
    # e2e: pinned host fields -> device, 10,000 steps, both fields -> host
    hu = [fields["f32"][0].cpu().pin_memory(), fields["f32"][1].cpu().pin_memory()]
    ho = [torch.empty_like(hu[0]).pin_memory(), torch.empty_like(hu[1]).pin_memory()]
    e2e = []

    def e2e_step():
        a.copy_(hu[0], non_blocking=True)
        bfield.copy_(hu[1], non_blocking=True)
        h.wave_step(a, bfield, dt, nsteps)
        ho[0].copy_(a, non_blocking=True)
        ho[1].copy_(bfield, non_blocking=True)

    for i in range(1 + args.steps):
        ctx.flush()
        t, _ = timed(e2e_step)
        if i >= 1:
            e2e.append(t)
    e2e_value = ctx.world * nc * nsteps / (ctx.max_over_ranks(statistics.mean(e2e)) / 1000.0)
    pk, kind = peaks()
    launch_s = statistics.mean(kern_ms) / 1000.0
    alg = LEAPFROG_BYTES_PER_DOF["f32"] * nc * nsteps
    achieved = alg / launch_s / 1e9
    return {"value": value, "ms_per_step": ms_per_step, "dtype": "f32", "num_cp": nc, "dt": dt,
            "tile": tile, "autotune_us_per_16_steps": tune,
            "us_per_time_step": 1000.0 * ms_per_step / nsteps,
            "fp64": {"ms_per_run": statistics.mean(f64), "us_per_time_step": 1000.0 * statistics.mean(f64) / nsteps,
                     "dof_steps_per_s": nc * nsteps / (statistics.mean(f64) / 1000.0),
                     "max_rel_diff_f32_vs_f64_after_run": diff},
            "roofline": {"bound": "hbm",
                         "kernel": "k_leapfrog<float, 2> (one launch per step in 32-step CUDA-graph chunks; bytes and "
                                   "time per 10,000-step wave_step call)",
                         "achieved": achieved, "peak": pk["hbm_gbs"], "peak_kind": kind, "unit": "GB/s",
                         "frac": achieved / pk["hbm_gbs"], "traffic": None,
                         "algorithmic_bytes_per_launch": alg, "avg_launch_us": launch_s * 1e6,
                         "launches_timed": len(kern_ms)},
            "e2e": {"value": e2e_value, "unit": "DOF-steps/s", "h2d_bytes_per_step": 2 * hu[0].numel() * 4,
                    "d2h_bytes_per_step": 2 * hu[0].numel() * 4},
            "gpu_launches": 3, "clocks": clocks}


def gpu_batched(ctx, args):
    from paper_2204_06083_gb300 import autotune
    import numpy as np
    import torch
    import eb_inputs as ei
    import paper_2204_06083_gb300 as eb
    nsteps = 50
    cfg = ei.star_batch(64, 0)
    grids = [ei.box_grid(2, nb) for nb, _ in cfg]
    lss = [ls for _, ls in cfg]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = eb.Batch(grids, lss)
    dts = [g.h for g in grids]
    B.heat_setup(dts, 1.0, vcycle_prec=eb.EB_F32)
    torch.cuda.synchronize()
    setup_ms = 1000.0 * (time.perf_counter() - t0)
    # the batched PCG in double-float (batch_set_outer_prec); FP64 beside it
    B.set_outer(eb.EB_DF64)
    tile, tune = tune_tiles(lambda: autotune.tune_batch(B, reps=5))
    u0 = B.zeros()
    f = B.zeros()
    ug = torch.zeros(max(B.num_cut, 1), dtype=torch.float64, device=ctx.dev)
    for g in range(B.count):
        X, Y = ei.grid_points(grids[g])
        B.view(u0, g).copy_(torch.tensor(ei.u_heat(X, Y, 0.0)))
        B.view(f, g).copy_(torch.tensor(-ei.f_heat(X, Y, 0.0)))
        xg = B.geometry(g).cuts()[3].cpu().numpy()
        ug[B.cut_off[g]:B.cut_off[g + 1]] = torch.tensor(ei.u_heat(xg[:, 0], xg[:, 1], 0.0))
    b1 = B.rhs(f, ug)
    u = B.zeros()

    def step():
        u.copy_(u0)
        stats = []
        for _ in range(nsteps):
            stats.append(B.heat_step(u, b1, rtol=RTOL, maxit=300))
        return stats

    res, ms_per_step, clocks = loop(ctx, args, step, torch.cuda.current_device())
    nc = B.num_cp
    value = ctx.world * nc * nsteps / (ms_per_step / 1000.0)
    launches = sum(st[0].launches for st in res[-1])
    B.set_profile(True)   # the roofline kernel's launches, in one more bench step
    ctx.flush()
    prof = step()
    B.set_profile(False)
    prof_ms = sum(st[0].prof_kernel_ms for st in prof)
    prof_n = sum(st[0].prof_launches for st in prof)
    iters = [max(s.iterations for s in st) for st in res[-1]]
    B.set_outer(eb.EB_F64)
    o64 = []
    for i in range(1 + args.steps):
        ctx.flush()
        t, st64 = timed(step)
        if i >= 1:
            o64.append(t)
    B.set_outer(eb.EB_DF64)
    fp64_outer = {"ms_per_time_step": statistics.mean(o64) / nsteps,
                  "dof_steps_per_s": nc * nsteps / (statistics.mean(o64) / 1000.0),
                  "max_iterations_per_time_step": [max(s.iterations for s in st) for st in st64]}
    # the plain FP64 AMG-PCG, geometry by geometry, on the first time step
    hs = [B.geometry(g) for g in range(B.count)]
    solvers = [eb.AMG(hs[g], 1.0 / dts[g]) for g in range(B.count)]
    us = [B.view(u0, g).contiguous() for g in range(B.count)]
    bs = [B.view(b1, g).contiguous() for g in range(B.count)]
    seq = []
    for i in range(1 + args.steps):
        uu = [v.clone() for v in us]
        ctx.flush()
        t, _ = timed(lambda: [solvers[g].heat_step(uu[g], bs[g], dts[g], theta=1.0, rtol=RTOL)
                              for g in range(B.count)])
        if i >= 1:
            seq.append(t)
    # e2e: pinned host u0 and b1 -> device, 50 steps, u -> host
    hu0 = u0.cpu().pin_memory()
    hb1 = b1.cpu().pin_memory()
    hout = torch.empty_like(hu0).pin_memory()
    db1 = torch.empty_like(b1)
    e2e = []

    def e2e_step():
        u.copy_(hu0, non_blocking=True)
        db1.copy_(hb1, non_blocking=True)
        for _ in range(nsteps):
            B.heat_step(u, db1, rtol=RTOL, maxit=300)
        hout.copy_(u, non_blocking=True)

    for i in range(1 + min(args.steps, 2)):
        ctx.flush()
        t, _ = timed(e2e_step)
        if i >= 1:
            e2e.append(t)
    e2e_value = ctx.world * nc * nsteps / (ctx.max_over_ranks(statistics.mean(e2e)) / 1000.0)
    pk, kind = peaks()
    avg_s = (prof_ms / prof_n) / 1000.0 if prof_n else float("nan")
    achieved = CHEB_BYTES_PER_DOF["f32"] * nc / avg_s / 1e9 if prof_n else None
    return {"value": value, "ms_per_step": ms_per_step,
            "dtype": "df64 outer (double-float: FP32 pairs; exit test on the FP64 true residual), f32 V-cycle",
            "num_cp": nc, "num_nodes": B.num_nodes, "setup_ms": setup_ms, "ms_per_time_step": ms_per_step / nsteps,
            "tile": tile, "autotune_us_per_vcycle": tune,
            "max_iterations_per_time_step": iters, "fp64_outer": fp64_outer,
            "sequential_fp64": {"ms_per_time_step": statistics.mean(seq),
                                "dof_per_s": nc / (statistics.mean(seq) / 1000.0)},
            "roofline": {"bound": "hbm", "kernel": "k_g_cheb_step<2, float, float> (batch view)",
                         "achieved": achieved, "peak": pk["hbm_gbs"], "peak_kind": kind, "unit": "GB/s",
                         "frac": (achieved / pk["hbm_gbs"]) if achieved else None, "traffic": None,
                         "algorithmic_bytes_per_launch": CHEB_BYTES_PER_DOF["f32"] * nc,
                         "avg_launch_us": avg_s * 1e6, "launches_timed": prof_n, "timing": PROF_NOTE},
            "e2e": {"value": e2e_value, "unit": "DOF/s", "h2d_bytes_per_step": 2 * hu0.numel() * 8,
                    "d2h_bytes_per_step": hu0.numel() * 8},
            "gpu_launches": launches, "clocks": clocks}


def gpu_learned(ctx, args):
    from paper_2204_06083_gb300 import autotune
    import numpy as np
    import torch
    import eb_inputs as ei
    import paper_2204_06083_gb300 as eb
    from paper_2204_06083_gb300 import learned
    ntrain, per, npairs, batch = 512, 8, 20000, 16
    t0 = time.perf_counter()
    geos = [(ei.box_grid(2, ntrain), ei.random_star(10000 + i)) for i in range(npairs // per)]
    store = learned.make_pairs(geos, per, seed=1)
    pairs_s = time.perf_counter() - t0
    net = eb.Net(learned.init_params(8))
    t0 = time.perf_counter()
    log = learned.train(net, store, steps=npairs // batch, batch=batch, lr=1e-3, seed=2, log_every=125)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del store
    grid, ls = ei.box_grid(2, 2048), ei.random_star(999)
    h = eb.EB(grid, ls)
    amg = eb.AMG(h)
    nc = h.info.num_cp
    tile, tune = tune_tiles(lambda: autotune.tune_amg(amg, reps=10))
    pts = ei.grid_points(grid)
    xg = h.cuts()[3].cpu().numpy()
    b = h.rhs(torch.tensor(ei.f_k1(*pts), device=ctx.dev), torch.tensor(ei.u_k1(xg[:, 0], xg[:, 1]), device=ctx.dev))
    x = torch.zeros_like(b)

    def step():
        x.zero_()
        return eb.solve_nn(amg, net, b, x=x, rtol=RTOL, maxit=400, mode=eb.EB_NN_PLAIN, allow_noconv=True)[1]

    sts, ms_per_step, clocks = loop(ctx, args, step, torch.cuda.current_device())
    value = ctx.world * nc / (ms_per_step / 1000.0)
    prof_ms, prof_n = profiled(ctx, args, lambda: eb.solve_nn(amg, net, b, x=x.zero_(), rtol=RTOL, maxit=400,
                                                              mode=eb.EB_NN_PLAIN, profile=2, allow_noconv=True)[1])
    compare = {}
    for name, fn in (("plain_fp64_amg_pcg", lambda: amg.solve(b, x=x, rtol=RTOL, maxit=400)[1]),
                     ("stage_energy_step", lambda: eb.solve_nn(amg, net, b, x=x, rtol=RTOL, maxit=400,
                                                               mode=eb.EB_NN_ENERGY, allow_noconv=True)[1])):
        tt = []
        for i in range(1 + args.steps):
            x.zero_()
            ctx.flush()
            t, st = timed(fn)
            if i >= 1:
                tt.append(t)
        compare[name] = {"time_to_tol_ms": statistics.mean(tt), "iterations": st.iterations,
                         "converged": bool(st.converged)}
    hb = b.cpu().pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    db = torch.empty_like(b)
    e2e = []

    def e2e_step():
        db.copy_(hb, non_blocking=True)
        x.zero_()
        eb.solve_nn(amg, net, db, x=x, rtol=RTOL, maxit=400, allow_noconv=True)
        hx.copy_(x, non_blocking=True)

    for i in range(1 + args.steps):
        ctx.flush()
        t, _ = timed(e2e_step)
        if i >= 1:
            e2e.append(t)
    e2e_value = ctx.world * nc / (ctx.max_over_ranks(statistics.mean(e2e)) / 1000.0)
    pk, kind = peaks()
    px = int(grid.n[0]) * int(grid.n[1])
    avg_s = (prof_ms / prof_n) / 1000.0 if prof_n else float("nan")
    return {"value": value, "ms_per_step": ms_per_step, "dtype": "f64 outer, bf16 CNN (f32 accumulate)",
            "num_cp": nc, "iterations": sts[-1].iterations, "converged": bool(sts[-1].converged),
            "tile": tile, "autotune_us_per_vcycle": tune,
            "time_to_tol_ms": ms_per_step, "compare": compare,
            "training": {"pairs": npairs, "pair_generation_s": pairs_s, "train_s": train_s, "adam_steps": npairs // batch,
                         "batch": batch, "loss_log": log},
            # the stage's network: one fused launch per application
            "roofline": net_roofline(avg_s, px, prof_n, PROF_NOTE, sustained=True),
            "e2e": {"value": e2e_value, "unit": "DOF/s", "h2d_bytes_per_step": hb.numel() * 8,
                    "d2h_bytes_per_step": hx.numel() * 8},
            "gpu_launches": sts[-1].launches, "clocks": clocks}


def net_roofline(avg_s, px, n, timing, sustained):
    """Roofline of the one-launch forward k_net_fwd: far above the ridge (73728
    tensor FLOP per 12 bytes of HBM traffic per pixel), so the tensor roof
    binds; its HBM figure rides along."""
    pk, kind = peaks()
    peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")) if sustained else pk.get("bf16_tflops")
    ok = n and avg_s == avg_s
    ach = NET_TENSOR_FLOP_PER_PX * px / avg_s / 1e12 if ok else None
    gbs = NET_BYTES_PER_PX * px / avg_s / 1e9 if ok else None
    return {"bound": "tensor", "kernel": "k_net_fwd (all six layers in one launch: layers 2-5 on tcgen05 with TMEM "
                                        "accumulators, activations kept in shared memory)",
            "achieved": ach, "peak": peak,
            "peak_kind": kind + (" bf16 sustained" if sustained else " bf16 burst"), "unit": "TFLOP/s",
            "frac": (ach / peak) if ach else None, "traffic": recorded_traffic("k_net_fwd"),
            "algorithmic_flops_per_launch": NET_TENSOR_FLOP_PER_PX * px,
            "all_layers_tflops": NET_FLOP_PER_PX * px / avg_s / 1e12 if ok else None,
            "avg_launch_us": avg_s * 1e6, "launches_timed": n, "timing": timing,
            "hbm": {"achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": (gbs / pk["hbm_gbs"]) if gbs else None,
                    "algorithmic_bytes_per_launch": NET_BYTES_PER_PX * px}}


def gpu_conv(ctx, args):
    import numpy as np
    import torch
    import eb_inputs as ei
    import paper_2204_06083_gb300 as eb
    from paper_2204_06083_gb300 import learned
    n = 2048
    h = eb.EB(ei.box_grid(2, n), ei.random_star(999))
    cp = ((h.classes() & eb.CODE_CP) != 0).float()
    rng = np.random.default_rng(0)
    inp = torch.empty((1, n, n, 2), dtype=torch.float32, device=ctx.dev)
    inp[0, :, :, 0] = torch.from_numpy(rng.standard_normal((n, n)).astype(np.float32)).cuda() * cp
    inp[0, :, :, 1] = cp
    out = torch.empty((1, n, n), dtype=torch.float32, device=ctx.dev)
    net = eb.Net(learned.init_params(8))

    def step():
        net.forward(inp, out)

    _, ms_per_step, clocks = loop(ctx, args, step, torch.cuda.current_device())
    px = n * n
    value = ctx.world * px / (ms_per_step / 1000.0)
    net.set_profile(True)  # the fused launch, in as many forwards right after the timed ones
    for _ in range(args.steps):
        ctx.flush()
        net.forward(inp, out)
    fz_ms, fz_n = net.profile()
    net.status()
    # the layer-by-layer launches on the same input, for comparison: the whole
    # forward and its 32 -> 32 convolution launches
    net.set_fused(False)
    ref_out = out.clone()
    net.forward(inp, out)
    same = bool(torch.equal(out, ref_out))
    net.profile()
    lay = []
    for _ in range(args.steps):
        ctx.flush()
        t, _ = timed(lambda: net.forward(inp, out))
        lay.append(t)
    conv_ms, conv_n = net.profile()
    net.set_profile(False)
    net.set_fused(True)
    net.status()
    hin = inp.cpu().pin_memory()
    hout = torch.empty_like(out, device="cpu").pin_memory()
    din = torch.empty_like(inp)
    e2e = []
    for i in range(1 + args.steps):
        ctx.flush()
        t, _ = timed(lambda: (din.copy_(hin, non_blocking=True), net.forward(din, out),
                              hout.copy_(out, non_blocking=True)))
        if i >= 1:
            e2e.append(t)
    e2e_value = ctx.world * px / (ctx.max_over_ranks(statistics.mean(e2e)) / 1000.0)
    pk, kind = peaks()
    fz_s = (fz_ms / fz_n) / 1000.0 if fz_n else float("nan")
    avg_s = (conv_ms / conv_n) / 1000.0 if conv_n else float("nan")
    achieved = CONV_FLOP_PER_PX * px / avg_s / 1e12 if conv_n else None
    peak = pk.get("bf16_tflops", pk.get("bf16_tflops_sustained"))
    hbm_ach = CONV_BYTES_PER_PX * px / avg_s / 1e9 if conv_n else None
    return {"value": value, "ms_per_step": ms_per_step, "dtype": "bf16 (f32 accumulate)",
            "roofline": net_roofline(fz_s, px, fz_n, "CUDA events around the fused launch, one forward after each "
                                     "512 MB L2 flush", sustained=False),
            "layered": {
                "ms_per_forward": statistics.mean(lay), "bitwise_equal_to_fused": same,
                "launches_per_forward": 6,
                # 144 FLOP per byte moved, below the ridge: HBM is the roof that binds a single convolution
                "conv_roofline": {
                    "bound": "hbm",
                    "kernel": "k_conv32_tma (32->32 implicit-GEMM conv: TMA-fed tcgen05 pipeline, TMEM)",
                    "achieved": hbm_ach, "peak": pk["hbm_gbs"], "peak_kind": kind, "unit": "GB/s",
                    "frac": (hbm_ach / pk["hbm_gbs"]) if hbm_ach else None,
                    "traffic": recorded_traffic("k_conv32_tma"),
                    "algorithmic_bytes_per_launch": CONV_BYTES_PER_PX * px, "avg_launch_us": avg_s * 1e6,
                    "launches_timed": conv_n,
                    "tensor": {"achieved": achieved, "peak": peak, "peak_kind": kind + " bf16 burst",
                               "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                               "algorithmic_flops_per_launch": CONV_FLOP_PER_PX * px}}},
            "e2e": {"value": e2e_value, "unit": "pixels/s", "h2d_bytes_per_step": hin.numel() * 4,
                    "d2h_bytes_per_step": hout.numel() * 4},
            "gpu_launches": 1, "clocks": clocks}


def _smoother_roofline(solver, nc, bytes_per_dof, note):
    """Level-0 smoothing step of the workload's hierarchy timed on its own
    (amg_time_kernel, DRAM-cold), against the measured HBM peak."""
    hbm = pk_hbm()
    cold = solver.time_smoother_step(0, ALONE_LAUNCHES, L2_CLEAR_BYTES)
    warm = solver.time_smoother_step(0, 4 * ALONE_LAUNCHES, 0)
    alg = bytes_per_dof * nc
    import paper_2204_06083_gb300 as eb
    cu = eb.time_copy_us(alg, ALONE_LAUNCHES, L2_CLEAR_BYTES)
    return {"size_matched_copy": {"copy_us": cu, "frac_of_copy": cu / cold},
            "bound": "hbm", "kernel": f"k_g_cheb_step (level-0 Chebyshev step, {note})",
            "achieved": alg / (cold * 1e-6) / 1e9, "peak": hbm, "peak_kind": "measured HBM copy (burst: kernel timed "
            "alone)", "unit": "GB/s", "frac": alg / (cold * 1e-6) / 1e9 / hbm, "traffic": None,
            "algorithmic_bytes_per_launch": alg, "avg_launch_us": cold, "timing": ALONE_NOTE, "warm_l2_us": warm,
            "warm_l2_frac": alg / (warm * 1e-6) / 1e9 / hbm}


def _e2e_loop(ctx, args, fn):
    ts = []
    for i in range(1 + args.steps):
        ctx.flush()
        t, _ = timed(fn)
        if i >= 1:
            ts.append(t)
    return ctx.max_over_ranks(statistics.mean(ts))


def gpu_paper(ctx, args, w):
    """The paper's experiments beyond the default workload, on the GPU path."""
    import numpy as np
    import torch
    import eb_inputs as ei
    import paper_2204_06083_gb300 as eb
    dev = ctx.dev
    extra = {}
    if w == "heat_cn":
        nsteps = 50
        grid, ls = ei.heat_disk(2048)
        h = eb.EB(grid, ls)
        h.set_beta(ei.beta_half_points(grid, ei.beta_heat_disk))
        dt, theta = grid.h, 0.5
        solver = eb.AMG(h, 1.0 / (theta * dt), vcycle_prec=eb.EB_F32)
        X, Y = ei.grid_points(grid)
        zc = torch.zeros(max(h.info.num_cut, 1), dtype=torch.float64, device=dev)
        bs = [h.rhs(torch.tensor(-ei.f_heat_disk(X, Y, k * dt), device=dev), zc) for k in range(nsteps + 1)]
        u0 = torch.tensor(ei.u_heat_disk(X, Y, 0.0), device=dev)
        u = torch.empty_like(u0)
        its = []

        def run(uu):
            out = []
            for k in range(nsteps):
                out.append(solver.heat_step(uu, bs[k + 1], dt, theta=theta, b0=bs[k], rtol=RTOL, maxit=300))
            return out

        def step():
            u.copy_(u0)
            return run(u)

        solver.set_outer(eb.EB_DF64)  # the solves in double-float; FP64 outer iteration timed beside
        res, ms, clocks = loop(ctx, args, step, torch.cuda.current_device())
        nc = h.info.num_cp
        value = ctx.world * nc * nsteps / (ms / 1000.0)
        solver.set_outer(eb.EB_F64)
        t64 = []
        for i in range(1 + args.steps):
            ctx.flush()
            t, r64 = timed(step)
            if i >= 1:
                t64.append(t)
        solver.set_outer(eb.EB_DF64)
        hu = u0.cpu().pin_memory()
        ho = torch.empty_like(hu).pin_memory()

        def e2e_step():
            u.copy_(hu, non_blocking=True)
            run(u)
            ho.copy_(u, non_blocking=True)

        e2e = ctx.world * nc * nsteps / (_e2e_loop(ctx, args, e2e_step) / 1000.0)
        nodes, _ = h.cp_data()
        nodes = nodes.cpu().numpy()
        err = float(np.abs(ho.numpy().reshape(-1)[nodes] - ei.u_heat_disk(X, Y, nsteps * dt).reshape(-1)[nodes]).max())
        extra = {"iterations_per_step": statistics.mean(st.iterations for st in res[-1]),
                 "max_err_vs_exact_at_t": err, "t_end": nsteps * dt,
                 "fp64_outer": {"ms_per_step": statistics.mean(t64),
                                "iterations_per_step": statistics.mean(st.iterations for st in r64)}}
        roof = _smoother_roofline(solver, nc, 28, "FP32, variable beta: x, b, d, beta_x, beta_y read, x, d written")
        launches = sum(st.launches for st in res[-1])
        e2e_bytes = (hu.numel() * 8, ho.numel() * 8)
    elif w == "wave_theta":
        nsteps, theta = 100, 1.0 / 12.0
        grid, ls = ei.disk_bessel(1602)
        h = eb.EB(grid, ls)
        dt = 0.85 * grid.h
        # FP32 V-cycle with the solves in double-float; the FP64 V-cycle with
        # the FP64 outer iteration timed beside
        solver = eb.AMG(h, 1.0 / (theta * dt * dt), vcycle_prec=eb.EB_F32)
        solver.set_outer(eb.EB_DF64)
        X, Y = ei.grid_points(grid)
        a0 = torch.tensor(ei.bessel_mode(X, Y, -dt), device=dev) * ((h.classes() & eb.CODE_CP) != 0)
        b0 = torch.tensor(ei.bessel_mode(X, Y, 0.0), device=dev) * ((h.classes() & eb.CODE_CP) != 0)
        ua, ub = torch.empty_like(a0), torch.empty_like(b0)

        def step():
            ua.copy_(a0)
            ub.copy_(b0)
            return solver.wave_theta_step(ua, ub, dt, theta, nsteps, rtol=RTOL, maxit=300)

        res, ms, clocks = loop(ctx, args, step, torch.cuda.current_device())
        nc = h.info.num_cp
        value = ctx.world * nc * nsteps / (ms / 1000.0)
        ha, hb_ = a0.cpu().pin_memory(), b0.cpu().pin_memory()
        oa, ob = torch.empty_like(ha).pin_memory(), torch.empty_like(hb_).pin_memory()

        def e2e_step():
            ua.copy_(ha, non_blocking=True)
            ub.copy_(hb_, non_blocking=True)
            solver.wave_theta_step(ua, ub, dt, theta, nsteps, rtol=RTOL, maxit=300)
            oa.copy_(ua, non_blocking=True)
            ob.copy_(ub, non_blocking=True)

        e2e = ctx.world * nc * nsteps / (_e2e_loop(ctx, args, e2e_step) / 1000.0)
        s64 = eb.AMG(h, 1.0 / (theta * dt * dt))
        t64 = []
        for i in range(1 + args.steps):
            ua.copy_(a0)
            ub.copy_(b0)
            ctx.flush()
            t, r64 = timed(lambda: s64.wave_theta_step(ua, ub, dt, theta, nsteps, rtol=RTOL, maxit=300))
            if i >= 1:
                t64.append(t)
        s64.close()
        extra = {"iterations_per_step": res[-1].iterations / nsteps, "dt_over_h": 0.85, "theta": theta,
                 "fp64_vcycle_fp64_outer": {"ms_per_step": statistics.mean(t64),
                                            "iterations_per_step": r64.iterations / nsteps}}
        roof = _smoother_roofline(solver, nc, 20, "FP32: x, b, d read, x, d written")
        launches = int(res[-1].launches)
        e2e_bytes = (2 * ha.numel() * 8, 2 * oa.numel() * 8)
    elif w == "helmholtz":
        grid, ls = ei.helmholtz_star(802)
        h = eb.EB(grid, ls)
        solver = eb.AMG(h, 0.0)
        sigma = -ei.HELMHOLTZ_OMEGA ** 2
        zc = torch.zeros(max(h.info.num_cut, 1), dtype=torch.float64, device=dev)
        b = h.rhs(torch.tensor(ei.hat_source(grid), device=dev), zc)
        x = torch.zeros_like(b)

        def step():
            x.zero_()
            return solver.minres(b, sigma, x=x, rtol=RTOL, maxit=20000)[1]

        res, ms, clocks = loop(ctx, args, step, torch.cuda.current_device())
        nc = h.info.num_cp
        value = ctx.world * nc / (ms / 1000.0)
        hb, hx = b.cpu().pin_memory(), torch.empty_like(b.cpu()).pin_memory()
        db = torch.empty_like(b)

        def e2e_step():
            db.copy_(hb, non_blocking=True)
            x.zero_()
            solver.minres(db, sigma, x=x, rtol=RTOL, maxit=20000)
            hx.copy_(x, non_blocking=True)

        e2e = ctx.world * nc / (_e2e_loop(ctx, args, e2e_step) / 1000.0)
        extra = {"iterations": res[-1].iterations, "true_rel_residual": res[-1].true_rel_residual,
                 "omega": ei.HELMHOLTZ_OMEGA}
        roof = _smoother_roofline(solver, nc, 40, "FP64 V-cycle of the Laplacian: x, b, d read, x, d written")
        launches = int(res[-1].launches)
        e2e_bytes = (hb.numel() * 8, hx.numel() * 8)
    elif w == "qoi":
        th = np.linspace(0.0, math.pi, 64, endpoint=False)
        cases = [ei.qoi_rotated(t) for t in th]
        grids = [g for g, _ in cases]
        B = eb.Batch(grids, [l for _, l in cases])
        B.heat_setup([math.inf] * len(cases), theta=1.0, vcycle_prec=eb.EB_F32)
        B.set_outer(eb.EB_DF64)  # the per-geometry PCG in double-float
        f, wq = B.zeros(), B.zeros()
        for g, gr in enumerate(grids):
            B.view(f, g).fill_(ei.QOI_F)
            B.view(wq, g).copy_(torch.tensor(ei.qoi_rect_weights(gr)))
        ug = torch.zeros(max(B.num_cut, 1), dtype=torch.float64, device=dev)
        b = B.rhs(f, ug)
        u = B.zeros()

        def step():
            u.zero_()
            st = B.heat_step(u, b, rtol=RTOL, maxit=500)
            return st, B.weighted_sum(wq, u)

        res, ms, clocks = loop(ctx, args, step, torch.cuda.current_device())
        nc = B.num_cp
        value = ctx.world * nc / (ms / 1000.0)
        hb, hq = b.cpu().pin_memory(), torch.empty(len(cases), dtype=torch.float64).pin_memory()
        db = torch.empty_like(b)

        def e2e_step():
            db.copy_(hb, non_blocking=True)
            u.zero_()
            B.heat_step(u, db, rtol=RTOL, maxit=500)
            hq.copy_(B.weighted_sum(wq, u), non_blocking=True)

        e2e = ctx.world * nc / (_e2e_loop(ctx, args, e2e_step) / 1000.0)
        q = hq.numpy()
        exact = np.array([ei.qoi_rotated_exact(t) for t in th])
        extra = {"geometries": len(cases), "qoi_max_rel_dev_from_closed_form": float(np.max(np.abs(q - exact) / np.abs(exact))),
                 "iterations": max(s.iterations for s in res[-1][0])}
        # the level-0 smoother launches of one more sweep, timed with events
        B.set_profile(True)
        ctx.flush()
        pst, _ = step()
        B.set_profile(False)
        pms, pn = pst[0].prof_kernel_ms, pst[0].prof_launches
        psec = (pms / pn) / 1000.0 if pn else float("nan")
        alg = CHEB_BYTES_PER_DOF["f32"] * nc
        roof = {"bound": "hbm", "kernel": "k_g_cheb_step<2, float, float> (level-0 Chebyshev step, batch view)",
                "achieved": alg / psec / 1e9, "peak": pk_hbm(), "peak_kind": "measured HBM copy (burst)",
                "unit": "GB/s", "frac": alg / psec / 1e9 / pk_hbm(), "traffic": None,
                "algorithmic_bytes_per_launch": alg, "avg_launch_us": psec * 1e6, "launches_timed": pn,
                "timing": PROF_NOTE + "; each bracketed launch carries the event pair's few microseconds"}
        launches = int(res[-1][0][0].launches)
        e2e_bytes = (hb.numel() * 8, hq.numel() * 8)
    elif w == "rs_w":
        grid, ls = ei.star_wave(2048)
        h = eb.EB(grid, ls)
        solver = eb.AMG(h, 0.0, coarsening=eb.EB_AMG_RS, cycle=2)
        X, Y = ei.grid_points(grid)
        xg = h.cuts()[3].cpu().numpy()
        b = h.rhs(torch.tensor(ei.f_k1(X, Y), device=dev), torch.tensor(ei.u_k1(xg[:, 0], xg[:, 1]), device=dev))
        x = torch.zeros_like(b)

        def step():
            x.zero_()
            return solver.solve(b, x=x, rtol=RTOL, maxit=300)[1]

        res, ms, clocks = loop(ctx, args, step, torch.cuda.current_device())
        nc = h.info.num_cp
        value = ctx.world * nc / (ms / 1000.0)
        hb, hx = b.cpu().pin_memory(), torch.empty_like(b.cpu()).pin_memory()
        db = torch.empty_like(b)

        def e2e_step():
            db.copy_(hb, non_blocking=True)
            x.zero_()
            solver.solve(db, x=x, rtol=RTOL, maxit=300)
            hx.copy_(x, non_blocking=True)

        e2e = ctx.world * nc / (_e2e_loop(ctx, args, e2e_step) / 1000.0)
        sa = eb.AMG(h, 0.0)
        xs = torch.zeros_like(b)
        tsa = []
        for i in range(1 + args.steps):
            xs.zero_()
            ctx.flush()
            t, st_sa = timed(lambda: sa.solve(b, x=xs, rtol=RTOL, maxit=300)[1])
            if i >= 1:
                tsa.append(t)
        extra = {"iterations": res[-1].iterations, "amg_levels": solver.rows,
                 "operator_complexity": solver.operator_complexity,
                 "sa_v_cycle": {"time_to_tol_ms": statistics.mean(tsa), "iterations": st_sa.iterations}}
        roof = _smoother_roofline(solver, nc, 40, "FP64: x, b, d read, x, d written")
        launches = int(res[-1].launches)
        e2e_bytes = (hb.numel() * 8, hx.numel() * 8)
    else:  # mixed
        grid, ls = ei.helmholtz_star(4096)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = eb.EB(grid, ls, closure=eb.EB_CLOSURE_MIXED)
        torch.cuda.synchronize()
        build_ms = 1000.0 * (time.perf_counter() - t0)
        t0 = time.perf_counter()
        h_line = eb.EB(grid, ls)
        torch.cuda.synchronize()
        build_line_ms = 1000.0 * (time.perf_counter() - t0)
        solver = eb.AMG(h, 0.0, vcycle_prec=eb.EB_F32)
        X, Y = ei.grid_points(grid)
        pts = h.sample_points().cpu().numpy()
        b = h.rhs(torch.tensor(ei.f_k1(X, Y), device=dev), torch.tensor(ei.u_k1(pts[:, 0], pts[:, 1]), device=dev))
        x = torch.zeros_like(b)

        def step():
            x.zero_()
            return solver.solve(b, x=x, rtol=RTOL, maxit=300, outer=eb.EB_DF64)[1]

        res, ms, clocks = loop(ctx, args, step, torch.cuda.current_device())
        nc = h.info.num_cp
        value = ctx.world * nc / (ms / 1000.0)
        hb, hx = b.cpu().pin_memory(), torch.empty_like(b.cpu()).pin_memory()
        db = torch.empty_like(b)

        def e2e_step():
            db.copy_(hb, non_blocking=True)
            x.zero_()
            solver.solve(db, x=x, rtol=RTOL, maxit=300, outer=eb.EB_DF64)
            hx.copy_(x, non_blocking=True)

        e2e = ctx.world * nc / (_e2e_loop(ctx, args, e2e_step) / 1000.0)
        nodes = h.cp_data()[0].cpu().numpy()
        err = float(np.abs(hx.numpy().reshape(-1)[nodes] - ei.u_k1(X, Y).reshape(-1)[nodes]).max())
        extra = {"iterations": res[-1].iterations, "num_rbf_cuts": h.info.num_rbf, "num_cuts": h.info.num_cut,
                 "build_mixed_ms": build_ms, "build_line_ms": build_line_ms, "max_err_vs_exact": err}
        roof = _smoother_roofline(solver, nc, 20, "FP32: x, b, d read, x, d written")
        launches = int(res[-1].launches)
        e2e_bytes = (hb.numel() * 8, hx.numel() * 8)
    dtype = ("df64 outer (double-float: FP32 pairs; exit test on the FP64 true residual), f32 V-cycle"
             if w in ("qoi", "mixed", "heat_cn", "wave_theta") else "f64 outer (V-cycle as stated in config)")
    line = {"value": value, "ms_per_step": ms, "dtype": dtype, "num_cp": nc,
            "roofline": roof, "e2e": {"value": e2e, "unit": UNITS[w], "h2d_bytes_per_step": e2e_bytes[0],
                                      "d2h_bytes_per_step": e2e_bytes[1]},
            "gpu_launches": launches, "clocks": clocks}
    line.update(extra)
    return line


def run_gpu(args):
    ctx = Ctx()
    w = args.workload
    if w == "poisson3d":
        body = gpu_poisson(ctx, args, 3)
    elif w == "poisson2d":
        body = gpu_poisson(ctx, args, 2)
    elif w == "wave":
        body = gpu_wave(ctx, args)
    elif w == "batched":
        body = gpu_batched(ctx, args)
    elif w == "conv":
        body = gpu_conv(ctx, args)
    elif w in PAPER_WORKLOADS:
        body = gpu_paper(ctx, args, w)
    else:
        body = gpu_learned(ctx, args)
    if ctx.rank != 0:
        ctx.close()
        return 0
    cpu = None
    if ctx.world == 1 and not args.no_cpu_baseline:
        v, sample, _ = cpu_oracle_sample(w)
        cpu = {"value": v, "unit": UNITS[w], "cores": 1, "kind": "oracle", "sample": sample + ", one thread",
               "same_config": w in ("poisson3d", "poisson2d"), "host": host_cpu()}
        if w == "poisson3d":
            va, procs, rec = oracle_poisson3d_all_cores()
            cpu["all_cores"] = {"value": va, "unit": UNITS[w], "cores": procs, "kind": "oracle",
                                "sample": (f"{procs} single-threaded oracle processes (one per host core, at most 16), "
                                           f"each solving the full workload once, timed solves started together; "
                                           f"aggregate DOF/s = sum N_C / slowest solve ({rec['wall_s']:.1f} s)")}
    line = {"metric": METRIC, "value": body.pop("value"), "unit": UNITS[w], "n_gpus": ctx.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": body.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": body.pop("dtype"),
            "data": "synthetic", "config": config_of(w)}
    line.update(body)
    line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="poisson3d", choices=WORKLOADS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-loop", action="store_true",
                    help="poisson workloads: timed solves check convergence on the host after every captured "
                         "iteration instead of looping on the device (for kernel-level profilers)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
