"""Benchmark of the JFNK hot path on the 160x160, p=3 isentropic vortex.

One step = one ROW3 (ROS34PW2) time step of the 2D Euler isentropic vortex
(strength 5, M = 0.5 at 45 degrees) on a periodic 160x160 uniform mesh of
[-5,5]^2 at p = 3 (1,638,400 DOFs): R(q^n), the element-Jacobi blocks at
shift 1/(gamma dt), four stage solves with GMRES(30) to tol_rel,linear = 1e-6
(the ROW tolerance of the paper's integrator comparison), and the update.
dt = 0.05 (CFL 13.6 with CFL = dt (|V|+c)(p+1)/h), i.e. 200 steps to t = 10.

value = DOF x GMRES iterations per second (whole job, all ranks).  Inputs are
resident in HBM; the working set (element blocks 0.84 GB, Krylov basis
0.42 GB) is ~10x the L2, so no explicit L2 flush is needed.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank runs an independent replica (the method has no
data-path exchange on one GPU): barrier + synchronize around the timed
region, max time over ranks, units summed over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX = 160
P = 3
SCHEME = 3
DT = 0.05
TOL_LIN = 1e-6
METRIC = "DOF*GMRES-iters/s (plain FP64 JFNK, ROW3 step, 160x160 p=3 vortex)"
UNIT = "DOF*iter/s"
WORKLOAD = "vortex-160x160-p3-ROW3-dt0.05-gmres30-tol1e-6"
FP64_PEAK_TFLOPS = 1.259  # 152 SMs x 4 FP64 flops/clk/SM x 2.07 GHz (nominal 1.25 TF)
FP32_PEAK_TFLOPS = 80.54  # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (CUDA cores)
REF_NX = 24               # oracle sample mesh (same p, scheme, CFL, tolerance)
REF_ARM_NX = 16           # smaller sample for the per-step reference arm


def _config(extra=None):
    c = {"workload": WORKLOAD, "mesh": f"{NX}x{NX}", "p": P, "ndof": NX * NX * 4 * (P + 1) ** 2,
         "scheme": "ROW3 (ROS34PW2)", "dt": DT, "cfl": round(DT * 3 * math.sqrt(2) * (P + 1) / (10.0 / NX), 2),
         "gmres": "GMRES(30), element-Jacobi, tol 1e-6", "fd_eps": "1e-7(1+||U||)/||z||",
         "l2": "inputs larger than L2 (blocks 0.84 GB + Krylov basis 0.42 GB)"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples during the timed region (read-only query)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
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
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ oracle --
ORACLE_SAMPLE = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import synthetic as S
from oracle.fr2d import Mesh
from oracle.jfnk import Problem
from oracle.steppers import SolverOpts, step_row
from oracle.tableaus import ROW
n, p, steps = {n}, {p}, {steps}
xe, ye = S.uniform_mesh(n)
X, Y = S.point_coords(xe, ye, p)
U = S.Vortex().state(X, Y)
prob = Problem(Mesh(xe, ye), p)
opts = SolverOpts(tol_lin={tol}, m=30, max_restarts=20)
out = []
for k in range(steps):
    t0 = time.perf_counter()
    U, st = step_row(prob, ROW[{scheme}](), {dt}, U, opts)
    out.append((time.perf_counter() - t0, st.gmres_iters))
print(json.dumps({{"ndof": prob.ndof, "steps": out}}))
"""

# Oracle samples.  C2 sample: ROW3 steps of the vortex on a coarser mesh at
# the benchmark's p, CFL 13.6 and tolerance (the unit is per DOF, so the rate
# is comparable); C1: the small configuration in full (20x20 p=2, ROW2, ten
# steps of dt = 0.05, GMRES(30) to 1e-8).
C2_SAMPLE = {"n": REF_NX, "p": P, "scheme": SCHEME, "tol": TOL_LIN, "dt": DT * (NX / REF_NX)}
C1_FULL = {"n": 20, "p": 2, "scheme": 2, "tol": 1e-8, "dt": 0.05}


def _oracle_procs(sample, steps, copies):
    """Start `copies` independent oracle processes (one host thread each)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    code = ORACLE_SAMPLE.format(root=ROOT, steps=steps, **sample)
    return [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                             text=True, env=env) for _ in range(copies)]


def run_oracle(sample, steps, copies=1):
    """Run the oracle sample in `copies` concurrent single-threaded processes
    (independent replicas, one per host core); returns (ndof, wall seconds
    of the slowest, per-copy lists of (seconds, iters) per step)."""
    t0 = time.perf_counter()
    procs = _oracle_procs(sample, steps, copies)
    runs = []
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        runs.append(json.loads(out.strip().splitlines()[-1]))
    wall = time.perf_counter() - t0
    return runs[0]["ndof"], wall, [r["steps"] for r in runs]


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


def cpu_baseline():
    """The oracle on the host: the C2 sample (one ROW3 step) on one thread and
    as one replica per host core; C1 in full on one thread and one replica per
    core.  value / cores: the all-core C2-sample rate (units summed over the
    replicas / wall time)."""
    cores = host_cores()
    res = {}
    for name, sample, steps in (("c2_sample", C2_SAMPLE, 1), ("c1_full", C1_FULL, 10)):
        nd, wall1, runs1 = run_oracle(sample, steps, 1)
        it1 = sum(i for _, i in runs1[0])
        ndN, wallN, runsN = run_oracle(sample, steps, cores)
        itN = sum(sum(i for _, i in r) for r in runsN)
        res[name] = {"ndof": nd, "gmres_iters": it1,
                     "single_thread": {"seconds": wall1, "value": nd * it1 / wall1},
                     "all_cores": {"replicas": cores, "seconds": wallN, "value": nd * itN / wallN}}
    c2 = res["c2_sample"]
    return {"value": c2["all_cores"]["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"oracle (NumPy FP64, one thread per process): one ROW3 step of the {REF_NX}x{REF_NX} "
                       f"p={P} vortex ({c2['ndof']} DOFs, CFL 13.6, tol 1e-6) as {cores} concurrent replicas "
                       f"(one per host core); single-thread rate and the C1 run (20x20 p=2 ROW2, 10 steps of "
                       f"0.05, tol 1e-8) in full alongside"),
            "single_thread_value": c2["single_thread"]["value"],
            "host": {"nproc": cores, "cpu": host_cpu_model()},
            "runs": res}


def reference_arm(args):
    """The oracle as it stands, timed on the host cores: each step runs one
    ROW3 step of the coarse vortex sample on every host core (independent
    replicas, one thread each)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = host_cores()
    sample = dict(C2_SAMPLE, n=REF_ARM_NX, dt=DT * (NX / REF_ARM_NX))
    secs, units, nd = 0.0, 0.0, None
    for k in range(args.warmup + args.steps):
        nd, wall, runs = run_oracle(sample, 1, cores)
        if k >= args.warmup:
            secs += wall
            units += sum(nd * sum(i for _, i in r) for r in runs)
    value = units / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": _config({"reference_sample": f"oracle ROW3 steps on the {REF_ARM_NX}x{REF_ARM_NX} p=3 vortex, "
                                               f"same CFL and tolerance, one replica per host core"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: one oracle ROW3 step of the {REF_ARM_NX}x{REF_ARM_NX} p={P} vortex "
                                   f"({nd} DOFs, same CFL 13.6, tol 1e-6) on each of {cores} host cores "
                                   f"(NumPy, one thread per process)",
                         "host": {"nproc": cores, "cpu": host_cpu_model()}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------ our arm --
def combine_ranks(dist, slowest, summed, device):
    """Whole-job figures of independent replicas: the maximum over ranks of
    each time in `slowest`, the sum over ranks of each work count in
    `summed`.  Every rank calls it (collective); dist None: one rank."""
    if dist is None:
        return list(slowest), list(summed)
    import torch
    t = torch.tensor(list(slowest), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor(list(summed), dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return [float(x) for x in t], [float(x) for x in u]


def our_arm(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    import paper_1904_04825_gb300 as fr
    import synthetic as S

    def barrier():
        if dist is not None:
            dist.barrier()

    prec = {"fp64": 0, "fp32": 1, "bf16": 2}[args.block_precision]
    kind, order = args.scheme[:-1], int(args.scheme[-1])
    if args.workload == "vortex":
        xe, ye = S.uniform_mesh(NX)
        X, Y = S.point_coords(xe, ye, P)
        U0 = S.Vortex().state(X, Y)
        p, dt, wall = P, (args.dt or DT), False
        opts = fr.default_opts(tol_lin=TOL_LIN, gmres_m=30, gmres_max_restarts=20, block_precision=prec,
                               jv_precision=1 if args.jv_precision == "fp32" else 0,
                               riemann=1 if args.riemann == "roe" else 0)
        wl = f"vortex-160x160-p3-{args.scheme.upper()}-dt{dt:g}-gmres30-tol{TOL_LIN:g}"
    elif args.workload == "tgv":
        # Taylor-Green vortex (Sec. 5): 64^3 hexahedra at p = 3, Re 1600, Ma 0.1,
        # dt = t_c / 25, tol_lin 1e-6; element-Jacobi blocks for p <= 3 (the
        # 320-row blocks of p = 3 are stored in FP32 unless BF16 is asked for)
        tg = S.TaylorGreen()
        p = args.p or 3
        if p == 3 and prec == 0:
            prec, args.block_precision = 1, "fp32"
        n3 = args.nx or 64
        edges3 = S.uniform_mesh3d(n3)
        X, Y, Z = S.point_coords3d(*edges3, p)
        U0 = tg.state(X, Y, Z)
        del X, Y, Z
        dt, wall = (args.dt or tg.t_c / 25.0), False
        opts = fr.default_opts(tol_lin=TOL_LIN, gmres_m=args.gmres_m, m_max=args.gmres_m, gmres_max_restarts=20,
                               block_precision=prec, mu=tg.mu, prandtl=tg.prandtl, precond=1 if p <= 3 else 0,
                               block_columns=1 if args.block_columns == "fp32" and p <= 3 else 0,
                               jv_precision=1 if args.jv_precision == "fp32" else 0)
        wl = (f"taylor-green-{n3}^3-p{p}-Re1600-Ma0.1-{args.scheme.upper()}-dt{dt:g}-gmres{args.gmres_m}"
              + ("" if p <= 3 else "-noprecond") + ("-fp32columns" if args.block_columns == "fp32" else ""))
    else:
        ch = S.Channel()
        cnx, cny = args.nx or 256, args.ny or 128
        xe = np.linspace(0.0, ch.lx, cnx + 1)
        ye = S.channel_y_edges(cny, first=1e-3, ratio=1.15)
        p = args.p or P
        X, Y = S.point_coords(xe, ye, p)
        U0 = ch.state(X, Y, seed=0)
        dt, wall = (args.dt or 1e-3), True
        opts = fr.default_opts(tol_lin=TOL_LIN, gmres_m=30, gmres_max_restarts=20, block_precision=prec,
                               mu=ch.mu, prandtl=ch.prandtl, body_force_x=ch.body_force,
                               wall_temperature=ch.temperature)
        wl = f"channel-{cnx}x{cny}-p{p}-Re1000-M0.2-{args.scheme.upper()}-dt{dt:g}"
    if prec:
        wl += f"-{args.block_precision}blocks"
    if args.jv_precision == "fp32":
        wl += "-fp32linearjv"
    if args.riemann == "roe":
        wl += "-roe"
    if args.workload == "tgv":
        ctx = fr.Context3D(*edges3, p, opts)
    else:
        ctx = fr.Context(xe, ye, p, opts, wall_y=wall)
    U = torch.from_numpy(U0).to(dev)
    del U0
    Uprev = torch.empty_like(U)
    tuned = None
    if not args.no_autotune:
        # launch configuration (vector-kernel grid, residual tile) measured on
        # full GMRES cycles at this step's shift, before any timing
        gam = {"row": {2: 0.43586652150845900, 3: 0.435866521508459, 4: 0.25}}.get(kind, {}).get(order, 0.5)
        vb, tv, ms_best, ms_def = fr.autotune(ctx, U, 1.0 / (gam * dt), reps=2)
        tuned = {"vec_blocks": vb, "tile_variant": tv, "cycle_ms": ms_best, "cycle_ms_default": ms_def}
    stream = torch.cuda.current_stream()
    ptc = fr.default_ptc_opts(tol_nl=1e-6, tol_lin=1e-1)
    nstep = [0]

    def one_step(Ucur):
        if kind == "row":
            st = fr.step_row(ctx, order, dt, Ucur)
        elif kind == "esdirk":
            st = fr.step_esdirk(ctx, order, dt, Ucur, ptc)
        else:
            st = fr.step_bdf2(ctx, dt, Ucur, Uprev, nstep[0] == 0, ptc)
        nstep[0] += 1
        return st

    # warm-up, with every kernel family timed to find the dominant one
    fr.fr_profile_begin(ctx)
    for _ in range(args.warmup):
        one_step(U)
    warm = fr.fr_profile_end(ctx)
    top = max(warm, key=lambda k: warm[k]["ms"])
    breakdown = {k: {"ms_per_step": v["ms"] / args.warmup, "launches_per_step": v["launches"] / args.warmup,
                     "tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12) if v["ms"] > 0 else None}
                 for k, v in warm.items()}

    # timed region: device-resident inputs, no per-launch instrumentation
    launches0 = fr.fr_kernel_launches()
    clocks = ClockSampler(dev)
    clocks.start()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters = 0
    e0.record(stream)
    for _ in range(args.steps):
        st = one_step(U)
        iters += st.gmres_iters
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = fr.fr_kernel_launches() - launches0

    # kernel timing pass: the same number of steps again, with CUDA events
    # around every launch of the dominant family on its launching stream
    fr.fr_profile_begin(ctx, [top])
    for _ in range(args.steps):
        one_step(U)
    torch.cuda.synchronize()
    prof = fr.fr_profile_end(ctx)[top]

    # end to end through the public API from pinned host memory
    host_in = torch.from_numpy(U.cpu().numpy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    Ud = torch.empty_like(U)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(args.steps):
        Ud.copy_(host_in, non_blocking=True)
        st = one_step(Ud)
        e2e_iters += st.gmres_iters
        host_out.copy_(Ud, non_blocking=True)
        torch.cuda.synchronize()
        host_in, host_out = host_out, host_in
    e2e_s = time.perf_counter() - t0

    ndof = ctx.ndof
    units = float(ndof) * iters
    e2e_units = float(ndof) * e2e_iters
    (ms, e2e_s), (units, e2e_units) = combine_ranks(dist, [ms, e2e_s], [units, e2e_units], dev)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # workload description from the context actually built
    m_used = ctx.opts.gmres_m
    nb = ctx.ndof // ctx.ne
    blk_bytes = ctx.ne * nb * nb * (8, 4, 2)[prec] if ctx.opts.precond else 0
    basis_bytes = (m_used + 1) * ctx.ndof * 8
    gmres_desc = (f"GMRES({m_used}), " + ("element-Jacobi" if ctx.opts.precond else "no preconditioner")
                  + f", tol {ctx.opts.tol_lin:g}")
    l2_desc = f"inputs larger than L2 (blocks {blk_bytes / 1e9:.2f} GB + Krylov basis {basis_bytes / 1e9:.2f} GB)"
    if args.workload == "vortex":
        cfl = round(dt * 3 * math.sqrt(2) * (p + 1) / (10.0 / NX), 2)
    elif args.workload == "tgv":   # (|v|max + c0)(p+1) dt / h with |v|max = V0, c0 = V0 / Ma
        cfl = round(dt * (1.0 + 10.0) * (p + 1) / (2 * math.pi / ctx.nx), 2)
    else:
        cfl = None
    avg_launch_s = prof["ms"] / max(prof["launches"], 1) * 1e-3
    work_flops = prof["flops"] / max(prof["launches"], 1)
    work_bytes = prof["bytes"] / max(prof["launches"], 1)
    achieved_tf = work_flops / avg_launch_s / 1e12
    achieved_gbs = work_bytes / avg_launch_s / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    alu_peak, alu_src = FP64_PEAK_TFLOPS, "FP64 FMA pipe: 152 SMs x 4 flops/clk x 2.07 GHz (derived, nominal 1.25 TF)"
    if top == "jv" and args.jv_precision == "fp32":
        alu_src += ("; the algorithmic count includes the linear parts, which this product runs in FP32, "
                    "so the fraction of the FP64 peak can exceed 1")
    if top == "invert" and prec:   # reduced-precision blocks are inverted in FP32 on the CUDA cores
        alu_peak, alu_src = FP32_PEAK_TFLOPS, "FP32 FMA: 152 SMs x 128 lanes x 2 flops x 2.07 GHz (derived)"
    roofline = {
        "kernel": top, "bound": "alu", "achieved": achieved_tf, "peak": alu_peak,
        "unit": "TFLOP/s", "frac": achieved_tf / alu_peak,
        "traffic": None,
        "peak_source": alu_src,
        "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"},
        "avg_launch_us": avg_launch_s * 1e6, "launches_timed": prof["launches"],
        "algorithmic_bytes_per_launch": work_bytes, "algorithmic_flops_per_launch": work_flops,
    }
    traffic_file = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(traffic_file) and args.workload == "vortex":   # captured on the vortex kernels
        try:
            tr = json.load(open(traffic_file)).get(top)
            if tr:
                roofline["traffic"] = tr["dram_bytes_per_launch"]
        except (OSError, ValueError):
            pass

    default_line = (prec == 0 and args.workload == "vortex" and args.scheme == "row3" and not args.dt
                    and args.jv_precision == "fp64" and args.riemann == "rusanov")
    t_end = None
    if world == 1 and default_line and not args.no_t_end:
        ctx.close()
        torch.cuda.empty_cache()
        plain = run_t_end(T_END_PLAIN, sample_clocks=True)
        mixed = run_t_end(T_END_MIXED, sample_clocks=True)
        t_end = {"t_end": 10.0, "plain_fp64": plain, "mixed": mixed,
                 "speedup": (plain["time_to_t_end_s"] / mixed["time_to_t_end_s"])
                 if "time_to_t_end_s" in plain and "time_to_t_end_s" in mixed else None,
                 "note": "both arms run one period of the 160x160 p=3 vortex through the public API "
                         "(wall time from the first step to the last, host waits included); E(rho), E(u) "
                         "by the Sec. 5.1 norm on the GPU"}

    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.workload == "vortex" and args.scheme == "row3":
        cpu = cpu_baseline()

    line = {
        "metric": METRIC if default_line else f"DOF*GMRES-iters/s ({wl})",
        "value": units / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": _config({"parallelism": f"replicas x{world}", "gmres_iters_per_step": iters / args.steps,
                           "p": p, "cfl": cfl, "gmres": gmres_desc, "l2": l2_desc,
                           "block_precision": args.block_precision, "jv_precision": args.jv_precision,
                           "workload": wl,
                           "scheme": args.scheme.upper(), "dt": dt, "ndof": ctx.ndof,
                           "mesh": f"{ctx.nx}x{ctx.ny}" + (f"x{ctx.nz}" if args.workload == "tgv" else ""),
                           "launch_config": tuned,
                           "kernel_timing": "roofline.avg_launch_us from a second pass of the same number of "
                                            "steps with CUDA events around each launch of the dominant family; "
                                            "the timed steps run without events"}),
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roofline,
        "kernel_breakdown": breakdown,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * ndof,
                "d2h_bytes_per_step": 8 * ndof},
        "time_to_t_end": t_end,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_t_end(cfg, autotune=True, sample_clocks=False):
    """Run the vortex workload to t_end through the public API and measure
    the wall time, GMRES iterations and the Sec. 5.1 errors E(rho), E(u)
    against the advected exact vortex (fr_vortex_error, on the GPU).
    cfg keys: scheme, cfl or dt, t_end, nx, p, box, tol, tol_lin, gmres_m,
    eps_fixed, block_precision, jv_precision, riemann, guess, precond_refresh."""
    import torch
    import paper_1904_04825_gb300 as fr
    import synthetic as S

    prec = {"fp64": 0, "fp32": 1, "bf16": 2}[cfg["block_precision"]]
    kind, order = cfg["scheme"][:-1], int(cfg["scheme"][-1])
    nx, p, L = cfg["nx"], cfg["p"], cfg["box"]
    box = (-L / 2, L / 2, -L / 2, L / 2)
    xe, ye = S.uniform_mesh(nx, box=box)
    X, Y = S.point_coords(xe, ye, p)
    U = torch.from_numpy(S.Vortex().state(X, Y, box=box)).cuda()
    del X, Y
    Uprev = torch.empty_like(U)
    h = L / nx
    dt = cfg.get("dt") or cfg["cfl"] * h / (3 * math.sqrt(2) * (p + 1))
    nsteps = int(round(cfg["t_end"] / dt))
    dt = cfg["t_end"] / nsteps
    tol = cfg["tol"]
    ctx = fr.Context(xe, ye, p, fr.default_opts(tol_lin=tol if kind == "row" else cfg["tol_lin"],
                                                gmres_m=cfg["gmres_m"], m_max=max(30, cfg["gmres_m"]),
                                                gmres_max_restarts=20,
                                                eps_fixed=cfg["eps_fixed"], block_precision=prec,
                                                guess=cfg["guess"], precond_refresh=cfg["precond_refresh"],
                                                jv_precision=1 if cfg["jv_precision"] == "fp32" else 0,
                                                riemann=1 if cfg["riemann"] == "roe" else 0))
    if autotune:
        fr.autotune(ctx, U, 1.0 / (0.5 * dt), reps=1)
    ptc = fr.default_ptc_opts(tol_nl=tol, tol_lin=cfg["tol_lin"])
    iters = 0
    bad = 0
    clocks = ClockSampler(torch.cuda.current_device()) if sample_clocks else None
    if clocks:
        clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    failed = None
    for k in range(nsteps):
        try:
            if kind == "ssprk":
                st = fr.step_ssprk3(ctx, dt, U)
            elif kind == "row":
                st = fr.step_row(ctx, order, dt, U)
            elif kind == "esdirk":
                st = fr.step_esdirk(ctx, order, dt, U, ptc)
            else:
                st = fr.step_bdf2(ctx, dt, U, Uprev, k == 0, ptc)
        except fr.FrError as e:  # e.g. an explicit step above its stability limit
            failed = {"step": k, "error": str(e)}
            break
        iters += st.gmres_iters
        bad += 0 if st.converged else 1
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop() if clocks else None
    out = {"workload": f"vortex-{nx}x{nx}-p{p}-box{L:g}", "scheme": cfg["scheme"].upper(), "dt": dt,
           "gmres_m": cfg["gmres_m"], "eps_fixed": cfg["eps_fixed"],
           "cfl": round(dt * 3 * math.sqrt(2) * (p + 1) / h, 2), "steps": nsteps,
           "tol": tol, "tol_lin": (tol if kind == "row" else cfg["tol_lin"]),
           "block_precision": cfg["block_precision"], "jv_precision": cfg["jv_precision"],
           "riemann": cfg["riemann"], "guess": cfg["guess"],
           "precond_refresh": cfg["precond_refresh"], "t_end": cfg["t_end"]}
    if failed:
        out["failed"] = failed
        ctx.close()
        return out
    err = fr.fr_vortex_error(ctx, U, cfg["t_end"])
    out.update({"time_to_t_end_s": wall, "E_rho": err["rho"], "E_u": err["u"], "gmres_iters": iters,
                "dof_iters_per_s": ctx.ndof * iters / wall, "unconverged_steps": bad})
    if clk is not None:
        out["clocks"] = clk
    ctx.close()
    return out


def _t_end_cfg(args):
    return {"scheme": args.scheme, "cfl": args.cfl, "dt": args.dt, "t_end": args.t_end, "nx": args.nx or NX,
            "p": args.p or P, "box": args.box, "tol": args.tol, "tol_lin": args.tol_lin, "gmres_m": args.gmres_m,
            "eps_fixed": args.eps_fixed, "block_precision": args.block_precision,
            "jv_precision": args.jv_precision, "riemann": args.riemann, "guess": args.guess,
            "precond_refresh": args.precond_refresh}


# The two arms of the time-to-t_end comparison on the 160^2 p=3 vortex, one
# period (t = 10): the plain FP64 method (ROW3 at CFL 13.6, FP64 blocks, zero
# guess, FP64 FD operator, Rusanov) and the mixed form (ROW4 at CFL 50, BF16
# blocks, previous-step guess, FP32 linear parts of the FD operator, the
# paper's Roe flux), both with GMRES(30) to 1e-6 and element-Jacobi.
T_END_PLAIN = {"scheme": "row3", "cfl": 13.6, "dt": None, "t_end": 10.0, "nx": NX, "p": P, "box": 10.0,
               "tol": TOL_LIN, "tol_lin": 1e-1, "gmres_m": 30, "eps_fixed": 0.0, "block_precision": "fp64",
               "jv_precision": "fp64", "riemann": "rusanov", "guess": 0, "precond_refresh": 0}
T_END_MIXED = dict(T_END_PLAIN, scheme="row4", cfl=50.0, block_precision="bf16", jv_precision="fp32",
                   riemann="roe", guess=1)


def t_end_arm(args):
    """Run the vortex workload to t_end; report wall time and E(rho), the L2
    density error against the advected exact vortex (Sec. 5.1 error norm)."""
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(run_t_end(_t_end_cfg(args), autotune=not args.no_autotune)))
    return 0


def tgv_t_end_arm(args):
    """Taylor-Green vortex to t_end (Sec. 5, the time-integrator study): the
    kinetic-energy dissipation rate eps = eps1 + eps3 (mu_v = 0) after every
    step of each implicit scheme against an SSPRK3 reference with
    dt = 2e-4 t_c on the same mesh and degree, and Error(eps) = RMS over the
    steps of eps_n - eps_ref,n; wall time (host waits included) and GMRES
    iterations per run.  ROW at tol_rel,linear = 1e-6, ESDIRK/BDF2 at
    tol_rel,nonlinear = 1e-6 with tol_rel,linear = 1e-1, GMRES(30),
    element-Jacobi blocks (FP32 storage at p = 3)."""
    import numpy as np
    import torch
    import paper_1904_04825_gb300 as fr
    import synthetic as S

    torch.cuda.set_device(0)
    tg = S.TaylorGreen()
    p, n3 = args.p or 3, args.nx or 16
    edges = S.uniform_mesh3d(n3)
    X, Y, Z = S.point_coords3d(*edges, p)
    U0 = torch.from_numpy(tg.state(X, Y, Z)).cuda()
    del X, Y, Z
    t_end = args.t_end * tg.t_c
    dt_ref = 2e-4 * tg.t_c
    divs = [int(x) for x in args.tgv_dt_divs.split(",")]
    dts = [tg.t_c / d for d in divs]
    n_ref = int(round(t_end / dt_ref))
    strides = [int(round(dt / dt_ref)) for dt in dts]
    for dt, st_ in zip(dts, strides):
        if abs(st_ * dt_ref - dt) > 1e-9 * dt:
            raise SystemExit(f"dt = {dt} is not a multiple of the reference step {dt_ref}")
    sample = math.gcd(*strides)
    gas = dict(mu=tg.mu, prandtl=tg.prandtl)

    def eps_of(ctx, U):
        e1, e3, _ = fr.fr_dissipation_rate(ctx, U, tg.rho0)
        return e1 + e3

    # reference: SSPRK3, eps sampled every `sample` steps
    ctx = fr.Context3D(*edges, p, fr.default_opts(precond=0, **gas))
    U = U0.clone()
    ref = {0: eps_of(ctx, U)}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(1, n_ref + 1):
        fr.step_ssprk3(ctx, dt_ref, U)
        if k % sample == 0:
            ref[k] = eps_of(ctx, U)
    torch.cuda.synchronize()
    ref_wall = time.perf_counter() - t0
    ctx.close()
    kmax = max(ref, key=ref.get)
    out = {"workload": f"taylor-green-{n3}^3-p{p}-Re1600-Ma0.1-to-{args.t_end:g}tc", "ndof": 5 * (p + 1) ** 3 * n3 ** 3,
           "block_columns": args.block_columns, "jv_precision": args.jv_precision,
           "reference": {"scheme": "SSPRK3", "dt": dt_ref, "steps": n_ref, "wall_s": ref_wall,
                         "eps_max": ref[kmax], "t_of_eps_max": kmax * dt_ref,
                         "eps_at": {f"{t:g}": ref[int(round(t * tg.t_c / dt_ref))]
                                    for t in (2.0, 4.0, 6.0, 8.0, 9.0, 10.0) if t <= args.t_end}},
           "runs": []}
    prec = 1 if p == 3 else 0
    schemes = (args.tgv_schemes or args.scheme).split(",")
    for dt, stride in zip(dts, strides):
        nsteps = n_ref // stride
        for sch in schemes:
            kind, order = sch[:-1], int(sch[-1])
            ctx = fr.Context3D(*edges, p, fr.default_opts(precond=1, block_precision=prec, tol_lin=1e-6 if kind == "row" else 1e-1,
                                                           gmres_m=30, m_max=30, gmres_max_restarts=20,
                                                           block_columns=1 if args.block_columns == "fp32" and prec else 0,
                                                           jv_precision=1 if args.jv_precision == "fp32" else 0,
                                                           **gas))
            ptc = fr.default_ptc_opts(tol_nl=1e-6, tol_lin=1e-1)
            U = U0.clone()
            Uprev = torch.empty_like(U)
            errs, iters, bad, failed = [], 0, 0, None
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(1, nsteps + 1):
                try:
                    if kind == "row":
                        st = fr.step_row(ctx, order, dt, U)
                    elif kind == "esdirk":
                        st = fr.step_esdirk(ctx, order, dt, U, ptc)
                    else:
                        st = fr.step_bdf2(ctx, dt, U, Uprev, k == 1, ptc)
                except fr.FrError as e:
                    failed = {"step": k, "error": str(e)}
                    break
                iters += st.gmres_iters
                bad += 0 if st.converged else 1
                errs.append(eps_of(ctx, U) - ref[k * stride])
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            run = {"scheme": sch.upper(), "dt_over_tc": dt / tg.t_c, "steps": nsteps, "wall_s": wall,
                   "gmres_iters": iters, "unconverged_steps": bad,
                   "error_eps": float(np.sqrt(np.mean(np.square(errs)))) if errs else None,
                   "eps_minus_ref_at": {f"{t:g}": errs[int(round(t * tg.t_c / dt)) - 1]
                                        for t in (8.0, 10.0) if t <= args.t_end and not failed}}
            if failed:
                run["failed"] = failed
            out["runs"].append(run)
            ctx.close()
            print(json.dumps(run), flush=True)
    print(json.dumps(out))
    return 0


def kernel_arm(args):
    """Time one kernel family alone on the full-size inputs (for per-kernel
    numbers and as a short, clean target for ncu captures)."""
    import torch
    import paper_1904_04825_gb300 as fr
    import synthetic as S

    torch.cuda.set_device(0)
    if args.kernel in ("mlp", "mlp_train"):
        return mlp_kernel_arm(args)
    prec = {"fp64": 0, "fp32": 1, "bf16": 2}[args.block_precision]
    if args.workload == "tgv":
        # the 3D operator on the Taylor-Green field (64^3 hexahedra, p = 3 by default)
        tg = S.TaylorGreen()
        p3, n3 = args.p or 3, args.nx or 64
        edges = S.uniform_mesh3d(n3)
        X, Y, Z = S.point_coords3d(*edges, p3)
        U = torch.from_numpy(tg.state(X, Y, Z)).cuda()
        del X, Y, Z
        blocks = args.kernel in ("factor", "apply") and p3 <= 3   # allocate the blocks only where timed
        if blocks and p3 == 3 and prec == 0:
            prec, args.block_precision = 1, "fp32"   # 320-row blocks are stored in FP32 or BF16
        ctx = fr.Context3D(*edges, p3, fr.default_opts(block_precision=prec, mu=tg.mu, prandtl=tg.prandtl,
                                                        precond=1 if blocks else 0, m_max=4, gmres_m=4,
                                                        block_columns=1 if blocks and args.block_columns == "fp32" else 0,
                                                        jv_precision=1 if args.jv_precision == "fp32" else 0))
    else:
        xe, ye = S.uniform_mesh(NX)
        X, Y = S.point_coords(xe, ye, P)
        U = torch.from_numpy(S.Vortex().state(X, Y)).cuda()
        ctx = fr.Context(xe, ye, P, fr.default_opts(block_precision=prec,
                                                    jv_precision=1 if args.jv_precision == "fp32" else 0))
    R = ctx.empty()
    fr.fr_residual(ctx, U, R)
    z = torch.from_numpy(S.random_vector(ctx.shape, 1)).cuda()
    y = ctx.empty()
    shift = 1.0 / (0.43586652150845900 * DT)
    if args.kernel in ("apply",):
        fr.ejacobi_factor(ctx, U, None, shift)
    run = {
        "residual": lambda: fr.fr_residual(ctx, U, R),
        "jv": lambda: fr.fr_jv(ctx, U, R, z, shift, y),
        "factor": lambda: fr.ejacobi_factor(ctx, U, None, shift),
        "apply": lambda: fr.ejacobi_apply(ctx, z, y),
    }[args.kernel]
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    # the staged blocks of the viscous and 3D contexts are inverted by
    # separate launches (family "invert"), timed alongside
    fams = [args.kernel] + (["invert"] if args.kernel == "factor" else [])
    fr.fr_profile_begin(ctx, fams)
    for _ in range(args.steps):
        run()
    torch.cuda.synchronize()
    prof = fr.fr_profile_end(ctx)

    def summary(pr):
        us = pr["ms"] / max(pr["launches"], 1) * 1e3
        return {"launches": pr["launches"], "avg_us": us,
                "tflops": pr["flops"] / max(pr["launches"], 1) / (us * 1e-6) / 1e12 if us > 0 else None,
                "gbs": pr["bytes"] / max(pr["launches"], 1) / (us * 1e-6) / 1e9 if us > 0 else None,
                "bytes_per_launch": pr["bytes"] / max(pr["launches"], 1),
                "flops_per_launch": pr["flops"] / max(pr["launches"], 1),
                "ms_per_call": pr["ms"] / args.steps}
    out = {"kernel": args.kernel, "workload": args.workload, "ndof": ctx.ndof,
           "block_precision": args.block_precision, "jv_precision": args.jv_precision}
    out.update(summary(prof[args.kernel]))
    if args.kernel == "factor" and prof["invert"]["launches"]:
        out["invert"] = summary(prof["invert"])
    print(json.dumps(out))
    return 0


def batch_arm(args):
    """Many independent problems: 64 vortex instances of uneven size (seeded
    centres, strengths and flow angles; meshes 32^2..128^2 of [-5,5]^2;
    p = 2, 3, 4), one step of dt for all per call (ROW4 by default).  Timed
    twice on the same instances: through the batch API (graph-replayed GMRES
    cycles for ROW, a host thread pool over instance streams for ESDIRK and
    BDF2) and instance after instance through the single-instance calls."""
    import numpy as np
    import torch
    import paper_1904_04825_gb300 as fr
    import synthetic as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    count = args.count
    scheme = args.scheme or "row4"
    kind, order = scheme[:-1], int(scheme[-1])
    prec = {"fp64": 0, "fp32": 1, "bf16": 2}[args.block_precision]
    dt = args.dt or DT
    inst = S.batch_instances(count, seed=0)
    meshes = [i.mesh() for i in inst]
    degrees = [i.p for i in inst]
    U0 = [i.state() for i in inst]
    tol = TOL_LIN if kind == "row" else 1e-1
    opts = fr.default_opts(tol_lin=tol, gmres_m=30, gmres_max_restarts=20, block_precision=prec)
    ptc = fr.default_ptc_opts(tol_nl=1e-6, tol_lin=1e-1)
    B = fr.Batch(meshes, degrees, opts)
    Ub = [torch.from_numpy(u).to(dev) for u in U0]
    Pb = [torch.empty_like(u) for u in Ub]
    singles = [fr.Context(xe, ye, p, opts) for (xe, ye), p in zip(meshes, degrees)]
    Us = [torch.from_numpy(u).to(dev) for u in U0]
    Ps = [torch.empty_like(u) for u in Us]
    ndofs = [m.ndof for m in B.members]
    stream = torch.cuda.current_stream()
    nb = [0]
    ns = [0]

    def timed(fn, steps):
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        units = 0.0
        e0.record(stream)
        for _ in range(steps):
            units += fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), units

    def batch_step(Ulist=Ub, Plist=Pb):
        if kind == "row":
            st = B.step_row(order, dt, Ulist)
        elif kind == "esdirk":
            st = B.step_esdirk(order, dt, Ulist, ptc)
        else:
            st = B.step_bdf2(dt, Ulist, Plist, nb[0] == 0, ptc)
        nb[0] += 1
        return float(sum(n * s.gmres_iters for n, s in zip(ndofs, st)))

    def seq_one(c, U, P):
        if kind == "row":
            return fr.step_row(c, order, dt, U)
        if kind == "esdirk":
            return fr.step_esdirk(c, order, dt, U, ptc)
        return fr.step_bdf2(c, dt, U, P, ns[0] == 0, ptc)

    def seq_step():
        u = float(sum(n * seq_one(c, U, P).gmres_iters for n, c, U, P in zip(ndofs, singles, Us, Ps)))
        ns[0] += 1
        return u

    t_cap = time.perf_counter()
    batch_step()  # captures the cycle graphs (ROW)
    capture_s = time.perf_counter() - t_cap
    for _ in range(args.warmup - 1):
        batch_step()
    for _ in range(args.warmup):
        seq_step()
    launches0 = fr.fr_kernel_launches()
    clocks = ClockSampler(dev)
    clocks.start()
    ms, units = timed(batch_step, args.steps)
    clk = clocks.stop()
    launches = fr.fr_kernel_launches() - launches0
    ms_seq, units_seq = timed(seq_step, args.steps)
    # the same batch with per-instance cycle kernels (no batched launches)
    nodes_batched = B.cycle_kernels()
    B.set_batched(False)
    for _ in range(2):
        batch_step()   # recaptures the cycle graphs
    nodes_per_instance = B.cycle_kernels()
    ms_pi, units_pi = timed(batch_step, args.steps)
    B.set_batched(True)
    batch_step()

    # end to end: every state from pinned host memory and back, each step
    host_in = [torch.from_numpy(u.cpu().numpy()).pin_memory() for u in Ub]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    Ud = [h.to(dev) for h in host_in]
    Pd = [torch.empty_like(u) for u in Ud]
    nb[0] = 0
    batch_step(Ud, Pd)  # new state buffers: capture outside the timed region
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_units = 0.0
    for _ in range(args.steps):
        for d, h in zip(Ud, host_in):
            d.copy_(h, non_blocking=True)
        e2e_units += batch_step(Ud, Pd)
        for d, h in zip(Ud, host_out):
            h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
        host_in, host_out = host_out, host_in
    e2e_s = time.perf_counter() - t0
    (ms, e2e_s, ms_seq), (units, e2e_units, units_seq) = combine_ranks(
        dist, [ms, e2e_s, ms_seq], [units, e2e_units, units_seq], dev)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    total = int(sum(ndofs))
    wl = (f"batch{count}-vortex-mesh32..128-p2..4-{scheme.upper()}-dt{dt:g}-gmres30-tol{tol:g}"
          + (f"-{args.block_precision}blocks" if prec else ""))
    line = {
        "metric": f"DOF*GMRES-iters/s ({wl})", "value": units / (ms * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl, "instances": count, "total_ndof": total,
                   "meshes": list(S.BATCH_MESHES), "degrees": list(S.BATCH_DEGREES),
                   "instances_recipe": "PCG64 seed 0: centre U([-2.5,2.5]^2), alpha U[3,6], theta U[0,2pi), "
                                       "mesh and p uniform",
                   "parallelism": f"replicas x{world}",
                   "l2": "working set of all instances ~10x the L2; no flush",
                   "graph_capture_s": capture_s},
        "sequential": {"value": units_seq / (ms_seq * 1e-3), "ms_per_step": ms_seq / args.steps,
                       "note": "same instances, one single-instance step call after another"},
        "speedup_vs_sequential": (units / ms) / (units_seq / ms_seq),
        "per_instance_cycles": {"value": units_pi / (ms_pi * 1e-3), "ms_per_step": ms_pi / args.steps,
                                "cycle_graph_kernels": nodes_per_instance,
                                "note": "same batch, every instance enqueuing its own cycle kernels"},
        "cycle_graph_kernels": nodes_batched,
        "gpu_launches": launches, "clocks": clk,
        "roofline": None,
        "roofline_note": "kernels run inside CUDA graphs; per-kernel event timing does not apply",
        "cpu_baseline": None,
        "e2e": {"value": e2e_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * total,
                "d2h_bytes_per_step": 8 * total},
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def guess_arm(args):
    """The learned initial guess at its workload: the stretched viscous
    channel (Re 1000, M 0.2, walls clustered to a first cell of 1e-3 with
    ratio 1.15) on a 384 x 192 mesh at p = 4 (7.4 M DOFs, 100 x 100 element
    blocks), ROW3 steps of dt with GMRES(30) to tol_lin = 1e-8.

    Training data: for each training seed s, the seeded perturbed channel
    state, one ROW3 step (which leaves the previous-step history) and a
    second step whose four stage solves are captured (features and targets
    of every 61st element, the offset rotating per stage).  The per-element
    MLP (300 -> 256 -> 256 -> 100) is trained by the library's FP32
    forward / backward / Adam kernels on random minibatches.  Evaluation:
    held-out seeds, two steps each with the zero guess, the previous-step
    guess and the learned guess (BF16 tensor-core inference); reported are
    the GMRES iterations and the wall time of the second step (the first has
    no history), all at the same absolute tolerance tol_lin * ||b||
    (--guess-tol)."""
    import numpy as np
    import torch
    import paper_1904_04825_gb300 as fr
    import synthetic as S

    torch.cuda.set_device(0)
    prec = {"fp64": 0, "fp32": 1, "bf16": 2}[args.block_precision]
    nx, ny, p = args.nx or 384, args.ny or 192, args.p or 4
    dt = args.dt or 1e-3
    ch = S.Channel()
    xe = np.linspace(0.0, ch.lx, nx + 1)
    ye = S.channel_y_edges(ny, first=1e-3, ratio=1.15)
    X, Y = S.point_coords(xe, ye, p)
    nb = 4 * (p + 1) ** 2
    ne = nx * ny
    stride = 61

    tol = args.guess_tol

    def opts(mode):
        return fr.default_opts(tol_lin=tol, gmres_m=30, gmres_max_restarts=60, block_precision=prec,
                               mu=ch.mu, prandtl=ch.prandtl, body_force_x=ch.body_force,
                               wall_temperature=ch.temperature, guess=mode)

    def state(seed):
        return torch.from_numpy(ch.state(X, Y, seed=seed)).cuda()

    ctx = {m: fr.Context(xe, ye, p, opts(m), wall_y=True) for m in (0, 1, 2)}
    train = list(range(1, args.train_seeds + 1))
    per_seed = 4 * ((ne + stride - 1) // stride)
    cap = per_seed * len(train)
    Xc = torch.empty((cap, 3 * nb), dtype=torch.float32, device="cuda")
    Tc = torch.empty((cap, nb), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    n = 0
    gen_iters = 0
    c1 = ctx[1]
    for s in train:
        U = state(s)
        fr.fr_reset_history(c1)
        gen_iters += fr.step_row(c1, 3, dt, U).gmres_iters
        fr.fr_set_stage_capture(c1, Xc[n:], Tc[n:], per_seed, stride)
        gen_iters += fr.step_row(c1, 3, dt, U).gmres_iters
        n += fr.fr_stage_capture_count(c1)
        fr.fr_set_stage_capture(c1, None, None, 0, 1)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    # floor of the stage solves: one GMRES(30) solve of the first stage's
    # system at a seeded state, 20 restarts, target 1e-12 (relres at exit)
    U = state(train[0])
    R0 = c1.empty()
    fr.fr_residual(c1, U, R0)
    shift = 1.0 / (0.435866521508459 * dt)
    fr.ejacobi_factor(c1, U, R0, shift)
    xg = torch.zeros_like(U)
    floor = fr.gmres_solve(c1, U, R0, shift, R0, xg, m=30, rtol=1e-12, max_restarts=20)

    # target normalisation: train on T / sigma (sigma = RMS of the captured
    # targets), so that the network's outputs and losses are of order one
    sigma = 1.0
    if args.normalize_targets:
        sigma = float(torch.sqrt((Tc[:n].double() ** 2).mean()))
        if sigma > 0.0:
            Tc[:n] /= sigma
        else:
            sigma = 1.0
    rng = np.random.default_rng(0)
    sizes = [3 * nb, 256, 256, nb]
    model = fr.MLP(3 * nb, 256, nb, max_batch=max(8192, ne))
    flat = []
    for a, b in zip(sizes[:-1], sizes[1:]):   # He-uniform weights, zero biases
        lim = math.sqrt(6.0 / a)
        flat.append(rng.uniform(-lim, lim, a * b).astype(np.float32))
        flat.append(np.zeros(b, np.float32))
    model.set_params(np.concatenate(flat))
    bs = 8192
    Yb = torch.empty((bs, nb), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    losses = []
    iters = args.train_iters
    for it in range(iters):
        idx = torch.from_numpy(rng.integers(0, n, bs)).cuda()
        xb, tb = Xc[idx].contiguous(), Tc[idx].contiguous()
        model.forward(xb, Yb)
        losses.append(model.backward(xb, tb))
        model.adam(1e-3 if it < iters * 2 // 3 else 3e-4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # loss of predicting no change, for scale (in the units trained on)
    Tz = Tc[:n]
    zero_loss = float((Tz.double() ** 2).sum(dim=1).mean() / 2 / nb)
    if sigma != 1.0:
        # the network was trained on targets / sigma: scaling the last layer
        # by sigma makes it predict the targets themselves
        flat = model.get_params()
        o3 = 3 * nb * 256 + 256 + 256 * 256 + 256
        flat[o3:] *= sigma
        model.set_params(flat)
    del Xc, Tc
    fr.fr_attach_guess_model(ctx[2], model)

    evals = list(range(10001, 10001 + args.eval_seeds))
    res = {m: {"iters": 0, "seconds": 0.0, "unconverged": 0} for m in (0, 1, 2)}
    for s in evals:
        for m in (0, 1, 2):
            c = ctx[m]
            U = state(s)
            fr.fr_reset_history(c)
            fr.step_row(c, 3, dt, U)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            st = fr.step_row(c, 3, dt, U)
            torch.cuda.synchronize()
            res[m]["seconds"] += time.perf_counter() - t1
            res[m]["iters"] += st.gmres_iters
            res[m]["unconverged"] += 0 if st.converged else 1
    tried, used = fr.fr_guess_stats(ctx[2])
    names = {0: "zero", 1: "previous_step", 2: "learned"}
    out = {"workload": f"learned-guess-channel-{nx}x{ny}-p{p}-ROW3-dt{dt:g}-tol{tol:g}-{args.block_precision}blocks",
           "ndof": ctx[0].ndof, "train_seeds": [train[0], train[-1]], "stage_solves_captured": 4 * len(train),
           "samples": n, "elem_stride": stride, "generation_s": gen_s, "generation_gmres_iters": gen_iters,
           "stage_solve_floor": {"relres": floor.relres, "iters": floor.iters, "target": 1e-12},
           "train_iters": iters, "minibatch": bs, "train_s": train_s,
           "loss_first": float(np.mean(losses[:10])), "loss_last": float(np.mean(losses[-50:])),
           "loss_zero_prediction": zero_loss, "target_rms": sigma if args.normalize_targets else None,
           "eval_seeds": [evals[0], evals[-1]],
           "second_step": {names[m]: {"gmres_iters_per_step": res[m]["iters"] / len(evals),
                                      "seconds_per_step": res[m]["seconds"] / len(evals),
                                      "unconverged": res[m]["unconverged"]} for m in (0, 1, 2)},
           "learned_guess_kept": [int(used), int(tried)]}
    print(json.dumps(out))
    for c in ctx.values():
        c.close()
    return 0


def mlp_kernel_arm(args):
    """The per-element guess MLP at the size of its largest workload: one
    inference (BF16 tensor cores, FP32 accumulate) or one training step
    (FP32 forward + backward + Adam) over the 73,728 elements of a 384x192
    p=4 mesh; features 3 x 100, two hidden layers of 256, 100 outputs."""
    import numpy as np
    import torch
    import paper_1904_04825_gb300 as fr

    n_in, n_h, n_out, M = 300, 256, 100, 384 * 192
    net = fr.MLP(n_in, n_h, n_out, M)
    rng = np.random.default_rng(0)
    flat = np.concatenate([rng.standard_normal(n).astype(np.float32) * 0.05 for n in [net.nparam]])
    net.set_params(flat)
    X = torch.from_numpy(rng.standard_normal((M, n_in)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.standard_normal((M, n_out)).astype(np.float32)).cuda()
    Yo = torch.empty((M, n_out), dtype=torch.float32, device="cuda")
    gemm_flops = 2.0 * M * (n_in * n_h + n_h * n_h + n_h * n_out)
    if args.kernel == "mlp":
        run = lambda: net.forward(X, Yo, bf16=True)
        flops = gemm_flops
    else:
        def run():
            net.forward(X, Yo, bf16=False)
            net.backward(X, T)
            net.adam()
        # forward, weight gradients of all layers, input gradients of layers 2 and 3
        flops = 2.0 * gemm_flops + 2.0 * M * (n_h * n_h + n_h * n_out)
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    out = {"kernel": args.kernel, "elements": M, "layers": [n_in, n_h, n_h, n_out], "ms": ms,
           "gflop": flops / 1e9, "tflops": flops / (ms * 1e-3) / 1e12}
    if args.kernel == "mlp":
        pk = peaks.get("bf16_tflops")
        out["bf16_peak_tflops"] = pk
        out["frac_of_measured_bf16"] = (out["tflops"] / pk) if pk else None
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", choices=["residual", "jv", "factor", "apply", "mlp", "mlp_train"], default=None,
                    help="time one kernel family alone on the full-size inputs")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-t-end", action="store_true",
                    help="default run: skip the plain-vs-mixed time-to-t_end comparison")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--block-precision", choices=["fp64", "fp32", "bf16"], default="fp64",
                    help="element-Jacobi block precision (fp64 = the plain method)")
    ap.add_argument("--block-columns", choices=["fp64", "fp32"], default="fp64",
                    help="arithmetic of the FD element-block columns (fp32: 3D with fp32/bf16 blocks)")
    ap.add_argument("--riemann", choices=["rusanov", "roe"], default="rusanov",
                    help="common inviscid flux (roe: the paper's; Euler only)")
    ap.add_argument("--jv-precision", choices=["fp64", "fp32"], default="fp64",
                    help="fp32: linear parts of the FD operator in FP32 (2D Euler and 3D)")
    ap.add_argument("--workload", choices=["vortex", "channel", "batch", "tgv", "guess"], default="vortex")
    ap.add_argument("--train-seeds", type=int, default=500, help="--workload guess: training seeds (4 stage solves each)")
    ap.add_argument("--eval-seeds", type=int, default=50, help="--workload guess: held-out seeds")
    ap.add_argument("--train-iters", type=int, default=3000, help="--workload guess: Adam steps")
    ap.add_argument("--guess-tol", type=float, default=1e-8, help="--workload guess: GMRES tolerance tol_lin")
    ap.add_argument("--normalize-targets", type=int, default=1, choices=[0, 1],
                    help="--workload guess: train on targets scaled to unit RMS (the last layer is rescaled after)")
    ap.add_argument("--count", type=int, default=64, help="--workload batch: number of instances")
    ap.add_argument("--scheme", default=None,
                    choices=["row2", "row3", "row4", "esdirk2", "esdirk3", "esdirk4", "bdf2", "ssprk3"])
    ap.add_argument("--dt", type=float, default=None)
    ap.add_argument("--t-end", type=float, default=None,
                    help="vortex: run to t_end, report time-to-t_end and E(rho); tgv: run to t_end t_c, "
                         "report Error(eps) against an SSPRK3 reference")
    ap.add_argument("--cfl", type=float, default=13.6)
    ap.add_argument("--tol", type=float, default=1e-6,
                    help="--t-end: tol_rel,linear for ROW, tol_rel,nonlinear for ESDIRK/BDF2")
    ap.add_argument("--tol-lin", type=float, default=1e-1, help="--t-end: ESDIRK/BDF2 GMRES tolerance")
    ap.add_argument("--guess", type=int, default=0, choices=[0, 1],
                    help="--t-end, ROW: stage-solve initial guess (0 zero, 1 previous step's)")
    ap.add_argument("--precond-refresh", type=int, default=0, choices=[0, 1, 2],
                    help="--t-end: ESDIRK/BDF2 element-Jacobi refresh (0 per stage + re-invert, 1 per iterate, 2 frozen)")
    ap.add_argument("--box", type=float, default=10.0, help="--t-end: side of the periodic square")
    ap.add_argument("--gmres-m", type=int, default=30, help="--t-end: GMRES restart length (<= 63; the paper's 60)")
    ap.add_argument("--eps-fixed", type=float, default=0.0, help="--t-end: fixed FD step (the paper's 1e-8)")
    ap.add_argument("--nx", type=int, default=None)
    ap.add_argument("--ny", type=int, default=None, help="--workload channel: cells across the channel")
    ap.add_argument("--p", type=int, default=None)
    ap.add_argument("--tgv-schemes", default=None,
                    help="--workload tgv --t-end: comma-separated schemes (default --scheme)")
    ap.add_argument("--tgv-dt-divs", default="25",
                    help="--workload tgv --t-end: time steps t_c / d for these d (comma-separated)")
    args = ap.parse_args()
    if args.scheme is None and args.workload != "batch":
        args.scheme = "row3"
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    if args.kernel:
        return kernel_arm(args)
    if args.t_end and args.workload == "tgv":
        return tgv_t_end_arm(args)
    if args.t_end:
        return t_end_arm(args)
    if args.workload == "batch":
        return batch_arm(args)
    if args.workload == "guess":
        return guess_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
