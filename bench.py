#!/usr/bin/env python
"""Benchmark of the GB300 preconditioned FR/CPR implicit hot path.

One step = one physical BDF2 step (Eq. unsteady_pre_discretized_3) of the isentropic
vortex on the periodic [0,10]^2 box, 64x64 quads, p = 3 (262,144 DOF), M = 0.05,
Re = 100 on the box length, dt = 0.01, driven to Res_m/Res_0 <= 1e-8 by the pseudo-time
Newton loop: residual, exact forward-mode JVP, element block-Jacobi blocks (built,
factored, applied), restarted GMRES with CGS2, Newton update.  Every step runs in the
library's CUDA kernels behind the C ABI; inputs are resident in HBM when the timed
region starts.

value  = DOF advanced per second by BDF2 steps (GDOF/s) = N_dof * steps / time, summed
         over ranks (replicas, weak scaling); sec_per_bdf2_step is its inverse per rank.
e2e    = the same metric with host buffers: every step copies q^n, q^c,n, q^c,n-1 from
         pinned host memory and q^n+1 back inside the timed region.
roofline: the dominant kernel class (largest share of device time over a profiled
         repetition of the timed steps): algorithmic flops (ALU-bound kernels, against the
         FP64 or FP32 pipe peak) or algorithmic DRAM bytes (streaming kernels, against the
         measured HBM copy bandwidth) over its CUDA-event duration.

--impl reference times the CPU oracle (numpy, FP64) on a bounded sample of the same
workload (the 16x16 sub-box at the same p, M, Re, dt: one BDF2 step per bench step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FR/CPR residual+JVP GDOF/s; sec per BDF2 step to 1e-8 (mixed vs FP64)"
UNIT = "GDOF/s"


# ------------------------------------------------------------------ roofline peaks
# ALU peaks from unit counts and the maximum SM clock (2.07 GHz): the FP64 pipe of a
# GB300 does 2 FMA per clock per SM, 152 SMs x 2 x 2 flop x 2.07 GHz = 1.26 TFLOP/s; the FP32
# SIMT pipe 152 x 128 x 2 x 2.07 GHz = 80.5 TFLOP/s.  HBM: the measured copy bandwidth.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
ALU_PEAK_SOURCE = ("nominal from unit counts and the maximum SM clock: FP64 152 SMs x 2 FMA/clk "
                   "x 2 flop x 2.07 GHz = 1.26 TFLOP/s; FP32 152 x 128 FMA/clk x 2 x 2.07 GHz = "
                   "80.5 TFLOP/s")
# Bound of each kernel class as ncu measured it: every FP64 kernel, the Gram-Schmidt
# reductions, vector updates and FP64 coarse levels included, saturates the FP64 pipe
# before DRAM (1 FMA per 8 bytes needs 1.7 TFLOP/s at full HBM bandwidth); the FP32/BF16
# block apply and FP32 coarse levels stream DRAM.
ALU_KINDS = {"trace", "face", "elem", "trace_jvp", "face_jvp", "elem_jvp", "block_jacobian",
             "block_factor", "geometry", "krylov_reduce", "vector", "linearize", "linear_apply",
             "linear_adjoint", "coarse"}


# DRAM bytes per launch of a kernel class from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum averaged over the captured launches; the summary under profiles/
# gives the command).  A class whose kernels changed since the capture is left out.
NCU_TRAFFIC = {
    # k_vdots / k_vaxdots / k_vaxpy<1> over the first GMRES(30) cycle of the 64x64 p=3
    # vortex (90 launches, nv = 1 .. 30): mean 34.8 MB per launch, equal to the
    # algorithmic (nv + 1) x 2.1 MB averaged over the cycle
    "krylov_reduce": 34.82e6,
}


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ replicas
def replica_throughput(t_rank: float, units_per_rank: float, world: int, dist, device):
    """Whole-job throughput of `world` replicas: the slowest rank's time (all-reduce MAX
    over the ranks, or the local time on one rank) and the units all ranks processed per
    second over it, in billions.  Returns (t_max, value)."""
    import torch
    t_max = t_rank
    if dist is not None and world > 1:
        tt = torch.tensor([t_rank], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    return t_max, units_per_rank * world / t_max / 1e9


def shard_cases(dofs, world: int):
    """Independent cases dealt to `world` ranks: largest first, each to the least loaded
    rank (DOF as the load, ties to the lower rank).  Deterministic; every case exactly
    once; each rank's list in case order."""
    load = [0] * world
    parts = [[] for _ in range(world)]
    for k in sorted(range(len(dofs)), key=lambda k: (-dofs[k], k)):
        r = min(range(world), key=lambda r: (load[r], r))
        parts[r].append(k)
        load[r] += dofs[k]
    return [sorted(p) for p in parts]


def sharded_throughput(t_rank: float, units_total: float, world: int, dist, device):
    """Throughput of a fixed set of units shared by `world` ranks (strong scaling): the
    slowest rank's time (all-reduce MAX) and all units per second over it, in billions.
    Returns (t_max, value)."""
    import torch
    t_max = t_rank
    if dist is not None and world > 1:
        tt = torch.tensor([t_rank], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    return t_max, units_total / t_max / 1e9


# ------------------------------------------------------------------ CPU oracle sample
# Per-step work profile of the headline steps (means over the timed steps of the GPU arm,
# two-level preconditioner, 64x64 p=3 vortex): the reference arm, which runs before any GPU
# measurement, prices these counts; the GPU arm prices its own.
STEP_PROFILE = {"newton": 3.2, "gmres": 228.0, "builds": 2.0, "restart": 30,
                "precond": "twolevel"}


def oracle_unit_costs(w, precond: str):
    """The oracle as it stands, timed per unit of a BDF2 step on a bounded sample: a
    16 x 16 sub-box of workload w's element size (same p, M, Re, dt), seconds per call of
    one residual, one exact Newton-operator product (complex step), one preconditioner
    build (element blocks by coloured complex steps and their inverses, plus for the
    two-level preconditioner the coloured Galerkin products and the hierarchy) and one
    preconditioner apply, and one CGS2 Arnoldi step at the mean basis size of a restart
    cycle.  Every unit is linear in the number of elements (the colour count does not
    grow with the mesh), so the costs are returned per DOF."""
    import numpy as np
    from oracle import physics as ph
    from oracle import residual as rs
    from oracle import solver as sv
    from oracle import twolevel as tl
    from paper_1903_06304_gb300 import inputs as inp
    n = 16
    h = (w.box[1] - w.box[0]) / w.nx
    c = inp.box_mesh(n, n, 0.0, n * h, 0.0, n * h)
    q = inp.random_perturbation(inp.uniform_state(n * n, w.p, w.mach, 0.8, 0.3), 3, 0.05, w.mach)
    prob = sv.Problem(rs.Mesh(n, n, c, np.zeros_like(c)), w.p, ph.Gas(mach=w.mach, re=w.re, kappa=w.kappa))
    a0_dt = 1.5 / w.dt
    x = inp.random_vector(q.shape, 4)
    dof = q.size

    def clock(fn, reps=1):
        t0 = time.perf_counter()
        for _ in range(reps):
            out = fn()
        return (time.perf_counter() - t0) / reps, out

    t_R, _ = clock(lambda: prob.R(q), 3)
    Aop = lambda v: sv.apply_A(prob, q, v, 1e-20, a0_dt)
    t_A, _ = clock(lambda: Aop(x), 3)
    if precond == "twolevel":
        t_build, pc = clock(lambda: tl.build(prob, q, 1e-20, a0_dt))
        t_M, _ = clock(lambda: pc.apply(x, Aop), 2)
    else:
        t_build, Binv = clock(lambda: np.linalg.inv(sv.block_jacobian(prob, q, 1e-20, a0_dt)))
        t_M, _ = clock(lambda: sv.block_apply(Binv, x), 3)
    j = w.restart // 2
    V = np.random.default_rng(5).standard_normal((j + 1, dof))
    wv = x.ravel()

    def arnoldi():
        h1 = V @ wv
        w2 = wv - V.T @ h1
        h2 = V @ w2
        return w2 - V.T @ h2

    t_arn, _ = clock(arnoldi, 3)
    return {"per_dof": {k: v / dof for k, v in (("residual", t_R), ("operator", t_A), ("build", t_build),
                                                 ("precond", t_M), ("arnoldi", t_arn))},
            "sample": f"{n}x{n} sub-box of the workload's element size, p={w.p}, {dof} DOF",
            "cores": 1}


def oracle_step_seconds(costs, profile, ndof):
    """Oracle seconds for one BDF2 step of ndof DOF with the given operation counts: a
    residual per Newton iteration (and one at the start), a preconditioner build per
    build, per GMRES iteration an operator product, a preconditioner apply and an Arnoldi
    step, and per restart cycle one more product and apply for the true residual."""
    c = costs["per_dof"]
    cycles = profile["gmres"] / profile["restart"] + profile["newton"]
    per_dof = ((profile["newton"] + 1) * c["residual"] + profile["builds"] * c["build"]
               + profile["gmres"] * (c["operator"] + c["precond"] + c["arnoldi"])
               + cycles * (c["operator"] + c["precond"]))
    return per_dof * ndof


def oracle_sample(w, profile):
    costs = oracle_unit_costs(w, profile["precond"])
    sec = oracle_step_seconds(costs, profile, w.dof)
    return {"value": w.dof / sec / 1e9, "unit": UNIT, "sec_per_step": sec, "dof": w.dof,
            "cores": costs["cores"], "kind": "oracle", "unit_costs_per_dof_s": costs["per_dof"],
            "profile": profile,
            "sample": ("oracle (numpy FP64, one thread) timed per unit on a bounded sample, the "
                       + costs["sample"] + ", scaled per DOF to the workload and priced with the "
                       f"step's counts (Newton {profile['newton']:.1f}, GMRES {profile['gmres']:.0f}, "
                       f"builds {profile['builds']:.1f}, {profile['precond']} preconditioner)")}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1903_06304_gb300 import inputs as inp
    w = inp.WORKLOADS[args.workload]
    prof = dict(STEP_PROFILE, precond=args.precond)
    times = []
    res = None
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = oracle_sample(w, prof)
        if k >= args.warmup:
            times.append(res["sec_per_step"])
    sec = sum(times) / len(times)
    value = w.dof / sec / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w.name, "note": res["sample"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["cores"],
                             "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def large_n_sweep(sizes, torch, fr, inp, flush):
    """Residual, dual and linearized JVP and VJP throughput on the benchmark geometry
    scaled to n x n elements (inputs far beyond L2): median of 10 calls each, with the
    FP64 rate from the library's algorithmic flop counts."""
    import numpy as np
    out = {}
    base = inp.NS_VORTEX_64
    for n in sizes:
        w = inp.Workload(f"vortex_{n}", n, n, base.p, base.mach, base.re, base.kappa, base.box,
                         ic="vortex", dt=base.dt)
        c, v, q = inp.make_case(w)
        T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")
        S = fr.Solver(fr.Config(p=w.p, mach=w.mach, re=w.re, kappa=w.kappa), n, n)
        S.update_mesh(T(c), T(v))
        qd = T(q)
        del c, v, q
        vec = torch.randn_like(qd)
        o = torch.empty_like(qd)
        S.linearize(qd, 1e-20, 1.5 / w.dt)
        res = {"dof": S.ndof}
        for name, fn in (("residual", lambda: S.residual(qd, o)),
                         ("jvp_dual", lambda: S.jvp(qd, vec, o, 1e-20, 1.5 / w.dt)),
                         ("jvp_linearized", lambda: S.apply_linear(vec, o)),
                         ("vjp", lambda: S.apply_linear(vec, o, transpose=True))):
            fn()
            torch.cuda.synchronize()
            S.profile_read(reset=True)
            ts = []
            for _ in range(10):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                ts.append((a, b))
            torch.cuda.synchronize()
            flops = sum(x["flops"] for x in S.profile_read(reset=True).values()) / 10
            t = statistics.median(a.elapsed_time(b) for a, b in ts) * 1e-3
            res[name] = {"gdofs": S.ndof / t / 1e9, "ms": t * 1e3,
                         "fp64_tflops": flops / t / 1e12, "fp64_frac": flops / t / 1e12 / FP64_PEAK_TFLOPS}
        out[f"{n}x{n}"] = res
        S.close()
        del qd, vec, o
        torch.cuda.empty_cache()
    return out


def march_inputs(w, nsteps, T):
    """Device copies of the mesh of every step of a march (corners and corner velocities at
    t = (k + 1) dt) for deforming workloads, made before any timed region; None for static
    meshes (one geometry for the whole march)."""
    if not w.deforming:
        return None
    from paper_1903_06304_gb300 import inputs as inp
    out = []
    for k in range(nsteps):
        c, v, _ = inp.make_case(w, t=(k + 1) * w.dt)
        out.append((T(c), T(v)))
    return out


class March:
    """State of a BDF2 march on the device: q^n, q^c,n, q^c,n-1 and the step index; a
    deforming mesh moves to t^(n+1) (the library's geometry kernel) before each step."""

    def __init__(self, S, q0, meshes, fr):
        import torch
        self.S, self.fr, self.meshes = S, fr, meshes
        self.q = q0.clone()
        self.qc_n = torch.empty_like(self.q)
        self.qc_nm1 = torch.empty_like(self.q)
        S.conservative(self.q, self.qc_n)
        self.qc_nm1.copy_(self.qc_n)
        self.k = 0

    def step(self):
        if self.meshes is not None:
            c, v = self.meshes[self.k]
            self.S.update_mesh(c, v)
        coeffs = self.fr.BDF1 if self.k == 0 else self.fr.BDF2
        st = self.S.bdf2_step(self.q, self.qc_n, self.qc_nm1, self.S.dt, coeffs=coeffs,
                              allow_unconverged=True)
        self.qc_nm1.copy_(self.qc_n)
        self.S.conservative(self.q, self.qc_n)
        self.k += 1
        return st.summary()

    def save(self):
        return (self.q.clone(), self.qc_n.clone(), self.qc_nm1.clone(), self.k)

    def restore(self, snap):
        q, a, b, k = snap
        self.q.copy_(q)
        self.qc_n.copy_(a)
        self.qc_nm1.copy_(b)
        self.k = k


def timed_steps(run, K, flush, barrier):
    """K steps with CUDA events around each on the current stream (L2 flushed before each,
    outside the events); returns per-step ms, stats and the library launches inside."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stats = []
    launches0 = run.S.kernel_launches
    barrier()
    for k in range(K):
        flush.zero_()
        ev[k][0].record()
        stats.append(run.step())
        ev[k][1].record()
    barrier()
    return [a.elapsed_time(b) for a, b in ev], stats, run.S.kernel_launches - launches0


def step_summary(stats):
    return {"converged": [s["converged"] for s in stats],
            "newton": [s["newton_iterations"] for s in stats],
            "gmres": [sum(s["gmres_iterations"]) for s in stats],
            "res_drop": [s["res_history"][-1] / s["res_history"][0] for s in stats]}


def low_mach_deforming_report(args, torch, fr, inp, T, flush):
    """The deforming 128 x 128, p = 3, M = 0.01 workload: the vortex march's first steps with
    the two-level preconditioner and each block precision (BF16 blocks also factored on
    the tensor cores), and free-stream preservation of the uniform stream on the moving
    mesh."""
    w = inp.NS_DEFORM_128
    c0, v0, q0 = inp.make_case(w, t=0.0)
    meshes = march_inputs(w, args.c3_steps, T)
    out = {"workload": w.name, "dof": w.dof, "newton_cap": args.c3_newton}

    def solver(prec, precond, tiles=1):
        factor = "tc_bf16" if prec == "bf16_tc" else "simt"
        prec = "bf16" if prec == "bf16_tc" else prec
        S = fr.Solver(fr.Config(p=w.p, mach=w.mach, re=w.re, kappa=w.kappa, prec=prec, factor=factor,
                                precond=precond, maxit_newton=args.c3_newton, restart=args.restart,
                                maxit_lin=args.maxit_lin, graphs=args.graphs, arnoldi_fused=args.arnoldi_fused, tiles=tiles,
                                apply_accum=args.apply_accum), w.nx, w.ny)
        S.dt = w.dt
        S.update_mesh(T(c0), T(v0))
        return S

    finals = {}
    for prec in ("fp64", "fp32", "bf16", "bf16_tc"):
        S = solver(prec, args.precond)
        run = March(S, T(q0), meshes, fr)
        ms, st, _ = timed_steps(run, args.c3_steps if prec == "fp32" else 1, flush, torch.cuda.synchronize)
        out[f"march_{prec}"] = dict(step_summary(st), sec_per_step=[m / 1e3 for m in ms])
        if prec == "fp64":
            # Res_m/Res_0 per Newton iteration of the first step: where it levels off
            h = st[0]["res_history"]
            out["march_fp64"]["res_history_step1"] = [float("%.3g" % (x / h[0])) for x in h]
        if prec != "fp32":
            finals[prec] = run.q.clone()
        else:
            r1 = March(S, T(q0), meshes, fr)
            r1.step()
            finals[prec] = r1.q.clone()
        S.close()
    dq = (finals["fp64"] - T(q0)).view(4, -1).abs().amax(dim=1)
    for prec in ("fp32", "bf16", "bf16_tc"):
        diff = (finals[prec] - finals["fp64"]).view(4, -1).abs().amax(dim=1)
        out[f"march_{prec}"]["state_diff_vs_fp64_step1"] = float((diff / dq).max())
    # free stream on the moving mesh
    S = solver("fp32", args.precond)
    qu = T(inp.uniform_state(w.ne, w.p, w.mach))
    R = torch.empty_like(qu)
    worst = 0.0
    for t in (0.05, 0.13, 0.21):
        c, v, _ = inp.make_case(w, t=t)
        S.update_mesh(T(c), T(v))
        S.residual(qu, R)
        worst = max(worst, float(R.abs().max()))
    out["free_stream_max_abs_residual"] = worst
    S.close()
    return out


def steady_ptc_study(args, torch, fr, inp, T):
    """Steady pseudo-transient continuation with SER (Eqs. steady_pre_discretized_1, SER)
    on a cylinder O-grid, the kind of study of Sec. 4.1 with a viscous body (the paper's
    inviscid slip-wall cylinder needs a wall condition not built here): 64 x 32 cells to 20
    diameters, p = 2, M = 0.1, Re = 20 on the diameter, impulsively started free stream,
    PTC to Res_m/Res_0 <= 1e-8 with GMRES(100); per variant the pseudo steps, GMRES
    iterations, wall time, final drop and drag coefficient C_d = F_x / (rho U^2 D / 2):
    tol_res 1e-3 / 1e-6 / 1e-9, the SER cap dtau_max 1e20 / 100 / 10, and kappa 1 / sqrt 5 / 3."""
    ni, nj, p, mach, re = 64, 32, 2, 0.1, 20.0
    c = inp.cylinder_ogrid(ni, nj, 20.0, 1e-2)
    v = 0.0 * c
    qi = inp.far_field_state(mach)
    q0 = inp.uniform_state(ni * nj, p, mach)
    # FP64 coarse levels, as on the NACA O-grid: the stretched grid at M = 0.1 is where FP32
    # coarse operators have given non-finite Krylov vectors
    base = dict(p=p, mach=mach, re=re, kappa=1.0, restart=100, maxit_lin=300, tol_res=1e-6,
                tol_pseudo=1e-8, maxit_newton=64, precond=args.precond, prec=args.prec,
                mg_prec="fp64")
    variants = [("tol_res=1e-3", {"tol_res": 1e-3}), ("tol_res=1e-6", {}), ("tol_res=1e-9", {"tol_res": 1e-9}),
                ("dtau_max=100", {"dtau_max": 100.0}), ("dtau_max=10", {"dtau_max": 10.0}),
                ("kappa=sqrt5", {"kappa": 5 ** 0.5}), ("kappa=3", {"kappa": 3.0})]
    out = {"workload": f"cylinder O-grid {ni}x{nj} p={p} M={mach} Re={re} (wall + far field)",
           "dof": 4 * ni * nj * (p + 1) ** 2}
    for name, over in variants:
        S = fr.Solver(fr.Config(**{**base, **over}), ni, nj, bc=("wall", "farfield"), q_inf=qi)
        S.update_mesh(T(c), T(v))
        q = T(q0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            st = S.ptc_solve(q, allow_unconverged=True).summary()
        except fr.FrError as e:
            out[name] = {"converged": False, "error": str(e)}
            S.close()
            continue
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        fx, _fy = S.wall_force(q)
        h = st["res_history"]
        out[name] = {"converged": st["converged"], "pseudo_steps": st["newton_iterations"],
                     "gmres_total": sum(st["gmres_iterations"]), "seconds": t1 - t0,
                     "res_drop": h[-1] / h[0], "c_d": 2.0 * fx}
        S.close()
    return out


def plunge_march_report(args, torch, fr, inp, T):
    """The plunging NACA 0012 of Sec. 4.4 in the benchmark's configuration: O-grid of
    ``--plunge-grid`` cells (256 x 96) to 20 chords, cosine clustering at the edges blended
    half with a uniform distribution, first cell 1e-3 chords; p = 3, Re = 1e4 on the chord,
    kappa = sqrt 5; rigid plunge y = 0.25 sin(k t), k = 1 (Sec. 4.4); dt = T/200; BDF1 then
    BDF2 from the impulsively started free stream, Newton to Res_m/Res_0 <= 1e-8 with
    GMRES(100), tol_res 1e-6 and the configured preconditioner.  Per Mach number: wall
    time, convergence, Newton and GMRES counts and C_l = 2 F_y, C_t = -2 F_x of each
    step (rho = U = c = 1).  With ``--plunge-periods P`` the march runs P periods and
    reports the last period's mean C_t, C_l rms and C_l max (Sec. 4.4's force table)."""
    import math
    ni, nj = (int(x) for x in args.plunge_grid.split("x"))
    p, re, kappa, h, k = 3, 1e4, 5 ** 0.5, 0.25, 1.0
    period = 2 * math.pi / k
    dt = period / 200
    ref = inp.naca_ogrid(ni, nj)
    nsteps = args.plunge_periods * 200 if args.plunge_periods > 0 else args.plunge_steps
    out = {"workload": f"naca0012_ogrid_{ni}x{nj}_p{p} plunge h={h} k={k} Re={re:g} dt=T/200",
           "dof": 4 * ni * nj * (p + 1) ** 2, "steps": nsteps, "precond": args.precond,
           "blocks": args.prec, "coarse": "fp64"}
    for mach in args.plunge_mach:
        qi = inp.far_field_state(mach)
        # FP64 coarse levels: on this stretched O-grid at M <= 0.1 the FP32 coarse
        # operators leave left-preconditioned GMRES a near-singular map, whose unconverged
        # Newton updates drive T negative within two iterations
        cfg = fr.Config(p=p, mach=mach, re=re, kappa=kappa, precond=args.precond, prec=args.prec,
                        mg_prec="fp64", restart=100, maxit_lin=100, tol_res=1e-6, tol_pseudo=1e-8,
                        maxit_newton=20, graphs=args.graphs, arnoldi_fused=args.arnoldi_fused)
        S = fr.Solver(cfg, ni, nj, bc=("wall", "farfield"), q_inf=qi)
        c0, v0 = inp.plunge(ref, 0.0, h, k)
        S.update_mesh(T(c0), T(v0))
        q = T(inp.uniform_state(ni * nj, p, mach))
        qn = torch.empty_like(q)
        S.conservative(q, qn)
        qm = qn.clone()
        rec = {"sec_per_step": [], "converged": [], "newton": [], "gmres": [], "c_l": [], "c_t": []}
        for n in range(nsteps):
            c1, v1 = inp.plunge(ref, (n + 1) * dt, h, k)
            S.update_mesh(T(c1), T(v1))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                st = S.bdf2_step(q, qn, qm, dt, coeffs=fr.BDF1 if n == 0 else fr.BDF2,
                                 allow_unconverged=True).summary()
            except fr.FrError as e:
                rec["error"] = f"step {n}: {e}"
                break
            torch.cuda.synchronize()
            rec["sec_per_step"].append(round(time.perf_counter() - t0, 4))
            qm.copy_(qn)
            S.conservative(q, qn)
            fx, fy = S.wall_force(q)
            rec["converged"].append(st["converged"])
            rec["newton"].append(st["newton_iterations"])
            rec["gmres"].append(sum(st["gmres_iterations"]))
            rec["c_l"].append(2.0 * fy)
            rec["c_t"].append(-2.0 * fx)
        S.close()
        if args.plunge_periods > 0 and len(rec["c_t"]) == nsteps:
            ct, cl = rec["c_t"][-200:], rec["c_l"][-200:]
            rec["last_period"] = {"c_t_mean": sum(ct) / 200,
                                  "c_l_rms": math.sqrt(sum(x * x for x in cl) / 200),
                                  "c_l_max": max(cl)}
            for key in ("sec_per_step", "newton", "gmres", "c_l", "c_t", "converged"):
                rec[key] = {"mean": sum(rec[key]) / nsteps, "n": nsteps} if key != "converged" \
                    else all(rec[key])
        out[f"M={mach:g}"] = rec
    return out


def plunge_adjoint_report(args, torch, fr, inp, T):
    """The discrete adjoint of the plunging-airfoil march (Sec. 3.2 march, Sec. 4.4 plunge):
    J = mean C_t over the first ``--adjoint-steps`` BDF steps of the ``--plunge-grid``
    O-grid at M = 0.2 (the configuration of ``plunging_naca``), its gradient in the plunge
    amplitude h and the Mach number by one reverse sweep (per step the wall-force
    gradient, the BDF coupling to the next two steps, the transposed GMRES solve with the
    transposed two-level preconditioner, and the parameter directional derivatives), timed
    against the forward march, and central differences of the whole march (h +- 1e-3 h,
    M +- 1e-3 M, the initial state held at the nominal free stream as in the adjoint's
    definition) as a check."""
    import math
    ni, nj = (int(x) for x in args.plunge_grid.split("x"))
    p, re, kappa, h, k, mach = 3, 1e4, 5 ** 0.5, 0.25, 1.0, 0.2
    dt = 2 * math.pi / k / 200
    K = args.adjoint_steps
    ref = inp.naca_ogrid(ni, nj)

    def mesh_at(t, hh):
        c1, v1 = inp.plunge(ref, t, 1.0, k)
        return ref + hh * (c1 - ref), hh * v1, c1 - ref, v1

    def solver(m, maxit_lin=100):
        cfg = fr.Config(p=p, mach=m, re=re, kappa=kappa, precond="twolevel", prec=args.prec,
                        mg_prec="fp64", restart=100, maxit_lin=maxit_lin, tol_res=1e-6,
                        tol_pseudo=1e-8, maxit_newton=20, graphs=args.graphs, arnoldi_fused=args.arnoldi_fused)
        return fr.Solver(cfg, ni, nj, bc=("wall", "farfield"), q_inf=inp.far_field_state(m))

    q_start = inp.uniform_state(ni * nj, p, mach)   # the nominal free stream, fixed

    def march(S, hh, m):
        c0, v0, _, _ = mesh_at(0.0, hh)
        S.update_mesh(T(c0), T(v0))
        q = T(q_start)
        qn = torch.empty_like(q)
        S.conservative(q, qn)
        qm = qn.clone()
        qs, J, conv = [q.clone()], 0.0, True
        for n in range(1, K + 1):
            c1, v1, _, _ = mesh_at(n * dt, hh)
            S.update_mesh(T(c1), T(v1))
            st = S.bdf2_step(q, qn, qm, dt, coeffs=fr.BDF1 if n == 1 else fr.BDF2,
                             allow_unconverged=True).summary()
            conv = conv and st["converged"]
            qm.copy_(qn)
            S.conservative(q, qn)
            qs.append(q.clone())
            J += -2.0 * S.wall_force(q)[0] / K
        return qs, J, conv

    coeffs = lambda n: fr.BDF1 if n == 1 else fr.BDF2
    S = solver(mach)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qs, J, conv = march(S, h, mach)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    S.close()
    S = solver(mach, maxit_lin=400)   # the adjoint solves: one linear system per step
    # reverse sweep
    wx = -2.0 / K
    dq_inf = (-2.0 / (inp.GAMMA * mach ** 3), 0.0, 0.0, 0.0)
    lam = [None] * (K + 3)
    grad = [0.0, 0.0]
    its = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for n in range(K, 0, -1):
        c, v, dc, dv = mesh_at(n * dt, h)
        cd, vd = T(c), T(v)
        S.update_mesh(cd, vd)
        g = torch.empty_like(qs[n])
        S.wall_force_vjp(qs[n], wx, 0.0, g)
        for m_, kk in ((n + 1, 1), (n + 2, 2)):
            if m_ <= K and coeffs(m_)[kk] != 0.0:
                S.conservative_vjp(qs[n], lam[m_], g, alpha=-coeffs(m_)[kk] / dt, beta=1.0)
        lam[n] = torch.empty_like(g)
        its.append(S.adjoint_solve(qs[n], g, lam[n], 0.0, coeffs(n)[0] / dt))
        wRh, Fh = S.param_jvp(qs[n], cd, vd, dcorners=T(dc), dvel=T(dv), w=lam[n], force=True)
        wRm, Fm = S.param_jvp(qs[n], cd, vd, dmach=1.0, dqinf=dq_inf, w=lam[n], force=True)
        grad[0] += wRh + wx * Fh[0]
        grad[1] += wRm + wx * Fm[0]
        for j, a in enumerate(coeffs(n)):
            if a != 0.0:
                grad[1] -= a / dt * S.conservative_dmach(qs[n - j], lam[n])
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    S.close()
    # central differences of the whole march
    eh, em = 1e-3 * h, 1e-3 * mach
    S = solver(mach)
    jh = [march(S, h + s * eh, mach)[1] for s in (1, -1)]
    S.close()
    jm = []
    for s in (1, -1):
        Sm = solver(mach + s * em)
        jm.append(march(Sm, h, mach + s * em)[1])
        Sm.close()
    fd = [(jh[0] - jh[1]) / (2 * eh), (jm[0] - jm[1]) / (2 * em)]
    return {"workload": f"naca0012_ogrid_{ni}x{nj}_p{p} plunge M={mach} h={h} k={k} dt=T/200",
            "steps": K, "J_mean_c_t": J, "forward_converged": conv,
            "dJ_dh": grad[0], "dJ_dM": grad[1], "fd_dJ_dh": fd[0], "fd_dJ_dM": fd[1],
            "rel_diff_h": abs(grad[0] - fd[0]) / max(abs(fd[0]), 1e-300),
            "rel_diff_M": abs(grad[1] - fd[1]) / max(abs(fd[1]), 1e-300),
            "sec_forward": t_fwd, "sec_reverse": t_adj, "adjoint_gmres_per_step": its[::-1],
            "note": "the differences carry the march's Newton tolerance (1e-8) over the step "
                    "1e-3 of the parameter, and the adjoint's GMRES tolerance (1e-6)"}


def gpu_arm(args):
    import numpy as np
    import torch

    from paper_1903_06304_gb300 import fr
    from paper_1903_06304_gb300 import inputs as inp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = inp.WORKLOADS[args.workload]
    corners, vel, q0 = inp.make_case(w)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    nsteps = args.startup + args.warmup + args.steps
    meshes = march_inputs(w, nsteps, T)

    def make_solver(prec, arith=None, precond=None, factor="simt"):
        cfg = fr.Config(p=w.p, mach=w.mach, re=w.re, kappa=w.kappa, prec=prec, factor=factor,
                        restart=args.restart, maxit_lin=args.maxit_lin, tol_res=w.tol_res,
                        tol_pseudo=w.tol_pseudo, maxit_newton=args.maxit_newton, lag=2,
                        line_search=args.line_search, graphs=args.graphs, arnoldi_fused=args.arnoldi_fused,
                        apply_accum=args.apply_accum, tiles=args.tiles, orthog=args.orthog,
                        krylov_arith=arith or args.krylov_arith, precond=precond or args.precond,
                        mg_prec=args.mg_prec, mg_sweeps=args.mg_sweeps, mg_omega=args.mg_omega)
        S = fr.Solver(cfg, w.nx, w.ny)
        S.dt = w.dt
        S.update_mesh(T(corners), T(vel))
        return S

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    # ---- the march: optional start-up steps (recorded, untimed; none by default), then
    # the warm-up steps, after which the march returns to the state before them: the timed
    # steps are the march's steps from its first on (from the first after the start-up)
    S = make_solver(args.prec)
    run = March(S, T(q0), meshes, fr)
    startup = []
    for _ in range(args.startup):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = run.step()
        torch.cuda.synchronize()
        startup.append((time.perf_counter() - t0, st))
    snap = run.save()
    for _ in range(args.warmup):
        run.step()
    run.restore(snap)
    clocks = ClockSampler(local)
    ms, stats, launches = timed_steps(run, args.steps, flush, barrier)
    clock_info = clocks.stop()
    t_rank = sum(ms) / 1e3
    dof = S.ndof
    t_max, value = replica_throughput(t_rank, dof * args.steps, world, dist, dev)
    ms_per_step = t_max * 1e3 / args.steps

    # ---- per-kernel device time over the same steps (profiling pass from the same state)
    run.restore(snap)
    S.profile(True)
    S.profile_read(reset=True)
    _ms_p, st_p, _ = timed_steps(run, args.steps, flush, barrier)
    prof = S.profile_read(reset=True)
    S.profile(False)
    hbm_gbs, hbm_src = hbm_peak()
    tot_ms = sum(v["ms"] for v in prof.values())
    kernels = {}
    for name, v in prof.items():
        if v["launches"] == 0:
            continue
        t_s = v["ms"] * 1e-3
        e = {"ms_total": v["ms"], "launches": v["launches"],
             "us_per_launch": 1e3 * v["ms"] / v["launches"],
             "share": v["ms"] / tot_ms if tot_ms else None}
        # FP32 coarse levels carry 0.5 flop per byte, far below the FP32 pipe's balance
        # (~12 flop/B): rated against HBM; FP64 coarse levels against the FP64 pipe
        alu = name in ALU_KINDS and not (name == "coarse" and args.mg_prec != "fp64")
        if alu or (name == "block_apply" and args.prec == "fp64"):
            fp32 = name == "block_factor" and args.prec != "fp64"
            peak = FP32_PEAK_TFLOPS if fp32 else FP64_PEAK_TFLOPS
            e.update(bound="alu", pipe="fp32" if fp32 else "fp64", unit="TFLOP/s",
                     achieved=v["flops"] / t_s / 1e12, peak=peak,
                     alg_per_launch=v["flops"] / v["launches"])
        else:
            e.update(bound="hbm", unit="GB/s", achieved=v["bytes"] / t_s / 1e9, peak=hbm_gbs,
                     alg_per_launch=v["bytes"] / v["launches"])
        e["frac"] = e["achieved"] / e["peak"]
        kernels[name] = e
    dominant = max(kernels, key=lambda k: kernels[k]["ms_total"])
    same_steps = [s["newton_iterations"] for s in st_p] == [s["newton_iterations"] for s in stats]

    # ---- end-to-end through host buffers, the same steps from the same state: each step
    # copies q^n, q^c,n, q^c,n-1 (and the step's mesh on a moving mesh) from pinned host
    # memory and q^n+1, q^c,n+1, q^c,n back
    e2e = None
    if not args.no_e2e:
        run.restore(snap)
        hq = torch.empty_like(run.q, device="cpu").pin_memory()
        hqn = torch.empty_like(hq).pin_memory()
        hqm = torch.empty_like(hq).pin_memory()
        hq.copy_(run.q)
        hqn.copy_(run.qc_n)
        hqm.copy_(run.qc_nm1)
        hmesh = None
        if meshes is not None:
            hmesh = [(c.cpu().pin_memory(), v.cpu().pin_memory()) for c, v in meshes]
        evs = []
        barrier()
        for k in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            run.q.copy_(hq, non_blocking=True)
            run.qc_n.copy_(hqn, non_blocking=True)
            run.qc_nm1.copy_(hqm, non_blocking=True)
            if hmesh is not None:
                c, v = meshes[run.k]
                c.copy_(hmesh[run.k][0], non_blocking=True)
                v.copy_(hmesh[run.k][1], non_blocking=True)
            run.step()
            hq.copy_(run.q, non_blocking=True)
            hqn.copy_(run.qc_n, non_blocking=True)
            hqm.copy_(run.qc_nm1, non_blocking=True)
            b.record()
            evs.append((a, b))
        barrier()
        t_e2e = sum(a.elapsed_time(b) for a, b in evs) / 1e3
        t_e2e, e2e_value = replica_throughput(t_e2e, dof * args.steps, world, dist, dev)
        nb = run.q.numel() * 8
        mb = 0 if meshes is None else 2 * meshes[0][0].numel() * 8
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": 3 * nb + mb, "d2h_bytes_per_step": 3 * nb,
               "same_steps_as_value": True}

    # ---- kernel throughput: residual and JVP at the start state of the timed steps
    run.restore(snap)
    if meshes is not None:
        S.update_mesh(*meshes[run.k])
    out = torch.empty_like(run.q)
    vec = torch.randn_like(run.q)

    def time_calls(fn, reps=50, flush_between=False):
        """Median device time of one call (CUDA events around each call), after 3 calls
        of warm-up; with flush_between the 256 MiB buffer is rewritten before each call."""
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        evs = []
        for _ in range(reps):
            if flush_between:
                flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in evs)

    calls = {
        "residual": lambda: S.residual(run.q, out),
        "jvp_dual": lambda: S.jvp(run.q, vec, out, 1e-20, 1.5 / w.dt),
        "jvp_linearized": lambda: S.apply_linear(vec, out),
        "vjp": lambda: S.apply_linear(vec, out, transpose=True),
    }
    S.linearize(run.q, 1e-20, 1.5 / w.dt)
    call_gdofs = {}
    for name, fn in calls.items():
        warm = time_calls(fn)
        cold = time_calls(fn, flush_between=True)
        call_gdofs[name] = {"warm_l2": dof / (warm * 1e-3) / 1e9,
                            "flushed_l2": dof / (cold * 1e-3) / 1e9, "median_of": 50}
    t_lin = time_calls(lambda: S.linearize(run.q, 1e-20, 1.5 / w.dt), reps=5)

    sweep = None
    if rank == 0 and not args.no_sweep:
        sweep = large_n_sweep(args.sweep, torch, fr, inp, flush)

    # ---- the plunging NACA 0012 O-grid (bounded mesh: wall below row 0, far field above
    # the last row), 256 x 96 elements at p = 3, Re = 1e4, kappa = sqrt(5): residual and
    # dual-number JVP per call, warm L2 and flushed
    ogrid = None
    if rank == 0 and not args.no_ogrid:
        ni, nj = 256, 96
        c_o, v_o = inp.plunge(inp.naca_ogrid(ni, nj), 0.3)
        qi = inp.far_field_state(w.mach)
        So = fr.Solver(fr.Config(p=3, mach=w.mach, re=1e4, kappa=5 ** 0.5), ni, nj,
                       bc=("wall", "farfield"), q_inf=qi)
        So.update_mesh(T(c_o), T(v_o))
        qo = T(inp.random_perturbation(inp.uniform_state(ni * nj, 3, w.mach), 7, 0.05, w.mach))
        vo = torch.randn_like(qo)
        oo = torch.empty_like(qo)
        ogrid = {"workload": "naca0012_ogrid_256x96_p3 (plunging, wall + far field)",
                 "dof": int(qo.numel())}
        for name, fn in (("residual", lambda: So.residual(qo, oo)),
                         ("jvp_dual", lambda: So.jvp(qo, vo, oo, 1e-20, 1.5 / w.dt))):
            warm = time_calls(fn)
            cold = time_calls(fn, flush_between=True)
            ogrid[name] = {"warm_l2": qo.numel() / (warm * 1e-3) / 1e9,
                           "flushed_l2": qo.numel() / (cold * 1e-3) / 1e9, "median_of": 50}
        So.close()

    # ---- GMRES iteration cost at the start state: a fixed count (tol_res 1e-30), so the
    # per-iteration time does not depend on the Newton history
    gm = {}
    for precond in ("block", "twolevel"):
        gm_cfg = fr.Config(p=w.p, mach=w.mach, re=w.re, kappa=w.kappa, prec=args.prec,
                           restart=args.restart, maxit_lin=120, tol_res=1e-30, graphs=args.graphs, arnoldi_fused=args.arnoldi_fused,
                           apply_accum=args.apply_accum, tiles=args.tiles, orthog=args.orthog,
                           krylov_arith=args.krylov_arith, precond=precond, mg_prec=args.mg_prec,
                           mg_sweeps=args.mg_sweeps, mg_omega=args.mg_omega)
        Sg = fr.Solver(gm_cfg, w.nx, w.ny)
        Sg.update_mesh(*(meshes[run.k] if meshes is not None else (T(corners), T(vel))))
        Sg.precond_build(run.q, 1e-20, 1.5 / w.dt)
        rhs = torch.empty_like(run.q)
        Sg.bdf_rhs(run.q, run.qc_n, run.qc_nm1, fr.BDF2, w.dt, rhs)
        xg = torch.empty_like(run.q)
        Sg.gmres(run.q, rhs, xg, 1e-20, 1.5 / w.dt)
        torch.cuda.synchronize()
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ga.record()
        its_g = Sg.gmres(run.q, rhs, xg, 1e-20, 1.5 / w.dt)
        gb.record()
        torch.cuda.synchronize()
        gm[precond] = 1e3 * ga.elapsed_time(gb) / its_g
        Sg.close()

    # ---- element-block inversion per method at the start state: device time of the
    # factorisation launch (event pair, profiling on), SIMT Gauss-Jordan against the
    # tensor-core blocked forms
    factor_ms = {}
    for prec, factor in (("fp32", "simt"), ("bf16", "tc_bf16"), ("fp32", "tc_bf16x3")):
        Sf = make_solver(prec, factor=factor)
        Sf.precond_build(run.q, 1e-20, 1.5 / w.dt)
        Sf.profile(True)
        Sf.profile_read(reset=True)
        for _ in range(3):
            Sf.precond_build(run.q, 1e-20, 1.5 / w.dt)
        pr = Sf.profile_read(reset=True)["block_factor"]
        Sf.profile(False)
        factor_ms[f"{factor}_{prec}"] = {"ms": pr["ms"] / max(1, pr["launches"]),
                                         "tflops": pr["flops"] / (pr["ms"] * 1e-3) / 1e12 if pr["ms"] else None}
        Sf.close()

    # ---- precision comparison: the timed steps again from the same state per block
    # precision (FP64 Krylov basis) and with FP32 blocks and the double-float basis; the
    # final state of each against the all-FP64 run (max over entries, relative to the
    # per-variable magnitude of the state change)
    compare = {}
    if not args.no_compare:
        finals = {}
        variants = {"fp64": ("fp64", "fp64", "simt"), "fp32": ("fp32", "fp64", "simt"),
                    "bf16": ("bf16", "fp64", "simt"), "fp32_df64_basis": ("fp32", "df64", "simt"),
                    "bf16_tensor_core": ("bf16", "fp64", "tc_bf16"),
                    "fp32_tensor_core_split": ("fp32", "fp64", "tc_bf16x3")}
        for name, (bprec, arith, factor) in variants.items():
            S2 = make_solver(bprec, arith, factor=factor)
            r2 = March(S2, snap[0], meshes, fr)
            r2.restore(snap)
            ms2, st2, _ = timed_steps(r2, args.steps, flush, torch.cuda.synchronize)
            finals[name] = r2.q.clone()
            compare[name] = {"sec_per_step": statistics.mean(ms2) / 1e3,
                             "newton": [s["newton_iterations"] for s in st2],
                             "gmres_total": [sum(s["gmres_iterations"]) for s in st2],
                             "converged": all(s["converged"] for s in st2)}
            S2.close()
        dq = (finals["fp64"] - snap[0]).view(4, -1).abs().amax(dim=1)
        for name in compare:
            diff = (finals[name] - finals["fp64"]).view(4, -1).abs().amax(dim=1)
            compare[name]["state_diff_vs_fp64"] = float((diff / dq).max())

    # the side reports: a failure in one of them is recorded in its entry, never ends the run
    def side_report(fn, *a):
        try:
            return fn(*a)
        except fr.FrError as e:
            torch.cuda.synchronize()
            return {"error": str(e)}

    low_mach = None
    if rank == 0 and not args.no_c3:
        low_mach = side_report(low_mach_deforming_report, args, torch, fr, inp, T, flush)
    ptc = None
    if rank == 0 and not args.no_ptc:
        ptc = side_report(steady_ptc_study, args, torch, fr, inp, T)
    plunge = None
    if rank == 0 and not args.no_plunge:
        plunge = side_report(plunge_march_report, args, torch, fr, inp, T)
    adjoint = None
    if rank == 0 and not args.no_adjoint:
        adjoint = side_report(plunge_adjoint_report, args, torch, fr, inp, T)

    # ---- CPU baseline (rank 0, N = 1 only): the oracle's unit costs priced with the
    # timed steps' own counts
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        profile = {"newton": statistics.mean(s["newton_iterations"] for s in stats),
                   "gmres": statistics.mean(sum(s["gmres_iterations"]) for s in stats),
                   "builds": statistics.mean(s["block_builds"] for s in stats),
                   "restart": args.restart, "precond": args.precond}
        res = oracle_sample(w, profile)
        cpu = {"value": res["value"], "unit": UNIT, "cores": res["cores"], "kind": "oracle",
               "sample": res["sample"], "sec_per_step": res["sec_per_step"]}

    dk = kernels[dominant]
    roof = {"kernel": dominant, "bound": dk["bound"], "achieved": dk["achieved"],
            "peak": dk["peak"], "unit": dk["unit"], "frac": dk["frac"],
            "peak_source": hbm_src if dk["bound"] == "hbm" else ALU_PEAK_SOURCE,
            "alg_per_launch": dk["alg_per_launch"], "us_per_launch": dk["us_per_launch"],
            "share": dk["share"], "traffic": NCU_TRAFFIC.get(dominant)}

    last = stats[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "mesh": f"{w.nx}x{w.ny} periodic [0,10]^2",
                   "deforming": w.deforming,
                   "p": w.p, "dof": dof, "mach": w.mach, "re_ref": w.re, "kappa": w.kappa,
                   "dt": w.dt, "tol_pseudo": w.tol_pseudo, "tol_res": w.tol_res,
                   "gmres": f"GMRES({args.restart}) left-preconditioned, {args.orthog}, "
                            f"{args.krylov_arith} basis, maxit {args.maxit_lin}, "
                            + ("fused Arnoldi step" if args.arnoldi_fused else "split Arnoldi passes"),
                   "newton": f"max {args.maxit_newton} iterations, backtracking {args.line_search} halvings",
                   "precond": f"{args.precond} ({args.prec} element blocks, {args.apply_accum} apply accumulation"
                              + (f", {args.mg_prec} coarse levels, {args.mg_sweeps} sweep(s) of"
                                 f" damping {args.mg_omega})" if args.precond == "twolevel" else ")"),
                   "march": f"timed steps {args.startup + 1}..{args.startup + args.steps} of the march "
                            f"({args.startup} start-up steps before; {args.warmup} warm-up steps run "
                            f"first from the same state, which is then restored)",
                   "l2": "256 MiB write between timed steps, outside the per-step events",
                   "tiles": S.tiles,
                   "parallelism": "replicas" if world > 1 else "single"},
        "startup_steps": {"count": args.startup,
                          "sec_per_step": [round(t, 4) for t, _ in startup],
                          **step_summary([s for _, s in startup])},
        "sec_per_bdf2_step": ms_per_step / 1e3,
        "converged_all": all(s["converged"] for s in stats),
        "newton_iterations": [s["newton_iterations"] for s in stats],
        "gmres_iterations_per_step": [sum(s["gmres_iterations"]) for s in stats],
        "res_drop_last": last["res_history"][-1] / last["res_history"][0],
        "residual_gdofs": call_gdofs["residual"]["warm_l2"],
        "jvp_gdofs": call_gdofs["jvp_dual"]["warm_l2"],
        "linearized_jvp_gdofs": call_gdofs["jvp_linearized"]["warm_l2"],
        "vjp_gdofs": call_gdofs["vjp"]["warm_l2"],
        "call_gdofs": call_gdofs,
        "large_n_sweep": sweep,
        "bounded_ogrid_gdofs": ogrid,
        "linearize_ms": t_lin,
        "us_per_gmres_iteration": gm,
        "precision_compare": compare,
        "block_factor_ms": factor_ms,
        "low_mach_deforming": low_mach,
        "steady_ptc_cylinder": ptc,
        "plunging_naca": plunge,
        "plunging_adjoint": adjoint,
        "kernels": kernels,
        "kernels_same_steps": same_steps,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clock_info,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    S.close()
    if dist is not None:
        dist.destroy_process_group()


def kernels_only(args):
    """Short fixed sequence for profiler captures: geometry, one residual, one JVP, a
    block build and one GMRES solve on the chosen workload (no timing, no JSON)."""
    import numpy as np
    import torch

    from paper_1903_06304_gb300 import fr
    from paper_1903_06304_gb300 import inputs as inp
    w = inp.WORKLOADS[args.workload]
    c, v, q = inp.make_case(w, t=0.13 if w.deforming else 0.0)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")
    S = fr.Solver(fr.Config(p=w.p, mach=w.mach, re=w.re, kappa=w.kappa, prec=args.prec,
                            factor=args.factor, restart=args.restart, maxit_lin=args.maxit_lin,
                            precond=args.precond, graphs=args.graphs, arnoldi_fused=args.arnoldi_fused), w.nx, w.ny)
    S.update_mesh(T(c), T(v))
    qd = T(q)
    out = torch.empty_like(qd)
    qc = torch.empty_like(qd)
    S.conservative(qd, qc)
    S.bdf_rhs(qd, qc, qc, fr.BDF1, w.dt, out)
    x = torch.empty_like(qd)
    for _ in range(args.steps):
        S.residual(qd, x)
        S.jvp(qd, out, x, 1e-20, 1.0 / w.dt)
    S.precond_build(qd, 1e-20, 1.0 / w.dt)
    its = S.gmres(qd, out, x, 1e-20, 1.0 / w.dt)
    torch.cuda.synchronize()
    print(f"kernels-only {w.name}: gmres {its} iterations, {S.kernel_launches} launches")
    S.close()


# ------------------------------------------------------------------ batched cases
def batch_arm(args):
    """Independent cases advanced together (fr_batch_*): the seeded batch recipe (mesh
    side 32..128, p in {2,3,4}, M in [0.01, 0.3], vortex or bump, Re = 100 on the box),
    one BDF2 step of every case per bench step; value = DOF of all cases x steps / time.
    On N ranks the cases are sharded (shard_cases), no data-path collective: each rank
    advances its own batch, the time is the slowest rank's (strong scaling)."""
    import numpy as np
    import torch
    from paper_1903_06304_gb300 import fr
    from paper_1903_06304_gb300 import inputs as inp
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    all_cs = inp.batch_cases(seed=0, ncases=args.batch_cases)
    dof_all = [4 * c.n * c.n * (c.p + 1) ** 2 for c in all_cs]
    parts = shard_cases(dof_all, world)
    # the partition is the same on every rank: all ranks refuse together, before any
    # process group exists, rather than leaving the others waiting in a collective
    if any(not part for part in parts):
        raise SystemExit(f"{len(all_cs)} cases cannot give each of {world} ranks one; use fewer ranks")
    mine = parts[rank]
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cs = [all_cs[k] for k in mine]
    cases = [fr.Case(c.p, c.n, c.n, c.mach, c.re, c.kappa) for c in cs]
    cfg = fr.Config(prec=args.prec, restart=args.restart, maxit_lin=args.maxit_lin,
                    maxit_newton=args.maxit_newton, lag=2, line_search=args.line_search,
                    graphs=args.graphs, arnoldi_fused=args.arnoldi_fused, apply_accum=args.apply_accum,
                    krylov_arith=args.krylov_arith, precond=args.precond, mg_prec=args.mg_prec)
    B = fr.Batch(cfg, cases)
    corners = np.zeros((B.ne, 4, 2))
    q = np.zeros(B.ndof)
    for k, bc in enumerate(cs):
        c, _v, qk = inp.make_batch_case(bc)
        corners[B.elem_slice(k)] = c
        q[B.case_slice(k)] = qk.ravel()
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    B.update_mesh(T(corners), T(np.zeros_like(corners)))
    qd = T(q)
    qc_n, qc_nm1 = torch.empty_like(qd), torch.empty_like(qd)
    B.conservative(qd, qc_n)
    qc_nm1.copy_(qc_n)
    dt = 0.01
    state = {"k": 0}

    def step():
        a = (1.0, -1.0, 0.0) if state["k"] == 0 else (1.5, -2.0, 0.5)
        st = B.bdf2_step(qd, qc_n, qc_nm1, [a + (dt,)] * len(cs), allow_unconverged=True)
        qc_nm1.copy_(qc_n)
        B.conservative(qd, qc_n)
        state["k"] += 1
        return st

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    launches0 = B.kernel_launches
    clocks = ClockSampler(local)
    ms, stats = [], []
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        stats.append(step())
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    barrier()
    clock_info = clocks.stop()
    launches = B.kernel_launches - launches0
    t, value = sharded_throughput(sum(ms) / 1e3, float(sum(dof_all) * args.steps), world, dist, dev)
    newton = [s.newton_iterations for st in stats for s in st]
    gmres = [sum(s.gmres_iterations[:s.newton_iterations]) for st in stats for s in st]
    conv = [s.converged for st in stats for s in st]
    # per-rank statistics summed (counts) or maxed over the ranks
    agg = torch.tensor([sum(conv), sum(newton), len(newton), sum(gmres), launches],
                       dtype=torch.float64, device=dev)
    mx = torch.tensor([max(newton), max(gmres)], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(agg)
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    n_conv, n_newton, n_rows, n_gmres, all_launches = agg.tolist()
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return
    out = {"metric": "batched BDF2 steps of independent cases (GDOF/s)", "impl": "ours",
           "value": value, "unit": "GDOF/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "strong", "dtype": "f64 (blocks %s)" % args.prec,
           "data": "synthetic",
           "config": {"workload": f"batch of {len(all_cs)} cases (seed 0)", "cases": len(all_cs),
                      "cases_rank0": len(cs), "groups_rank0": B.num_groups, "dof": sum(dof_all),
                      "elements": sum(c.n * c.n for c in all_cs),
                      "prec": args.prec, "precond": args.precond, "restart": args.restart,
                      "maxit_lin": args.maxit_lin,
                      "maxit_newton": args.maxit_newton, "line_search": args.line_search,
                      "graphs": args.graphs, "l2": "256 MiB flush between steps",
                      "parallelism": f"cases sharded over {world} ranks" if world > 1 else "single"},
           "cases_converged_per_step": n_conv / args.steps,
           "newton_iterations": {"mean": n_newton / n_rows, "max": int(mx[0])},
           "gmres_iterations": {"mean": n_gmres / n_rows, "max": int(mx[1])},
           "gpu_launches": int(all_launches), "clocks": clock_info}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--startup", type=int, default=0,
                    help="BDF2 steps of the march (recorded, untimed) before the timed ones")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ns_vortex_64x64_p3")
    ap.add_argument("--prec", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--factor", default="simt", choices=["simt", "tc_bf16", "tc_bf16x3"],
                    help="block inversion of --kernels-only: SIMT or on the tensor cores")
    ap.add_argument("--mg-prec", dest="mg_prec", default="fp32", choices=["fp32", "fp64"],
                    help="arithmetic of the two-level preconditioner's coarse levels")
    ap.add_argument("--mg-sweeps", dest="mg_sweeps", type=int, default=2, choices=[1, 2],
                    help="smoothing sweeps per coarse level and direction")
    ap.add_argument("--mg-omega", dest="mg_omega", type=float, default=0.8,
                    help="damping of the coarse block-Jacobi sweeps (0.8: the fastest of "
                         "0.7 .. 1.0 with 1 or 2 sweeps on the benchmark workload)")
    ap.add_argument("--arnoldi-fused", dest="arnoldi_fused", type=int, default=0, choices=[0, 1, 2, 4],
                    help="each Arnoldi step in one launch with bounded barriers (1: part size "
                         "chosen by occupancy; 2, 4: pairs per thread) or as split passes (0)")
    ap.add_argument("--precond", default="twolevel", choices=["block", "twolevel"],
                    help="element block Jacobi, or with the P1 coarse correction")
    ap.add_argument("--no-c3", dest="no_c3", action="store_true",
                    help="skip the deforming 128x128 M = 0.01 report")
    ap.add_argument("--no-ptc", dest="no_ptc", action="store_true",
                    help="skip the steady PTC study on the cylinder O-grid")
    ap.add_argument("--no-plunge", dest="no_plunge", action="store_true",
                    help="skip the plunging NACA 0012 march")
    ap.add_argument("--plunge-steps", dest="plunge_steps", type=int, default=3)
    ap.add_argument("--plunge-periods", dest="plunge_periods", type=int, default=0,
                    help="march whole periods (200 steps each) and report the last one's forces")
    ap.add_argument("--plunge-mach", dest="plunge_mach", type=lambda t: [float(x) for x in t.split(",")],
                    default=[0.05, 0.1, 0.2, 0.3])
    ap.add_argument("--plunge-grid", dest="plunge_grid", default="256x96")
    ap.add_argument("--no-adjoint", dest="no_adjoint", action="store_true",
                    help="skip the plunging march's discrete adjoint")
    ap.add_argument("--adjoint-steps", dest="adjoint_steps", type=int, default=4)
    ap.add_argument("--c3-steps", dest="c3_steps", type=int, default=3)
    ap.add_argument("--c3-newton", dest="c3_newton", type=int, default=20,
                    help="Newton cap of the deforming 128x128 M = 0.01 steps")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--maxit-lin", dest="maxit_lin", type=int, default=100)
    ap.add_argument("--maxit-newton", dest="maxit_newton", type=int, default=40)
    ap.add_argument("--line-search", dest="line_search", type=int, default=0,
                    help="backtracking halvings per Newton update (0: plain Newton)")
    ap.add_argument("--apply-accum", dest="apply_accum", default="df64", choices=["df64", "fp32"],
                    help="block-apply arithmetic with FP32/BF16-stored inverses")
    ap.add_argument("--no-ogrid", action="store_true",
                    help="skip the bounded NACA O-grid residual / JVP timings")
    ap.add_argument("--krylov-arith", dest="krylov_arith", default="fp64", choices=["fp64", "df64"],
                    help="Krylov basis and Gram-Schmidt arithmetic: FP64, or FP32 pairs "
                         "(double-float on the FP32 pipe)")
    ap.add_argument("--orthog", default="cgs2", choices=["cgs2", "cgs"],
                    help="Arnoldi orthogonalisation: CGS2, or one classical pass (PETSc's default)")
    ap.add_argument("--tiles", type=int, default=1, choices=[0, 1, 2],
                    help="elements per CTA of the point kernels: 1 or 2 fixed (1, the library's "
                         "default: reproducible arithmetic), 0 autotuned at set-up by timing (the "
                         "two shapes contract the same formulas into FMAs differently)")
    ap.add_argument("--graphs", type=int, default=1,
                    help="replay GMRES chunks from captured CUDA graphs (1) or launch each kernel (0)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep", type=lambda t: [int(x) for x in t.split(",")], default=[256, 512, 1024],
                    help="mesh sides of the large-N kernel throughput sweep")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--batch-cases", dest="batch_cases", type=int, default=0,
                    help="run the batched-cases workload with this many cases instead")
    ap.add_argument("--kernels-only", action="store_true",
                    help="short fixed call sequence for profiler captures")
    args = ap.parse_args()
    if args.kernels_only:
        kernels_only(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    elif args.batch_cases > 0:
        batch_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
