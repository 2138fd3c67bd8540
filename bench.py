#!/usr/bin/env python
"""Benchmark: matrix-free operator apply throughput (GDoF/s) with its roofline, and the
time of an implicit heat-step solve in fp64 vs mixed fp32/fp64 precision.

One step = one application of the linearised incompressible Navier-Stokes (Oseen) operator,
Q2 velocity / Q1 pressure on a uniform 64^3 mesh (6,714,692 DoFs), fp64, with density and
viscosity from a tanh-smoothed level set (1000:1, 100:1) and a seeded convection field: gather,
Gauss-point values and gradients, pointwise physics, integration and scatter-add, all in the
library's CUDA kernels.  Inputs are resident in HBM; L2 is flushed between timed steps.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference] [--no-solve]
Under torchrun (N > 1) every rank runs an independent replica on its own GPU.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GDoF/s of matrix-free operator apply & %HBM roofline; CG solve time FP64 vs mixed"
WORKLOAD = "oseen_q2q1_interface_64"
HBM_FALLBACK_GBS = 6800.0
FP64_PEAK_TFLOPS = 1.25      # GB300 FP64 (vector and tensor) rate of the profiling recipe's table
# Algorithmic flops of one Oseen Q2/Q1 cell apply as each kernel variant performs it (FMA = 2).
# The 1D sweeps skip the exact zeros and ones of the tables (the middle Gauss point is the middle
# node; D[1][1] = 0): a value sweep costs 9 lines x 2 points x 5 = 90, an integration sweep
# 9 x 10 = 90, a collocation derivative 5 (3 at the middle point), a test accumulation along one
# line 6 (4 at the middle point).
# Gauss-point loop outside, on Gauss-point coefficients with the weight and the powers of h folded
# in (w h^2 rho beta tabulated, so the value terms are multiply-adds only): value sweeps 3 x 270,
# 27 points x 159 (pressure 15, 9 gradients 39, value terms 24, symmetric stress 15 with 2 mu formed
# once, 3 test accumulations 48, continuity 18), nodal pressure and continuity scaling 16,
# integration sweeps 3 x 270 = 5929.
# Component loop outside: pressure at the Gauss points and its test terms 891, three velocity
# components x (value sweeps 270 + 27 points x 80) = 7290, integration sweeps and scaling 899.
OSEEN_FLOPS_PER_CELL = {"component-outer": 891 + 7290 + 899, "qpoint-outer": 810 + 27 * 159 + 16 + 810}
# Algorithmic HBM bytes of one fp64 Oseen apply: read u, write v (16 B per DoF), the nodal
# level set and convection field the coefficients come from (4 x 8 B per velocity node).
OSEEN_BYTES_PER_VEL_NODE = 4 * 8


def max_over_ranks(seconds, dist=None, device="cpu"):
    """The slowest rank's timed-region duration (every rank calls this)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, world, seconds):
    """Whole-job throughput in G units/s: every rank processes units_per_rank per step
    (independent replicas, weak scaling), timed by the slowest rank."""
    return units_per_rank * steps * world / seconds / 1e9


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons every 100 ms while running (the timed
    region starts after the first sample has arrived)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 3.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def kernel_hash():
    h = hashlib.sha256()
    for f in ("apply_f64.cu", "apply_kernels.cuh", "cellops.cuh", "scalar_local.cuh", "df64.cuh"):
        with open(os.path.join(ROOT, "paper_2501_18781_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    kh = kernel_hash()
    for line in open(p):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == workload and parts[1] == kh:
            return float(parts[2])
    return None


def build_oseen(ctx, n=64):
    import numpy as np
    import torch
    import synthetic as syn
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    wl = syn.scaled(syn.OSEEN_INTERFACE, n)
    p = wl.params
    mesh = Mesh.uniform(ctx, n, wl.lo, wl.hi)
    mu, mp = DofMap(mesh, 2, 0b011111), DofMap(mesh, 1, 0)
    x = mu.coords()
    t1, t2 = syn.wavy_plane_phases(wl.seed)
    phi = syn.initial_level_set(syn.wavy_plane_distance(*x.T, t1, t2), wl.eps)
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    sigma = 1.0 / (p["dt_cfl"] * wl.h)
    op = Operator(ctx, "oseen", [mu, mp], sigma=sigma, rho_l=p["rho_l"], rho_g=p["rho_g"], mu_l=p["mu_l"],
                  mu_g=p["mu_g"], eps=wl.eps)
    op.set_field("phi", torch.tensor(phi, device="cuda"))
    op.set_field("beta", torch.tensor(beta.ravel(), device="cuda"))
    op.autotune()   # set-up: picks the fp64 kernel variant (component- or Gauss-point-outer)
    return op, mu, mp, mesh


def time_apply(op, src, dst, steps, warmup, flush):
    import torch
    for _ in range(warmup):
        op.apply(src, dst)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        op.apply(src, dst)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return times


def _event_ms(fn, reps=5, flush=None):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def _apply_rates(op, n, nrhs, flush, reps=5):
    """GDoF/s (DoF x RHS per second) of the fp64, double-float and fp32 applies."""
    import torch
    import synthetic as syn
    u = torch.tensor(syn.uniform_pm1(1, n * nrhs), device="cuda")
    u32 = u.float()
    v, v32 = torch.empty_like(u), torch.empty_like(u32)
    out = {}
    for name, fn in (("f64", lambda: op.apply(u, v, nrhs=nrhs)),
                     ("df64", lambda: op.apply(u, v, nrhs=nrhs, arith="df64")),
                     ("f32", lambda: op.apply(u32, v32, nrhs=nrhs))):
        ms = _event_ms(fn, reps, flush)
        out[name] = {"ms": ms, "gdofs": n * nrhs / ms / 1e6, "variant": op.variant}
    return out


def _packed_rates(op, n, nrhs, flush, reps=5):
    """G DoF.RHS/s of the packed 16-bit applies (fp32 vectors, pairs of right-hand sides per thread)."""
    import torch
    import synthetic as syn
    u = torch.tensor(syn.uniform_pm1(1, n * nrhs), device="cuda").float()
    v = torch.empty_like(u)
    out = {}
    for arith in ("f16", "bf16"):
        ms = _event_ms(lambda: op.apply(u, v, nrhs=nrhs, arith=arith), reps, flush)
        out[arith] = {"ms": ms, "gdofs": n * nrhs / ms / 1e6, "variant": op.variant}
    return out


def workload_suite(ctx, flush):
    """One bounded measurement per benchmark workload (the parity tests cover their numerics)."""
    import numpy as np
    import torch
    import synthetic as syn
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    res = {}
    # Helmholtz 16^3 (L2-resident: launch-latency bound), Jacobi-CG in a CUDA graph
    wl = syn.HELMHOLTZ_SPHERE
    p = wl.params
    m = DofMap(Mesh.uniform(ctx, wl.n, wl.lo, wl.hi), 2, 0)
    x = m.coords()
    phi = syn.initial_level_set(syn.sphere_distance(*x.T), wl.eps)
    op = Operator(ctx, "helmholtz", [m], mass_coef=p["mass"], a_liquid=p["a_liquid"], a_gas=p["a_gas"])
    op.set_field("phi", torch.tensor(phi, device="cuda"))
    op.autotune()
    b = torch.tensor(syn.uniform_pm1(1, m.n_dofs), device="cuda")
    r = {"n_dofs": m.n_dofs, "apply": _apply_rates(op, m.n_dofs, 1, None, reps=20)}
    for g in (False, True):
        op.solve(b, solver="cg", precond="jacobi", use_graph=g)
        t0 = time.perf_counter()
        _, info = op.solve(b, solver="cg", precond="jacobi", use_graph=g)
        r["cg_jacobi_graph" if g else "cg_jacobi"] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                                                      "rel_residual": info["rel_residual"]}
    res[wl.name] = r
    # heat-step adjoint on 64^3: forward + adjoint GMRES and both gradients
    wl = syn.HEAT_ADJOINT
    p = wl.params
    m = DofMap(Mesh.uniform(ctx, wl.n, wl.lo, wl.hi), 2, 1 << 4)
    x = m.coords()
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    kq = syn.kq_field(m.n_cells * 27, wl.seed, p["k0"])
    op = Operator(ctx, "heat", [m], rhocp=p["rhocp"], dt=p["dt"], k0=p["k0"], t_boil=p["t_boil"])
    op.set_field("beta", torch.tensor(beta.ravel(), device="cuda"))
    op.set_field("k_qpoint", torch.tensor(kq, device="cuda"))
    ztop = wl.hi[2]
    lz = p["laser"]
    th_prev = syn.heat_initial_temperature(*x.T, lz["radius"], ztop) - p["t_ref"]
    target = syn.heat_target_temperature(*x.T, ztop, wl.seed + 4) - p["t_ref"]
    tp, tt = torch.tensor(th_prev, device="cuda"), torch.tensor(target, device="cuda")
    lzt = (lz["power"], lz["radius"], lz["x0"], lz["y0"], lz["absorptivity"])
    kw = dict(solver="gmres", precond="jacobi", tol=1e-10, restart=50)
    op.heat_step_gradient(lzt, tp, tt, p["box_half"], p["box_depth"], **kw)
    t0 = time.perf_counter()
    J, g, gk, _, _ = op.heat_step_gradient(lzt, tp, tt, p["box_half"], p["box_depth"], **kw)
    torch.cuda.synchronize()
    res[wl.name] = {"n_dofs": m.n_dofs, "gradient_seconds": time.perf_counter() - t0, "J": J,
                    "dJ_dlaser": g, "apply": _apply_rates(op, m.n_dofs, 1, flush)}
    # adaptive octree reinitialisation, 8 right-hand sides batched per launch, mixed precision
    wl = syn.REINIT_OCTREE
    d = lambda X, Y, Z: syn.deformed_sphere_distance(X, Y, Z, wl.seed)
    leaves = syn.refine_band_leaves(wl.n, wl.levels, d, wl.eps)
    mesh = Mesh.octree(ctx, wl.n, wl.levels, leaves)
    m = DofMap(mesh, 2, 0)
    x = m.coords()
    phi = syn.initial_level_set(syn.deformed_sphere_distance(*x.T, wl.seed), wl.eps)
    hmin = 1.0 / (wl.n << wl.levels)
    op = Operator(ctx, "reinit", [m], eps=wl.eps, dtau=0.5 * hmin)
    op.set_field("phi", torch.tensor(phi, device="cuda"))
    op.autotune()
    B = torch.tensor(np.concatenate([syn.uniform_pm1(s, m.n_dofs) for s in range(1, wl.nrhs + 1)]), device="cuda")
    r = {"n_dofs": m.n_dofs, "cells": m.n_cells, "hanging_nodes": m.n_constraints, "nrhs": wl.nrhs,
         "apply_batched": _apply_rates(op, m.n_dofs, wl.nrhs, flush, reps=3),
         "apply_single": _apply_rates(op, m.n_dofs, 1, flush, reps=3),
         "apply_batched_packed16": _packed_rates(op, m.n_dofs, wl.nrhs, flush, reps=3)}
    kw = dict(solver="defect_correction", precond="chebyshev", tol=1e-10, use_graph=True)
    op.solve(B, nrhs=wl.nrhs, **kw)
    t0 = time.perf_counter()
    _, info = op.solve(B, nrhs=wl.nrhs, **kw)
    torch.cuda.synchronize()
    r["mixed_solve_8rhs"] = {"seconds": time.perf_counter() - t0, "inner_iterations": info["iterations"],
                             "outer": info["outer_iterations"], "rel_residual": info["rel_residual"],
                             "status": info["status"]}
    for arith in ("bf16", "f16"):
        op.solve(B, nrhs=wl.nrhs, inner_arith=arith, **kw)
        t0 = time.perf_counter()
        _, info = op.solve(B, nrhs=wl.nrhs, inner_arith=arith, **kw)
        torch.cuda.synchronize()
        r[f"mixed_solve_8rhs_inner_{arith}"] = {"seconds": time.perf_counter() - t0,
                                                "inner_iterations": info["iterations"],
                                                "outer": info["outer_iterations"], "rel_residual": info["rel_residual"],
                                                "status": info["status"]}
    res[wl.name] = r
    return res


def heat_solve_comparison(ctx, n=128):
    """Implicit heat step on n^3 Q2 cells: fp64 CG with Chebyshev(4)-Jacobi vs fp32 inner CG
    (same preconditioner in fp32) inside fp64 defect correction, both to 1e-10."""
    import numpy as np
    import torch
    import synthetic as syn
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    wl = syn.scaled(syn.HEAT_LASER, n)
    p = wl.params
    mesh = Mesh.uniform(ctx, n, wl.lo, wl.hi)
    m = DofMap(mesh, 2, 1 << 4)
    x = m.coords()
    T_prev = syn.heat_initial_temperature(*x.T, p["laser"]["radius"], wl.hi[2])
    op = Operator(ctx, "heat", [m], rhocp=p["rhocp"], dt=p["dt"], k0=p["k0"], t_boil=p["t_boil"], coef_mode=1)
    op.set_field("t_prev", torch.tensor(T_prev, device="cuda"))
    b = torch.tensor(syn.uniform_pm1(1, m.n_dofs), device="cuda")
    b[torch.tensor(m.export(cell_map=False, constraints=False, coords=False)["dirichlet"], device="cuda")] = 0
    out = {"workload": wl.name, "n_dofs": m.n_dofs, "tol": 1e-10}
    for name, kw in (("fp64", dict(solver="cg", precond="chebyshev")),
                     ("mixed", dict(solver="defect_correction", precond="chebyshev", inner_tol=1e-4,
                                    inner_maxit=100))):
        op.solve(b, tol=1e-10, use_graph=True, **kw)          # set-up + warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = op.solve(b, tol=1e-10, use_graph=True, **kw)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                     "outer": info["outer_iterations"], "rel_residual": info["rel_residual"],
                     "status": info["status"]}
    out["speedup_mixed_over_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    return out


def cpu_oracle_apply(n_sample, budget_s=8.0):
    """The oracle (assembled CSR from full-quadrature element matrices) applied on the host:
    returns GDoF/s of its SpMV on an n_sample^3 instance of the same workload."""
    import numpy as np
    import synthetic as syn
    from oracle import assemble as asm
    from oracle import mesh as omesh
    wl = syn.scaled(syn.OSEEN_INTERFACE, n_sample)
    p = wl.params
    dmu = omesh.uniform_dofmap(n_sample, wl.lo, wl.hi, 2, 0b011111)
    dmp = omesh.uniform_dofmap(n_sample, wl.lo, wl.hi, 1, 0)
    x = dmu.dof_coords()
    t1, t2 = syn.wavy_plane_phases(wl.seed)
    phi = syn.initial_level_set(syn.wavy_plane_distance(*x.T, t1, t2), wl.eps)
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    A = asm.oseen_matrix(dmu, dmp, phi, beta, 1.0 / (p["dt_cfl"] * wl.h), p["rho_l"], p["rho_g"], p["mu_l"],
                         p["mu_g"])
    u = syn.uniform_pm1(1, A.shape[0])
    A @ u
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        A @ u
        reps += 1
    dt = time.perf_counter() - t0
    return A.shape[0] * reps / dt / 1e9, A.shape[0], reps, dt


def cpu_oracle_workloads():
    """The oracle as it stands on the host (one core, scipy CSR): assembly, SpMV and Jacobi-CG to
    1e-10 on the Helmholtz 16^3 workload (35,937 DoFs) -- the CPU side of the solve comparison."""
    import numpy as np
    import synthetic as syn
    from oracle import assemble as asm
    from oracle import krylov
    from oracle import mesh as omesh
    wl = syn.HELMHOLTZ_SPHERE
    p = wl.params
    t0 = time.perf_counter()
    dm = omesh.uniform_dofmap(wl.n, wl.lo, wl.hi, 2)
    phi = syn.initial_level_set(syn.sphere_distance(*dm.dof_coords().T), wl.eps)
    A = asm.helmholtz_matrix(dm, phi, p["mass"], p["a_liquid"], p["a_gas"])
    t_asm = time.perf_counter() - t0
    b = syn.uniform_pm1(1, dm.n_dofs)
    A @ b
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < 2.0:
        A @ b
        reps += 1
    t_spmv = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    _, its, res = krylov.cg(lambda v: A @ v, b, krylov.jacobi(A.diagonal()), tol=1e-10)
    t_cg = time.perf_counter() - t0
    return {"workload": wl.name, "n_dofs": dm.n_dofs, "cores": 1, "assembly_seconds": t_asm,
            "spmv_gdofs": dm.n_dofs / t_spmv / 1e9, "cg_jacobi_seconds": t_cg, "cg_iterations": its,
            "rel_residual": res}


def reference_arm(args, rank, world):
    out = {"impl": "reference", "metric": METRIC, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic"}
    if rank != 0:
        return None
    import numpy as np
    import synthetic as syn
    from oracle import assemble as asm
    from oracle import mesh as omesh
    n_sample = 12
    wl = syn.scaled(syn.OSEEN_INTERFACE, n_sample)
    p = wl.params
    dmu = omesh.uniform_dofmap(n_sample, wl.lo, wl.hi, 2, 0b011111)
    dmp = omesh.uniform_dofmap(n_sample, wl.lo, wl.hi, 1, 0)
    x = dmu.dof_coords()
    t1, t2 = syn.wavy_plane_phases(wl.seed)
    phi = syn.initial_level_set(syn.wavy_plane_distance(*x.T, t1, t2), wl.eps)
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    A = asm.oseen_matrix(dmu, dmp, phi, beta, 1.0 / (p["dt_cfl"] * wl.h), p["rho_l"], p["rho_g"], p["mu_l"],
                         p["mu_g"])
    u = syn.uniform_pm1(1, A.shape[0])
    for _ in range(args.warmup):
        A @ u
    t0 = time.perf_counter()
    for _ in range(args.steps):
        A @ u
    dt = time.perf_counter() - t0
    val = A.shape[0] * args.steps / dt / 1e9
    out.update(value=val, ms_per_step=dt / args.steps * 1e3,
               config={"workload": WORKLOAD, "sample": wl.name, "n_dofs": int(A.shape[0]),
                       "note": "oracle: assembled-CSR SpMV of a 12^3 instance (assembly untimed)"},
               cpu_baseline={"value": val, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                             "sample": f"{wl.name}: assembled CSR SpMV, {args.steps} steps"},
               e2e={"value": val, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
    return out


def oseen_solve(ctx, op, mu, mp):
    """The Oseen saddle-point solve to 1e-10: flexible GMRES(50) with the block upper-triangular
    preconditioner (fp32 inner applies), a seeded right-hand side with zero Dirichlet rows."""
    import numpy as np
    import torch
    import synthetic as syn
    b = syn.uniform_pm1(1, op.n)
    d = mu.export(cell_map=False, constraints=False, coords=False)["dirichlet"]
    b[np.concatenate([np.tile(d, 3), np.zeros(mp.n_dofs, bool)])] = 0
    bt = torch.tensor(b, device="cuda")
    kw = dict(solver="gmres", precond="block_triangular", restart=50, maxit=400, tol=1e-10, velocity_steps=10,
              schur_tol=0.1, schur_maxit=30)
    out = {"solver": "fgmres(50) + block-triangular (fp32 inner)", "tol": 1e-10}
    for key, graph in (("seconds_direct", False), ("seconds", True)):
        op.solve(bt, use_graph=graph, **kw)                        # set-up + warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = op.solve(bt, use_graph=graph, **kw)
        torch.cuda.synchronize()
        out[key] = time.perf_counter() - t0
    out.update(iterations=info["iterations"], rel_residual=info["rel_residual"], status=info["status"],
               preconditioner="replayed CUDA graph", schur_steps_per_call=info["inner_steps"] / info["iterations"])
    return out


def meltpool_oseen(ctx, n, flush, darcy_c=None):
    """The Oseen workload with the melt-pool terms switched on (three-phase rho/mu, Darcy damping,
    trace-corrected stress) and a hot spot across the interface.  The paper damps with C = 1e12
    kg/(m^3 s) at a time step of 0.01 us (rho_l / dt = 4.1e11): C / (rho_l sigma) = 2.45.  The
    unit-cube workload has sigma = 1/dt = 2n, so C is scaled to keep that ratio (C = 1e12 * 1e-8 *
    sigma); the unscaled 1e12 makes even a direct solve stall at a 1e-7 relative residual here.
    Solid below T_s far from the spot.  fp64 and fp32 apply rates and the FGMRES solve to 1e-10 with
    the interface source loads as right-hand side."""
    import numpy as np
    import torch
    import synthetic as syn
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    from paper_2501_18781_gb300._lib import MF_OSEEN_DARCY, MF_OSEEN_THREE_PHASE, MF_OSEEN_TRACE_CORRECTION
    wl = syn.scaled(syn.OSEEN_INTERFACE, n)
    p = wl.params
    mesh = Mesh.uniform(ctx, n, wl.lo, wl.hi)
    mu, mp = DofMap(mesh, 2, 0b011111), DofMap(mesh, 1, 0)
    x = mu.coords()
    t1, t2 = syn.wavy_plane_phases(wl.seed)
    phi = syn.initial_level_set(syn.wavy_plane_distance(*x.T, t1, t2), wl.eps)
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    T = syn.interface_temperature(*x.T, t_base=1500.0)
    sigma = 1.0 / (p["dt_cfl"] * wl.h)
    if darcy_c is None:
        darcy_c = 1e12 * 1e-8 * sigma
    op = Operator(ctx, "oseen", [mu, mp], sigma=sigma, rho_l=p["rho_l"], rho_g=p["rho_g"],
                  mu_l=p["mu_l"], mu_g=p["mu_g"], eps=wl.eps, rho_s=p["rho_l"], mu_s=p["mu_l"], t_solidus=1933.0,
                  t_liquidus=2200.0, darcy_c=darcy_c, darcy_b=1.0,
                  oseen_flags=MF_OSEEN_THREE_PHASE | MF_OSEEN_DARCY | MF_OSEEN_TRACE_CORRECTION)
    fields = [torch.tensor(phi, device="cuda"), torch.tensor(beta.ravel(), device="cuda"), torch.tensor(T, device="cuda")]
    op.set_field("phi", fields[0])
    op.set_field("beta", fields[1])
    op.set_field("t_prev", fields[2])
    u = torch.tensor(syn.uniform_pm1(1, op.n), device="cuda")
    v = torch.empty_like(u)
    u32, v32 = u.float(), torch.empty(op.n, dtype=torch.float32, device="cuda")
    ms64 = _event_ms(lambda: op.apply(u, v), 10, flush)
    ms32 = _event_ms(lambda: op.apply(u32, v32), 10, flush)
    # right-hand side: the interface loads of this temperature field (hybrid recoil force in the
    # momentum rows, evaporative dilation in the continuity rows)
    ev, ti = syn.EVAPORATION, syn.TI64
    src = op.interface_sources(fields[2], ev["p_amb"], ev["h_v"], ev["molar_mass"], ev["t_boil"],
                               ti["rho_l"] * ti["cp_l"], ti["rho_g"] * ti["cp_g"], outputs=("u", "p"))
    bt = torch.cat([src["u"], src["p"]])
    kw = dict(solver="gmres", precond="block_triangular", restart=50, maxit=400, tol=1e-10, use_graph=True)
    op.solve(bt, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, info = op.solve(bt, **kw)
    torch.cuda.synchronize()
    return {"workload": f"oseen_meltpool_{n}", "variant": op.variant, "darcy_c": darcy_c,
            "apply_f64": {"ms": ms64, "gdofs": op.n / ms64 / 1e6}, "apply_f32": {"ms": ms32, "gdofs": op.n / ms32 / 1e6},
            "solve": {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                      "rel_residual": info["rel_residual"], "status": info["status"]}}


def build_meltpool_step(ctx, n=64):
    """The melt-pool step workload on the 600 um box (n^3 cells): maps, the seeded state (fp64
    device tensors) and the MeltPoolStep with every term switched on."""
    import numpy as np
    import torch
    import synthetic as syn
    from paper_2501_18781_gb300 import DofMap, MeltPoolStep, Mesh
    from paper_2501_18781_gb300._lib import MF_OSEEN_DARCY, MF_OSEEN_THREE_PHASE, MF_OSEEN_TRACE_CORRECTION
    wl = syn.scaled(syn.MELTPOOL_STEP, n)
    p, ti, ev = wl.params, syn.TI64, syn.EVAPORATION
    mesh = Mesh.uniform(ctx, n, wl.lo, wl.hi)
    maps = [DofMap(mesh, 2, 0b011111), DofMap(mesh, 1, 0), DofMap(mesh, 2, 0), DofMap(mesh, 2, 1 << 4)]
    x = maps[0].coords()
    state = {k: torch.tensor(np.ascontiguousarray(v.ravel()), device="cuda")
             for k, v in syn.meltpool_state(*x.T, wl.seed, wl.lo, wl.hi, wl.eps, u_max=p["u_max"]).items()}
    sol, dar, st = p["solid"], p["darcy"], p["surface_tension"]
    step = MeltPoolStep(
        ctx, maps,
        evaporation=dict(mass_flux="knight", p_ambient=ev["p_amb"], latent_heat=ev["h_v"], molar_mass=ev["molar_mass"],
                         t_boil=ev["t_boil"], sticking=ev["sticking"], gas_constant=8.314),
        laser=p["laser"], gravity=p["gravity"], dt=p["dt"], eps=wl.eps, rho_l=ti["rho_l"], rho_g=ti["rho_g"],
        mu_l=ti["mu_l"], mu_g=ti["mu_g"], rhocp_l=ti["rho_l"] * ti["cp_l"], rhocp_g=ti["rho_g"] * ti["cp_g"],
        k_l=ti["k_l"], k_g=ti["k_g"], oseen_flags=MF_OSEEN_THREE_PHASE | MF_OSEEN_DARCY | MF_OSEEN_TRACE_CORRECTION,
        rho_s=sol["rho_s"], mu_s=sol["mu_s"], t_solidus=sol["t_solidus"], t_liquidus=sol["t_liquidus"],
        darcy_c=dar["C"], darcy_b=dar["b"], alpha0=st["alpha0"], alpha1=st["alpha1"], t_alpha=st["t_alpha"],
        alpha_res=st["alpha_res"], reinit_steps=p["reinit_steps"], dtau=p["dtau_cells"] * wl.h, tol=p["tol"],
        flow_tol=p["flow_tol"], maxit=500, reinit_mixed=p["reinit_mixed"], flow_velocity_steps=p["flow_velocity_steps"],
        flow_schur_maxit=p["flow_schur_maxit"], flow_schur_tol=p["flow_schur_tol"])
    return wl, maps, state, step


def meltpool_step(ctx, n=64, reps=3):
    """One step of the melt-pool algorithm on the 600 um box (64^3 cells: 2.1M Q2 nodes per field,
    6.7M velocity-pressure DoFs): predictors, level-set advection (GMRES) with the variant-1
    transport velocity, 2 reinitialisation steps (CG), two-phase heat with laser and evaporative
    cooling (GMRES), melt-pool Navier-Stokes with surface tension, recoil and Darcy damping
    (FGMRES, block-triangular).  The same state is advanced reps times after one warm-up step."""
    import torch
    wl, maps, state, step = build_meltpool_step(ctx, n)
    p = wl.params
    step.advance(state)
    torch.cuda.synchronize()
    runs = []
    for _ in range(reps):
        t0 = time.perf_counter()
        _, info = step.advance(state)
        torch.cuda.synchronize()
        runs.append((time.perf_counter() - t0, info))
    wall, info = sorted(runs, key=lambda r: r[0])[len(runs) // 2]
    nu, npr = maps[0].n_dofs, maps[1].n_dofs
    return {"workload": wl.name, "n_u": nu, "n_p": npr, "unknowns_per_step": 5 * nu + npr, "ms_per_step": wall * 1e3,
            "stage_seconds": dict(zip(("advection", "reinit", "heat", "flow", "total"), info["seconds"])),
            "iterations": {k: info[k + "_iterations"] for k in ("advection", "reinit", "heat", "flow")},
            "rel_residuals": {k: info[k + "_residual"] for k in ("advection", "reinit", "heat", "flow")},
            "status": info["status"], "tol": p["tol"], "flow_tol": p["flow_tol"]}


def qk_flops_per_cell(k):
    """Sum-factorised Q_k Helmholtz apply, P = k + 1: 3 interpolation sweeps, 3 collocation
    derivatives, 3 transposed derivatives and 3 transposed sweeps of P^4 multiply-adds each, and
    about 10 flops per Gauss point for the pointwise work."""
    P = k + 1
    return 2 * 12 * P ** 4 + 10 * P ** 3


def helmholtz_qk(ctx, flush):
    """Q3 on 64^3 and Q4 on 48^3 cells (193^3 = 7,189,057 DoFs each), the sphere coefficient
    a = 1 + 999 H(phi): fp64 and fp32 applies with the L2 flushed."""
    import torch
    import synthetic as syn
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    out = {}
    for k, n in ((3, 64), (4, 48)):
        m = DofMap(Mesh.uniform(ctx, n), k, 0)
        eps = 1.0 / (2 * n)
        phi = torch.tensor(syn.initial_level_set(syn.sphere_distance(*m.coords().T), eps), device="cuda")
        op = Operator(ctx, "helmholtz", [m], mass_coef=1.0, a_liquid=1000.0, a_gas=1.0, eps=eps)
        op.set_field("phi", phi)
        fl = qk_flops_per_cell(k) * m.n_cells
        r = {"cells": m.n_cells, "n_dofs": m.n_dofs, "flops_per_cell": qk_flops_per_cell(k)}
        for dt in (torch.float64, torch.float32):
            u = torch.tensor(syn.uniform_pm1(1, m.n_dofs), device="cuda").to(dt)
            v = torch.empty_like(u)
            op.apply(u, v)
            ms = _event_ms(lambda: op.apply(u, v), 10, flush)
            r["f64" if dt == torch.float64 else "f32"] = {"ms": ms, "gdofs": m.n_dofs / ms / 1e6,
                                                          "tflops": fl / ms / 1e9, "variant": op.variant}
        r["f64"]["frac_of_fp64_peak"] = r["f64"]["tflops"] / FP64_PEAK_TFLOPS
        if k == 3:
            # the tensor-core kernel: 2 dense products of 2 x 64 x 256 flops per cell, three split terms
            u = torch.tensor(syn.uniform_pm1(1, m.n_dofs), device="cuda").float()
            v = torch.empty_like(u)
            op.apply(u, v, arith="tc")
            ms = _event_ms(lambda: op.apply(u, v, arith="tc"), 10, flush)
            dense = 3 * 2 * 2 * 64 * 256 * m.n_cells
            r["tc_bf16x3"] = {"ms": ms, "gdofs": m.n_dofs / ms / 1e6, "tensor_tflops": dense / ms / 1e9,
                              "sum_factorised_tflops_equiv": fl / ms / 1e9, "variant": op.variant}
            # solves to 1e-10: fp64 Jacobi-CG; defect correction with fp32 Chebyshev-CG inner solves on
            # the CUDA cores or on the tensor cores
            b = torch.tensor(syn.uniform_pm1(2, m.n_dofs), device="cuda")
            # (this contrast-1000 problem needs ~1750 Jacobi-CG iterations in fp64: the inner solves get
            # room to reach their 1e-4)
            runs = {"fp64_cg_jacobi": dict(solver="cg", precond="jacobi"),
                    "mixed_inner_f32": dict(solver="defect_correction", precond="chebyshev", inner_arith="f32",
                                            inner_maxit=3000),
                    "mixed_inner_tensor_cores": dict(solver="defect_correction", precond="chebyshev",
                                                     inner_arith="tc", inner_maxit=3000)}
            r["solve"] = {}
            for name, kw in runs.items():
                op.solve(b, tol=1e-10, **kw)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, info = op.solve(b, tol=1e-10, **kw)
                torch.cuda.synchronize()
                r["solve"][name] = {"seconds": time.perf_counter() - t0, "iterations": info["iterations"],
                                    "outer": info["outer_iterations"], "rel_residual": info["rel_residual"],
                                    "status": info["status"]}
        out[f"q{k}"] = r
    return out


def interface_sources_timing(ctx, op, mu, flush, reps=10):
    """The fused interface-source kernel (evaporative dilation, cooling and hybrid recoil loads)
    on the Oseen mesh, Knight's mass flux, a hot spot across the interface."""
    import torch
    import synthetic as syn
    ev, ti = syn.EVAPORATION, syn.TI64
    T = torch.tensor(syn.interface_temperature(*mu.coords().T), device="cuda")
    args = (T, ev["p_amb"], ev["h_v"], ev["molar_mass"], ev["t_boil"], ti["rho_l"] * ti["cp_l"], ti["rho_g"] * ti["cp_g"])
    op.interface_sources(*args)
    ms = _event_ms(lambda: op.interface_sources(*args), reps, flush)
    return {"ms": ms, "cells_per_s": mu.n_cells / ms * 1e3, "gdofs": op.n / ms / 1e6,
            "outputs": "recoil force (3 n_u), dilation (n_p), cooling (n_u)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--suite", action="store_true", help="also measure the other benchmark workloads")
    ap.add_argument("--meltpool-step", action="store_true", help="also time one melt-pool algorithm step")
    ap.add_argument("--qk", action="store_true", help="also time the Q3 / Q4 Helmholtz applies")
    ap.add_argument("--n", type=int, default=64)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = reference_arm(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    ctx = Context(local)
    op, mu, mp, mesh = build_oseen(ctx, args.n)
    n = op.n
    ncells = mu.n_cells
    import synthetic as syn
    src = torch.tensor(syn.uniform_pm1(1, n), device="cuda")
    dst = torch.empty_like(src)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    # warm-up and set-up (Gauss-point coefficient tables) outside the timed region
    for _ in range(args.warmup):
        op.apply(src, dst)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ctx.launch_count()
    with ClockSampler(local) as clocks:
        times = time_apply(op, src, dst, args.steps, 0, flush)
    launches = ctx.launch_count() - l0
    total = sum(times)
    total = max_over_ranks(total, dist, "cuda")
    value = whole_job_rate(n, args.steps, world, total)
    mean = total / args.steps

    # end to end through the public API: pinned host input -> device -> apply -> host output
    hsrc = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hsrc.copy_(src.cpu())
    hdst = torch.empty(n, dtype=torch.float64, pin_memory=True)
    dsrc = torch.empty_like(src)
    for _ in range(2):
        dsrc.copy_(hsrc, non_blocking=True)
        op.apply(dsrc, dst)
        hdst.copy_(dst, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        dsrc.copy_(hsrc, non_blocking=True)
        op.apply(dsrc, dst)
        hdst.copy_(dst, non_blocking=True)
    e1.record()
    e1.synchronize()
    e2e_t = e0.elapsed_time(e1) / 1e3
    e2e = {"value": n * args.steps * world / e2e_t / 1e9, "unit": "GDoF/s",
           "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8}

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", HBM_FALLBACK_GBS)
    flops = OSEEN_FLOPS_PER_CELL["qpoint-outer" if "qpoint-outer" in op.variant else "component-outer"] * ncells
    alg_bytes = 16 * n + OSEEN_BYTES_PER_VEL_NODE * mu.n_dofs
    achieved = flops / mean / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"oseen_q2q1_interface_{args.n}", "n_dofs": n, "cells": ncells,
                   "velocity": "Q2 x 3", "pressure": "Q1", "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed between timed steps (256 MB write)", "variant": op.variant},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": ncu_traffic(f"oseen_q2q1_interface_{args.n}"),
                     "flops_per_launch": flops, "peak_source": "GB300 FP64 rate of the profiling recipe"},
        "hbm_roofline": {"achieved": alg_bytes / mean / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg_bytes / mean / 1e9 / hbm, "bytes_per_launch": alg_bytes,
                         "peak_source": "MEASURED_PEAKS.json" if "hbm_gbs" in peaks else "fallback"},
        "e2e": e2e, "gpu_launches": launches, "clocks": clocks.summary(),
    }
    # the same apply in fp32 (context for the mixed-precision solver)
    src32, dst32 = src.float(), torch.empty(n, dtype=torch.float32, device="cuda")
    t32 = time_apply(op, src32, dst32, max(5, args.steps // 2), 3, flush)
    out["fp32_apply"] = {"value": n / (sum(t32) / len(t32)) / 1e9, "unit": "GDoF/s",
                         "ms_per_step": sum(t32) / len(t32) * 1e3}
    out["df64_apply"] = {"value": n / (_event_ms(lambda: op.apply(src, dst, arith="df64"), 5, flush) / 1e3) / 1e9,
                         "unit": "GDoF/s", "note": "fp64 vectors, double-float cell arithmetic on the fp32 pipes"}
    if rank == 0:
        out["interface_sources"] = interface_sources_timing(ctx, op, mu, flush)
    if not args.no_solve and rank == 0:
        out["solve"] = heat_solve_comparison(ctx)
        out["oseen_solve"] = oseen_solve(ctx, op, mu, mp)
    if args.suite and rank == 0:
        out["workloads"] = workload_suite(ctx, flush)
        out["workloads"]["oseen_meltpool"] = meltpool_oseen(ctx, args.n, flush)
    if args.suite and rank == 0 and world == 1:
        out.setdefault("workloads", {})["cpu_oracle_helmholtz_16"] = cpu_oracle_workloads()
    if (args.suite or args.qk) and rank == 0:
        out.setdefault("workloads", {})["helmholtz_qk"] = helmholtz_qk(ctx, flush)
    if (args.suite or args.meltpool_step) and rank == 0:
        out.setdefault("workloads", {})["meltpool_step"] = meltpool_step(ctx, args.n)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, nd, reps, dt = cpu_oracle_apply(16)
        out["cpu_baseline"] = {"value": v, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                               "sample": f"oseen_q2q1_interface_16 ({nd} DoFs): assembled-CSR SpMV x {reps} "
                                         f"in {dt:.1f} s (assembly untimed)"}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
