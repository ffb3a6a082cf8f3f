#!/usr/bin/env python
"""Benchmark of the hierarchical Chebyshev-collocation solve on B300.

Workload (one "step"): the 257^3 heterogeneous two-phase problem solved by
hierarchical refinement 65^3 -> 129^3 -> 257^3 with modal prolongation
(seeded non-overlapping spheres, radii U(0.08, 0.15), 20% volume fraction,
K_incl / K_matrix = 100, f = 0, Dirichlet u = x on x = +-1, zero-flux Neumann
elsewhere), mixed precision (FP32 inner LGMRES, FP64 refinement), stopping at
a preconditioned relative residual of 1e-12.  The metric is the time to
solve; the same line reports the operator apply throughput (GDOF/s) in FP32
and FP64, the plain-FP64 time to solve, the roofline of the dominant
kernel, an end-to-end time through the public API with host buffers, and
(rank 0) the FP64 CPU oracle's own hierarchical solve of the same workload,
run once on the host cores: its measured time is the CPU baseline and its
solution gives the relative L2 error of the GPU solutions at every level.

``--impl reference`` runs that oracle solve alone (the reference arm).
Multi-GPU: independent replicas (the single-grid solve does not shard).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "257³ time-to-solve at rel.err≤1e-8 and apply GDOF/s, mixed vs FP64, same B300"
BC = [0, 0, 1, 1, 1, 1]   # x faces Dirichlet, y and z faces Neumann


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--levels", default="65,129,257")
    ap.add_argument("--contrast", type=float, default=100.0)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the oracle's hierarchical solve (CPU baseline and parity)")
    ap.add_argument("--reorth", type=int, default=0, help="Gram-Schmidt twice per Arnoldi step")
    ap.add_argument("--inner-rtol", type=float, default=1e-4)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--workload", default="hierarchy", choices=["hierarchy", "batch", "newton"],
                    help="hierarchy: the 257^3 hierarchical solve (the metric); batch: 16 uneven "
                         "lognormal Picard instances solved concurrently (a secondary line); newton: the "
                         "paper's Table 1 nonlinear problem by hierarchical Newton (a secondary line)")
    ap.add_argument("--use-graph", type=int, default=0)
    ap.add_argument("--batch-mode", type=int, default=1, choices=[1, 2],
                    help="--workload batch: 1 lockstep, 2 one concurrent solver per instance")
    ap.add_argument("--picard-steps", type=int, default=60,
                    help="--workload batch: Picard iteration limit (the batch converges in 30)")
    ap.add_argument("--coarse-rtol", type=float, default=1e-2,
                    help="relative tolerance of the hierarchy's coarse levels, whose solutions only "
                         "start the next level (0: the finest level's 1e-12)")
    ap.add_argument("--ncu-step", action="store_true",
                    help="after the warm-up, run one step between cudaProfilerStart/Stop and exit "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--pmat", type=int, default=0, choices=[0, 1],
                    help="FP32 preconditioner matrices: 0 rounded to TF32 (the library default, two "
                         "tensor-core products per step), 1 to FP32 accuracy (three products)")
    ap.add_argument("--recycle", type=int, default=0,
                    help="carry LGMRES augmentation vectors across refinement steps (1) or not (0)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 16-instance batch keys")
    ap.add_argument("--no-newton", action="store_true", help="skip the Table 1 Newton keys")
    ap.add_argument("--route32", default="auto", choices=["auto", "transform", "tensor"],
                    help="operator-apply routes: auto = the library's autotuner times every "
                         "route each axis allows and keeps the fastest (per precision); "
                         "transform / tensor force the FP32 route of every axis")
    ap.add_argument("--fdm-only", type=int, default=0, metavar="BITS",
                    help="only time the preconditioner at the finest level (profiling)")
    ap.add_argument("--apply-only", type=int, default=0, metavar="BITS",
                    help="only time cheb_apply at the finest level in FP32 (32) or FP64 (64); "
                         "for profiling")
    return ap.parse_args()


def max_over_ranks(value, world, device="cuda"):
    """The largest of the ranks' values (the interval of the slowest replica);
    one process returns its own.  Every rank must call it (a collective)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------

def x_boundary(X, Y, Z):
    return X, (np.ones_like(X), 0 * X, 0 * X), 0 * X


def host_level(n, spheres, contrast, nodes):
    """K and b of one level on the host, sampled at the given node arrays."""
    import workloads as W
    X, Y, Z = W.mesh(*nodes)
    K = W.two_phase_conductivity(X, Y, Z, spheres, 1.0, contrast)
    faces = W.face_values(BC, nodes[0], nodes[1], nodes[2], x_boundary)
    return K, faces


def set_routes(p, route32):
    """Routes of the plan's axes: chosen by the autotuner (``auto``), or the
    FP32 route of every axis that allows it forced to ``tensor`` or
    ``transform``."""
    import paper_2606_21410_b300 as P
    if route32 == "auto":
        return p.autotune(None)
    want = P.ROUTE_TENSOR if route32 == "tensor" else P.ROUTE_TRANSFORM
    for a in range(p.dim):
        try:
            p.set_route32(a, want)
        except P.ChebError:
            pass
    return None


def setup_gpu(levels, contrast, route32="transform"):
    import torch
    import paper_2606_21410_b300 as P
    import workloads as W
    sp = W.sphere_packing(0)
    plans, Ks, bs, hostK, hostb = [], [], [], [], []
    for n in levels:
        p = P.Plan((n, n, n), bc=BC)
        p.chosen_routes = set_routes(p, route32)
        K, faces = host_level(n, sp, contrast, [p.nodes(0), p.nodes(1), p.nodes(2)])
        Kd = torch.from_numpy(K).cuda()
        bd = p.rhs(torch.zeros(p.shape, dtype=torch.float64, device="cuda"),
                   [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in faces])
        plans.append(p)
        Ks.append(Kd)
        bs.append(bd)
        hostK.append(torch.from_numpy(K).pin_memory())
        hostb.append(bd.cpu().pin_memory())
    return plans, Ks, bs, hostK, hostb


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                smax.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# oracle timing (cpu baseline / reference arm)
# ----------------------------------------------------------------------------

def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_levels(levels, contrast):
    """Per-level oracle grids, K and b, each sampled on the oracle's own nodes."""
    import oracle as O
    sp = None
    import workloads as W
    sp = W.sphere_packing(0)
    grids, Ks, bs = [], [], []
    for n in levels:
        g = O.Grid((n,) * 3, bc=BC)
        K, faces = host_level(n, sp, contrast, [g.nodes(0), g.nodes(1), g.nodes(2)])
        grids.append(g)
        Ks.append(K)
        bs.append(O.rhs(np.zeros(g.shape), faces, g))
    return grids, Ks, bs


def oracle_hierarchy(levels, contrast):
    """The FP64 CPU oracle's hierarchical solve of the workload (Alg. 4 with
    barycentric prolongation and preconditioned GMRES, rtol 1e-12), timed on
    the host cores.  Returns (solutions, infos, e_ref, seconds)."""
    import oracle as O
    grids, Ks, bs = oracle_levels(levels, contrast)
    t0 = time.perf_counter()
    us, infos, eref = O.solve_hierarchy(Ks, bs, grids, rtol=1e-12)
    return us, infos, eref, time.perf_counter() - t0


def oracle_sample_text(levels, infos, seconds):
    its = [i["iterations"] for i in infos]
    return (f"the whole workload once, not sampled: the oracle's hierarchical solve "
            f"{'->'.join(f'{n}^3' for n in levels)} (dense Kronecker apply, constant-K "
            f"preconditioner, GMRES(50) to a preconditioned relative residual of 1e-12, "
            f"{its} iterations per level, {seconds:.1f} s)")


def run_reference(args):
    """Reference arm: the FP64 CPU oracle solving the same workload.  One
    oracle solve takes minutes, so the timed region is one complete solve
    (steps = 1); the warm-up steps are bounded samples (one oracle operator
    application plus one preconditioner application at the coarsest level)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    levels = [int(v) for v in args.levels.split(",")]
    import oracle as O
    grids, Ks, bs = oracle_levels(levels[:1], args.contrast)
    M = O.FDMPreconditioner(grids[0], O.geometric_mean(Ks[0]))
    for _ in range(args.warmup):
        M(O.apply(bs[0], Ks[0], grids[0]))
    us, infos, eref, v = oracle_hierarchy(levels, args.contrast)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world,
        "steps": 1, "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(levels, args.contrast),
        "iterations_per_level": [i["iterations"] for i in infos], "e_ref": eref,
        "rel_residual_per_level": [i["rel_residual"] for i in infos],
        "cpu_baseline": {"value": v, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": oracle_sample_text(levels, infos, v)},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": ("one oracle solve takes minutes on the host cores, so the timed region is one "
                 "complete solve (steps = 1) instead of the requested steps"),
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# DRAM traffic of a kernel from a committed ncu summary
# ----------------------------------------------------------------------------

def _sha256(path):
    h = hashlib.sha256()
    with open(path, "rb") as f:
        h.update(f.read())
    return h.hexdigest()


def profile_record(kernel, workload):
    """Counters of `kernel` on `workload` from a ``traffic-record:`` line of a
    summary under profiles/ (one ncu capture: DRAM bytes read + written per
    launch, and for FP64 kernels the executed FP64 flops per launch).  The
    record names the kernel's source files and their SHA-256 at capture time
    ("sources": [{"path", "sha256"}, ...], or one "source" / "source_sha256");
    when any of them has changed since, the counters no longer describe the
    kernel and are reported as null."""
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            if not line.startswith("traffic-record:"):
                continue
            try:
                rec = json.loads(line.split(":", 1)[1])
            except ValueError:
                continue
            if rec.get("kernel") != kernel or rec.get("workload") != workload:
                continue
            srcs = rec.get("sources") or [{"path": rec.get("source"), "sha256": rec.get("source_sha256")}]
            fresh = all(s.get("path") and os.path.exists(os.path.join(ROOT, s["path"])) and
                        _sha256(os.path.join(ROOT, s["path"])) == s.get("sha256") for s in srcs)
            return {"bytes_per_launch": rec.get("dram_bytes_per_launch") if fresh else None,
                    "fp64_flops_per_launch": rec.get("fp64_flops_per_launch") if fresh else None,
                    "summary": os.path.relpath(path, ROOT), "fresh": fresh,
                    "capture": rec.get("capture")}
    return {"bytes_per_launch": None, "fp64_flops_per_launch": None, "summary": None, "fresh": False,
            "capture": None}


def apply_only(args, n):
    """Time cheb_apply alone (profiling helper): u smooth, K the sphere field."""
    import torch
    import paper_2606_21410_b300 as P
    import workloads as W
    bits = args.apply_only or args.fdm_only
    dt = torch.float32 if bits == 32 else torch.float64
    p = P.Plan((n, n, n), bc=BC)
    set_routes(p, args.route32)
    X, Y, Z = p.mesh()
    K = torch.from_numpy(W.two_phase_conductivity(X, Y, Z, W.sphere_packing(0), 1.0,
                                                  args.contrast)).to("cuda", dt)
    u = torch.from_numpy(np.sin(X + 2 * Y) * np.cos(Z)).to("cuda", dt)
    out = torch.empty_like(u)

    def op():
        if args.fdm_only:
            p.precond_apply(u, 1.5, out, matrices=args.pmat)
        else:
            p.apply(K, u, out)
    for _ in range(max(3, args.warmup)):
        op()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        op()
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    wb = 4 if dt == torch.float32 else 8
    rec = {"op": "fdm" if args.fdm_only else "apply", "bits": bits, "n": n, "ms": t * 1e3,
           "gdofs": n ** 3 / t / 1e9}
    if args.fdm_only:
        rec["tflops_12m4"] = 12.0 * (n - 2) ** 4 / t / 1e12
    else:
        rec["gbs_11words"] = 11 * wb * n ** 3 / t / 1e9
    print(json.dumps(rec), flush=True)


def batch_run(steps=1, warmup=1, use_graph=0, batch_mode=1, picard_steps=60, ncu_step=False):
    """The batched configuration: 16 instances, sizes U{33..97} (seed 1),
    K = K0 (1 + 0.5 |grad u|^2) with lognormal K0 (sigma 0.5, correlation 0.2),
    Dirichlet u = x on x = +-1 and z = -1, Neumann 0 elsewhere; relaxed Picard
    (omega 0.5) to a relative change of 1e-9, inner mixed-precision solves; all
    instances concurrently (cheb_picard_batched).  Returns a summary dict."""
    import torch
    import paper_2606_21410_b300 as P
    import workloads as W
    bc = [0, 0, 1, 1, 0, 1]
    sizes = W.batch_sizes(1)
    plans, K0, bs = [], [], []
    for i, n in enumerate(sizes):
        p = P.Plan((n, n, n), bc=bc)
        X, Y, Z = p.mesh()
        K0.append(torch.from_numpy(W.lognormal_conductivity(X, Y, Z, seed=1000 + i)).cuda())
        faces = W.face_values(bc, p.nodes(0), p.nodes(1), p.nodes(2), x_boundary)
        bs.append(p.rhs(torch.zeros(p.shape, dtype=torch.float64, device="cuda"),
                        [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in faces]))
        plans.append(p)
    kw = dict(beta=0.5, tol=1e-9, maxit=picard_steps, omega=0.5, mode=1, rtol=1e-10, use_graph=use_graph,
              batch_mode=batch_mode)
    for _ in range(max(1, warmup)):
        us, infos, its = P.picard_batched(plans, K0, bs, check_status=False, **kw)
    torch.cuda.synchronize()
    if ncu_step:
        torch.cuda.profiler.start()
        P.picard_batched(plans, K0, bs, check_status=False, **kw)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return {"profiled": True}
    l0 = P.lib.cheb_launch_count()
    t0 = time.perf_counter()
    for _ in range(steps):
        us, infos, its = P.picard_batched(plans, K0, bs, check_status=False, **kw)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    dofs = sum(n ** 3 for n in sizes)
    mode_name = {1: "lockstep (batched passes, per-instance mask, step graphs)",
                 2: "concurrent (one solver per instance)"}[batch_mode]
    return {"workload": f"16 uneven lognormal Picard instances, {mode_name}", "sizes": sizes, "dofs": dofs,
            "s_per_batch": dt, "gdofs_solved_per_s": dofs / dt / 1e9, "picard_iters": its,
            "inner_iterations": [i["iterations"] for i in infos],
            "status": [i["status"] for i in infos], "use_graph": use_graph, "batch_mode": batch_mode,
            "graph_captures": infos[0]["graph_captures"],
            "gpu_launches_per_batch": (P.lib.cheb_launch_count() - l0) // steps}


# the paper's Table 1 (Sec. 3.4; Python/scipy, FP64, MacBook Pro M2 CPU):
# N -> (max error against the exact temperature, wall seconds); context only
PAPER_TABLE1 = {4: (7.352339e-2, 0.035), 8: (4.903119e-4, 0.114), 16: (6.270730e-9, 0.873),
                32: (1.272603e-9, 2.008), 64: (8.182031e-10, 47.908), 128: (7.737196e-10, 557.870),
                256: (7.734714e-10, 5245.951)}


def newton_table(Ns=(4, 8, 16, 32, 64, 128, 256), mode=1):
    """The paper's manufactured nonlinear heat problem (Sec. 3.4, Table 1):
    k(T) = 1 / (1 + T/2) on (0,1)^3, T = 2 (exp(Phi/2) - 1), Dirichlet T = 0
    on x = 0 and y = 0, flux data on the other faces; hierarchical Newton
    (prolonged guess per level, cheb_newton_solve).  Per level: Newton steps,
    LGMRES iterations, max error against the exact T, e_ref, and the level's
    wall time (the paper's printed error and M2 time beside it)."""
    import torch
    import paper_2606_21410_b300 as P
    import workloads as W
    alpha = 0.5
    bc = [0, 2, 0, 2, 2, 2]
    sol = lambda X, Y, Z: W.paper_nonlinear_3d(X, Y, Z, alpha)
    rows, prev = [], None
    total = 0.0
    for N in Ns:
        p = P.Plan((N + 1,) * 3, (0, 0, 0), (1, 1, 1), bc)
        X, Y, Z = p.mesh()
        T, _, f = sol(X, Y, Z)
        faces = W.face_values(bc, p.nodes(0), p.nodes(1), p.nodes(2), sol, k_fn=W.reciprocal_conductivity(alpha))
        b = p.rhs(torch.from_numpy(f).cuda(), [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in faces])
        K0 = torch.ones(p.shape, dtype=torch.float64, device="cuda")
        u = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if prev is not None:
            P.prolong(prev[0], p, prev[1], u)
        guess = u.clone() if prev is not None else None
        u, info, its, d = p.newton_solve(K0, b, u, alpha=alpha, tol=1e-13, maxit=30, mode=mode,
                                         inner_rtol=1e-6, check_status=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        total += dt
        err = float(np.abs(u.cpu().numpy() - T).max())
        rows.append({"N": N, "newton_steps": its, "lgmres_iterations": info["iterations"], "max_error": err,
                     "e_ref": P.rel_diff(p, u, guess) if guess is not None else None,
                     "seconds": dt, "status": info["status"],
                     "paper_max_error": PAPER_TABLE1[N][0], "paper_seconds_m2_cpu": PAPER_TABLE1[N][1]})
        prev = (p, u)
    return {"workload": "paper Table 1: nonlinear heat, hierarchical Newton N = 4 .. 256, flux faces",
            "mode": "mixed" if mode == 1 else "fp64", "levels": rows, "total_seconds": total}


def batch_workload(args):
    print(json.dumps(batch_run(args.steps, args.warmup, args.use_graph, args.batch_mode, args.picard_steps,
                               args.ncu_step)), flush=True)


def workload_config(levels, contrast):
    return {"workload": f"two-phase spheres, hierarchical {'->'.join(f'{n}^3' for n in levels)}, "
                        f"K_incl/K_matrix={contrast:g}, mixed FP32/FP64, finest level to rtol 1e-12",
            "levels": levels, "precond": "FDM (constant-K fast diagonalization)",
            "lgmres": "restart 30, augment 3", "l2": "inputs larger than L2 (257^3 FP64 = 136 MB)"}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2606_21410_b300 as P
    lib = P.lib
    levels = [int(v) for v in args.levels.split(",")]
    if args.apply_only or args.fdm_only:
        apply_only(args, levels[-1])
        return
    if args.workload == "batch":
        batch_workload(args)
        return
    if args.workload == "newton":
        print(json.dumps(newton_table()), flush=True)
        return
    plans, Ks, bs, hostK, hostb = setup_gpu(levels, args.contrast, args.route32)
    opts = dict(mode=1, rtol=1e-12, reorth=args.reorth, inner_rtol=args.inner_rtol,
                restart=args.restart, use_graph=args.use_graph, recycle=args.recycle,
                coarse_rtol=args.coarse_rtol, precond_matrices=args.pmat)
    stream = torch.cuda.current_stream()

    def step():
        return P.solve_hierarchy(plans, Ks, bs, **opts)

    for _ in range(max(3, args.warmup)):
        us, infos, eref = step()
    torch.cuda.synchronize()
    if args.ncu_step:
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- timed region
    import ctypes as C
    l0 = lib.cheb_launch_count()
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            us, infos, eref = step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = lib.cheb_launch_count() - l0
    elapsed = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
    per_step = elapsed / args.steps

    # ---- phase split from one more step with the event profiler on (outside
    # the timed region: the events add host work).  GPU time not inside any
    # instrumented phase is idle time (host synchronisation, launch gaps).
    lib.cheb_profile_enable(1)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    step()
    p1.record(stream)
    torch.cuda.synchronize()
    ms = (C.c_double * 8)()
    cnt = (C.c_longlong * 8)()
    lib.cheb_profile_read(ms, cnt)
    lib.cheb_profile_enable(0)
    prof_step_ms = p0.elapsed_time(p1)
    phase = {nm: {"ms": ms[i], "count": cnt[i]} for i, nm in enumerate(
        ["apply64", "apply32", "prec64", "prec32", "orth64", "orth32", "prolong", "other"])}
    phase["idle"] = {"ms": prof_step_ms - sum(ms[i] for i in range(8)), "count": 0}
    phase["profiled_step_ms"] = prof_step_ms

    # ---- apply throughput at the finest level
    pf, nf = plans[-1], levels[-1]
    ntot = nf ** 3

    def time_apply(dtype, reps=20):
        K = Ks[-1].to(dtype)
        u = us[-1].to(dtype)
        out = torch.empty_like(u)
        for _ in range(3):
            pf.apply(K, u, out)
        torch.cuda.synchronize()
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            pf.apply(K, u, out)
        b2.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b2) / 1e3 / reps

    t32 = time_apply(torch.float32)
    t64 = time_apply(torch.float64)
    apply = {"fp32_gdofs": ntot / t32 / 1e9, "fp64_gdofs": ntot / t64 / 1e9,
             "fp32_ms": t32 * 1e3, "fp64_ms": t64 * 1e3}

    # ---- apply at every level with the solve's routes, L2 flushed before each
    # timed apply (65^3 and 129^3 fields fit in the 126 MB L2)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB

    def time_apply_cold(l, dtype, reps=10):
        K = Ks[l].to(dtype)
        u = us[l].to(dtype)
        out = torch.empty_like(u)
        plans[l].apply(K, u, out)
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plans[l].apply(K, u, out)
            b2.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b2) / 1e3
        return tot / reps

    apply_levels = []
    for l, n in enumerate(levels):
        ta32, ta64 = time_apply_cold(l, torch.float32), time_apply_cold(l, torch.float64)
        apply_levels.append({
            "n": n, "fp32_routes": [plans[l].route32(a) for a in range(3)],
            "fp64_routes": [plans[l].route(a) for a in range(3)],
            "fp32_ms": ta32 * 1e3, "fp64_ms": ta64 * 1e3,
            "fp32_gdofs": n ** 3 / ta32 / 1e9, "fp64_gdofs": n ** 3 / ta64 / 1e9,
            "fp32_gbs_3word": 12.0 * n ** 3 / ta32 / 1e9, "fp32_gbs_11word": 44.0 * n ** 3 / ta32 / 1e9,
            "fp64_gbs_3word": 24.0 * n ** 3 / ta64 / 1e9})
    del flush

    # ---- measured FMA peaks of the CUDA cores, clocks sampled meanwhile
    fma = {}
    with ClockSampler(local) as clk_fma:
        for nm, prec in (("fp64", P.FP64), ("fp32", P.FP32)):
            tf, msl = C.c_double(), C.c_double()
            P.check(lib.cheb_fma_peak(prec, C.byref(tf), C.byref(msl)), "cheb_fma_peak")
            fma[nm + "_tflops"] = tf.value
    fma["clocks"] = clk_fma.summary()
    # FP64 apply (transform route, FP64-pipe bound) against the FP64 peak:
    # executed FP64 flops per launch from one ncu capture of the kernel
    rec64 = profile_record("tf_pass_kernel<double>", f"fp64 apply {nf}^3")
    fl64 = rec64["fp64_flops_per_launch"]
    fp64_roof = {"bound": "alu", "kernel": f"tf_pass_kernel<double> ({pf.dim} launches per apply)",
                 "unit": "TFLOP/s", "peak": fma["fp64_tflops"],
                 "peak_source": "measured FP64 FMA throughput (cheb_fma_peak, this run)",
                 "achieved": (fl64 * pf.dim / t64 / 1e12) if fl64 else None,
                 "frac": (fl64 * pf.dim / t64 / 1e12 / fma["fp64_tflops"]) if fl64 else None,
                 "flops_source": rec64["summary"], "flops_fresh": rec64["fresh"],
                 "dram_bytes_per_launch": rec64["bytes_per_launch"],
                 "apply_ms": t64 * 1e3}

    # ---- plain FP64 comparison solve
    fp64 = None
    if not args.no_fp64:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u64, infos64, _ = P.solve_hierarchy(plans, Ks, bs, mode=0, rtol=1e-12, check_status=False,
                                            restart=args.restart, coarse_rtol=args.coarse_rtol)
        torch.cuda.synchronize()
        fp64 = {"time_to_solve_s": time.perf_counter() - t0,
                "iterations": [i["iterations"] for i in infos64],
                "status": [i["status"] for i in infos64],
                "rel_diff_mixed_vs_fp64": P.rel_diff(pf, u64[-1], us[-1])}

    # ---- end to end through the public API with host buffers
    torch.cuda.synchronize()
    out_host = torch.empty(plans[-1].shape, dtype=torch.float64).pin_memory()
    t0 = time.perf_counter()
    Kd2 = [k.to("cuda", non_blocking=True) for k in hostK]
    bd2 = [b.to("cuda", non_blocking=True) for b in hostb]
    ue, _, _ = P.solve_hierarchy(plans, Kd2, bd2, **opts)
    out_host.copy_(ue[-1], non_blocking=True)
    torch.cuda.synchronize()
    e2e_t = max_over_ranks(time.perf_counter() - t0, world)
    h2d = sum(k.numel() * 8 + b.numel() * 8 for k, b in zip(hostK, hostb))
    d2h = out_host.numel() * 8

    # ---- the batched configuration (secondary keys of the line)
    batch = None
    if not args.no_batch:
        batch = batch_run(steps=1, warmup=1, batch_mode=1)
        batch_c = batch_run(steps=1, warmup=1, batch_mode=2)
        batch["concurrent_s_per_batch"] = batch_c["s_per_batch"]
        batch["concurrent_gpu_launches_per_batch"] = batch_c["gpu_launches_per_batch"]
        # batch_mode AUTO picks lockstep for >= 32 instances or <= 200k points each
        mean = batch["dofs"] / len(batch["sizes"])
        batch["auto_mode"] = "lockstep" if len(batch["sizes"]) >= 32 or mean <= 2e5 else "concurrent"
    newton = None
    if not args.no_newton:
        newton_table(Ns=(4, 8, 16))            # warm-up of the level plans' kernels
        newton = newton_table()

    # ---- finest-level timing of the preconditioner (the dominant phase)
    def time_prec(dtype, matrices, reps=10):
        r = bs[-1].to(dtype)
        out = torch.empty_like(r)
        kref = float(infos[-1]["kref"])
        for _ in range(3):
            pf.precond_apply(r, kref, out, matrices=matrices)
        torch.cuda.synchronize()
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            pf.precond_apply(r, kref, out, matrices=matrices)
        b2.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b2) / 1e3 / reps

    tp32 = time_prec(torch.float32, args.pmat)
    apply["fdm_fp32_ms"] = tp32 * 1e3
    apply["fdm_fp32_ms_fp32_matrices"] = time_prec(torch.float32, 1) * 1e3
    apply["fdm_fp32_ms_tf32_matrices"] = time_prec(torch.float32, 0) * 1e3

    # ---- roofline of the dominant kernel: the FP32 operator apply (the
    # largest single-kernel share of the solve; the Arnoldi dot/axpy work is
    # split over two kernels).  Unit: one apply at the finest level, timed with
    # CUDA events on the plan stream around 20 applies right after the timed
    # region (the level-mixed per-apply time inside the timed solve, from the
    # phase profiler, is reported beside it).  Algorithmic bytes per apply,
    # the floor of the operator: read u, read K, write Au = 3 FP32 words per
    # DOF; the three-pass schedule (x pass reads u, K and writes the output,
    # the y and z passes also read the accumulated output) moves 11 words.
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6400.0)
    bf16 = peaks.get("bf16_tflops", 1800.0)
    tensor_route = all(pf.route32(a) == P.ROUTE_TENSOR for a in range(pf.dim))
    launches_per_apply = 2 * pf.dim if tensor_route else pf.dim
    kernel = "dense_pass_kernel" if tensor_route else "tf_pass_kernel<float>"
    floor_bytes = 3 * 4 * ntot
    achieved = floor_bytes / t32 / 1e9
    tr = profile_record(kernel, f"fp32 apply {nf}^3")
    traffic = tr["bytes_per_launch"]
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic,
            "kernel": (f"{kernel} ({launches_per_apply} launches per apply; "
                       + ("tcgen05 split-TF32 dense derivative)" if tensor_route else "FFT transform route)")),
            "unit_of_work": f"one FP32 operator apply at {nf}^3 ({ntot} DOF)",
            "algorithmic_bytes_per_apply": floor_bytes,
            "algorithmic_bytes_per_launch": floor_bytes / launches_per_apply,
            "achieved_11word_model_gbs": 11 * 4 * ntot / t32 / 1e9,
            "frac_11word_model": 11 * 4 * ntot / t32 / 1e9 / hbm,
            "dram_gbs": (traffic * launches_per_apply / t32 / 1e9) if traffic else None,
            "traffic_source": tr["summary"], "traffic_capture": tr["capture"],
            "traffic_fresh": tr["fresh"],
            "peak_source": ("measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks
                            else "fallback 6400 GB/s"),
            "apply_ms_finest": t32 * 1e3,
            "apply_ms_timed_solve_all_levels": (phase["apply32"]["ms"] / phase["apply32"]["count"])
            if phase["apply32"]["count"] else None}
    if tensor_route:
        flops = 2.0 * ntot * nf * 2 * pf.dim  # dense-D products of one apply (2 per axis)
        roof["tensor_tflops_dense_d"] = flops / t32 / 1e12
        roof["tensor_frac_split_tf32"] = 3.0 * flops / t32 / 1e12 / (bf16 * 1.1 / 2.25)
    # preconditioner contractions beside it (tcgen05, tensor bound)
    m = nf - 2
    fl = 12.0 * m ** 4
    tf32_peak = bf16 * (1.1 / 2.25)
    prec_roof = {"bound": "tensor", "kernel": "umma_tf32x3_rot_kernel (FDM contractions, 6 per application)",
                 "achieved": fl / tp32 / 1e12, "peak": tf32_peak, "unit": "TFLOP/s",
                 "frac": fl / tp32 / 1e12 / tf32_peak,
                 "peak_source": "measured bf16 burst x 1.1/2.25 (nominal TF32/BF16 ratio)",
                 "note": "whole preconditioner time; the contractions issue %d TF32 MMAs per useful flop "
                         "(%s matrices)" % (2 if args.pmat == 0 else 3, "TF32" if args.pmat == 0 else "FP32")}

    # ---- the oracle's hierarchical solve on the host cores: CPU baseline and
    # the relative L2 error of the GPU solutions at every level
    cpu, parity = None, None
    if rank == 0 and not args.no_cpu:
        uo, io, eref_o, t_or = oracle_hierarchy(levels, args.contrast)
        us_h = [u.cpu().numpy() for u in us]
        parity = {"rel_err_vs_oracle_mixed": [float(np.linalg.norm(a - b) / np.linalg.norm(b))
                                               for a, b in zip(us_h, uo)],
                  "oracle_iterations": [i["iterations"] for i in io],
                  "oracle_rel_residual": [i["rel_residual"] for i in io],
                  "oracle_e_ref": eref_o}
        if fp64 is not None:
            u64h = [u.cpu().numpy() for u in u64]
            parity["rel_err_vs_oracle_fp64"] = [float(np.linalg.norm(a - b) / np.linalg.norm(b))
                                                for a, b in zip(u64h, uo)]
        cpu = {"value": t_or, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
               "sample": oracle_sample_text(levels, io, t_or)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": per_step, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": per_step * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
            "config": dict(workload_config(levels, args.contrast),
                           coarse_levels_rtol=args.coarse_rtol or 1e-12, recycle=args.recycle,
                           inner_rtol=args.inner_rtol,
                           precond_matrices="tf32" if args.pmat == 0 else "fp32"),
            "solves_per_s": world * args.steps / elapsed,
            "iterations_per_level": [i["iterations"] for i in infos],
            "seconds_per_level": [i["seconds"] for i in infos],
            "refinements_per_level": [i["refinements"] for i in infos],
            "rel_residual": infos[-1]["rel_residual"], "e_ref": eref,
            "apply": apply, "apply_levels": apply_levels, "fp64": fp64, "phase_ms_per_step": phase,
            "routes_per_level": [p.chosen_routes for p in plans],
            "roofline": roof, "prec_roofline": prec_roof, "fp64_apply_roofline": fp64_roof,
            "fma_peaks": fma, "batch": batch, "newton_table1": newton,
            "fp32_routes_finest": [pf.route32(a) for a in range(pf.dim)],
            "rel_err_vs_oracle": parity["rel_err_vs_oracle_mixed"][-1] if parity else None,
            "oracle_parity": parity,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_t, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
