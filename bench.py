#!/usr/bin/env python
"""Benchmark: OSRC-preconditioned PMCHWT solves/s on one GB300.

Workload (one step = one solve): unit sphere, level-5 icosphere (10242
vertices, 20480 flat triangles), k_ext = 20, k_int = 26, rho_int/rho_ext =
1.5, unit plane wave along +z (other directions on other ranks), P1 Galerkin,
FP32 matrix-free far field + FP64 Sauter-Schwab near-field CSR, OSRC with
N_Pade = 4 and theta = pi/3 (interior wavenumber), GMRES without restart to a
preconditioned relative residual of 1e-5.  The right-hand side is resident
in HBM when the timed region starts; the problem set-up (near field, mass and
stiffness matrices, Pade constants) is resident state built before it.  L2
is flushed (a 512 MiB buffer is written) before every timed solve.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded row sample of the same workload instead.
"""
from __future__ import annotations

import argparse
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

WORKLOAD = "sphere10242"
METRIC = "OSRC-PMCHWT solves/s to 1e-5 residual"
UNIT = "solves/s"
TOL = 1e-5
# FP32 flops (FMA = 2) of one far-field point pair, both wavenumbers, as the
# factored evaluation of the far kernel performs it: 32 FMA, 14 MUL, 5 ADD
# (distance, 1/r and 1/r^2, (y - x).n_x, k r for both k, cos and sin of both
# phases scaled by 1/r, then the V, D-normal (scale k0^2 taken out per source
# triangle), D-curl, H and T/K accumulations); 5 MUFU operations (1 rsqrt,
# 2 sin, 2 cos) and their argument scaling come on top and are not counted.
FLOPS_PER_PAIR = 83
# nominal count for a per-operator evaluation (V, K, T, D separately per
# wavenumber), reported beside the main figure
FLOPS_PER_PAIR_NOMINAL = 176
# executed FP32 flops per far point pair of the several-right-hand-side far
# kernel: shared per pair (distance, 1/r, 1/r^2, (y - x).n_x, k r, scaled cos
# and sin, the V / D-normal / D-curl / H combinations with the K and D-normal
# triangle factors folded in, and negated imaginary parts: 16 FMA, 22 MUL,
# 5 ADD), plus per right-hand side the four complex multiply-adds into u1, u2
# (16 FMA)
FLOPS_PER_PAIR_MULTI_SHARED = 59
FLOPS_PER_PAIR_MULTI_RHS = 32
# GMRES iterations of this workload (measured on the GPU path; the oracle's
# unrestarted GMRES needs the same count within +-2 at smaller sizes): used
# to turn the oracle's sampled matvec rate into solves/s
REF_ITERATIONS = 47
# DRAM bytes (read + write) of one far_kernel<0, 0, 0> launch at this
# workload, from one ncu capture of this command (dram__bytes_read.sum
# 15,393,536 + dram__bytes_write.sum 2,816, the ncu summary of the far kernel
# kept with the profiles); to be retaken whenever the far kernel changes
FAR_TRAFFIC_BYTES = 15396352


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--serve-route", default="both", choices=["both", "matrix_free", "hybrid"],
                    help="serving legs to run")
    ap.add_argument("--serve-deadline", type=float, default=None, metavar="S",
                    help="stop the serving leg S seconds after its first submission (unfinished "
                         "requests are reported as such)")
    ap.add_argument("--serve-progress", default=None, metavar="FILE",
                    help="append one JSON line per finished request to FILE")
    ap.add_argument("--serve-requests", type=int, default=2,
                    help="requests of the seeded Poisson stream in the serving legs, at their stated "
                         "sizes (0: skip; 50 for the full measurement, about 20 minutes)")
    ap.add_argument("--dense-rhs", type=int, default=128,
                    help="right-hand sides of the batched dense leg (ellipsoid8000; 0: skip)")
    ap.add_argument("--dense-matfree-rhs", type=int, default=1,
                    help="right-hand sides of the same workload solved matrix-free for comparison")
    ap.add_argument("--multi-rhs", default="8,16",
                    help="right-hand-side counts of the lockstep (several right-hand sides per "
                         "far-field launch) leg on the headline mesh ('' to skip)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the far-field apply on the 80000-vertex bumpy ellipsoid")
    ap.add_argument("--no-objects", action="store_true",
                    help="skip the four-sphere multiple-scattering solve")
    ap.add_argument("--profile-case", choices=["far-small", "far-multi-small", "precond-small", "dense-short",
                                               "dense-small", "gemm"],
                    help="instead of the benchmark: run one small case for profiler captures "
                         "(far-small: far-field applies on a 2562-vertex sphere, plain then "
                         "large-ka; far-multi-small: the same with 8 right-hand sides per apply; "
                         "precond-small: five OSRC preconditioner applies on it; "
                         "dense-short: ellipsoid8000, 128 right-hand sides, one "
                         "refinement of 120 inner iterations; dense-small: the same on a "
                         "3000-vertex ellipsoid, 24 inner iterations; gemm: three tensor-core "
                         "GEMMs at M 16000, N 256, K 32000)")
    ap.add_argument("--sponge-sweep", action="store_true",
                    help="instead of the benchmark: GMRES iterations of the four formulations on "
                         "the level-2 Menger sponge at 0.5 and 1 MHz")
    ap.add_argument("--precond-sweep", action="store_true",
                    help="instead of the benchmark: GMRES iterations vs frequency on the "
                         "10242-vertex sphere for the OSRC, mass-only and Calderon preconditioners")
    ap.add_argument("--large-ks", default="15,30,45,60", help="k_ext values of --large-sweep")
    ap.add_argument("--large-maxit", type=int, default=600, help="GMRES cap of --large-sweep")
    ap.add_argument("--large-sweep", type=int, default=0, metavar="NV",
                    help="instead of the benchmark: GMRES iterations vs ka on the bumpy "
                         "ellipsoid with NV vertices, k_ext in {15, 30, 45, 60}")
    return ap.parse_args()


# --------------------------------------------------------------------------
# distributed plumbing (one process per GPU; no data-path collective)
# --------------------------------------------------------------------------
class Dist:
    def __init__(self, want_cuda=True):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist

            backend = "nccl" if (want_cuda and torch.cuda.is_available()) else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, v):
        if self.pg is None:
            return v
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v):
        if self.pg is None:
            return v
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpus):
        self.gpus = gpus
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            out = self.parse(f, self.gpus)
        os.unlink(self.path)
        return out

    @staticmethod
    def parse(lines, gpus):
        """Median and maximum SM clock and the throttle reasons seen, from
        nvidia-smi CSV lines of QUERY (no header, no units) for the GPUs in
        gpus; lines of other GPUs and unreadable lines are skipped."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                idx = int(parts[0])
            except ValueError:
                continue
            if idx not in gpus:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                pass
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            return None
    return None


def run_ours(args, D):
    import numpy as np
    import torch

    import __graft_entry__

    if D.rank == 0 or D.world == 1:
        __graft_entry__.build()
    D.barrier()
    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import plane_wave_dirs, workload

    torch.cuda.set_device(D.local)
    dev = torch.device("cuda", D.local)
    W = workload(WORKLOAD)
    t_setup = time.perf_counter()
    S = B.Solver(W["verts"], W["tris"], W["k_ext"], W["k_int"], W["rho_ratio"], device=D.local)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    d = np.array([[0.0, 0.0, 1.0]]) if D.rank == 0 else plane_wave_dirs(1, seed=100 + D.rank)
    b = S.rhs_planewave(d)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        x, info = S.solve(b, tol=TOL, maxit=1000)
    torch.cuda.synchronize()

    B.osrc_profile_enable(S.pb, True)
    launches0 = S.launches()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(list(range(max(1, D.world))) if D.rank == 0 else [])
    D.barrier()
    torch.cuda.synchronize()
    if D.rank == 0:
        clocks.start()
    infos = []
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        x, info = S.solve(b, tol=TOL, maxit=1000)
        evs[k][1].record(stream)
        infos.append(info.as_dict())
    torch.cuda.synchronize()
    D.barrier()
    clk = clocks.stop() if D.rank == 0 else None
    launches = S.launches() - launches0
    far_n, far_ms = B.osrc_far_kernel_stats(S.pb)
    B.osrc_profile_enable(S.pb, False)
    step_ms = [a.elapsed_time(e) for a, e in evs]
    total_ms = D.max(sum(step_ms))
    solves = D.sum(args.steps)
    value = solves / (total_ms / 1000.0)

    # end to end through the C ABI with host buffers (pinned), copies inside
    n2 = 2 * S.nv
    hb = torch.empty((1, n2), dtype=torch.complex128, pin_memory=True)
    hb.copy_(b.cpu())
    hx = torch.empty((1, n2), dtype=torch.complex128, pin_memory=True)
    hbn, hxn = hb.numpy(), hx.numpy()
    B.osrc_gmres_solve(S.pb, hbn, hxn, 1, TOL, 1000, host_buffers=True)
    D.barrier()
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.osrc_gmres_solve(S.pb, hbn, hxn, 1, TOL, 1000, host_buffers=True)
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = D.max(sum(e2e_t))
    e2e_value = solves / e2e_total
    sol_diff = float(np.linalg.norm(hxn.ravel() - x.cpu().numpy().ravel()) /
                     np.linalg.norm(x.cpu().numpy().ravel()))

    field = run_field(S, x, W, B) if D.world == 1 else None
    # accuracy of the timed solve: error against the Mie series of the
    # penetrable sphere (the workload is the unit sphere), and the weak
    # residual b - B x kept for the oracle's row check in the CPU leg
    xs = x.cpu().numpy().ravel()
    bs = b.cpu().numpy().ravel()
    r_gpu = bs - S.apply(x).cpu().numpy().ravel()
    accuracy = solution_error_vs_mie(W, xs, d[0]) if D.rank == 0 else None
    # the same solve run until the true weak residual is also below TOL: GMRES
    # to a tighter preconditioned residual, scaled from the timed solve's ratio
    tight = None
    if D.world == 1:
        ratio = max(1.0, infos[-1]["true_residual"] / max(infos[-1]["precond_residual"], 1e-300))
        tol2 = max(1e-10, 0.5 * TOL / ratio)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x2, info2 = S.solve(b, tol=tol2, maxit=1000)
        e1.record(stream)
        torch.cuda.synchronize()
        tight = {"precond_tol": tol2, "iterations": info2.iterations,
                 "precond_residual": info2.precond_residual, "true_residual": info2.true_residual,
                 "solve_ms": e0.elapsed_time(e1),
                 "solves_per_s": 1000.0 / e0.elapsed_time(e1),
                 "solution_error_vs_mie": solution_error_vs_mie(W, x2.cpu().numpy().ravel(), d[0])}
        del x2
    # measured FP32 throughput of this GPU (denominator beside the derived one)
    fclk = ClockSampler(list(range(max(1, D.world))) if D.rank == 0 else [])
    fclk.start()
    ffma_tf, ffma2_tf = B.osrc_fp32_peak(5)
    fclk_res = fclk.stop()
    far_pairs = B.osrc_far_pairs(S.pb)
    far_avg_ms = far_ms / max(far_n, 1)
    achieved = FLOPS_PER_PAIR * far_pairs / (far_avg_ms * 1e-3) / 1e12
    props = torch.cuda.get_device_properties(dev)
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    mean_info = {k: infos[-1][k] for k in ("iterations", "precond_residual", "true_residual",
                                           "inner_iterations_max")}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": D.world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": "sphere10242: unit sphere, level-5 icosphere, 10242 vertices / 20480 "
                        "triangles, k_ext 20, k_int 26, rho ratio 1.5, plane wave +z",
            "path": "FP32 matrix-free far field + FP64 Sauter-Schwab near CSR (n_ss 4), "
                    "FP64 CG mass solve and batched COCG OSRC (N_Pade 4, theta pi/3, tol 1e-10), "
                    "FP64 CGS2 GMRES without restart",
            "tol": TOL, "rhs_per_rank": 1, "l2": "flushed (512 MiB write) before every step",
            "setup_s": round(t_setup, 3), "parallelism": f"replicas x{D.world}",
            **mean_info,
            "residual_reading": "tol 1e-5 applies to the preconditioned relative residual "
                                "|P M^-1 (b - B x)| / |P M^-1 b| (GMRES convention); the true weak "
                                "residual |b - B x| / |b| is reported beside it, and "
                                "true_residual_1e-5 gives the same solve run until that one is "
                                "below 1e-5 too",
            "solution_error_vs_mie": accuracy,
            "true_residual_1e-5": tight,
        },
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n2 * 16,
                "d2h_bytes_per_step": n2 * 16, "solution_rel_diff_vs_device_run": sol_diff},
        "gpu_launches": int(launches),
        "roofline": {
            "bound": "alu", "kernel": "far_kernel",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": FAR_TRAFFIC_BYTES, "traffic_unit": "bytes per launch (ncu)",
            "flops_per_unit": FLOPS_PER_PAIR, "units_per_launch": far_pairs,
            "unit_def": "far point pair (test point, source point of triangles sharing no "
                        "vertex), both wavenumbers",
            "achieved_nominal_176": FLOPS_PER_PAIR_NOMINAL * far_pairs / (far_avg_ms * 1e-3) / 1e12,
            "avg_launch_ms": far_avg_ms, "launches_timed": far_n,
            "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x "
                          f"{sm_max:.0f} MHz (derived; no FP32 entry in MEASURED_PEAKS.json)",
            "peak_measured_ffma": ffma_tf, "peak_measured_ffma2": ffma2_tf,
            "peak_measured_sm_mhz": fclk_res.get("sm_mhz"),
            "frac_of_measured_ffma": achieved / ffma_tf,
            "peak_measured_basis": "osrc_fp32_peak: independent FFMA (FP32x2 FMA) chains, "
                                   "2048 threads per SM, no memory traffic, best of 5 launches, "
                                   "SM clock sampled while it ran",
        },
    }
    if field is not None:
        out["field"] = field
    peaks = measured_peaks()
    if peaks is not None:
        out["measured_peaks_file"] = True
    S.close()
    # single-GPU legs: only when one GPU runs the bench (a multi-GPU run
    # measures the replicated headline solve and holds the other GPUs for it only)
    single = D.world == 1
    if single:
        out["small_dense"] = run_small_dense(D.local)
    if args.multi_rhs and single:
        out["multi_rhs"] = run_multi(args.multi_rhs, D.local, value)
    if args.dense_rhs > 0 and single:
        out["dense_batched"] = run_dense(args.dense_rhs, args.dense_matfree_rhs, D.local)
    if not args.no_large and single:
        out["large"] = run_large(D.local)
    if not args.no_objects and single:
        out["four_spheres"] = run_four_spheres(D.local)
    if args.serve_requests > 0 and single:
        if args.serve_route in ("both", "matrix_free"):
            out["serving"] = run_serving(args.serve_requests, D.local, progress=args.serve_progress,
                                         deadline=args.serve_deadline)
        if args.serve_route in ("both", "hybrid"):
            out["serving_batched"] = run_serving(args.serve_requests, D.local, route="hybrid",
                                                 progress=args.serve_progress, deadline=args.serve_deadline)
    out["_solution"] = (xs, bs, r_gpu) if D.rank == 0 else None
    return out, (infos[-1]["iterations"] if infos else REF_ITERATIONS)


# --------------------------------------------------------------------------
# several right-hand sides, matrix-free: GMRES in lockstep, one far-field
# launch per iteration for up to 8 right-hand sides
# --------------------------------------------------------------------------
def run_multi(spec, device, single_value):
    import numpy as np
    import torch

    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import plane_wave_dirs, workload

    dev = torch.device("cuda", device)
    W = workload(WORKLOAD)
    S = B.Solver(W["verts"], W["tris"], W["k_ext"], W["k_int"], W["rho_ratio"], device=device)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    res = []
    try:
        for R in [int(v) for v in str(spec).split(",") if v.strip()]:
            dirs = np.vstack([[0.0, 0.0, 1.0], plane_wave_dirs(R - 1, seed=21)]) if R > 1 else \
                np.array([[0.0, 0.0, 1.0]])
            b = S.rhs_planewave(dirs)
            S.solve(b, tol=TOL, maxit=1000)                      # warm-up (workspaces)
            B.osrc_profile_enable(S.pb, True)
            l0 = S.launches()
            flush.zero_()
            clk = ClockSampler([0])
            clk.start()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, info = S.solve(b, tol=TOL, maxit=1000)
            e1.record(stream)
            torch.cuda.synchronize()
            c = clk.stop()
            ms = e0.elapsed_time(e1)
            n_l, far_ms = B.osrc_far_kernel_stats(S.pb)
            n_rhs = B.osrc_far_kernel_rhs(S.pb)
            B.osrc_profile_enable(S.pb, False)
            pairs = B.osrc_far_pairs(S.pb)
            flops = (FLOPS_PER_PAIR_MULTI_SHARED * n_l + FLOPS_PER_PAIR_MULTI_RHS * n_rhs) * pairs
            achieved = flops / (far_ms * 1e-3) / 1e12
            peak = 152 * 128 * 2 * (c.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
            # the same right-hand sides one at a time would take R / single_value s
            res.append({
                "right_hand_sides": R, "solves_per_s": R / (ms * 1e-3), "solve_ms": ms,
                "speedup_vs_one_at_a_time": (R / (ms * 1e-3)) / single_value,
                "iterations_sum": info.total_iterations, "iterations_last": info.iterations,
                "precond_residual_last": info.precond_residual,
                "true_residual_last": info.true_residual, "converged": bool(info.converged),
                "gpu_launches": int(S.launches() - l0),
                "far_kernel": {"launches": n_l, "rhs_processed": n_rhs, "total_ms": far_ms,
                               "share_of_solve": far_ms / ms,
                               "ms_per_rhs_apply": far_ms / max(n_rhs, 1),
                               "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                               "frac": achieved / peak, "bound": "alu",
                               "flops_per_unit": f"{FLOPS_PER_PAIR_MULTI_SHARED} per launch + "
                                                 f"{FLOPS_PER_PAIR_MULTI_RHS} per right-hand side",
                               "units_per_launch": pairs},
                "clocks": c,
            })
            del x, b
    finally:
        S.close()
    return {"workload": "sphere10242 (the headline mesh and physics), R plane waves: +z and seeded "
                        "directions", "path": "GMRES in lockstep over the right-hand sides; far field "
                        "of up to 8 right-hand sides per launch sharing each point pair's geometry "
                        "and sine / cosine", "tol": TOL, "l2": "flushed before the timed solve",
            "runs": res}


# --------------------------------------------------------------------------
# batched dense leg: blocks of right-hand sides on the tensor cores
# --------------------------------------------------------------------------
DENSE_WORKLOAD = "ellipsoid8000"
DENSE_TOL = 1e-6
FALLBACK_BF16_TFLOPS = 1900.0


def run_dense(nrhs, n_matfree, device):
    """Ellipsoid (1, 0.7, 0.5), 8000 vertices / 15996 triangles, k_ext 15,
    k_int 36, rho ratio 1.9, nrhs plane waves (seeded directions): FP64 dense
    assembly, explicit BF16 preconditioner matrix, batched solve (BF16
    tensor-core far field + exact near field, FP32 inner GMRES, outer
    refinement to 1e-6).  The same right-hand sides, first n_matfree of them,
    are also solved one at a time by the FP32 matrix-free path to the same
    true residual for comparison."""
    import numpy as np
    import torch

    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import workload

    dev = torch.device("cuda", device)
    W = workload(DENSE_WORKLOAD)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = B.Solver(W["verts"], W["tris"], W["k_ext"], W["k_int"], W["rho_ratio"], device=device,
                 precision=B.OSRC_FP64_DENSE, dense_assembly=B.OSRC_ASSEMBLE_FF)
    torch.cuda.synchronize()
    t_assembly = time.perf_counter() - t0
    out = {}
    try:
        b = S.rhs_planewave(W["dirs"][:nrhs])
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.osrc_dense_precond_build(S.pb, tol=1e-3, maxit=500)
        torch.cuda.synchronize()
        t_pbuild = time.perf_counter() - t0
        kw = dict(tol=DENSE_TOL, max_refine=10, inner_tol=1e-3, inner_maxit=400)
        B.osrc_dense_batched_solve(S.pb, b, x, **kw)           # warm-up (workspace, clocks)
        flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = B.osrc_dense_batched_solve(S.pb, b, x, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        t_solve = e0.elapsed_time(e1) / 1000.0
        launches = S.launches()
        # one FP64 GEMV of the assembled system (single right-hand side)
        xv = b[0:1].contiguous()
        S.apply(xv)
        e0.record(stream)
        for _ in range(5):
            S.apply(xv)
        e1.record(stream)
        torch.cuda.synchronize()
        gemv_ms = e0.elapsed_time(e1) / 5
        # tensor-core GEMM of the inner products at this shape, timed alone
        Mp, Kp, N = (S.nv * 2 + 127) // 128 * 128, (4 * S.nv + 63) // 64 * 64, 2 * ((nrhs + 7) // 8 * 8)
        gA = torch.randn(Mp, Kp, device=dev).to(torch.bfloat16)
        gB = torch.randn(N, Kp, device=dev).to(torch.bfloat16)
        gC = torch.empty(Mp, N, device=dev, dtype=torch.float32)
        gE = torch.zeros(1, device=dev, dtype=torch.int32)
        gW = torch.empty(max(B.osrc_gemm_bf16_ws_bytes(Mp, N, Kp), 16), dtype=torch.uint8, device=dev)
        for _ in range(3):
            B.osrc_gemm_bf16(gA, gB, gC, gE, ws=gW)
        reps = 20
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(reps):
            B.osrc_gemm_bf16(gA, gB, gC, gE, ws=gW)
        g1.record(stream)
        torch.cuda.synchronize()
        gemm_ms = g0.elapsed_time(g1) / reps
        gemm_tf = 2.0 * Mp * N * Kp / (gemm_ms * 1e-3) / 1e12
        peaks = measured_peaks() or {}
        hbm_peak = peaks.get("hbm_gbs") or 6800.0
        peak = peaks.get("bf16_tflops")
        basis = "measured burst (MEASURED_PEAKS.json)"
        if not peak:
            peak, basis = FALLBACK_BF16_TFLOPS, "fallback 1.9 PFLOP/s burst (no MEASURED_PEAKS.json)"
        del gA, gB, gC, gW
        out = {
            "workload": f"{DENSE_WORKLOAD}: ellipsoid (1, 0.7, 0.5), {S.nv} vertices, k_ext "
                        f"{W['k_ext']:g}, k_int {W['k_int']:g}, rho ratio {W['rho_ratio']:g}, "
                        f"{nrhs} plane waves (seed 1)",
            "path": "dense assembly in float-float (FP64 storage); explicit BF16 P M^-1 matrix; "
                    "inner GMRES (FP32, CGS) on "
                    "BF16 tcgen05 far field + exact near field; float-float outer residual",
            "tol": DENSE_TOL, "right_hand_sides": nrhs,
            "solves_per_s": nrhs / t_solve,
            "solves_per_s_incl_setup": nrhs / (t_solve + t_assembly + t_pbuild),
            "solve_s": t_solve, "assembly_s": t_assembly, "precond_build_s": t_pbuild,
            "fp64_gemv_ms": gemv_ms,
            "refinements": info["refinements"], "inner_iterations": info["inner_iterations"],
            "residual": info["residual"], "gpu_launches": int(launches),
            "gemm": {"bound": "tensor", "M": Mp, "N": N, "K": Kp, "avg_ms": gemm_ms,
                     "achieved": gemm_tf, "peak": peak, "unit": "TFLOP/s", "frac": gemm_tf / peak,
                     "peak_basis": basis,
                     # 2 N flops per byte of A (BF16) is below the ridge of this part (bf16 peak
                     # / HBM bandwidth, about 280): the product is bound by streaming A
                     "hbm_view": {"bound": "hbm", "a_bytes": Mp * Kp * 2,
                                  "achieved_gbs": Mp * Kp * 2 / (gemm_ms * 1e-3) / 1e9,
                                  "peak_gbs": hbm_peak,
                                  "frac": Mp * Kp * 2 / (gemm_ms * 1e-3) / 1e9 / hbm_peak,
                                  "flops_per_a_byte": N, "ridge": peak / hbm_peak * 1e3}},
        }
        # the FP32 matrix-free path on the same right-hand sides, one at a time
        if n_matfree > 0:
            S.close()
            S = B.Solver(W["verts"], W["tris"], W["k_ext"], W["k_int"], W["rho_ratio"], device=device)
            t_mf, its, rel, tres = 0.0, [], [], []
            for r in range(n_matfree):
                br = b[r:r + 1].contiguous()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                xr, inf = S.solve(br, tol=DENSE_TOL, maxit=1000)
                torch.cuda.synchronize()
                t_mf += time.perf_counter() - t0
                its.append(inf.iterations)
                tres.append(inf.true_residual)
                rel.append(float(torch.linalg.norm(xr - x[r:r + 1]) / torch.linalg.norm(x[r:r + 1])))
            out["matrix_free"] = {
                "right_hand_sides": n_matfree, "solves_per_s": n_matfree / t_mf,
                "iterations": its, "tol": DENSE_TOL, "true_residual": max(tres),
                "solution_rel_diff_vs_batched": max(rel),
                "note": "FP32 matrix-free GMRES, preconditioned residual 1e-6; the batched "
                        "path's tolerance is on the true residual",
            }
            out["speedup_vs_matrix_free"] = out["solves_per_s"] / out["matrix_free"]["solves_per_s"]
    finally:
        S.close()
    return out


# --------------------------------------------------------------------------
# field on the paper's grid (Sec. 3.2): 101 x 101 points on a square of 6 radii
# in the plane z = 0, error of the amplitude against the Mie series
# --------------------------------------------------------------------------
def mie_total_field(k0, k1, rho, a, pts):
    """Total field of the penetrable sphere (radius a, rho = rho_int/rho_ext)
    for the plane wave exp(i k0 z), by the Mie series."""
    import numpy as np
    from scipy.special import eval_legendre, spherical_jn, spherical_yn

    r = np.linalg.norm(pts, axis=1)
    cth = np.where(r > 0, pts[:, 2] / np.where(r > 0, r, 1.0), 1.0)
    L = int(max(k0, k1) * max(a, r.max()) + 4 * (k1 * a) ** (1 / 3) + 20)
    out = r > a
    ro, ri = np.where(out, r, a), np.where(out, a, r)
    u = np.zeros(len(r), dtype=complex)
    for l in range(L):
        j0, j0p = spherical_jn(l, k0 * a), spherical_jn(l, k0 * a, True)
        h0 = j0 + 1j * spherical_yn(l, k0 * a)
        h0p = j0p + 1j * spherical_yn(l, k0 * a, True)
        j1, j1p = spherical_jn(l, k1 * a), spherical_jn(l, k1 * a, True)
        al = ((k1 / rho) * j1p * j0 - k0 * j1 * j0p) / (k0 * j1 * h0p - (k1 / rho) * j1p * h0)
        ext = spherical_jn(l, k0 * ro) + al * (spherical_jn(l, k0 * ro) + 1j * spherical_yn(l, k0 * ro))
        inn = (j0 + al * h0) / j1 * spherical_jn(l, k1 * ri)
        u += (2 * l + 1) * 1j ** l * np.where(out, ext, inn) * eval_legendre(l, cth)
    return u


def mie_traces(k0, k1, rho, a, cth):
    """phi = gamma_D u_tot and psi = gamma_N^+ u_tot on the sphere of radius a
    for the plane wave exp(i k0 d.x), cth = cos of the angle to d (Mie
    series of the penetrable sphere)."""
    import numpy as np
    from scipy.special import eval_legendre, spherical_jn, spherical_yn

    L = int(k0 * a + 4 * (k0 * a) ** (1 / 3) + 15)
    phi = np.zeros_like(cth, dtype=complex)
    psi = np.zeros_like(cth, dtype=complex)
    for l in range(L):
        j0, j0p = spherical_jn(l, k0 * a), spherical_jn(l, k0 * a, True)
        h0 = j0 + 1j * spherical_yn(l, k0 * a)
        h0p = j0p + 1j * spherical_yn(l, k0 * a, True)
        j1, j1p = spherical_jn(l, k1 * a), spherical_jn(l, k1 * a, True)
        al = ((k1 / rho) * j1p * j0 - k0 * j1 * j0p) / (k0 * j1 * h0p - (k1 / rho) * j1p * h0)
        P = eval_legendre(l, cth)
        phi += (2 * l + 1) * 1j ** l * (j0 + al * h0) * P
        psi += k0 * (2 * l + 1) * 1j ** l * (j0p + al * h0p) * P
    return phi, psi


def p1_mass(verts, tris):
    """Sparse P1 mass matrix |t|/12 (1 + delta_ab) of a flat-triangle mesh
    (for error norms)."""
    import numpy as np
    import scipy.sparse as sp

    p0, p1, p2 = (verts[tris[:, i]] for i in range(3))
    area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1)
    rows = np.repeat(tris, 3, axis=1).ravel()
    cols = np.tile(tris, (1, 3)).ravel()
    loc = np.array([2, 1, 1, 1, 2, 1, 1, 1, 2], dtype=float) / 12.0
    vals = (area[:, None] * loc[None, :]).ravel()
    nv = verts.shape[0]
    return sp.coo_matrix((vals, (rows, cols)), shape=(nv, nv)).tocsr()


def solution_error_vs_mie(W, x, d):
    """Mass-weighted relative errors of psi and phi at the vertices against
    the Mie series (unit sphere workloads), and of [psi; phi] together."""
    import numpy as np

    v, t = W["verts"], W["tris"]
    nv = v.shape[0]
    rad = np.linalg.norm(v, axis=1)
    cth = (v @ np.asarray(d, dtype=float)) / rad
    phi, psi = mie_traces(W["k_ext"], W["k_int"], W["rho_ratio"], 1.0, cth)
    M = p1_mass(v, t)

    def werr(a, e):
        dd = a - e
        return float(np.sqrt(np.real(np.vdot(dd, M @ dd)) / np.real(np.vdot(e, M @ e))))

    e_psi, e_phi = werr(x[:nv], psi), werr(x[nv:], phi)
    both = float(np.sqrt((np.real(np.vdot(x[:nv] - psi, M @ (x[:nv] - psi))) +
                          np.real(np.vdot(x[nv:] - phi, M @ (x[nv:] - phi)))) /
                         (np.real(np.vdot(psi, M @ psi)) + np.real(np.vdot(phi, M @ phi)))))
    return {"psi": e_psi, "phi": e_phi, "both": both,
            "note": "mass-weighted relative error of the P1 coefficients at the vertices "
                    "against the Mie series: discretisation error of the mesh, not solver error"}


def run_field(S, x, W, B):
    import numpy as np
    import torch

    g = np.linspace(-3.0, 3.0, 101)
    X, Y = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    tp = torch.tensor(pts, device=x.device)
    S.field(x, tp, B.OSRC_INC_PLANEWAVE, [0.0, 0.0, 1.0])
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    u, reg = S.field(x, tp, B.OSRC_INC_PLANEWAVE, [0.0, 0.0, 1.0])
    e1.record(stream)
    torch.cuda.synchronize()
    u = u.cpu().numpy()
    ue = mie_total_field(W["k_ext"], W["k_int"], W["rho_ratio"], 1.0, pts)
    r = np.linalg.norm(pts, axis=1)
    h = B.osrc_mesh_mean_edge(S.mesh)
    away = np.abs(r - 1.0) > 2.0 * h

    def err(m):
        return float(np.linalg.norm(np.abs(u[m]) - np.abs(ue[m])) / np.linalg.norm(np.abs(ue[m])))

    return {"grid": "101 x 101 points, [-3, 3]^2 in the plane z = 0 (the paper's 3 cm square "
                    "around a 5 mm sphere)", "eval_ms": e0.elapsed_time(e1),
            "amplitude_l2_error_vs_mie": err(np.ones(len(r), dtype=bool)),
            "amplitude_l2_error_vs_mie_away_from_surface": err(away),
            "surface_band": "points within two mean edge lengths of the surface left out",
            "points_inside": int(reg.sum().item())}


# --------------------------------------------------------------------------
# small dense leg (level-3 icosphere, FP64 dense, GMRES to 1e-8) and the large
# far-field apply (80000-vertex bumpy ellipsoid, k 60 / 144)
# --------------------------------------------------------------------------
SMALL_WORKLOAD = "sphere642"
LARGE_WORKLOAD = "bumpy80000"
# FP32 flops per far point pair of the large-ka (centred) variant: the 83 of the
# plain kernel less its 2 MUL for k r, plus 21 for the phase from the centroid
# distance (3 ADD for the offsets, r^2 - r_c^2 in 2 x (1 MUL + 2 FMA) + 1 FMA,
# 1 ADD and 1 MUL for r - r_c, one FMA per wavenumber for the phase)
FLOPS_PER_PAIR_CENTRED = 102


def run_small_dense(device):
    """Unit sphere, level-3 icosphere (642 vertices), k 2 / 3, rho 1.5, plane
    wave +z: FP64 dense assembly and OSRC GMRES to 1e-8 (set-up included)."""
    import torch

    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import workload

    W = workload(SMALL_WORKLOAD)
    times = []
    for _ in range(2):  # the first pass warms up the library
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = B.Solver(W["verts"], W["tris"], W["k_ext"], W["k_int"], W["rho_ratio"], device=device,
                     precision=B.OSRC_FP64_DENSE)
        b = S.rhs_planewave(W["dirs"][:1])
        x, info = S.solve(b, tol=1e-8, maxit=500)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        S.close()
    return {"workload": f"{SMALL_WORKLOAD}: level-3 icosphere, 642 vertices, k 2 / 3, rho 1.5, "
                        "plane wave +z", "tol": 1e-8, "solve_incl_setup_s": times[-1],
            "iterations": info.iterations, "true_residual": info.true_residual}


def run_large(device):
    """Bumpy ellipsoid (2, 1, 1) + 32 bumps, 80000 vertices / 159996 triangles,
    k 60 / 144, rho 1.9, point source at (3, 0, 0): one weak-form apply of the
    permuted PMCHWT operator (large-ka far kernel + near field), timed."""
    import torch

    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import workload

    W = workload(LARGE_WORKLOAD)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = B.Solver(W["verts"], W["tris"], W["k_ext"], W["k_int"], W["rho_ratio"], device=device)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    try:
        x = S.rhs_pointsource(W["src"])
        S.apply(x)
        B.osrc_profile_enable(S.pb, True)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        e0.record(stream)
        for _ in range(reps):
            S.apply(x)
        e1.record(stream)
        torch.cuda.synchronize()
        apply_s = e0.elapsed_time(e1) / 1000.0 / reps
        far_n, far_ms = B.osrc_far_kernel_stats(S.pb)
        B.osrc_profile_enable(S.pb, False)
        pairs = B.osrc_far_pairs(S.pb)
        far_avg = far_ms / max(far_n, 1)
        achieved = FLOPS_PER_PAIR_CENTRED * pairs / (far_avg * 1e-3) / 1e12
        props = torch.cuda.get_device_properties(torch.device("cuda", device))
        peak = props.multi_processor_count * 128 * 2 * 2070.0 * 1e6 / 1e12
        return {
            "workload": f"{LARGE_WORKLOAD}: bumpy ellipsoid (2, 1, 1), {S.nv} vertices, k "
                        f"{W['k_ext']:g} / {W['k_int']:g}, rho {W['rho_ratio']:g}, point source "
                        "(3, 0, 0)",
            "setup_s": t_setup, "apply_s": apply_s, "rows_per_s": 2 * S.nv / apply_s,
            "far_kernel": {"variant": "centred (float-float centroid phase)", "avg_ms": far_avg,
                           "pairs": pairs, "flops_per_pair": FLOPS_PER_PAIR_CENTRED,
                           "achieved_tflops": achieved, "peak_tflops": peak,
                           "frac": achieved / peak},
        }
    finally:
        S.close()


# --------------------------------------------------------------------------
# four spheres (Sec. 3.5): radius 1 (5 mm), centres (+-3, +-1.5, 0), two
# fat-like and two bone-like interiors, water outside, 0.5 and 1 MHz
# --------------------------------------------------------------------------
C_WATER, C_FAT, C_BONE = 1500.0, 1450.0, 3600.0
RHO_FAT, RHO_BONE = 0.95, 1.9


def four_spheres(level=4):
    import numpy as np

    from paper_2104_04609_gb300.inputs import icosphere

    v, t = icosphere(level)
    centres = [(-3.0, -1.5, 0.0), (-3.0, 1.5, 0.0), (3.0, -1.5, 0.0), (3.0, 1.5, 0.0)]
    V = np.vstack([v + np.array(c) for c in centres])
    T = np.vstack([t + i * len(v) for i in range(4)])
    return V, T


def run_four_spheres(device):
    """Multiple scattering at four disjoint spheres (level-4 icospheres, 10248
    vertices in all): the spheres at x < 0 fat-like (c 1450 m/s, rho ratio
    0.95), at x > 0 bone-like (c 3600 m/s, rho ratio 1.9), k_int = k_ext c_water
    / c_object; plane wave along +x; GMRES to 1e-5."""
    import torch

    from paper_2104_04609_gb300 import binding as B

    V, T = four_spheres()
    res = []
    for f_mhz in (0.5, 1.0):
        k0 = 2.0 * math.pi * f_mhz * 1e6 / C_WATER * 5e-3  # radius 5 mm = 1
        kin = [k0 * C_WATER / C_FAT] * 2 + [k0 * C_WATER / C_BONE] * 2
        rho = [RHO_FAT] * 2 + [RHO_BONE] * 2
        S = B.Solver(V, T, k0, None, None, device=device, objects=(kin, rho))
        try:
            b = S.rhs_planewave([[1.0, 0.0, 0.0]])
            S.solve(b, tol=TOL, maxit=1000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, info = S.solve(b, tol=TOL, maxit=1000)
            torch.cuda.synchronize()
            res.append({"frequency_mhz": f_mhz, "k_ext": k0, "iterations": info.iterations,
                        "solve_s": time.perf_counter() - t0, "true_residual": info.true_residual})
        finally:
            S.close()
    return {"workload": "four spheres (radius 1 = 5 mm) at (+-3, +-1.5, 0), level-4 icospheres, "
                        "10248 vertices; two fat-like, two bone-like; plane wave +x; tol 1e-5",
            "runs": res}


# --------------------------------------------------------------------------
# serving leg: continuous batching on a seeded Poisson stream
# --------------------------------------------------------------------------
# hybrid route of the serving leg: requests with several right-hand sides on
# meshes up to this many vertices take the batched mixed-precision dense
# solve (the assembled FP64 system of 2 n_v x 2 n_v entries and its BF16
# copies stay within a few tens of GB); larger or single-right-hand-side
# requests stay matrix-free
SERVE_DENSE_MAX_NV = 12000


def serving_workload(n_req):
    """The first n_req requests of the seeded stream (rate 50/s, seed 2) at
    their stated sizes: spheres and ellipsoids (Fibonacci hulls) of 2k-40k
    vertices, ka in [5, 40] (a = largest semi-axis), k_int = k_ext / c_ratio,
    1-16 plane waves."""
    import numpy as np

    from paper_2104_04609_gb300.inputs import fibonacci_hull, plane_wave_dirs, serving_requests

    out = []
    for r in serving_requests(1000, 50.0, seed=2)[:n_req]:
        v, t = fibonacci_hull(r["n_v"])
        v = v * np.asarray(r["axes"])[None, :]
        a = max(r["axes"])
        k_ext = r["ka"] / a
        out.append(dict(t=r["t"], verts=v, tris=t, k_ext=k_ext, k_int=k_ext / r["c_ratio"],
                        rho=r["rho_ratio"], ka=r["ka"], n_v=r["n_v"],
                        dirs=plane_wave_dirs(r["nrhs"], seed=r["seed"] % (2 ** 31))))
    return out


def run_serving(n_req, device, route="matrix_free", progress=None, deadline=None):
    """route "matrix_free": every request FP32 matrix-free (a request with
    several right-hand sides runs GMRES in lockstep over them, one far-field
    launch per iteration for all); "hybrid": requests with several
    right-hand sides on meshes of at most SERVE_DENSE_MAX_NV vertices take the
    batched mixed-precision dense solve (tolerance on the true residual), the
    rest stay matrix-free.  Requests are submitted at their Poisson arrival
    times (offered load 50/s); the loop serves them with 4 slots."""
    import numpy as np
    import torch

    from paper_2104_04609_gb300 import binding as B

    work = serving_workload(n_req)
    total_mem = torch.cuda.get_device_properties(device).total_memory
    ctx = B.osrc_create(device, int(0.7 * total_mem))
    sv = B.osrc_server_create(ctx, 4)
    try:
        t0 = time.perf_counter()
        ids = []
        for w in work:
            delay = t0 + w["t"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            p = B.osrc_params_default(k_ext=w["k_ext"], k_int=w["k_int"], rho_ratio=w["rho"])
            w["route"] = "matrix-free" if len(w["dirs"]) == 1 else "lockstep"
            if route == "hybrid" and len(w["dirs"]) >= 2 and w["n_v"] <= SERVE_DENSE_MAX_NV:
                p.precision = B.OSRC_FP64_DENSE
                p.dense_assembly = B.OSRC_ASSEMBLE_FF
                w["route"] = "dense batched"
            ids.append(B.osrc_server_submit(sv, w["verts"], w["tris"], p, w["dirs"], tol=TOL,
                                            maxit=1000))
        t_sub = time.perf_counter() - t0
        lat, que, its, ok, per = [], [], 0, 0, []
        unfinished = 0
        for rid, w in zip(ids, work):
            wait = 3600.0 if deadline is None else max(0.0, deadline - (time.perf_counter() - t0))
            B.osrc_server_wait(sv, rid, wait)
            done, st, l, info = B.osrc_server_poll(sv, rid)
            if not done:
                unfinished += 1
            if done:
                lat.append(l)
                que.append(info["ms_queued"])
                its += info["total_iterations"]
                ok += 1 if st == B.OSRC_OK else 0
                per.append({"n_v": w["n_v"], "ka": round(w["ka"], 2), "rhs": len(w["dirs"]),
                            "route": w["route"], "latency_s": round(l / 1e3, 3),
                            "queued_s": round(info["ms_queued"] / 1e3, 3),
                            "iterations": info["total_iterations"], "status": int(st)})
                if progress:  # one line per finished request, for long runs
                    with open(progress, "a") as f:
                        f.write(json.dumps({"t_s": time.perf_counter() - t0, **per[-1]}) + "\n")
        t1 = time.perf_counter()
        stats = B.osrc_server_get_stats(sv)
    finally:
        B.osrc_server_destroy(sv)
        B.osrc_destroy(ctx)
    nrhs = sum(p["rhs"] for p in per)
    lat, que = np.asarray(lat), np.asarray(que)
    span = max(work[-1]["t"], 1e-9)
    wall = t1 - t0
    if unfinished:  # censored: the unfinished requests' latency is at least the deadline
        lat = np.concatenate([lat, np.full(unfinished, 1e3 * wall)])
    return {
        "route": route, "requests": len(work), "finished_requests": len(per),
        "unfinished_at_deadline": unfinished, "deadline_s": deadline,
        "right_hand_sides_solved": nrhs, "converged_requests": ok,
        "offered_requests_per_s": len(work) / span, "served_requests_per_s": len(per) / wall,
        "solves_per_s": nrhs / wall, "wall_s": wall, "submit_span_s": t_sub,
        "right_hand_sides_submitted": sum(len(w["dirs"]) for w in work),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max()),
                       "note": "unfinished requests count with the deadline as their latency (a lower "
                               "bound)" if unfinished else "all requests finished"},
        "queued_ms": {"p50": float(np.percentile(que, 50)), "p99": float(np.percentile(que, 99))},
        "queueing_share_of_latency": float(que.sum() / max(np.asarray(lat[:len(que)]).sum(), 1e-9)),
        "gmres_iterations": its, "max_active": 4, "active_peak": stats["active_peak"],
        "cache_hits": stats["cache_hits"], "cache_misses": stats["cache_misses"],
        "mem_peak_bytes": stats["mem_peak"], "block_requests": stats["batched_jobs"],
        "per_request": per,
        "sample": f"first {len(work)} requests of the seeded Poisson stream (50/s, seed 2) at their "
                  f"stated sizes (2k-40k vertices, ka 5-40, 1-16 right-hand sides, no caps); "
                  f"the offered load far exceeds what one GPU serves, so latency is mostly "
                  f"queueing (queued = submit to first GPU work); saturation throughput = "
                  f"solves_per_s",
    }


# --------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# --------------------------------------------------------------------------
class OracleTimer:
    """Times the FP64 CPU oracle on rows of the same matvec: each row of the
    permuted PMCHWT matrix at both wavenumbers, assembled and applied."""

    def __init__(self):
        import numpy as np

        import oracle as O
        from paper_2104_04609_gb300.inputs import workload

        self.O = O
        self.W = workload(WORKLOAD)
        self.nv = self.W["verts"].shape[0]
        rng = np.random.default_rng(0)
        self.x = rng.standard_normal(2 * self.nv) + 1j * rng.standard_normal(2 * self.nv)
        self.rng = np.random.default_rng(1)
        self.threads = O.lib().orc_num_threads()
        self.t_osrc = None

    def rows(self, nrows):
        W = self.W
        rows = self.rng.choice(self.nv, nrows, replace=False)
        t0 = time.perf_counter()
        R1, R2 = self.O.pmchwt_rows(W["verts"], W["tris"], W["k_ext"], W["k_int"],
                                    W["rho_ratio"], rows, nss=4)
        _ = R1 @ self.x, R2 @ self.x
        return time.perf_counter() - t0

    def osrc_time(self):
        """One strong-form mass solve + OSRC apply with the oracle's sparse LU."""
        if self.t_osrc is None:
            import numpy as np

            W = self.W
            O = self.O
            M, Sm = O.mass_stiffness(W["verts"], W["tris"])
            R = O.mean_edge_length(W["verts"], W["tris"])
            ke = O.damped_wavenumber(W["k_int"], R)
            solver = O._ShiftedSolver(M, Sm)
            u = self.x
            O.osrc_apply(M, Sm, u[: self.nv], u[self.nv:], W["k_int"], ke, 4, math.pi / 3, solver)
            t0 = time.perf_counter()
            y = O.strong_apply(M, u)
            O.osrc_apply(M, Sm, y[: self.nv], y[self.nv:], W["k_int"], ke, 4, math.pi / 3, solver)
            self.t_osrc = time.perf_counter() - t0
        return self.t_osrc

    def calibrate(self, seconds):
        t = self.rows(8)
        per_row = t / 8
        return max(8, min(self.nv, int(seconds / max(per_row, 1e-6))))

    def solves_per_s(self, nrows, t_rows, iterations):
        t_matvec = t_rows / nrows * self.nv
        t_solve = (iterations + 1) * t_matvec + iterations * self.osrc_time()
        return 1.0 / t_solve


def cpu_baseline(iterations, seconds, solution=None):
    T = OracleTimer()
    n = T.calibrate(seconds)
    t = T.rows(n)
    v = T.solves_per_s(n, t, iterations)
    check = oracle_row_residual(T, solution) if solution is not None else None
    return {"value": v, "unit": UNIT, "cores": T.threads, "kind": "oracle",
            "oracle_row_check": check,
            "sample": f"{n} of {T.nv} rows of one permuted-PMCHWT matvec (both wavenumbers, "
                      f"6x6 rule + Sauter-Schwab n_ss 4) in {t:.1f} s, plus one sparse-LU "
                      f"mass solve + OSRC apply; scaled to (iterations + 1) matvecs and "
                      f"{iterations} preconditioner applies per solve ({iterations} GMRES "
                      f"iterations)"}


def oracle_row_residual(T, solution, nrows=96):
    """The GPU solution of the timed solve checked by the FP64 oracle on
    sampled rows: the oracle's weak residual (R x - b)[rows] relative to
    b[rows], and the oracle's rows of B x against the GPU's (the residuals of
    both on the same rows)."""
    import numpy as np

    xs, bs, r_gpu = solution
    W = T.W
    nv = T.nv
    rows = np.random.default_rng(11).choice(nv, nrows, replace=False)
    R1, R2 = T.O.pmchwt_rows(W["verts"], W["tris"], W["k_ext"], W["k_int"], W["rho_ratio"], rows, nss=4)
    idx = np.concatenate([rows, nv + rows])
    Bx_orc = np.concatenate([R1 @ xs, R2 @ xs])
    r_orc = bs[idx] - Bx_orc
    Bx_gpu = bs[idx] - r_gpu[idx]
    return {"rows": 2 * nrows,
            "oracle_weak_residual": float(np.linalg.norm(r_orc) / np.linalg.norm(bs[idx])),
            "gpu_weak_residual_same_rows": float(np.linalg.norm(r_gpu[idx]) / np.linalg.norm(bs[idx])),
            "Bx_rel_diff_oracle_vs_gpu": float(np.linalg.norm(Bx_orc - Bx_gpu) / np.linalg.norm(Bx_orc)),
            "note": f"{nrows} vertex rows of both block rows, FP64 oracle (6x6 rule + "
                    f"Sauter-Schwab n_ss 4), applied to the GPU's solution"}


def cpu_other_configs(out, seconds=4.0):
    """The oracle on the other workloads beside the GPU numbers of this run:
    the full small dense solve, sampled rows of the assembled ellipsoid system
    (assembly + one GEMV, extrapolated to all rows), sampled rows of the large
    operator (rows/s)."""
    import numpy as np

    import oracle as O
    from paper_2104_04609_gb300.inputs import workload

    res = {}
    if "small_dense" in out:
        W = workload(SMALL_WORKLOAD)
        t0 = time.perf_counter()
        P = O.Problem(W["verts"], W["tris"], W["k_ext"], W["k_int"], W["rho_ratio"], nss=4)
        b = P.rhs()
        P.solve_gmres(b, tol=1e-8)
        t = time.perf_counter() - t0
        g = out["small_dense"]["solve_incl_setup_s"]
        res["sphere642_solve"] = {"oracle_s": t, "gpu_s": g, "speedup": t / g,
                                  "sample": "full FP64 dense assembly + OSRC GMRES to 1e-8"}

    def rows_rate(name, nss=4):
        W = workload(name)
        nv = W["verts"].shape[0]
        rng = np.random.default_rng(5)
        x = rng.standard_normal(2 * nv) + 1j * rng.standard_normal(2 * nv)
        n = 2
        while True:
            rows = rng.choice(nv, n, replace=False)
            t0 = time.perf_counter()
            R1, R2 = O.pmchwt_rows(W["verts"], W["tris"], W["k_ext"], W["k_int"], W["rho_ratio"],
                                   rows, nss=nss)
            _ = R1 @ x, R2 @ x
            t = time.perf_counter() - t0
            if t > seconds / 4 or n >= nv:
                return nv, n, t
            n = min(nv, n * 4)

    if "dense_batched" in out:
        nv, n, t = rows_rate(DENSE_WORKLOAD)
        t_all = t / n * nv
        d = out["dense_batched"]
        g = d["assembly_s"] + d["fp64_gemv_ms"] * 1e-3
        res["ellipsoid8000_assembly_gemv"] = {
            "oracle_s": t_all, "gpu_s": g, "speedup": t_all / g,
            "sample": f"{n} of {nv} vertex rows (both block rows) assembled and applied in "
                      f"{t:.1f} s, extrapolated to all rows"}
    if "large" in out:
        nv, n, t = rows_rate(LARGE_WORKLOAD)
        r = 2 * n / t
        gr = out["large"]["rows_per_s"]
        res["bumpy80000_rows"] = {"oracle_rows_per_s": r, "gpu_rows_per_s": gr, "speedup": gr / r,
                                  "sample": f"{n} of {nv} vertex rows (both block rows) in {t:.1f} s"}
    return res


def run_reference(args, D):
    if D.world > 1 and D.rank != 0:
        return None
    import __graft_entry__

    from oracle import build as orcbuild

    orcbuild.build()
    T = OracleTimer()
    per_step = max(1.0, min(args.cpu_seconds, 20.0))
    n = T.calibrate(per_step)
    for _ in range(args.warmup):
        T.rows(max(8, n // 8))
    times = [T.rows(n) for _ in range(args.steps)]
    vals = [T.solves_per_s(n, t, REF_ITERATIONS) for t in times]
    value = statistics.mean(vals)
    ms_per_step = 1000.0 / value
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": D.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": "sphere10242: unit sphere, level-5 icosphere, 10242 vertices / "
                               "20480 triangles, k_ext 20, k_int 26, rho ratio 1.5, plane wave +z",
                   "path": "FP64 CPU oracle (C + OpenMP, numpy/scipy)", "tol": TOL,
                   "timing": f"extrapolated: each step times a row sample of one matvec and "
                             f"scales it to a whole solve of {REF_ITERATIONS} iterations"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": T.threads, "kind": "oracle",
                         "sample": f"each step: {n} of {T.nv} rows of one matvec, scaled to "
                                   f"{REF_ITERATIONS + 1} matvecs + {REF_ITERATIONS} "
                                   f"preconditioner applies per solve"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return out


def large_sweep(nv, device=0, maxit=600, ks=(15.0, 30.0, 45.0, 60.0)):
    """GMRES iteration count vs frequency on the bumpy ellipsoid (point source
    at (3, 0, 0), k_int = 2.4 k_ext, rho 1.9, tol 1e-5): one JSON line per k.
    With nv = 80000 and k_ext = 60 this is the large workload's full solve."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import bumpy_ellipsoid

    v, t = bumpy_ellipsoid(nv)
    for k0 in ks:
        S = B.Solver(v, t, k0, k0 * 3600.0 / 1500.0, 1.9, device=device)
        try:
            b = S.rhs_pointsource([[3.0, 0.0, 0.0]])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, info = S.solve(b, tol=TOL, maxit=maxit, raise_on_nonconvergence=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            print(json.dumps({"mesh": f"bumpy ellipsoid (2, 1, 1), {S.nv} vertices",
                              "k_ext": k0, "k_int": k0 * 2.4, "ka": 2.0 * k0,
                              "iterations": info.iterations, "converged": bool(info.converged),
                              "precond_residual": info.precond_residual,
                              "true_residual": info.true_residual, "solve_s": dt}), flush=True)
        finally:
            S.close()


def precond_sweep(device=0, maxit=800):
    """Iteration counts of the paper's comparison (Sec. 3.3): unit sphere
    (level-5 icosphere, 10242 vertices), k_int = 1.3 k_ext, rho 1.5, plane wave,
    tol 1e-5, for PMCHWT with OSRC, mass-only and Calderon preconditioning and
    the Mueller formulation with mass preconditioning."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import icosphere

    v, t = icosphere(5)
    kinds = (("osrc", B.OSRC_PRECOND_OSRC, B.OSRC_PMCHWT), ("mass", B.OSRC_PRECOND_MASS, B.OSRC_PMCHWT),
             ("calderon", B.OSRC_PRECOND_CALDERON, B.OSRC_PMCHWT),
             ("muller", B.OSRC_PRECOND_MASS, B.OSRC_MULLER))
    for k0 in (5.0, 10.0, 20.0):
        for name, code, form in kinds:
            S = B.Solver(v, t, k0, 1.3 * k0, 1.5, device=device, precond=code, formulation=form)
            try:
                b = S.rhs_planewave([[0.0, 0.0, 1.0]])
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                x, info = S.solve(b, tol=TOL, maxit=maxit, raise_on_nonconvergence=False)
                torch.cuda.synchronize()
                print(json.dumps({"mesh": "unit sphere, 10242 vertices", "k_ext": k0,
                                  "k_int": 1.3 * k0, "precond": name,
                                  "iterations": info.iterations, "converged": bool(info.converged),
                                  "true_residual": info.true_residual,
                                  "solve_s": time.perf_counter() - t0}), flush=True)
            finally:
                S.close()


def profile_case(name, device=0):
    """Small fixed workloads for ncu captures (see --profile-case)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import ellipsoid, icosphere, plane_wave_dirs, workload

    if name == "far-small":
        v, t = icosphere(4)
        for k0, k1 in ((20.0, 26.0), (40.0, 100.0)):
            S = B.Solver(v, t, k0, k1, 1.5, device=device)
            x = S.rhs_planewave([[0.0, 0.0, 1.0]])
            for _ in range(3):
                S.apply(x)
            torch.cuda.synchronize()
            S.close()
        return
    if name == "far-multi-small":
        # several-right-hand-side far field on icosphere(4): three applies of 8
        # right-hand sides at k 20 / 26 (plain), then three at k 40 / 100 (centred)
        v, t = icosphere(4)
        for k0, k1 in ((20.0, 26.0), (40.0, 100.0)):
            S = B.Solver(v, t, k0, k1, 1.5, device=device)
            x = S.rhs_planewave(plane_wave_dirs(8, seed=3))
            for _ in range(3):
                S.apply(x)
            torch.cuda.synchronize()
            S.close()
        return
    if name == "precond-small":
        # OSRC preconditioner (mass solve + 2 N_Pade + 1 shifted systems) on icosphere(4), five applies
        v, t = icosphere(4)
        S = B.Solver(v, t, 20.0, 26.0, 1.5, device=device)
        x = S.rhs_planewave([[0.0, 0.0, 1.0]])
        for _ in range(5):
            S.precond(x)
        torch.cuda.synchronize()
        S.close()
        return
    if name == "gemm":
        # the tensor-core GEMM alone at the batched path's shape for ellipsoid8000
        # (M 16000, N 2 x 128, K 32000; 1 GB of A), three launches
        M, N, K = 16000, 256, 32000
        A = torch.randn(M, K, device=f"cuda:{device}").to(torch.bfloat16)
        Bm = torch.randn(N, K, device=f"cuda:{device}").to(torch.bfloat16)
        C = torch.empty(M, N, device=f"cuda:{device}")
        err = torch.zeros(1, dtype=torch.int32, device=f"cuda:{device}")
        ws = torch.empty(max(B.osrc_gemm_bf16_ws_bytes(M, N, K), 16), dtype=torch.uint8, device=f"cuda:{device}")
        for _ in range(3):
            B.osrc_gemm_bf16(A, Bm, C, err, ws=ws)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        return
    if name == "dense-short":
        W = workload(DENSE_WORKLOAD)
        v, t, k0, k1, rho, dirs, maxit = W["verts"], W["tris"], W["k_ext"], W["k_int"], W["rho_ratio"], \
            W["dirs"][:128], 120
    else:
        v, t = ellipsoid(3000)
        k0, k1, rho, dirs, maxit = 15.0, 36.0, 1.9, plane_wave_dirs(128, seed=1), 24
    S = B.Solver(v, t, k0, k1, rho, device=device, precision=B.OSRC_FP64_DENSE,
                 dense_assembly=B.OSRC_ASSEMBLE_FF)
    try:
        b = S.rhs_planewave(dirs)
        x = torch.zeros_like(b)
        B.osrc_dense_precond_build(S.pb, tol=1e-3, maxit=500)
        info = B.osrc_dense_batched_solve(S.pb, b, x, tol=1e-6, max_refine=1, inner_tol=1e-3,
                                          inner_maxit=maxit, raise_on_nonconvergence=False)
        torch.cuda.synchronize()
        print(json.dumps(info), flush=True)
    finally:
        S.close()


def sponge_sweep(device=0, maxit=400):
    """The non-smooth domain of Sec. 3.4: level-2 Menger sponge, edge 2 (10 mm),
    bone-like interior (c 3600 m/s, rho ratio 1.9) in water, plane wave +x,
    tol 1e-5; faces split so that there are about six or more elements per
    exterior wavelength (sub 3 at 0.5 MHz, 5 at 1 MHz)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import menger_sponge

    kinds = (("osrc", B.OSRC_PRECOND_OSRC, B.OSRC_PMCHWT), ("mass", B.OSRC_PRECOND_MASS, B.OSRC_PMCHWT),
             ("calderon", B.OSRC_PRECOND_CALDERON, B.OSRC_PMCHWT),
             ("muller", B.OSRC_PRECOND_MASS, B.OSRC_MULLER))
    for f_mhz, sub in ((0.5, 3), (1.0, 5)):
        v, t = menger_sponge(2, sub, edge=2.0)
        k0 = 2.0 * math.pi * f_mhz * 1e6 / C_WATER * 5e-3
        for name, code, form in kinds:
            S = B.Solver(v, t, k0, k0 * C_WATER / C_BONE, RHO_BONE, device=device, precond=code,
                         formulation=form)
            try:
                b = S.rhs_planewave([[1.0, 0.0, 0.0]])
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                x, info = S.solve(b, tol=TOL, maxit=maxit, raise_on_nonconvergence=False)
                torch.cuda.synchronize()
                print(json.dumps({"mesh": f"level-2 Menger sponge, {S.nv} vertices",
                                  "frequency_mhz": f_mhz, "k_ext": k0, "formulation": name,
                                  "iterations": info.iterations, "converged": bool(info.converged),
                                  "true_residual": info.true_residual,
                                  "solve_s": time.perf_counter() - t0}), flush=True)
            finally:
                S.close()


def main():
    args = parse()
    if args.sponge_sweep:
        sponge_sweep()
        return
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.large_sweep > 0:
        large_sweep(args.large_sweep, maxit=args.large_maxit,
                    ks=[float(k) for k in args.large_ks.split(",") if k.strip()])
        return
    if args.precond_sweep:
        precond_sweep()
        return
    if args.impl == "reference":
        D = Dist(want_cuda=False)
        out = run_reference(args, D)
        if out is not None:
            print(json.dumps(out), flush=True)
        D.close()
        return
    D = Dist(want_cuda=True)
    out, iters = run_ours(args, D)
    solution = out.pop("_solution", None)
    if D.rank == 0:
        if D.world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(iters, args.cpu_seconds, solution)
            out["cpu_baseline"]["other_workloads"] = cpu_other_configs(out)
            chk = out["cpu_baseline"].get("oracle_row_check")
            if chk is not None:
                out["config"]["oracle_row_residual"] = chk["oracle_weak_residual"]
        print(json.dumps(out), flush=True)
    D.close()


if __name__ == "__main__":
    main()
