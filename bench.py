#!/usr/bin/env python
"""Benchmark: solves/s of the dynamic-OT inexact proximal ALM at KKT <= 1e-6.

One step = one complete solve (Algorithm 2 from q = alpha = beta = 0 until
eta_dot <= tol at a check) of a seeded synthetic 2D 256^2 x 64 Gaussian-mixture
transport problem, with its inputs already resident in HBM.  The mixed-precision
path is the product; the FP64 path is solved once on the same GPU for the
"mixed vs FP64" comparison.  Multi-GPU: independent replicas (one process per
GPU, no collective on the data path), value = all solves / max wall time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  --impl reference times the CPU oracle (the
plain FP64 restatement under oracle/) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s at KKT<=1e-6, mixed vs FP64 on same GPU; p50/p99 latency; %HBM peak"
WORKLOAD = "mix256"
WORKLOAD_DESCS = {
    "mix256": ("2D DOT 256x256 cells x 64 time steps, seeded mixtures of 1-5 Gaussians "
               "(means U[0.15,0.85]^2, sigma U[0.03,0.12], Dirichlet weights), pdf < 1e-4 -> 0"),
    "obst128": ("2D DOT with obstacles, 128x128 cells x 32 time steps, seeded mixtures as mix256 zeroed on "
                "a mask of 3-6 rectangles covering 8-12% of cells, obstacle weight 1e-6"),
    "mix3d64": ("3D DOT 64^3 cells x 32 time steps, seeded mixtures of 2-4 anisotropic Gaussians "
                "(sigma U[0.05,0.15]^3), floor 1e-4"),
    "gauss32": "2D DOT 32x32 cells x 16 time steps, Gaussians sigma 0.1 at (0.3,0.3), (0.7,0.7) + floor 1e-3",
    "mix1024": ("2D DOT 1024x1024 cells x 32 time steps (the scalability case), seeded mixtures as mix256"),
}
WORKLOAD_SEEDS = {"mix256": 1002, "obst128": 1003, "mix3d64": 1004, "gauss32": None, "mix1024": 1005,
                  "ex1": None, "ex2": None, "ex3": None, "ex4": None}
# Iterations the FP64 recurrence (GPU FP64 path == oracle, lock-step tested) needs to reach
# eta_dot <= 1e-6 on the seed-1002 instance of this workload; converts the oracle's
# seconds per iteration into solves/s in the reference arm.  Measured by this script's
# own arm ("fp64" -> "iterations" in its JSON line).
ORACLE_ITERS_PER_SOLVE = {"mix256": 11120}   # the FP64 recurrence to eta <= 1e-6, checks every 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--maxit", type=int, default=40000)
    ap.add_argument("--check-every", type=int, default=10,
                    help="stopping measures and penalty rule every this many iterations")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison solve")
    ap.add_argument("--fp64-maxit", type=int, default=40000)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="end-to-end solves through the public API with host buffers, on the timed steps' instances (-1: as many as --steps)")
    ap.add_argument("--workload", default=WORKLOAD, choices=["mix256", "gauss32", "obst128", "mix3d64", "mix1024",
                                                                "ex1", "ex2", "ex3", "ex4"])
    ap.add_argument("--serve", type=int, default=0,
                    help="serve the first SERVE requests of the seeded serving stream (2D grids "
                         "{32^2x16, 64^2x32, 128^2x32, 256^2x64}, Poisson arrivals, 20%% masked) through "
                         "the continuous-batching server and print its JSON line instead")
    ap.add_argument("--rate", type=float, default=200.0, help="arrivals per second of the serving stream")
    ap.add_argument("--serve-multilevel", type=int, default=0,
                    help="serve large requests with the multilevel warm start over this many coarse levels")
    ap.add_argument("--serve-ml-masked", action="store_true",
                    help="also warm-start requests with obstacles")
    ap.add_argument("--serve-ml-min-nodes", type=int, default=500000,
                    help="requests with at least this many nodes get the multilevel warm start")
    ap.add_argument("--serve-maxit", type=int, default=300000,
                    help="iteration limit of each served request (obstacle instances need ~1e5 at tol 1e-6)")
    ap.add_argument("--multilevel", type=int, default=0,
                    help="solve every timed instance with the multilevel strategy over this many coarse levels")
    ap.add_argument("--coarse-tol", type=float, default=0.0,
                    help="tolerance of the coarse levels (0: the paper's max(tol*10^-v, 1e-6))")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="run this many iterations of one solve (no stopping checks) and exit: a short, "
                         "fixed launch sequence for ncu; prints no JSON")
    return ap.parse_args()


def run_profile_case(args):
    """A fixed launch sequence for profilers: one context, N iterations, no checks."""
    import torch
    from paper_2505_05424_gb300 import workloads as W
    from paper_2505_05424_gb300 import _native
    _native.build()
    spec, r0, r1, m = W.workload(args.workload)
    s = make_solver(spec, r0, r1, m, args.prec, check_every=0)
    s.dot_solve(0.0, args.profile_iters)
    torch.cuda.synchronize()
    print(f"profile case: {args.workload} {args.prec} {args.profile_iters} iterations, "
          f"{s.launch_count()} launches", file=sys.stderr)
    s.close()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
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
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- algorithmic bytes of one launch per kernel ---------------------------------

def algorithmic_bytes(name: str, D: int, T: int, N: int, prec: str) -> float:
    """Compulsory DRAM bytes of one launch of `name` (natural, unpadded counts)."""
    P = N ** D
    nc, n0 = (T + 1) * P, T * P
    nf = (T + 1) * N ** (D - 1) * (N - 1)          # faces of one spatial axis
    K = 4 * D + 2
    if prec == "fp64":
        w, ws, wf = 8, 8, 8                        # q/z, multipliers, phi
    else:
        w, ws, wf = 4, 8, 8                        # FP32 q/z, two-float multipliers and phi
    nq = n0 + D * nf
    table = {
        "assemble_b": (w + ws) * nq + w * nc,
        "cone_project": w * nq + ws * K * n0 + w * K * n0,
        "update_q0_alpha0": wf * nc + 2 * w * n0 + 2 * ws * n0 + ws * n0 + w * n0 + ws * n0,
        "update_qd_alphad": wf * nc + 4 * w * n0 + 4 * ws * n0 + ws * nf + w * nf + ws * nf,
        "update_beta": w * nq + w * K * n0 + 2 * ws * K * n0,
        "dct_axis": 2 * (8 if prec == "fp64" else 4) * nc,
        "poisson_residual": 3 * 4 * nc,
        "poisson_combine": (4 + 4 + 8) * nc,
        "dct_scale": 2 * (8 if prec == "fp64" else 4) * nc,
        # lines 3-6 fused: read q, alpha/sigma, beta/sigma (iteration k) and phi; write
        # q, alpha/sigma, beta/sigma (k+1) and the next iteration's residual r (FP32)
        "fused_cone_update": 2 * (w + ws) * nq + 2 * ws * K * n0 + wf * nc + w * nc,
        # D = 3 face pass: read alpha_d/sigma, phi, beta/sigma, z and the new q_0,
        # alpha_0/sigma; write q_d, alpha_d/sigma, beta/sigma and the residual r
        "face_beta_residual": 2 * (w + ws) * D * nf + wf * nc + w * K * n0 + 2 * ws * K * n0 + (w + ws) * n0
                              + w * nc,
    }
    if prec != "fp64" and D == 3:
        # D = 3 cone pass: read q, beta/sigma, phi, alpha_0/sigma; write z, q_0, alpha_0/sigma
        table["cone_project"] = w * nq + ws * K * n0 + wf * nc + w * K * n0 + w * n0 + 2 * ws * n0
    return float(table.get(name, 0.0))


# DRAM bytes (read + write) of one launch from a stored ncu capture of the kernel on
# the named workload, with the SHA-256 prefix of the kernel source it was taken on:
# the figure is reported only while that source is unchanged (else traffic = null).
NCU_TRAFFIC = {("fused_cone_update", "mix256", "mixed"):
               (603.940096e6 + 472.039424e6, "k_fused2d.cu", "1800e29b4d940626")}


def stored_traffic(kernel: str, workload: str, prec: str):
    """(bytes, note) of the stored ncu DRAM traffic, or (None, reason)."""
    import hashlib
    ent = NCU_TRAFFIC.get((kernel, workload, prec))
    if ent is None:
        return None, "no stored ncu capture for this kernel and workload"
    nbytes, src, sha = ent
    path = os.path.join(ROOT, "paper_2505_05424_gb300", "csrc", src)
    with open(path, "rb") as fh:
        cur = hashlib.sha256(fh.read()).hexdigest()[:16]
    if cur != sha:
        return None, f"{src} changed since the stored ncu capture"
    return nbytes, f"stored ncu capture (dram__bytes_read.sum + dram__bytes_write.sum), {src} sha256 {sha}"


# ---- replicas: one process per GPU, independent solves, no data-path collective --

def replica_seed(base: int, step: int, rank: int) -> int:
    """Seed of the instance a rank solves at a step: ranks never share an instance."""
    return base + step + 1000 * rank


def replica_max_ms(elapsed_ms: float, dist=None, device=None) -> float:
    """The slowest rank's timed region (the job ends when every replica has)."""
    if dist is None:
        return float(elapsed_ms)
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, steps: int, max_ms: float) -> float:
    """Whole-job solves/s: all ranks' solves over the slowest rank's time."""
    return world * steps / (max_ms / 1e3)


def make_solver(spec, r0, r1, mask, prec, **kw):
    from paper_2505_05424_gb300.solver import DotSolver
    return DotSolver(spec.D, spec.T, spec.N, r0, r1, mask=mask, prec=prec, **kw)


def run_ours(args):
    import torch
    from paper_2505_05424_gb300 import workloads as W
    from paper_2505_05424_gb300 import _native

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _native.build()
    _native.load()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wl = args.workload
    spec = W.workload(wl)[0]
    base_seed = WORKLOAD_SEEDS[wl]

    def instance(step):
        if base_seed is None:
            return W.workload(wl)[1:]
        return W.workload(wl, replica_seed(base_seed, step, rank))[1:]

    stream = torch.cuda.current_stream(dev)
    # warm-up solves
    for w in range(args.warmup):
        r0, r1, m = instance(w)
        s = make_solver(spec, r0, r1, m, args.prec, check_every=args.check_every)
        s.dot_solve(args.tol, args.maxit)
        s.close()
    # inputs resident in HBM before the timed region; the last timed solve brackets
    # every kernel with CUDA events on the solver's stream (the per-kernel durations
    # of the roofline), the others replay each check period from a CUDA graph
    solvers = []
    for k in range(args.steps):
        r0, r1, m = instance(k)
        s = make_solver(spec, r0, r1, m, args.prec, check_every=args.check_every)
        s.dot_profile(k == args.steps - 1)
        solvers.append(s)
    launches0 = sum(s.launch_count() for s in solvers)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    lat, iters, etas, objs = [], [], [], []
    ev0.record(stream)
    level_iters = []
    for s in solvers:
        t0 = time.perf_counter()
        if args.multilevel > 0:
            rc, its = s.dot_solve_multilevel(args.multilevel, args.tol, args.maxit, args.coarse_tol)
            level_iters.append(its)
        else:
            rc = s.dot_solve(args.tol, args.maxit)
        lat.append((time.perf_counter() - t0) * 1e3)
        kk = s.dot_kkt()
        iters.append(int(kk["iterations"]))
        etas.append(kk["eta_dot"])
        objs.append(-2.0 * kk["primal_obj"] / spec.N ** spec.D)   # W2^2 = -2 |X_i| <c, phi>
        if rc != 0:
            print(json.dumps({"warning": f"solve did not converge (rc={rc})", "eta": kk["eta_dot"]}),
                  file=sys.stderr)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed_ms = replica_max_ms(ev0.elapsed_time(ev1), dist, dev)
    gpu_launches = sum(s.launch_count() for s in solvers) - launches0
    prof = {}
    for s in solvers:
        for k, (ms, n) in s.dot_profile_read().items():
            a = prof.setdefault(k, [0.0, 0])
            a[0] += ms
            a[1] += n
    for s in solvers:
        s.close()
    value = replica_value(world, args.steps, elapsed_ms)
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    peaks, peak_src = load_peaks()
    # dominant kernel by total time in the timed region
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dname, (dms, dn) = dom[0], dom[1]
    per_launch_ms = dms / max(dn, 1)
    abytes = algorithmic_bytes(dname, spec.D, spec.T, spec.N, args.prec)
    if dname in ("dct_axis", "dct_tcgen05"):
        M = spec.N
        flops = 2.0 * M * (spec.T + 1) * spec.N ** spec.D * (3 if dname == "dct_tcgen05" else 1)
        tf32_peak = peaks.get("bf16_tflops_sustained", 1700.0) * (1.1 / 2.25)
        achieved = flops / (per_launch_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": tf32_peak, "unit": "TFLOP/s",
                "frac": achieved / tf32_peak, "traffic": None, "kernel": dname,
                "peak_source": f"{peak_src} bf16 sustained x tf32/bf16 nominal ratio 1.1/2.25"}
    else:
        achieved = abytes / (per_launch_ms / 1e3) / 1e9
        hbm = peaks.get("hbm_gbs", 6800.0)
        traffic, traffic_src = stored_traffic(dname, wl, args.prec)
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": traffic, "traffic_source": traffic_src,
                "kernel": dname,
                "per_launch_ms": round(per_launch_ms, 5), "algorithmic_bytes": abytes,
                "peak_source": f"{peak_src} (of measured copy bandwidth)" if peak_src == "measured" else peak_src}

    kernels = {k: {"ms_total": round(v[0], 3), "launches": v[1],
                   "ms_per_launch": round(v[0] / max(v[1], 1), 5),
                   "GBps": (round(algorithmic_bytes(k, spec.D, spec.T, spec.N, args.prec)
                                  / (v[0] / max(v[1], 1) / 1e3) / 1e9, 1)
                            if algorithmic_bytes(k, spec.D, spec.T, spec.N, args.prec) > 0 and v[1] else None)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0]) if v[1]}

    # e2e through the public API with host buffers: create (H2D) -> solve -> get (D2H),
    # on the same instances as the timed steps (so the two numbers differ by the
    # end-to-end costs only)
    e2e_lat, e2e_iters = [], []
    h2d = d2h = 0
    n_e2e = args.steps if args.e2e_steps < 0 else args.e2e_steps
    for k in range(n_e2e):
        r0, r1, m = instance(k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = make_solver(spec, r0, r1, m, args.prec, check_every=args.check_every)
        s.dot_solve(args.tol, args.maxit)
        rho, mm, phi, obj, kk = s.dot_get()
        torch.cuda.synchronize()
        e2e_lat.append(time.perf_counter() - t0)
        e2e_iters.append(int(kk["iterations"]))
        s.close()
        h2d = r0.nbytes + r1.nbytes + (0 if m is None else m.size)
        d2h = rho.nbytes + sum(a.nbytes for a in mm) + phi.nbytes + 8 * 12
    e2e_value = world * len(e2e_lat) / sum(e2e_lat) if e2e_lat else None

    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.prec == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"{wl}: {WORKLOAD_DESCS[wl]}", "D": spec.D, "T": spec.T, "N": spec.N,
                   "tol": args.tol, "prec": args.prec, "check_every": args.check_every, "tau": 1.9,
                   "l2": "inputs larger than L2 (per-solve state > 129 MB)", "seeds": f"{base_seed}+step",
                   "parallelism": f"replicas{world}"},
        "iterations": iters, "eta_dot": etas, "objective": objs,
        "multilevel": ({"levels": args.multilevel, "coarse_tol": args.coarse_tol or "paper",
                        "iterations_per_level_finest_first": level_iters}
                       if args.multilevel > 0 else None),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "it_per_s": round(sum(iters) / (elapsed_ms / 1e3), 1),
        "clocks": clk, "gpu_launches": int(gpu_launches),
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "iterations": e2e_iters,
                "seeds": f"{base_seed}+step (the timed steps' instances)" if base_seed is not None else None},
        "roofline": roof, "kernels": kernels,
    }

    # FP64 path on the same GPU, same instance as step 0
    fp64_iters = None
    if not args.no_fp64 and args.prec == "mixed":
        r0, r1, m = instance(0)
        s = make_solver(spec, r0, r1, m, "fp64", check_every=args.check_every)
        s.dot_solve(args.tol, 20)          # warm the kernels
        s.close()
        s = make_solver(spec, r0, r1, m, "fp64", check_every=args.check_every)
        s.dot_profile(True)       # the FP64 path launches kernel by kernel either way
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = s.dot_solve(args.tol, args.fp64_maxit)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        kk = s.dot_kkt()
        fprof = s.dot_profile_read()
        s.close()
        fp64_iters = int(kk["iterations"])
        out["fp64"] = {"solves_per_s": (1.0 / dt) if rc == 0 else None, "seconds": round(dt, 3),
                       "iterations": fp64_iters, "eta_dot": kk["eta_dot"], "converged": rc == 0,
                       "ms_per_iter": round(dt * 1e3 / max(fp64_iters, 1), 3),
                       "objective": -2.0 * kk["primal_obj"] / spec.N ** spec.D,
                       "kernels": {k: {"ms_total": round(v[0], 1), "launches": v[1],
                                       "ms_per_launch": round(v[0] / v[1], 4)}
                                   for k, v in sorted(fprof.items(), key=lambda kv: -kv[1][0]) if v[1]}}
        if rc == 0:
            # the same instance on both paths (timed step 0 of the mixed run)
            out["mixed_vs_fp64"] = round(dt / (lat[0] / 1e3), 3)
            out["mixed_vs_fp64_instance"] = f"seed {base_seed}" if base_seed is not None else wl

    if not args.no_cpu and wl == WORKLOAD:
        out["cpu_baseline"] = cpu_baseline(fp64_iters or (iters[0] if iters else None), wl)
    print(json.dumps(out))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def oracle_seconds_per_iteration(n_iter: int, wl: str = WORKLOAD):
    """Time n_iter oracle iterations (plain FP64 C, OpenMP) on the workload's default instance."""
    import oracle as O
    from paper_2505_05424_gb300 import workloads as W
    O.build()
    spec, r0, r1, m = W.workload(wl)
    g = O.Grid(spec.D, spec.T, [spec.N] * spec.D)
    prob = O.Problem(g, r0, r1, m)
    st = O.State.zeros(g)
    t0 = time.perf_counter()
    for _ in range(n_iter):
        O.iterate(prob, st)
    return (time.perf_counter() - t0) / n_iter


def cpu_baseline(iters_per_solve, wl: str = WORKLOAD):
    cores = len(os.sched_getaffinity(0))
    spi = oracle_seconds_per_iteration(2, wl)
    val = (1.0 / (spi * iters_per_solve)) if iters_per_solve else None
    return {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"2 oracle iterations of {wl} ({spi:.2f} s/iteration, OpenMP on {cores} threads); "
                      f"solves/s = 1 / (s/iteration x {iters_per_solve} iterations to eta<=1e-6)"}


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    wl = args.workload
    iters = ORACLE_ITERS_PER_SOLVE.get(wl) if args.check_every == 10 else None
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable": "iterations-per-solve of the workload not recorded"}))
        return
    for _ in range(args.warmup):
        oracle_seconds_per_iteration(1, wl)
    per = [oracle_seconds_per_iteration(1, wl) for _ in range(args.steps)]
    spi = float(np.mean(per))
    cores = len(os.sched_getaffinity(0))
    val = 1.0 / (spi * iters)
    out = {"metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": spi * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"{wl}: {WORKLOAD_DESCS.get(wl, wl)}", "tol": args.tol},
           "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                            "sample": f"each step = 1 oracle iteration; solves/s = 1/(s/it x {iters})"},
           "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


SERVE_GRIDS = ((32, 16), (64, 32), (128, 32), (256, 64))


def serving_stream(n: int, rate: float, seed: int = 5005):
    """The first n requests of the seeded serving stream: (arrival s, N, T, seed, masked)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        N, T = SERVE_GRIDS[int(rng.integers(0, len(SERVE_GRIDS)))]
        out.append((t, N, T, 50000 + i, bool(rng.random() < 0.2)))
    return out


def run_serve(args):
    """Serve the stream through DotServer; latency = completion - submission."""
    import torch
    from paper_2505_05424_gb300 import workloads as W
    from paper_2505_05424_gb300 import _native
    from paper_2505_05424_gb300.solver import DotServer
    _native.build()
    _native.load()
    torch.cuda.init()
    reqs = serving_stream(args.serve, args.rate)
    inputs = [W.mixture_pair(W.GridSpec(2, T, N), sd, obstacles=m) for (_, N, T, sd, m) in reqs]
    # warm-up: one solve per grid (kernel attributes, graph capture paths)
    with DotServer() as srv:
        ids = [srv.submit(2, T, N, *W.mixture_pair(W.GridSpec(2, T, N), 7)[:2], tol=args.tol, maxit=40,
                          keep_fields=False) for (N, T) in SERVE_GRIDS]
        for i in ids:
            srv.wait(i)
    clocks = ClockSampler(0)
    srv = DotServer(multilevel=args.serve_multilevel, multilevel_min_nodes=args.serve_ml_min_nodes,
                    multilevel_masked=args.serve_ml_masked)
    clocks.start()
    t0 = time.perf_counter()
    ids = []
    for (ta, N, T, sd, m), (r0, r1, mask) in zip(reqs, inputs):
        dt = ta - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(srv.submit(2, T, N, r0, r1, mask=mask, tol=args.tol, maxit=args.serve_maxit, keep_fields=False))
    status = [srv.wait(i) for i in ids]
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    res = [srv.result(i) for i in ids]
    stats = srv.stats()
    srv.close()
    lat = np.array([r["times"][2] - r["times"][0] for r in res]) * 1e3
    qwait = np.array([r["times"][1] - r["times"][0] for r in res]) * 1e3
    t_first = min(r["times"][0] for r in res)
    t_last = max(r["times"][2] for r in res)
    per_grid = {}
    for (ta, N, T, sd, m), l, r in zip(reqs, lat, res):
        d = per_grid.setdefault(f"{N}^2x{T}", {"n": 0, "lat": [], "iters": []})
        d["n"] += 1
        d["lat"].append(float(l))
        d["iters"].append(int(r["kkt"]["iterations"]))
    for k, d in per_grid.items():
        d["p50_ms"] = float(np.percentile(d["lat"], 50))
        d["p99_ms"] = float(np.percentile(d["lat"], 99))
        d["mean_iters"] = float(np.mean(d["iters"]))
        del d["lat"], d["iters"]
    out = {"metric": "serving: solves/s and p50/p99 latency, seeded stream of mixed 2D grids, KKT<=1e-6",
           "value": round(len(ids) / (t_last - t_first), 4), "unit": "solves/s", "n_gpus": 1,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"serving stream, first {len(ids)} requests, Poisson arrivals at {args.rate}/s, "
                                  "grids uniform over 32^2x16, 64^2x32, 128^2x32, 256^2x64, 20% with rectangle "
                                  "obstacles, seeded mixtures (seed 50000+i)", "tol": args.tol,
                      "maxit": args.serve_maxit, "multilevel": args.serve_multilevel,
                      "multilevel_min_nodes": args.serve_ml_min_nodes,
                      "multilevel_masked": bool(args.serve_ml_masked),
                      "arrivals_span_s": round(reqs[-1][0], 3) if reqs else 0.0},
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "queue_p50": float(np.percentile(qwait, 50)), "queue_p99": float(np.percentile(qwait, 99))},
           "converged": int(sum(1 for s_ in status if s_ == 0)), "requests": len(ids),
           "wall_s": round(wall, 3), "per_grid": per_grid, "server": stats, "clocks": clk}
    print(json.dumps(out))


def main():
    args = parse()
    if args.profile_iters > 0:
        run_profile_case(args)
        return
    if args.serve > 0:
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
