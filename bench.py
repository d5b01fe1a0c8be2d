#!/usr/bin/env python3
"""EXCMG benchmark on one GB300: finest-grid unknowns/s of the complete EXCMG solve.

Headline workload (default): the mixed-precision solve of Poisson on [0,1]^3 with
1024 x 512 x 512 cells (hx = 1/1024, hy = hz = 1/512), u = r^(5/3), f = (40/9) r^(-1/3),
g = u; 8 grids from 8 x 4 x 4; CG tolerance 1e-9 on levels >= 2 (||f_h|| reading "lift"),
DSOLVE on the two coarsest; float32 inner CG with float64 iterative refinement on grids
of >= 2^21 nodes.  One step = one complete excmg_solve (all levels, extrapolation,
interpolation, CG) through the C-ABI.  The plain FP64 solve of the same workload is
timed beside it, and both errors are stated against the exact solution and against
the FP64 discretisation error (FP64 at tolerance 1e-13).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload c3|c2|c1|c4|c5] [--no-extras] [--no-cpu-baseline]

Prints one JSON line (rank 0).  value = finest-grid interior unknowns solved per second
summed over ranks (each rank solves its own copy: independent problems, weak scaling,
no collective on the data path).  e2e = the same metric through the C-ABI with f and g
in pinned host memory and u copied back to pinned host memory inside the timed region
(four ways of moving the data; the fastest reported, all listed).

--impl reference times the FP64 CPU oracle (the plain numpy restatement of the paper in
oracle/) on the host cores, each step a bounded sample of the same workload extrapolated
to the complete solve (the oracle's complete solve of the headline workload takes
minutes and ~25 GB), and prints the same JSON line with "impl": "reference".
"""
import os

# the CPU oracle baseline is timed single-threaded (numpy BLAS included)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_v] = "1"

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import multiprocessing  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1507_05063_gb300 import problems as P  # noqa: E402

METRIC = "EXCMG finest-grid unknowns/s at stated L2 error, mixed vs FP64; CG HBM GB/s"
WORKLOADS = {
    # name: (problem, L, N, N0, eps, eps_coarse, precision)
    "c3": ("r53", (1.0, 1.0, 1.0), (1024, 512, 512), (8, 4, 4), 1e-9, 1e-12, "mixed"),
    "c2": ("exp3", (1.0, 1.0, 1.0), (512, 256, 128), (8, 4, 2), 1e-9, 1e-12, "fp64"),
    "c1": ("sin3", (1.0, 1.0, 1.0), (32, 32, 32), (4, 4, 4), 1e-8, 1e-12, "fp64"),
}
DESCRIPTION = {
    "c3": "1024x512x512 cells on [0,1]^3 (hx=1/1024, hy=hz=1/512), u=r^(5/3), f=(40/9) r^(-1/3), "
          "g=u; 8 grids from 8x4x4; eps 1e-9 (levels>=2, ||f_h|| = ||b|| with the lift), DSOLVE "
          "direct on the two coarsest; MIXED: float32 CG inside float64 refinement on grids of "
          ">= 2^21 nodes",
    "c2": "512x256x128 cells on [0,1]^3 (hx=1/512, hy=1/256, hz=1/128), u=exp(x+y+z), f=3u, g=u; "
          "7 grids from 8x4x2; eps 1e-9 / DSOLVE direct",
    "c1": "32^3 cells on [0,1]^3, u=sin(pi x)sin(pi y)sin(pi z), f=-3pi^2 u, g=0; 4 grids from 4^3; "
          "eps 1e-8 / DSOLVE direct",
}

# Algorithmic bytes and float64 operations per node of one launch of each kernel kind
# (streams the method must move; halo re-reads excluded).  DP ops count FMA, MUL and
# ADD as one each: they take one issue slot of the FP64 pipe.
ALGO = {
    "spmv_f64": {"bytes": 32.0, "dp_ops": 16.0},     # r, p_old in; p, q out
    "update_f64": {"bytes": 48.0, "dp_ops": 3.0},    # x, p, r, q in; x, r out
    "spmv_f32": {"bytes": 16.0, "dp_ops": 0.0},
    "update_f32": {"bytes": 24.0, "dp_ops": 0.0},
    # u, f in; r out.  DP ops: per plane 12 (19-point C/T terms), per node 2 (combine),
    # 6 (twice the RHS), 1 (r), 1 (r.r), 1 (b.b; the lift terms only near the boundary)
    "residual": {"bytes": 24.0, "dp_ops": 23.0},
    # per fine node: ~4.4 FMA for the three quartic passes (odd positions only), ~1 for
    # the extrapolated lattice (separable corner sums + one FMA per grid-2h node)
    "exp_finite": {"bytes": 8.0 * (1 + 1 / 8 + 1 / 64), "dp_ops": 5.4},
    "init": {"bytes": 8.0, "dp_ops": 0.0},
    # MIXED refinement: u += e / s (u in and out, e in and zeroed): 8 + 4 + 8 + 4
    "correct": {"bytes": 24.0, "dp_ops": 1.0},
    "exp_true": {"bytes": 8.0 * (2 + 1 / 8), "dp_ops": 4.0},
    # persistent CG: per node and CG step (the two fused bodies above)
    "cg_f64": {"bytes": 80.0, "dp_ops": 19.0},
    "cg_f32": {"bytes": 40.0, "dp_ops": 0.0},
    "cg_cluster_f64": {"bytes": 0.0, "dp_ops": 25.0},
    "cg_cluster_f32": {"bytes": 0.0, "dp_ops": 0.0},
    "cg_resident_f64": {"bytes": 24.0, "dp_ops": 25.0},
    "dsolve": {"bytes": 24.0, "dp_ops": 72.0},
    "prolong_cmp": {"bytes": 8.0 * (1 + 1 / 8 + 1 / 64), "dp_ops": 3.0},
    # compact gradient: u in, three components out; the one-sided formulas, the
    # right-hand side and the Thomas sweeps of every line in three directions (per node
    # and direction: a difference, a product and an FMA forward, an FMA back)
    "grad": {"bytes": 32.0, "dp_ops": 12.0},
}
KERNEL_SYMBOL = {"spmv_f64": "k_dir_spmv_dot<double>", "update_f64": "k_update_dot<double>",
                 "spmv_f32": "k_dir_spmv_dot<float>", "update_f32": "k_update_dot<float>",
                 "residual": "k_residual", "exp_finite": "k_exp_finite", "init": "k_boundary_init",
                 "correct": "k_add_correction", "exp_true": "k_exp_true",
                 "cg_f64": "k_cg_persistent<double>",
                 "cg_f32": "k_cg_persistent<float> (tensor-copy staged)",
                 "cg_cluster_f64": "k_cg_cluster<double>", "cg_cluster_f32": "k_cg_cluster<float>",
                 "cg_resident_f64": "k_cg_resident", "dsolve": "k_dsolve",
                 "prolong_cmp": "k_prolong_cmp", "grad": "k_grad_x + k_grad_strided"}
KERNEL_SOURCE = {"spmv_f64": "cg_kernels.cu", "update_f64": "cg_kernels.cu",
                 "spmv_f32": "cg_kernels.cu", "update_f32": "cg_kernels.cu",
                 "residual": "cg_kernels.cu", "exp_finite": "transfer_kernels.cu",
                 "init": "transfer_kernels.cu", "correct": "cg_kernels.cu",
                 "exp_true": "transfer_kernels.cu", "cg_f64": "cg_kernels.cu",
                 "cg_f32": "cg_kernels.cu", "cg_cluster_f64": "cluster_cg.cu",
                 "cg_cluster_f32": "cluster_cg.cu", "cg_resident_f64": "resident_cg.cu",
                 "dsolve": "dsolve_kernels.cu", "prolong_cmp": "transfer_kernels.cu",
                 "grad": "grad_kernels.cu"}
# FP64 issue rate: 2 DFMA per clock per SM x 152 SMs x 2.07 GHz (maximum SM clock).
DP_PEAK_GOPS = 2 * 152 * 2.070


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash(fname):
    with open(os.path.join(ROOT, "paper_1507_05063_gb300", "csrc", fname), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def recorded_traffic(kind, workload):
    """Per-node DRAM bytes of a kernel on this workload from a committed ncu summary, if
    the kernel source is unchanged since (profiles/ncu_traffic.txt: kind workload
    bytes_per_node source_sha)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == kind and parts[1] == workload:
            if parts[3] == source_hash(KERNEL_SOURCE[kind]):
                return float(parts[2])
    return None


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.file.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def interior_unknowns(N):
    return (N[0] - 1) * (N[1] - 1) * (N[2] - 1)


def host_cpu():
    """The host's CPU model and logical core count, for the CPU baseline's record."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key, _, val = line.partition(":")
                if key.strip().lower() == "model name":
                    model = val.strip()
                    break
    except OSError:
        pass
    if model is None:  # Arm hosts list no model name in /proc/cpuinfo
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            model = next((ln.split(":", 1)[1].strip() for ln in out.splitlines()
                          if ln.lower().startswith("model name")), None)
        except (OSError, subprocess.SubprocessError):
            pass
    import platform
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


# ------------------------------------------------------------------------------------
# The FP64 CPU oracle as a timed baseline.  Its complete solve of the headline workload
# takes minutes and ~25 GB, so a bounded sample is timed and extrapolated: the oracle's
# own cascade on the coarse levels (run in full), and on the finest levels its
# EXP_finite, its CG routine's set-up (b, ||f_h||, r) and one CG step, timed on one grid
# and scaled by node count, times the per-level CG step counts of the oracle's complete
# solve (tests/golden/oracle_c3.txt, written by a script that runs only the oracle).
# ------------------------------------------------------------------------------------

def oracle_iters(wl):
    """Per-level CG step counts of the oracle's complete solve of the workload."""
    if wl != "c3":
        return None
    path = os.path.join(ROOT, "tests", "golden", "oracle_c3.txt")
    with open(path) as fh:
        for line in fh:
            if line.startswith("iters "):
                return [int(v) for v in line.split()[1].split(",")]
    raise RuntimeError("oracle_c3.txt holds no iteration counts")


def oracle_level_costs(wl, Ns):
    """Seconds of the oracle's EXP_finite onto the grid Ns (of the workload's box and
    problem), of its CG routine with zero steps (set-up) and with one step."""
    import oracle as O
    name, L = WORKLOADS[wl][0], WORKLOADS[wl][1]
    f, g, u = P.make_inputs(P.PROBLEMS[name], Ns)
    h = O.meshsizes(L, Ns)
    u2, u4 = np.ascontiguousarray(u[::2, ::2, ::2]), np.ascontiguousarray(u[::4, ::4, ::4])
    t0 = time.perf_counter()
    w = O.with_boundary(O.exp_finite(u2, u4), g)
    t_pro = time.perf_counter() - t0
    del u2, u4
    t0 = time.perf_counter()
    O.cg(w, f, h, 0.0, fixed_iters=0)
    t_set = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.cg(w, f, h, 0.0, fixed_iters=1)
    t_one = time.perf_counter() - t0
    return {"N": list(Ns), "nodes": int(np.prod([n + 1 for n in Ns])), "prolong_s": t_pro,
            "cg_setup_s": t_set, "cg_step_s": max(t_one - t_set, 0.0)}


def oracle_coarse_seconds(wl, k):
    """The oracle's complete cascade on the workload's levels 0 .. k (its own step
    counts), timed."""
    import oracle as O
    name, L, N, N0, eps, epsc, _ = WORKLOADS[wl]
    s = 2 ** (len(O.level_sizes(N, N0)) - 1 - k)
    Nk = tuple(n // s for n in N)
    f, g, _ = P.make_inputs(P.PROBLEMS[name], Nk)
    t0 = time.perf_counter()
    res = O.excmg(f, g, L, Nk, N0, eps=eps, eps_coarse=epsc, dsolve="dense", want_utilde=False)
    return time.perf_counter() - t0, res["iters"]


def oracle_estimate(wl, sample_level, coarse_upto):
    """Estimated seconds of the oracle's complete solve: levels 0 .. coarse_upto run in
    full; each finer level l costs (nodes_l / nodes_s) x (EXP_finite + CG set-up +
    iters_l x CG step) from the costs timed on grid `sample_level`."""
    import oracle as O
    name, L, N, N0, eps, epsc, _ = WORKLOADS[wl]
    sizes = O.level_sizes(N, N0)
    iters = oracle_iters(wl)
    t_coarse, it_coarse = oracle_coarse_seconds(wl, coarse_upto)
    c = oracle_level_costs(wl, sizes[sample_level])
    total = t_coarse
    per_level = []
    for l in range(coarse_upto + 1, len(sizes)):
        nodes = int(np.prod([n + 1 for n in sizes[l]]))
        sc = nodes / c["nodes"]
        t = sc * (c["prolong_s"] + c["cg_setup_s"] + iters[l] * c["cg_step_s"])
        per_level.append({"level": l, "N": list(sizes[l]), "iters": iters[l], "seconds": t})
        total += t
    return {"seconds": total, "coarse_seconds": t_coarse, "coarse_levels": coarse_upto + 1,
            "coarse_iters": it_coarse, "sample_costs": c, "extrapolated_levels": per_level,
            "iters": iters}


def _oracle_worker(args):
    wl, sample_level, coarse_upto = args
    return oracle_estimate(wl, sample_level, coarse_upto)["seconds"]


def oracle_all_cores(wl, sample_level, coarse_upto, procs):
    """The same estimate run in `procs` concurrent processes (every host core busy with
    its own copy of the sample): whole-host throughput = procs x unknowns / the mean
    estimated solve time under that load."""
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(procs) as pool:
        secs = pool.map(_oracle_worker, [(wl, sample_level, coarse_upto)] * procs)
    n = interior_unknowns(WORKLOADS[wl][2])
    return {"cores": procs, "value": procs * n / float(np.mean(secs)), "unit": "unknowns/s",
            "seconds_per_solve_mean": float(np.mean(secs))}


def cpu_baseline_c3(all_cores=True):
    est = oracle_estimate("c3", sample_level=7, coarse_upto=5)
    n = interior_unknowns(WORKLOADS["c3"][2])
    out = {"value": n / est["seconds"], "unit": "unknowns/s", "cores": 1, "kind": "oracle",
           "sample": "the FP64 oracle (numpy, one thread): its complete cascade on levels 0-5 "
                     "(8x4x4 .. 256x128x128) timed in full; on 1024x512x512 its EXP_finite, its CG "
                     "set-up (b, ||f_h||, r) and one CG step timed; levels 6-7 extrapolated by node "
                     "count to the per-level step counts of the oracle's complete solve "
                     "(tests/golden/oracle_c3.txt); DSOLVE dense",
           "estimated_solve_seconds": est["seconds"], "detail": est, "host": host_cpu()}
    if all_cores:
        procs = os.cpu_count() or 1
        ac = oracle_all_cores("c3", sample_level=6, coarse_upto=5, procs=procs)
        ac["sample"] = (f"{procs} concurrent copies of the same estimate, each timing its finest-level "
                        "costs on 512x256x256 (memory for one copy per core) and scaling them by node count")
        out["all_cores"] = ac
    return out


# ------------------------------------------------------------------------------------
# N ranks: independent replicas
# ------------------------------------------------------------------------------------

class Replicas:
    """The N ranks of a run: each solves its own copy of the workload (independent
    problems, no collective on the data path); they meet only at the barriers around the
    timed region and in the max of their times.  `dist` is torch.distributed (or None for
    one rank); the max travels in a float64 tensor on `device`."""

    def __init__(self, world, device, dist=None):
        self.world, self.device, self.dist = world, device, dist

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, v):
        if self.world == 1:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def rate(self, units_per_rank, steps, ms):
        """Whole-job throughput: the units all ranks processed over the slowest rank's time
        (ms, already the max over ranks)."""
        return units_per_rank * self.world * steps / (ms / 1e3)


# ------------------------------------------------------------------------------------
# --impl reference: the oracle, bounded samples
# ------------------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = args.workload if args.workload in WORKLOADS else "c3"
    name, L, N, N0, eps, epsc, prec = WORKLOADS[wl]
    n = interior_unknowns(N)
    steps_total = max(args.steps, 1) + max(args.warmup, 0)
    if wl == "c3":
        # each step a bounded sample: finest-level costs timed on a grid sized so that the
        # whole run takes a few minutes (the finest grid itself when the budget allows)
        budget = 150.0 / steps_total
        sample_level, coarse_upto = (7, 5) if budget >= 60 else ((6, 5) if budget >= 12 else (5, 4))
        kind = (f"each step: the oracle's cascade on levels 0-{coarse_upto} in full, its costs on a "
                f"finer level (EXP_finite, CG set-up, one CG step) timed on level {sample_level} and "
                f"extrapolated by node count to levels {coarse_upto + 1}-7 with the step counts of its "
                "complete solve (tests/golden/oracle_c3.txt)")
        est = lambda: oracle_estimate(wl, sample_level, coarse_upto)["seconds"]  # noqa: E731
    else:
        import oracle as O
        f, g, _ = P.make_inputs(P.PROBLEMS[name], N)
        kind = "each step: one complete oracle EXCMG solve of the workload"

        def est():
            t0 = time.perf_counter()
            O.excmg(f, g, L, N, N0, eps=eps, eps_coarse=epsc, dsolve="dense", want_utilde=False)
            return time.perf_counter() - t0
    for _ in range(max(args.warmup, 0)):
        est()
    t = sum(est() for _ in range(max(args.steps, 1)))
    value = n * max(args.steps, 1) / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (closed-form f, g on the host)",
            "config": {"workload": DESCRIPTION[wl], "unknowns": n},
            "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                             "sample": kind + " (numpy, float64, one thread)", "host": host_cpu()},
            "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------

def errors(uh, u):
    return {"L2_rms": float(np.sqrt(np.mean((uh - u) ** 2))), "Linf": float(np.max(np.abs(uh - u)))}


def timed_solves(X, torch, stream, k, fd, gd, L, N0, ws, ud, **opts):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    res = None
    launches = 0
    for _ in range(k):
        res = X.solve(fd, gd, L, N0, ws=ws, out=ud, **opts)
        launches += res["stats"]["launches"]
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b), res, launches


def kernel_table(prof, hbm_peak):
    total = sum(v["ms"] for v in prof.values())
    kernels = {}
    for kind, v in prof.items():
        a = ALGO[kind]
        t = v["ms"] / 1e3
        gbs = a["bytes"] * v["nodes"] / t / 1e9 if t > 0 else 0.0
        gops = a["dp_ops"] * v["nodes"] / t / 1e9 if t > 0 else 0.0
        t_hbm = a["bytes"] / (hbm_peak * 1e9)
        t_alu = a["dp_ops"] / (DP_PEAK_GOPS * 1e9)
        kernels[kind] = {"share": v["ms"] / total if total else 0.0, "ms": v["ms"],
                         "launches": v["launches"], "avg_launch_us": 1e3 * v["ms"] / v["launches"],
                         "GB_s": gbs, "Gdpop_s": gops, "bound": "alu" if t_alu > t_hbm else "hbm"}
    return kernels


def roofline_of(kind, k, prof, hbm_peak, peak_kind, workload):
    nodes_per_launch = prof[kind]["nodes"] / prof[kind]["launches"]
    traffic = recorded_traffic(kind, workload)
    if k["bound"] == "alu":
        roof = {"bound": "alu", "achieved": k["Gdpop_s"], "peak": DP_PEAK_GOPS, "unit": "G DP-op/s",
                "frac": k["Gdpop_s"] / DP_PEAK_GOPS,
                "peak_source": "derived: 2 FP64 FMA per clock per SM x 152 SMs x 2.07 GHz"}
    else:
        roof = {"bound": "hbm", "achieved": k["GB_s"], "peak": hbm_peak, "unit": "GB/s",
                "frac": k["GB_s"] / hbm_peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    roof.update({"kernel": KERNEL_SYMBOL[kind], "share_of_step": k["share"],
                 "traffic": traffic * nodes_per_launch if traffic is not None else None,
                 "algorithmic_bytes_per_launch": ALGO[kind]["bytes"] * nodes_per_launch,
                 "dp_ops_per_launch": ALGO[kind]["dp_ops"] * nodes_per_launch,
                 "avg_launch_us": k["avg_launch_us"],
                 "timing": "CUDA events around every launch on the solve's stream, in a profiled "
                           "repeat of the step after the timed region"})
    return roof


def e2e_modes(X, torch, args, stream, f, g, L, N0, ws, fd, uh_ref, opts, ranks):
    """The headline metric through the C-ABI with host buffers, four ways."""
    f_pin = torch.from_numpy(f).pin_memory()
    g_pin = torch.from_numpy(g).pin_memory()
    u_pins = [torch.empty(f.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    fd2, gd2 = torch.empty_like(fd), torch.empty_like(fd)
    ud_pair = [torch.empty_like(fd), torch.empty_like(fd)]
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = args.steps

    def region(body):
        ranks.barrier()
        torch.cuda.synchronize()
        e2.record(stream)
        body()
        e3.record(stream)
        torch.cuda.synchronize()
        ranks.barrier()
        return ranks.max(e2.elapsed_time(e3))

    def copy_then_solve():
        for _ in range(K):
            fd2.copy_(f_pin, non_blocking=True)
            gd2.copy_(g_pin, non_blocking=True)
            X.solve(fd2, gd2, L, N0, ws=ws, out=ud_pair[0], **opts)
            u_pins[0].copy_(ud_pair[0], non_blocking=True)
    ms_copy = region(copy_then_solve)
    assert np.array_equal(u_pins[0].numpy(), uh_ref), "e2e solution differs from the device-resident one"

    def in_place():
        for _ in range(K):
            X.solve(f_pin, g_pin, L, N0, ws=ws, out=ud_pair[0], **opts)
            u_pins[0].copy_(ud_pair[0], non_blocking=True)
    u_pins[0].zero_()
    ms_zc = region(in_place)
    assert np.array_equal(u_pins[0].numpy(), uh_ref), "in-place solution differs"

    copy_stream, up_stream = torch.cuda.Stream(), torch.cuda.Stream()

    def in_place_pipelined():
        solved = [torch.cuda.Event(), torch.cuda.Event()]
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        for k in range(K):
            b = k % 2
            if k >= 2:
                stream.wait_event(copied[b])  # the copy of step k - 2 has left ud_pair[b]
            X.solve(f_pin, g_pin, L, N0, ws=ws, out=ud_pair[b], **opts)
            solved[b].record(stream)
            copy_stream.wait_event(solved[b])
            with torch.cuda.stream(copy_stream):
                u_pins[b].copy_(ud_pair[b], non_blocking=True)
            copied[b].record(copy_stream)
        for b in range(min(2, K)):
            stream.wait_event(copied[b])
    for t in u_pins:
        t.zero_()
    ms_pipe = region(in_place_pipelined)
    for b in range(min(2, K)):
        assert np.array_equal(u_pins[b].numpy(), uh_ref), "pipelined solution differs"

    fd_pair, gd_pair = [fd2, torch.empty_like(fd)], [gd2, torch.empty_like(fd)]

    def copy_pipelined():
        solved = [torch.cuda.Event(), torch.cuda.Event()]
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        uploaded = [torch.cuda.Event(), torch.cuda.Event()]
        for ev in solved + copied:
            ev.record(stream)

        def upload(k):
            b = k % 2
            up_stream.wait_event(solved[b])  # step k - 2 is done with these buffers
            with torch.cuda.stream(up_stream):
                fd_pair[b].copy_(f_pin, non_blocking=True)
                gd_pair[b].copy_(g_pin, non_blocking=True)
            uploaded[b].record(up_stream)
        upload(0)
        for k in range(K):
            b = k % 2
            if k + 1 < K:
                upload(k + 1)
            stream.wait_event(uploaded[b])
            stream.wait_event(copied[b])
            X.solve(fd_pair[b], gd_pair[b], L, N0, ws=ws, out=ud_pair[b], **opts)
            solved[b].record(stream)
            copy_stream.wait_event(solved[b])
            with torch.cuda.stream(copy_stream):
                u_pins[b].copy_(ud_pair[b], non_blocking=True)
            copied[b].record(copy_stream)
        for b in range(min(2, K)):
            stream.wait_event(copied[b])
    for t in u_pins:
        t.zero_()
    ms_cpipe = region(copy_pipelined)
    for b in range(min(2, K)):
        assert np.array_equal(u_pins[b].numpy(), uh_ref), "copy-pipelined solution differs"

    def copy_f_pipelined():
        # as copy_pipelined, but only f is uploaded: g stays in page-locked host memory,
        # where the solve reads nothing but its boundary nodes (the Dirichlet data of each
        # level)
        solved = [torch.cuda.Event(), torch.cuda.Event()]
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        uploaded = [torch.cuda.Event(), torch.cuda.Event()]
        for ev in solved + copied:
            ev.record(stream)

        def upload(k):
            b = k % 2
            up_stream.wait_event(solved[b])
            with torch.cuda.stream(up_stream):
                fd_pair[b].copy_(f_pin, non_blocking=True)
            uploaded[b].record(up_stream)
        upload(0)
        for k in range(K):
            b = k % 2
            if k + 1 < K:
                upload(k + 1)
            stream.wait_event(uploaded[b])
            stream.wait_event(copied[b])
            X.solve(fd_pair[b], g_pin, L, N0, ws=ws, out=ud_pair[b], **opts)
            solved[b].record(stream)
            copy_stream.wait_event(solved[b])
            with torch.cuda.stream(copy_stream):
                u_pins[b].copy_(ud_pair[b], non_blocking=True)
            copied[b].record(copy_stream)
        for b in range(min(2, K)):
            stream.wait_event(copied[b])
    for t in u_pins:
        t.zero_()
    ms_fpipe = region(copy_f_pipelined)
    for b in range(min(2, K)):
        assert np.array_equal(u_pins[b].numpy(), uh_ref), "f-copy-pipelined solution differs"
    # boundary nodes of every level (each level reads the Dirichlet data at its own nodes)
    n_bnd_levels, Nl = 0, [f.shape[2] - 1, f.shape[1] - 1, f.shape[0] - 1]
    while all(a >= b for a, b in zip(Nl, N0)):
        n_bnd_levels += (Nl[0] + 1) * (Nl[1] + 1) * (Nl[2] + 1) - (Nl[0] - 1) * (Nl[1] - 1) * (Nl[2] - 1)
        Nl = [a // 2 for a in Nl]
    modes = {"copy": {"ms_per_step": ms_copy / K, "h2d_bytes_per_step": f.nbytes + g.nbytes,
                      "how": "f and g copied to the device (cudaMemcpyAsync), then the solve"},
             "in_place": {"ms_per_step": ms_zc / K, "h2d_bytes_per_step": f.nbytes + 8 * n_bnd_levels,
                          "how": "the solve reads f and g's boundary from page-locked host memory"},
             "in_place_pipelined": {"ms_per_step": ms_pipe / K, "h2d_bytes_per_step": f.nbytes + 8 * n_bnd_levels,
                                    "how": "as in_place; step i's solution is copied back on a second "
                                           "stream while step i + 1 solves"},
             "copy_pipelined": {"ms_per_step": ms_cpipe / K, "h2d_bytes_per_step": f.nbytes + g.nbytes,
                                "how": "f and g copied to the device on an upload stream while the "
                                       "previous step solves; the solution copied back on a download "
                                       "stream while the next step solves"},
             "copy_f_pipelined": {"ms_per_step": ms_fpipe / K, "h2d_bytes_per_step": f.nbytes + 8 * n_bnd_levels,
                                  "how": "as copy_pipelined, but only f is copied: the solve reads g's "
                                         "boundary nodes (each level's Dirichlet data) from page-locked "
                                         "host memory"}}
    best = min(modes, key=lambda k: modes[k]["ms_per_step"])
    n_unk = interior_unknowns((f.shape[2] - 1, f.shape[1] - 1, f.shape[0] - 1))
    ms = modes[best]["ms_per_step"] * K
    return {"value": ranks.rate(n_unk, K, ms), "unit": "unknowns/s",
            "h2d_bytes_per_step": modes[best]["h2d_bytes_per_step"], "d2h_bytes_per_step": f.nbytes,
            "ms_per_step": ms / K, "mode": best, "modes": modes}


def cg_rates(X, torch, wl, hbm_peak, steps=20):
    """Finest-grid CG step rates: `steps` fixed float64 steps (the persistent engine) and
    one float32 inner solve of `steps` steps (the tensor-copy engine), profiled."""
    name, L, N = WORKLOADS[wl][0], WORKLOADS[wl][1], WORKLOADS[wl][2]
    f, g, _ = P.make_inputs(P.PROBLEMS[name], N)
    fd = torch.from_numpy(f).cuda()
    u0 = torch.from_numpy(g).cuda()
    u0[1:-1, 1:-1, 1:-1] = 0.0
    out = {}
    for prec in ("mixed", "fp64"):
        best = None
        for _ in range(3):
            u = u0.clone()
            if prec == "fp64":
                st = X.cg(fd, u, L, eps=0.0, fixed_iters=[steps], profile=1)
            else:
                st = X.cg(fd, u, L, precision="mixed", mixed_min_nodes=1, eps=1e-300, inner_tol=1e-30,
                          max_iter=steps, max_refine=1, profile=1, allow_not_converged=True)
            kind = "cg_f64" if prec == "fp64" else "cg_f32"
            pr = st["profile"][kind]
            if best is None or pr["ms"] < best[0]:
                best = (pr["ms"], pr["nodes"], st["iters"][0], kind)
        ms, node_steps, it, kind = best
        t_it = ms / it
        nodes = node_steps / it
        byt = ALGO[kind]["bytes"] * nodes
        r = {"kernel": KERNEL_SYMBOL[kind], "steps": it, "ms_per_iter": t_it,
             "unknown_iters_per_s": nodes / (t_it / 1e3), "bytes_per_unknown_iter": ALGO[kind]["bytes"],
             "GB_s": byt / (t_it / 1e3) / 1e9, "frac_hbm": byt / (t_it / 1e3) / 1e9 / hbm_peak}
        if prec == "fp64":
            r["Gdpop_s"] = ALGO[kind]["dp_ops"] * nodes / (t_it / 1e3) / 1e9
            r["frac_alu"] = r["Gdpop_s"] / DP_PEAK_GOPS
        out[prec] = r
    del fd, u0
    return out


def utilde_grad_rates(X, torch, u_dev, L, hbm_peak, reps=5):
    """EXP_true (u~_h from u_h and u_2h) and the compact gradient on the headline grid,
    timed with CUDA events over `reps` launches each (the solution's coarse grid is
    stood in for by u_h at the coarse nodes: the kernels' cost does not depend on the
    values)."""
    N = (u_dev.shape[2] - 1, u_dev.shape[1] - 1, u_dev.shape[0] - 1)
    nodes = float(u_dev.numel())
    u2 = u_dev[::2, ::2, ::2].contiguous()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for kind, fn in (("exp_true", lambda: X.exp_true(u_dev, u2, L)), ("grad", lambda: X.grad(u_dev, L))):
        fn()
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            r = fn()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        del r
        gbs = ALGO[kind]["bytes"] * nodes / (ms / 1e3) / 1e9
        gops = ALGO[kind]["dp_ops"] * nodes / (ms / 1e3) / 1e9
        out[kind] = {"kernel": KERNEL_SYMBOL[kind], "ms_per_call": ms, "nodes": nodes,
                     "bytes_per_node": ALGO[kind]["bytes"], "dp_ops_per_node": ALGO[kind]["dp_ops"],
                     "GB_s": gbs, "frac_hbm": gbs / hbm_peak, "Gdpop_s": gops, "frac_alu": gops / DP_PEAK_GOPS,
                     "grid": list(N), "timing": "CUDA events, includes the call's closing synchronisation"}
    return out


def extra_c2(X, torch, stream, hbm_peak, cg_finest):
    """The 512x256x128 workload: FP64 and MIXED solves (after their tuning pass), the
    finest-grid CG step rates, per-level tolerance, and the prolongation ablation (what
    EXP_finite saves)."""
    name, L, N, N0, eps, epsc, _ = WORKLOADS["c2"]
    f, g, u = P.make_inputs(P.PROBLEMS[name], N)
    fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    ud = torch.empty_like(fd)
    n = interior_unknowns(N)
    out = {"workload": DESCRIPTION["c2"], "unknowns": n}
    for prec in ("fp64", "mixed"):
        kw = dict(eps=eps, eps_coarse=epsc, precision=prec)
        ws = X.workspace(X.solve_workspace_bytes(L, N, N0, **kw), fd.device)
        X.solve(fd, gd, L, N0, ws=ws, out=ud, autotune=1, **kw)
        # the float32 engine's shapes for this grid: a MIXED tuning solve with float32 CG
        # on every level from 2 up
        X.solve(fd, gd, L, N0, out=ud, autotune=1, precision="mixed", mixed_min_nodes=1, eps=eps,
                eps_coarse=epsc)
        for _ in range(3):
            X.solve(fd, gd, L, N0, ws=ws, out=ud, **kw)
        ms, res, _ = timed_solves(X, torch, stream, 10, fd, gd, L, N0, ws, ud, **kw)
        out[prec] = {"value": n / (ms / 10 / 1e3), "ms_per_step": ms / 10,
                     "iters_per_level": res["stats"]["iters"],
                     "refinements_per_level": res["stats"]["refinements"],
                     "error_vs_exact": errors(ud.cpu().numpy(), u)}
    tol = {}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for tag, kw in (("uniform_1e-9", dict(eps=eps)), ("uniform_1e-13", dict(eps=1e-13)),
                    ("per_level_1e-13_x4", dict(eps=1e-13, eps_ratio=4.0)),
                    ("per_level_1e-13_x16", dict(eps=1e-13, eps_ratio=16.0)),
                    ("per_level_1e-13_x64", dict(eps=1e-13, eps_ratio=64.0))):
        o2 = dict(eps_coarse=epsc, precision="fp64", **kw)
        X.solve(fd, gd, L, N0, out=ud, want_utilde=True, **o2)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(3):
            r2 = X.solve(fd, gd, L, N0, out=ud, want_utilde=True, **o2)
        b.record(stream)
        torch.cuda.synchronize()
        uh2, ut2 = ud.cpu().numpy(), r2["ut"].cpu().numpy()
        tol[tag] = {"ms_per_solve": a.elapsed_time(b) / 3, "iters_per_level": r2["stats"]["iters"],
                    "u_Linf": float(np.max(np.abs(uh2 - u))), "u_tilde_Linf": float(np.max(np.abs(ut2 - u)))}
    out["tolerance_per_level"] = tol
    if "512x256x128" not in cg_finest:
        cg_finest["512x256x128"] = cg_rates(X, torch, "c2", hbm_peak)
    abl = {}
    for kind in ("quartic", "quadratic", "linear"):
        o2 = dict(eps=eps, eps_coarse=epsc, precision="fp64", prolong=kind)
        X.solve(fd, gd, L, N0, out=ud, **o2)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(3):
            r2 = X.solve(fd, gd, L, N0, out=ud, **o2)
        b.record(stream)
        torch.cuda.synchronize()
        abl[kind] = {"ms_per_solve": a.elapsed_time(b) / 3, "iters_per_level": r2["stats"]["iters"],
                     "u_Linf": float(np.max(np.abs(ud.cpu().numpy() - u)))}
    out["prolong_ablation"] = abl
    return out


def extra_c1(X, torch, stream):
    name, L, N, N0, eps, epsc, _ = WORKLOADS["c1"]
    f, g, u = P.make_inputs(P.PROBLEMS[name], N)
    fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    ud = torch.empty_like(fd)
    kw = dict(eps=eps, eps_coarse=epsc, precision="fp64")
    ws = X.workspace(X.solve_workspace_bytes(L, N, N0, **kw), fd.device)
    for _ in range(3):
        X.solve(fd, gd, L, N0, ws=ws, out=ud, **kw)
    ms, res, _ = timed_solves(X, torch, stream, 50, fd, gd, L, N0, ws, ud, **kw)
    r = X.solve(fd, gd, L, N0, ws=ws, out=ud, want_utilde=True, **kw)
    gx, gy, gz = (t.cpu().numpy() for t in X.grad(ud, L))
    ex, ey, ez = P.exact_gradient(P.PROBLEMS[name], N)
    ge = max(float(np.max(np.abs(gx - ex))), float(np.max(np.abs(gy - ey))), float(np.max(np.abs(gz - ez))))
    return {"workload": DESCRIPTION["c1"], "value": interior_unknowns(N) / (ms / 50 / 1e3),
            "ms_per_step": ms / 50, "iters_per_level": res["stats"]["iters"],
            "error_vs_exact": errors(ud.cpu().numpy(), u),
            "u_tilde_Linf": float(np.max(np.abs(r["ut"].cpu().numpy() - u))), "grad_Linf": ge}


def run_batched(X, torch, reps=2):
    """64 independent problems (sizes from {32,64,128,256}^3 cells, random aspect,
    trig-sum right-hand sides, seed 20151507), solved together by excmg_solve_batched and
    one after another by excmg_solve, FP64 and MIXED, at the same tolerance.  value =
    interior unknowns of all problems per second."""
    seed, nprob, eps = 20151507, 64, 1e-8
    grids = P.batched_grids(nprob, seed)
    probs, n_unk = [], 0
    for i, (L, N, N0) in enumerate(grids):
        f, g, u = P.make_inputs(P.trig_sum(seed + i, K=8, L=L), N, L)
        probs.append((L, N, N0, f, g, u))
        n_unk += interior_unknowns(N)
    fds = [torch.from_numpy(p[3]).cuda() for p in probs]
    gds = [torch.from_numpy(p[4]).cuda() for p in probs]
    batch = [X.BatchedProblem(L, N, N0, fd, gd) for (L, N, N0, _, _, _), fd, gd in zip(probs, fds, gds)]
    out = {"workload": "64 problems, sizes {32,64,128,256}^3 cells drawn per direction, h_d in {1/N, 2/N}, "
                       "trig-sum f (K=8), g=0, seed 20151507; eps 1e-8, eps_coarse 1e-10",
           "n_problems": nprob, "unknowns": n_unk, "sizes": [list(p[1]) for p in probs]}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def err(us):
        return max(float(np.max(np.abs(uu.cpu().numpy() - p[5]))) / max(float(np.max(np.abs(p[5]))), 1e-300)
                   for uu, p in zip(us, probs))
    for prec in ("fp64", "mixed"):
        kw = dict(eps=eps, eps_coarse=1e-10, precision=prec)
        res = X.solve_batched(batch, **kw)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            res = X.solve_batched(batch, **kw)
        b.record()
        torch.cuda.synchronize()
        ms_b = a.elapsed_time(b) / reps
        # the same problems one by one (one workspace, sized for the largest)
        need = max(X.solve_workspace_bytes(p[0], p[1], p[2], **kw) for p in probs)
        ws = X.workspace(need, fds[0].device)
        outs = [torch.empty_like(fd) for fd in fds]
        for (L, N, N0, _, _, _), fd, gd, uo in zip(probs, fds, gds, outs):
            X.solve(fd, gd, L, N0, ws=ws, out=uo, **kw)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            for (L, N, N0, _, _, _), fd, gd, uo in zip(probs, fds, gds, outs):
                X.solve(fd, gd, L, N0, ws=ws, out=uo, **kw)
        b.record()
        torch.cuda.synchronize()
        ms_s = a.elapsed_time(b) / reps
        out[prec] = {"batched": {"value": n_unk / (ms_b / 1e3), "ms_per_batch": ms_b, "status": res["status"],
                                 "max_rel_err_vs_exact": err(res["u"])},
                     "sequential": {"value": n_unk / (ms_s / 1e3), "ms_per_batch": ms_s,
                                    "max_rel_err_vs_exact": err(outs)}}
        del ws, outs
    out["batched_over_sequential"] = {p: out[p]["sequential"]["ms_per_batch"] / out[p]["batched"]["ms_per_batch"]
                                      for p in ("fp64", "mixed")}
    return out


def run_adjoint(X, torch, steps=3):
    """Source recovery on a 256^3 cube (a sample of the 20-step run): L = ||u(f) - u_t||^2,
    u_t the solution for a seeded trig-sum source; `steps` gradient steps on f with dL/df
    from excmg_adjoint through torch.autograd and an exact line search (L is quadratic in
    f); FP64 and MIXED; seconds per step."""
    from paper_1507_05063_gb300.autograd import excmg_solve
    torch.cuda.empty_cache()  # the larger workloads' cached blocks
    N, N0, L = (256, 256, 256), (4, 4, 4), (1.0, 1.0, 1.0)
    ft, g, _ = P.make_inputs(P.trig_sum(20150705, K=8), N)
    gd = torch.from_numpy(g).cuda()
    out = {"workload": "adjoint source recovery on 256^3 (trig-sum target, seed 20150705), eps 1e-10",
           "steps": steps}
    for prec in ("fp64", "mixed"):
        # one workspace for every solve of the loop (the adjoint sizes its own)
        ws = X.workspace(X.solve_workspace_bytes(L, N, N0, eps=1e-10, eps_coarse=1e-12, precision=prec),
                         gd.device)
        kw = dict(eps=1e-10, eps_coarse=1e-12, precision=prec, ws=ws)
        ut = X.solve(torch.from_numpy(ft).cuda(), gd, L, N0, **kw)["u"]
        # one untimed forward and backward: the allocator's first requests of this size
        fw = torch.zeros_like(ut).requires_grad_(True)
        ((excmg_solve(fw, gd, L, N0, **kw) - ut) ** 2).sum().backward()
        del fw
        torch.cuda.synchronize()
        f = torch.zeros_like(ut)
        losses, t_fwd, t_adj = [], 0.0, 0.0
        t0 = time.perf_counter()
        for _ in range(steps):
            f.requires_grad_(True)
            a = time.perf_counter()
            u = excmg_solve(f, gd, L, N0, **kw)
            loss = ((u - ut) ** 2).sum()
            torch.cuda.synchronize()
            t_fwd += time.perf_counter() - a
            a = time.perf_counter()
            loss.backward()
            torch.cuda.synchronize()
            t_adj += time.perf_counter() - a
            d = f.grad.detach()
            with torch.no_grad():
                Jd = X.solve(d, gd, L, N0, **kw)["u"] - X.solve(torch.zeros_like(d), gd, L, N0, **kw)["u"]
                t = float(((u - ut).detach() * Jd).sum() / (Jd * Jd).sum())
                f = f.detach() - t * d
            losses.append(float(loss.detach()))
        total = time.perf_counter() - t0
        out[prec] = {"losses": losses, "monotone": all(b < a for a, b in zip(losses, losses[1:])),
                     "seconds_per_step": total / steps, "seconds_forward": t_fwd / steps,
                     "seconds_adjoint": t_adj / steps}
    return out


def _setup_gpu():
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05063_gb300 import excmg as X
    return torch, X


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS) + ["c4", "c5"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other configurations")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload in ("c4", "c5"):
        torch, X = _setup_gpu()
        print(json.dumps(run_batched(X, torch) if args.workload == "c4" else run_adjoint(X, torch, 20)),
              flush=True)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05063_gb300 import excmg as X

    wl = args.workload
    name, L, N, N0, eps, epsc, prec = WORKLOADS[wl]
    f, g, u_exact = P.make_inputs(P.PROBLEMS[name], N)
    n_unk = interior_unknowns(N)
    fd = torch.from_numpy(f).to(device)
    gd = torch.from_numpy(g).to(device)
    ud = torch.empty_like(fd)
    opts = dict(eps=eps, eps_coarse=epsc, precision=prec)
    ws = X.workspace(X.solve_workspace_bytes(L, N, N0, **opts), device)
    stream = torch.cuda.current_stream()
    ranks = Replicas(world, device, dist if world > 1 else None)

    # the launch-shape tuning pass (options.autotune = 1) for both precisions' levels, once;
    # every later solve uses its cache
    other = "fp64" if prec == "mixed" else "mixed"
    o_opts = dict(opts, precision=other)
    ws_o = X.workspace(X.solve_workspace_bytes(L, N, N0, **o_opts), device)
    uo = torch.empty_like(fd)
    X.solve(fd, gd, L, N0, ws=ws, out=ud, autotune=1, **opts)
    X.solve(fd, gd, L, N0, ws=ws_o, out=uo, autotune=1, **o_opts)
    for _ in range(max(args.warmup, 0)):
        X.solve(fd, gd, L, N0, ws=ws, out=ud, **opts)

    # ---- timed region: inputs resident in HBM (each finest array >= 136 MB > 129 MB L2)
    clocks = Clocks(local)
    ranks.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # an NVTX range around the timed solves, so that a profiler can capture them alone
    # (ncu --nvtx --nvtx-include "excmg_timed/")
    torch.cuda.nvtx.range_push("excmg_timed")
    ms, res, launches = timed_solves(X, torch, stream, args.steps, fd, gd, L, N0, ws, ud, **opts)
    torch.cuda.nvtx.range_pop()
    ranks.barrier()
    clk = clocks.stop()
    ms = ranks.max(ms)
    stats = res["stats"]
    value = ranks.rate(n_unk, args.steps, ms)
    uh = ud.cpu().numpy()
    err = errors(uh, u_exact)

    # ---- profiled repeat (events around every launch; not the timed region) and the
    # finest-grid CG step rates, in the memory state of the timed region
    prof = X.solve(fd, gd, L, N0, ws=ws, out=ud, profile=1, **opts)["stats"]["profile"]
    hbm_peak, peak_kind = load_peaks()
    cg_finest = {}
    if not args.no_extras and wl in ("c3", "c2"):
        try:
            cg_finest[{"c3": "1024x512x512", "c2": "512x256x128"}[wl]] = cg_rates(X, torch, wl, hbm_peak)
        except Exception as ex:  # keep the line; record what failed
            cg_finest["error"] = repr(ex)

    # ---- the other precision at the same tolerance, and the discretisation error
    for _ in range(2):
        X.solve(fd, gd, L, N0, ws=ws_o, out=uo, **o_opts)
    k_o = max(3, args.steps // 4)
    ms_o, res_o, _ = timed_solves(X, torch, stream, k_o, fd, gd, L, N0, ws_o, uo, **o_opts)
    ms_o = ranks.max(ms_o)
    err_o = errors(uo.cpu().numpy(), u_exact)
    del ws_o
    r13 = X.solve(fd, gd, L, N0, out=uo, eps=1e-13, eps_coarse=1e-13, precision="fp64")
    err_disc = errors(uo.cpu().numpy(), u_exact)
    mixed_err, fp64_err = (err, err_o) if prec == "mixed" else (err_o, err)
    accuracy = {
        "eps": eps, "rhs_norm": "lift",
        "mixed": mixed_err, "fp64": fp64_err,
        "fp64_eps_1e-13": dict(err_disc, iters_per_level=r13["stats"]["iters"],
                               note="FP64 at tolerance 1e-13: the discretisation error of the scheme"),
        "mixed_over_fp64_same_eps": {k: mixed_err[k] / fp64_err[k] for k in mixed_err},
        "mixed_over_discretisation": {k: mixed_err[k] / err_disc[k] for k in mixed_err},
        "fp64_over_discretisation": {k: fp64_err[k] / err_disc[k] for k in fp64_err}}
    # equal error at the discretisation level: both precisions at tolerance 1e-13
    tight = {"eps": 1e-13}
    for p_ in ("mixed", "fp64"):
        kw = dict(eps=1e-13, eps_coarse=1e-13, precision=p_)
        ws_t = X.workspace(X.solve_workspace_bytes(L, N, N0, **kw), device)
        X.solve(fd, gd, L, N0, ws=ws_t, out=uo, **kw)
        ms_t, res_t, _ = timed_solves(X, torch, stream, 2, fd, gd, L, N0, ws_t, uo, **kw)
        e_t = errors(uo.cpu().numpy(), u_exact)
        tight[p_] = {"value": n_unk / (ms_t / 2 / 1e3), "ms_per_step": ms_t / 2, "error_vs_exact": e_t,
                     "iters_per_level": res_t["stats"]["iters"],
                     "refinements_per_level": res_t["stats"]["refinements"]}
        del ws_t
    tight["mixed_over_fp64_error"] = {k: tight["mixed"]["error_vs_exact"][k] / tight["fp64"]["error_vs_exact"][k]
                                      for k in err_disc}
    tight["mixed_speedup_over_fp64"] = tight["fp64"]["ms_per_step"] / tight["mixed"]["ms_per_step"]
    accuracy["equal_error_eps_1e-13"] = tight
    del uo

    # ---- end to end through the C-ABI with host buffers
    e2e = e2e_modes(X, torch, args, stream, f, g, L, N0, ws, fd, uh, opts, ranks)

    kernels = kernel_table(prof, hbm_peak)
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    roof = roofline_of(dom, kernels[dom], prof, hbm_peak, peak_kind, wl)
    roof_cg = roofline_of("cg_f32", kernels["cg_f32"], prof, hbm_peak, peak_kind, wl) if "cg_f32" in kernels else None

    line = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == "mixed" else "f64",
            "data": "synthetic (closed-form f, g evaluated on the host in float64)",
            "config": {"workload": DESCRIPTION[wl], "unknowns": n_unk, "grid": list(N),
                       "levels": stats["levels"], "iters_per_level": stats["iters"],
                       "refinements_per_level": stats["refinements"],
                       "relres_finest": stats["relres"][-1], "precision": prec,
                       "parallelism": f"{world} independent replica(s)",
                       "l2": "inputs larger than L2 (each finest-level array 2.2 GB > 129 MB L2)"},
            "accuracy": accuracy,
            other: {"value": ranks.rate(n_unk, k_o, ms_o), "ms_per_step": ms_o / k_o,
                    "iters_per_level": res_o["stats"]["iters"],
                    "refinements_per_level": res_o["stats"]["refinements"]},
            "mixed_speedup_over_fp64": ((ms_o / k_o) / (ms / args.steps)) if prec == "mixed"
            else ((ms / args.steps) / (ms_o / k_o)),
            "gpu_launches": launches, "clocks": clk, "roofline": roof, "roofline_cg_f32": roof_cg,
            "kernels": kernels, "e2e": e2e}
    del e2e

    if not args.no_extras:
        extras = {"cg_finest": cg_finest}
        try:
            extras["utilde_and_gradient"] = utilde_grad_rates(X, torch, ud, L, hbm_peak)
        except Exception as ex:
            extras["utilde_and_gradient"] = {"error": repr(ex)}
        del ws
        torch.cuda.empty_cache()
        for key, fn in (("c2", lambda: extra_c2(X, torch, stream, hbm_peak, cg_finest)),
                        ("c1", lambda: extra_c1(X, torch, stream)),
                        ("c4_batched", lambda: run_batched(X, torch)), ("c5_adjoint", lambda: run_adjoint(X, torch))):
            try:
                extras[key] = fn()
            except Exception as ex:
                extras[key] = {"error": repr(ex)}
            torch.cuda.empty_cache()
        line["extras"] = extras
    line["tuning"] = {"how": "options.autotune = 1 on the first solve of each workload and precision: "
                             "candidate slab depths per level timed with CUDA events, the fastest cached "
                             "per (level grid, engine class, device) and used by every later solve",
                      "levels": X.tuning_entries()}

    if rank == 0 and world == 1 and not args.no_cpu_baseline and wl == "c3":
        line["cpu_baseline"] = cpu_baseline_c3()
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        t0 = time.perf_counter()
        ores = O.excmg(f, g, L, N, N0, eps=eps, eps_coarse=epsc, dsolve="dense", want_utilde=False)
        secs = time.perf_counter() - t0
        uo_ = ores["u"][-1]
        line["cpu_baseline"] = {"value": n_unk / secs, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                                "sample": "one complete oracle EXCMG solve of the same workload "
                                          "(numpy float64, single thread)", "seconds": secs,
                                "iters_per_level": ores["iters"], "host": host_cpu(),
                                "gpu_vs_oracle_rel_linf": float(np.max(np.abs(uh - uo_)) / np.max(np.abs(uo_)))}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
