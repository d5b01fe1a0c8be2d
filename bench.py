#!/usr/bin/env python3
"""EXCMG benchmark: finest-grid unknowns/s of the FP64 EXCMG solve on one GB300.

Workload (default): Poisson on [0,1]^3 with 512 x 256 x 128 cells (hx = 1/512,
hy = 1/256, hz = 1/128), u = exp(x+y+z), f = 3u, g = u; 7 grids from 8 x 4 x 2; CG
tolerance 1e-9 on levels >= 2 and 1e-12 on the two coarsest; FP64.  One step = one
complete excmg_solve (all levels, extrapolation, interpolation, CG) through the C-ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  value = finest-grid interior unknowns solved per second
summed over ranks (each rank solves its own copy: independent problems, weak scaling,
no collective on the data path).  e2e = the same metric through the C-ABI with the
inputs in pinned host memory and the solution copied back to pinned host memory inside
the timed region; measured both with f and g copied to the device first and with the
solve reading them in place over the host link, the faster reported (both listed).
"""
import os

# the CPU oracle baseline is timed single-threaded
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_v] = "1"

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
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
    # name: (problem, L, N, N0, eps, eps_coarse)
    "c2": ("exp3", (1.0, 1.0, 1.0), (512, 256, 128), (8, 4, 2), 1e-9, 1e-12),
    "c1": ("sin3", (1.0, 1.0, 1.0), (32, 32, 32), (4, 4, 4), 1e-8, 1e-12),
    "c3": ("r53", (1.0, 1.0, 1.0), (1024, 512, 512), (8, 4, 4), 1e-9, 1e-12),
}
PRECISION = {"c1": "fp64", "c2": "fp64", "c3": "mixed"}
DESCRIPTION = {
    "c2": "FP64 EXCMG, [0,1]^3, 512x256x128 cells (hx=1/512, hy=1/256, hz=1/128), "
          "u=exp(x+y+z), f=3u, g=u; 7 grids from 8x4x2; eps 1e-9 (levels>=2), 1e-12 (two coarsest)",
    "c1": "FP64 EXCMG, [0,1]^3, 32^3 cells, u=sin(pi x)sin(pi y)sin(pi z), f=-3pi^2 u, g=0; "
          "4 grids from 4^3; eps 1e-8 / 1e-12",
    "c3": "MIXED EXCMG (float32 CG inside float64 refinement on grids of >= 2^21 nodes), "
          "[0,1]^3, 1024x512x512 cells, u=r^(5/3), f=(40/9) r^(-1/3), g=u; "
          "8 grids from 8x4x4; eps 1e-9 / 1e-12",
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
    "correct": {"bytes": 24.0, "dp_ops": 1.0},
    "exp_true": {"bytes": 8.0 * (2 + 1 / 8), "dp_ops": 4.0},
    # persistent CG: per node and CG step (the two fused bodies above)
    "cg_f64": {"bytes": 80.0, "dp_ops": 19.0},
    "cg_f32": {"bytes": 40.0, "dp_ops": 0.0},
    # all CG steps of a small grid in one thread-block cluster, vectors in shared memory
    # (single-reduction recurrence): per node-step p, s, x, r 4 + stencil 19 + r.r, w.r 2
    "cg_cluster_f64": {"bytes": 0.0, "dp_ops": 25.0},
    "cg_cluster_f32": {"bytes": 0.0, "dp_ops": 0.0},
    # all CG steps of a mid-size grid, vectors resident in the blocks' shared memory: the
    # same 25 operations; global traffic = the published r, s, w of every node (24 B)
    "cg_resident_f64": {"bytes": 24.0, "dp_ops": 25.0},
    # DSOLVE by the sine transform: b in, x and the check residual out; per unknown
    # 2 (mx + my + mz) FMA for the transforms (~25 on the workloads' 16x8x4 grid), the
    # division, and the 19-point check
    "dsolve": {"bytes": 24.0, "dp_ops": 72.0},
    # comparison prolongations (tri-quadratic after extrapolation, or trilinear): the
    # same streams as EXP_finite; ~3 (quadratic) or ~1.5 (linear) FMA per fine node
    "prolong_cmp": {"bytes": 8.0 * (1 + 1 / 8 + 1 / 64), "dp_ops": 3.0},
}
KERNEL_SYMBOL = {"spmv_f64": "k_dir_spmv_dot<double>", "update_f64": "k_update_dot<double>",
                 "spmv_f32": "k_dir_spmv_dot<float>", "update_f32": "k_update_dot<float>",
                 "residual": "k_residual", "exp_finite": "k_exp_finite", "init": "k_boundary_init",
                 "correct": "k_add_correction", "exp_true": "k_exp_true",
                 "cg_f64": "k_cg_persistent<double>", "cg_f32": "k_cg_persistent<float>",
                 "cg_cluster_f64": "k_cg_cluster<double>", "cg_cluster_f32": "k_cg_cluster<float>",
                 "cg_resident_f64": "k_cg_resident", "dsolve": "k_dsolve",
                 "prolong_cmp": "k_prolong_cmp"}
KERNEL_SOURCE = {"spmv_f64": "cg_kernels.cu", "update_f64": "cg_kernels.cu",
                 "spmv_f32": "cg_kernels.cu", "update_f32": "cg_kernels.cu",
                 "residual": "cg_kernels.cu", "exp_finite": "transfer_kernels.cu",
                 "init": "transfer_kernels.cu", "correct": "cg_kernels.cu",
                 "exp_true": "transfer_kernels.cu", "cg_f64": "cg_kernels.cu",
                 "cg_f32": "cg_kernels.cu", "cg_cluster_f64": "cluster_cg.cu",
                 "cg_cluster_f32": "cluster_cg.cu", "cg_resident_f64": "resident_cg.cu",
                 "dsolve": "dsolve_kernels.cu", "prolong_cmp": "transfer_kernels.cu"}
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


def oracle_solve_seconds(wl, f, g):
    """One complete oracle EXCMG solve of the workload; returns (seconds, u)."""
    import oracle as O
    name, L, N, N0, eps, epsc = WORKLOADS[wl]
    t0 = time.perf_counter()
    res = O.excmg(f, g, L, N, N0, eps=eps, eps_coarse=epsc, dsolve="dense", want_utilde=False)
    return time.perf_counter() - t0, res


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


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name, L, N, N0, eps, epsc = WORKLOADS[args.workload]
    f, g, _ = P.make_inputs(P.PROBLEMS[name], N)
    for _ in range(args.warmup):
        oracle_solve_seconds(args.workload, f, g)
    t = 0.0
    for _ in range(args.steps):
        dt, _ = oracle_solve_seconds(args.workload, f, g)
        t += dt
    n = interior_unknowns(N)
    value = n * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (closed-form f, g on the host)",
            "config": {"workload": DESCRIPTION[args.workload], "unknowns": n},
            "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                             "sample": "each step: one complete oracle EXCMG solve of the workload "
                                       "(numpy, float64, single thread)", "host": host_cpu()},
            "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS) + ["c4", "c5"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip mixed / CG-rate extras")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload in ("c4", "c5"):
        {"c4": run_batched, "c5": run_adjoint}[args.workload](args)
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

    name, L, N, N0, eps, epsc = WORKLOADS[args.workload]
    f, g, u_exact = P.make_inputs(P.PROBLEMS[name], N)
    n_unk = interior_unknowns(N)
    fd = torch.from_numpy(f).to(device)
    gd = torch.from_numpy(g).to(device)
    ud = torch.empty_like(fd)
    prec = PRECISION[args.workload]
    opts = dict(eps=eps, eps_coarse=epsc, precision=prec)
    ws = X.workspace(X.solve_workspace_bytes(L, N, N0, **opts), device)
    stream = torch.cuda.current_stream()

    ranks = Replicas(world, device, dist if world > 1 else None)
    barrier = ranks.barrier
    max_over_ranks = ranks.max

    for _ in range(max(args.warmup, 0)):
        X.solve(fd, gd, L, N0, ws=ws, out=ud, **opts)

    # ---- timed region: inputs resident in HBM
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        res = X.solve(fd, gd, L, N0, ws=ws, out=ud, **opts)
        launches += res["stats"]["launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms)
    stats = res["stats"]
    value = ranks.rate(n_unk, args.steps, ms)

    # ---- accuracy of the timed solution (host evaluation)
    uh = ud.cpu().numpy()
    err_l2 = float(np.sqrt(np.mean((uh - u_exact) ** 2)))
    err_linf = float(np.max(np.abs(uh - u_exact)))

    # ---- end to end through the C-ABI with host buffers
    f_pin = torch.from_numpy(f).pin_memory()
    g_pin = torch.from_numpy(g).pin_memory()
    u_pin = torch.empty(f.shape, dtype=torch.float64).pin_memory()
    fd2, gd2, ud2 = torch.empty_like(fd), torch.empty_like(gd), torch.empty_like(fd)
    barrier()
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        fd2.copy_(f_pin, non_blocking=True)
        gd2.copy_(g_pin, non_blocking=True)
        X.solve(fd2, gd2, L, N0, ws=ws, out=ud2, **opts)
        u_pin.copy_(ud2, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_copy = max_over_ranks(e2.elapsed_time(e3))
    assert np.array_equal(u_pin.numpy(), uh), "e2e solution differs from the device-resident one"
    # the same with f and g left in page-locked host memory: the kernels read f (and g's
    # boundary nodes, the only ones the solver reads) over the host link while they run
    u_pin.zero_()
    barrier()
    torch.cuda.synchronize()
    e2.record(stream)
    for _ in range(args.steps):
        X.solve(f_pin, g_pin, L, N0, ws=ws, out=ud2, **opts)
        u_pin.copy_(ud2, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_zc = max_over_ranks(e2.elapsed_time(e3))
    assert np.array_equal(u_pin.numpy(), uh), "zero-copy solution differs from the device-resident one"
    # in place and pipelined: step i's solution goes back to the host on a copy stream
    # while step i + 1 solves (two device solution buffers, two host buffers)
    copy_stream = torch.cuda.Stream()
    ud_pair = [ud2, torch.empty_like(fd)]
    u_pins = [u_pin, torch.empty(f.shape, dtype=torch.float64).pin_memory()]
    for b in u_pins:
        b.zero_()
    solved = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    barrier()
    torch.cuda.synchronize()
    e2.record(stream)
    for k in range(args.steps):
        b = k % 2
        if k >= 2:
            stream.wait_event(copied[b])  # the copy of step k - 2 has left ud_pair[b]
        X.solve(f_pin, g_pin, L, N0, ws=ws, out=ud_pair[b], **opts)
        solved[b].record(stream)
        copy_stream.wait_event(solved[b])
        with torch.cuda.stream(copy_stream):
            u_pins[b].copy_(ud_pair[b], non_blocking=True)
        copied[b].record(copy_stream)
    for b in range(2):
        stream.wait_event(copied[b])
    e3.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_pipe = max_over_ranks(e2.elapsed_time(e3))
    for b in range(min(2, args.steps)):
        assert np.array_equal(u_pins[b].numpy(), uh), "pipelined solution differs from the device-resident one"
    # copies pipelined: step i + 1's f and g go to the device on an upload stream while
    # step i solves, and step i's solution comes back on a download stream while step
    # i + 1 solves (two device buffers of f, g and u; the uploads of step i + 1 are
    # enqueued before the call of step i, which returns when step i is done)
    up_stream = torch.cuda.Stream()
    fd_pair = [fd2, torch.empty_like(fd)]
    gd_pair = [gd2, torch.empty_like(gd)]
    uploaded = [torch.cuda.Event(), torch.cuda.Event()]
    for b in u_pins:
        b.zero_()

    def upload(k):
        b = k % 2
        up_stream.wait_event(solved[b])  # step k - 2 is done with these buffers
        with torch.cuda.stream(up_stream):
            fd_pair[b].copy_(f_pin, non_blocking=True)
            gd_pair[b].copy_(g_pin, non_blocking=True)
        uploaded[b].record(up_stream)
    solved = [torch.cuda.Event(), torch.cuda.Event()]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    for ev in solved + copied:
        ev.record(stream)
    barrier()
    torch.cuda.synchronize()
    e2.record(stream)
    upload(0)
    for k in range(args.steps):
        b = k % 2
        if k + 1 < args.steps:
            upload(k + 1)
        stream.wait_event(uploaded[b])
        stream.wait_event(copied[b])  # the download of step k - 2 has left ud_pair[b]
        X.solve(fd_pair[b], gd_pair[b], L, N0, ws=ws, out=ud_pair[b], **opts)
        solved[b].record(stream)
        copy_stream.wait_event(solved[b])
        with torch.cuda.stream(copy_stream):
            u_pins[b].copy_(ud_pair[b], non_blocking=True)
        copied[b].record(copy_stream)
    for b in range(2):
        stream.wait_event(copied[b])
    e3.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_cpipe = max_over_ranks(e2.elapsed_time(e3))
    for b in range(min(2, args.steps)):
        assert np.array_equal(u_pins[b].numpy(), uh), "pipelined solution differs from the device-resident one"
    n_bnd = int(np.prod(f.shape)) - int(np.prod([s - 2 for s in f.shape]))
    e2e_modes = {"copy": {"ms_per_step": ms_copy / args.steps, "h2d_bytes_per_step": f.nbytes + g.nbytes,
                          "how": "f and g copied to the device (cudaMemcpyAsync), then the solve"},
                 "in_place": {"ms_per_step": ms_zc / args.steps, "h2d_bytes_per_step": f.nbytes + 8 * n_bnd,
                              "how": "the solve reads f and g's boundary from page-locked host memory"},
                 "in_place_pipelined": {"ms_per_step": ms_pipe / args.steps,
                                        "h2d_bytes_per_step": f.nbytes + 8 * n_bnd,
                                        "how": "as in_place; step i's solution is copied back on a second "
                                               "stream while step i + 1 solves"},
                 "copy_pipelined": {"ms_per_step": ms_cpipe / args.steps,
                                    "h2d_bytes_per_step": f.nbytes + g.nbytes,
                                    "how": "f and g copied to the device on an upload stream while the "
                                           "previous step solves; the solution copied back on a download "
                                           "stream while the next step solves"}}
    best = min(e2e_modes, key=lambda k: e2e_modes[k]["ms_per_step"])
    ms_e2e = e2e_modes[best]["ms_per_step"] * args.steps
    e2e_value = ranks.rate(n_unk, args.steps, ms_e2e)
    h2d = e2e_modes[best]["h2d_bytes_per_step"]
    d2h = f.nbytes

    # ---- profiled repeat (events around every launch; not the timed region)
    prof = X.solve(fd, gd, L, N0, ws=ws, out=ud, profile=1, **opts)["stats"]["profile"]
    total_prof = sum(v["ms"] for v in prof.values())
    hbm_peak, peak_kind = load_peaks()
    kernels = {}
    for kind, v in prof.items():
        a = ALGO[kind]
        t = v["ms"] / 1e3
        gbs = a["bytes"] * v["nodes"] / t / 1e9 if t > 0 else 0.0
        gops = a["dp_ops"] * v["nodes"] / t / 1e9 if t > 0 else 0.0
        t_hbm = a["bytes"] / (hbm_peak * 1e9)
        t_alu = a["dp_ops"] / (DP_PEAK_GOPS * 1e9)
        kernels[kind] = {"share": v["ms"] / total_prof if total_prof else 0.0,
                         "ms": v["ms"], "launches": v["launches"],
                         "avg_launch_us": 1e3 * v["ms"] / v["launches"],
                         "GB_s": gbs, "Gdpop_s": gops,
                         "bound": "alu" if t_alu > t_hbm else "hbm"}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    dk = kernels[dom]
    launches_dom = prof[dom]["launches"]
    nodes_per_launch = prof[dom]["nodes"] / launches_dom  # node-steps for persistent CG
    traffic = recorded_traffic(dom, args.workload)
    if dk["bound"] == "alu":
        roof = {"bound": "alu", "achieved": dk["Gdpop_s"], "peak": DP_PEAK_GOPS,
                "unit": "G DP-op/s", "frac": dk["Gdpop_s"] / DP_PEAK_GOPS}
    else:
        roof = {"bound": "hbm", "achieved": dk["GB_s"], "peak": hbm_peak, "unit": "GB/s",
                "frac": dk["GB_s"] / hbm_peak}
    roof.update({"kernel": KERNEL_SYMBOL[dom], "share_of_step": dk["share"],
                 "traffic": traffic * nodes_per_launch if traffic is not None else None,
                 "algorithmic_bytes_per_launch": ALGO[dom]["bytes"] * nodes_per_launch,
                 "avg_launch_us": dk["avg_launch_us"], "peak_source": peak_kind,
                 "timing": "CUDA events around every launch on the solve's stream, in a "
                           "profiled repeat of the step after the timed region"})

    line = {"metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32+f64",
            "data": "synthetic (closed-form f, g evaluated on the host in float64)",
            "config": {"workload": DESCRIPTION[args.workload], "unknowns": n_unk,
                       "levels": stats["levels"], "iters_per_level": stats["iters"],
                       "relres_finest": stats["relres"][-1],
                       "error_vs_exact": {"L2_rms": err_l2, "Linf": err_linf},
                       "parallelism": f"{world} independent replica(s)",
                       "precision": prec,
                       "l2": "inputs larger than L2 (each finest-level array >= 136 MB > 129 MB L2)"},
            "gpu_launches": launches, "clocks": clk, "roofline": roof, "kernels": kernels,
            "e2e": {"value": e2e_value, "unit": "unknowns/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e / args.steps,
                    "mode": best, "modes": e2e_modes}}

    if not args.no_extras:
        line.update(extras(X, torch, device, L, N, N0, fd, gd, u_exact, opts, err_l2, err_linf,
                           hbm_peak, args, world))

    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload != "c3":
        secs, ores = oracle_solve_seconds(args.workload, f, g)
        uo = ores["u"][-1]
        line["cpu_baseline"] = {"value": n_unk / secs, "unit": "unknowns/s", "cores": 1,
                                "kind": "oracle",
                                "sample": "one complete oracle EXCMG solve of the same workload "
                                          "(numpy float64, single thread)",
                                "seconds": secs, "iters_per_level": ores["iters"],
                                "host": host_cpu(),
                                "gpu_vs_oracle_rel_linf": float(np.max(np.abs(uh - uo)) / np.max(np.abs(uo)))}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _setup_gpu():
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05063_gb300 import excmg as X
    return torch, X


def run_batched(args):
    """64 independent problems (sizes from {32,64,128,256}^3 cells, random aspect),
    solved together by excmg_solve_batched; MIXED (float32 inner solves, float64
    refinement) and FP64.  value = interior unknowns of all problems per second."""
    torch, X = _setup_gpu()
    seed, nprob, eps = 20151507, 64, 1e-8
    grids = P.batched_grids(nprob, seed)
    probs, n_unk = [], 0
    for i, (L, N, N0) in enumerate(grids):
        f, g, u = P.make_inputs(P.trig_sum(seed + i, K=8, L=L), N, L)
        probs.append((L, N, N0, f, g, u))
        n_unk += interior_unknowns(N)
    batch = [X.BatchedProblem(L, N, N0, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
             for L, N, N0, f, g, _ in probs]
    out = {"metric": METRIC, "unit": "unknowns/s", "workload": "batched", "n_problems": nprob,
           "unknowns": n_unk, "eps": eps, "sizes": [list(p[1]) for p in probs]}
    for prec in ("mixed", "fp64"):
        for _ in range(max(1, args.warmup)):
            res = X.solve_batched(batch, eps=eps, precision=prec, eps_coarse=1e-10)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(1, args.steps // 4)
        a.record()
        for _ in range(k):
            res = X.solve_batched(batch, eps=eps, precision=prec, eps_coarse=1e-10)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / k
        errs = [float(np.max(np.abs(u.cpu().numpy() - p[5]))) / max(float(np.max(np.abs(p[5]))), 1e-300)
                for u, p in zip(res["u"], probs)]
        out[prec] = {"value": n_unk / (ms / 1e3), "ms_per_batch": ms, "status": res["status"],
                     "max_rel_err_vs_exact": max(errs),
                     "max_relres_finest": max(st["relres"][-1] for st in res["stats"])}
    print(json.dumps(out), flush=True)


def run_adjoint(args):
    """Source recovery on a 256^3 cube: L = ||u(f) - u_t||^2 with u_t the solution for a
    seeded trig-sum source; 20 gradient steps on f with dL/df from excmg_adjoint through
    torch.autograd and an exact line search (L is quadratic in f)."""
    torch, X = _setup_gpu()
    from paper_1507_05063_gb300.autograd import excmg_solve
    N, N0, L = (256, 256, 256), (4, 4, 4), (1.0, 1.0, 1.0)
    ft, g, _ = P.make_inputs(P.trig_sum(20150705, K=8), N)
    gd = torch.from_numpy(g).cuda()
    out = {"metric": METRIC, "workload": "adjoint source recovery 256^3", "steps": 20}
    for prec in ("fp64", "mixed"):
        kw = dict(eps=1e-10, eps_coarse=1e-12, precision=prec)
        ut = X.solve(torch.from_numpy(ft).cuda(), gd, L, N0, **kw)["u"]
        f = torch.zeros_like(ut)
        losses, t_fwd, t_adj = [], 0.0, 0.0
        t0 = time.perf_counter()
        for _ in range(20):
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
        out[prec] = {"loss_first": losses[0], "loss_last": losses[-1],
                     "monotone": all(b < a for a, b in zip(losses, losses[1:])),
                     "seconds_total": total, "seconds_forward": t_fwd, "seconds_adjoint": t_adj}
    print(json.dumps(out), flush=True)


def extras(X, torch, device, L, N, N0, fd, gd, u_exact, opts, err_l2, err_linf, hbm_peak, args,
           world):
    """Mixed-precision EXCMG on the same workload, and the finest-grid CG rates."""
    out = {}
    n_unk = interior_unknowns(N)
    stream = torch.cuda.current_stream()
    other = "fp64" if opts["precision"] == "mixed" else "mixed"
    opts = {k: v for k, v in opts.items() if k != "precision"}
    ws_m = X.workspace(X.solve_workspace_bytes(L, N, N0, precision=other, **opts), device)
    um = torch.empty_like(fd)
    for _ in range(2):
        X.solve(fd, gd, L, N0, ws=ws_m, out=um, precision=other, **opts)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = max(3, args.steps // 2)
    a.record(stream)
    for _ in range(k):
        rm = X.solve(fd, gd, L, N0, ws=ws_m, out=um, precision=other, **opts)
    b.record(stream)
    torch.cuda.synchronize()
    msm = a.elapsed_time(b) / k
    uhm = um.cpu().numpy()
    e2m = float(np.sqrt(np.mean((uhm - u_exact) ** 2)))
    eim = float(np.max(np.abs(uhm - u_exact)))
    out[other] = {"value": n_unk * world / (msm / 1e3), "ms_per_step": msm,
                    "iters_per_level": rm["stats"]["iters"],
                    "refinements_per_level": rm["stats"]["refinements"],
                    "error_vs_exact": {"L2_rms": e2m, "Linf": eim},
                    "error_ratio_vs_headline": {"L2": e2m / err_l2, "Linf": eim / err_linf}}
    # finest-grid CG rates: fixed 20 iterations from the solution, profiled
    rates = {}
    for prec in ("fp64", "mixed"):
        u0 = um.clone()
        st = X.cg(fd, u0, L, eps=0.0 if prec == "fp64" else 1e-30, fixed_iters=[20] if prec == "fp64" else None,
                  precision=prec, inner_tol=1e-30, max_iter=20, max_refine=1, profile=1,
                  allow_not_converged=True)
        pr = st["profile"]
        kind = "cg_f64" if prec == "fp64" else "cg_f32"
        if kind not in pr:
            continue
        steps = st["iters"][0]
        node_steps = pr[kind]["nodes"]
        t_it = pr[kind]["ms"] / max(steps, 1)
        nodes = node_steps / max(steps, 1)
        byt = ALGO[kind]["bytes"] * nodes
        rates[prec] = {"kernel": KERNEL_SYMBOL[kind], "steps": steps, "ms_per_iter": t_it,
                       "unknown_iters_per_s": nodes / (t_it / 1e3),
                       "GB_s": byt / (t_it / 1e3) / 1e9, "frac_hbm": byt / (t_it / 1e3) / 1e9 / hbm_peak,
                       "bytes_per_unknown_iter": ALGO[kind]["bytes"]}
        if prec == "fp64":
            ops = ALGO[kind]["dp_ops"] * nodes
            rates[prec]["Gdpop_s"] = ops / (t_it / 1e3) / 1e9
            rates[prec]["frac_alu"] = rates[prec]["Gdpop_s"] / DP_PEAK_GOPS
    out["cg_finest"] = rates
    # per-level tolerance (eps_ratio r: level l stops at eps * r^(levels-1-l)): a uniform
    # eps leaves the finest grid's algebraic error above the sixth-order error of u~.
    # Time, steps and accuracy of uniform and per-level settings, FP64, same workload.
    tol = {}
    for tag, kw in (("uniform_1e-9", dict(eps=opts["eps"])),
                    ("uniform_1e-13", dict(eps=1e-13)),
                    ("per_level_1e-13_x4", dict(eps=1e-13, eps_ratio=4.0)),
                    ("per_level_1e-13_x16", dict(eps=1e-13, eps_ratio=16.0)),
                    ("per_level_1e-13_x64", dict(eps=1e-13, eps_ratio=64.0))):
        o2 = dict(opts, **kw)
        for _ in range(2):
            X.solve(fd, gd, L, N0, out=um, want_utilde=True, precision="fp64", **o2)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(3):
            r2 = X.solve(fd, gd, L, N0, out=um, want_utilde=True, precision="fp64", **o2)
        b.record(stream)
        torch.cuda.synchronize()
        uh2, ut2 = um.cpu().numpy(), r2["ut"].cpu().numpy()
        tol[tag] = {"ms_per_solve": a.elapsed_time(b) / 3, "iters_per_level": r2["stats"]["iters"],
                    "u_Linf": float(np.max(np.abs(uh2 - u_exact))),
                    "u_tilde_Linf": float(np.max(np.abs(ut2 - u_exact)))}
    out["tolerance_per_level"] = tol
    # prolongation ablation (the prolong option): EXP_finite against extrapolation +
    # tri-quadratic and against the trilinear cascadic-multigrid start, same workload and
    # tolerance; the finest grid's CG step count is what EXP_finite saves
    abl = {}
    for kind in ("quartic", "quadratic", "linear"):
        o2 = dict(opts, prolong=kind)
        for _ in range(2):
            X.solve(fd, gd, L, N0, out=um, precision="fp64", **o2)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(3):
            r2 = X.solve(fd, gd, L, N0, out=um, precision="fp64", **o2)
        b.record(stream)
        torch.cuda.synchronize()
        abl[kind] = {"ms_per_solve": a.elapsed_time(b) / 3, "iters_per_level": r2["stats"]["iters"],
                     "u_Linf": float(np.max(np.abs(um.cpu().numpy() - u_exact)))}
    out["prolong_ablation"] = abl
    return out


if __name__ == "__main__":
    main()
