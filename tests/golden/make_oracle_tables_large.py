"""Writes oracle_tables_large.txt (the "lift" reading of ||f_h|| in the stopping test of
Algorithm 1) and oracle_tables_large_forcing.txt (the "forcing" reading): the FP64
oracle's EXCMG errors and per-level CG step counts on the meshes of paper_tables_gpu.txt
(64^3 ... 256^3; Example 4: 128x64x32 ... 512x256x128), at each example's tolerance and
coarsest grid (Section 5), DSOLVE dense.

Calls only the oracle and the closed-form inputs; the runs are independent and go to a
pool of worker processes (lift: a few minutes; forcing: tens of minutes, its finest
grids take many more CG steps).
Usage: python tests/golden/make_oracle_tables_large.py [lift|forcing] [workers]
"""
import multiprocessing
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1507_05063_gb300 import problems as P  # noqa: E402

# tolerance stated by each example's tables, and its coarsest grid (Section 5)
SETUP = {"ex1": (1e-14, (4, 4, 4)), "ex2": (1e-14, (4, 4, 4)), "ex3": (1e-11, (4, 4, 4)),
         "ex4": (1e-9, (8, 4, 2)), "ex5": (1e-12, (4, 4, 4)), "ex6": (1e-13, (4, 4, 4))}
MESHES = {ex: [(n, n, n) for n in (64, 128, 256)] for ex in SETUP}
MESHES["ex4"] = [(128, 64, 32), (256, 128, 64), (512, 256, 128)]


OUT = {"lift": "oracle_tables_large.txt", "forcing": "oracle_tables_large_forcing.txt"}


def errors(name, N, reading="lift"):
    eps, N0 = SETUP[name]
    prob = P.PROBLEMS[name]
    f, g, u = P.make_inputs(prob, N)
    res = O.excmg(f, g, (1.0, 1.0, 1.0), N, N0, eps=eps, eps_coarse=eps, dsolve="dense",
                  rhs_norm=reading)
    uh, ut, w = res["u"][-1], res["ut"][-1], res["w"][-1]
    gx, gy, gz = O.gradient(uh, res["h"][-1])
    ex, ey, ez = P.exact_gradient(prob, N)
    vals = {
        ("L2", "u"): O.l2_norm(uh - u), ("Linf", "u"): O.linf_norm(uh - u),
        ("L2", "grad"): O.grad_l2_norm(gx - ex, gy - ey, gz - ez),
        ("Linf", "grad"): O.grad_linf_norm(gx - ex, gy - ey, gz - ez),
        ("L2", "ut"): O.l2_norm(ut - u), ("Linf", "ut"): O.linf_norm(ut - u),
        ("L2", "w"): O.l2_norm(w - uh), ("Linf", "w"): O.linf_norm(w - uh),
    }
    return vals, res["iters"]


def _run(job):
    name, N, reading = job
    vals, iters = errors(name, N, reading)
    mesh = "x".join(str(n) for n in N)
    out = [f"{name} {mesh} {norm} {qty} {v:.6e}" for (norm, qty), v in vals.items()]
    out.append(f"{name} {mesh} iters {','.join(str(i) for i in iters)}")
    print(out[-1], flush=True)
    return out


def main():
    reading = sys.argv[1] if len(sys.argv) > 1 else "lift"
    workers = int(sys.argv[2]) if len(sys.argv) > 2 else 1
    lines = [f"# FP64 oracle (oracle/excmg_oracle.py, DSOLVE dense, ||f_h|| reading '{reading}')",
             "# on the meshes of paper_tables_gpu.txt; written by make_oracle_tables_large.py.",
             "# Rows: example mesh norm quantity value  |  example mesh iters c0,c1,... (per level)"]
    jobs = [(name, N, reading) for name in sorted(SETUP) for N in MESHES[name]]
    if workers > 1:
        with multiprocessing.get_context("spawn").Pool(workers) as pool:
            results = pool.map(_run, jobs, chunksize=1)
    else:
        results = [_run(j) for j in jobs]
    for r in results:
        lines.extend(r)
    with open(os.path.join(HERE, OUT[reading]), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
