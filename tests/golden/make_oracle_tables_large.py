"""Writes oracle_tables_large.txt: the FP64 oracle's EXCMG errors and per-level CG step
counts on the meshes of paper_tables_gpu.txt (64^3 ... 256^3; Example 4: 128x64x32 ...
512x256x128), at each example's tolerance and coarsest grid (Section 5), DSOLVE dense.

Calls only the oracle and the closed-form inputs; a few minutes on one CPU core.
Usage: python tests/golden/make_oracle_tables_large.py
"""
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


def errors(name, N):
    eps, N0 = SETUP[name]
    prob = P.PROBLEMS[name]
    f, g, u = P.make_inputs(prob, N)
    res = O.excmg(f, g, (1.0, 1.0, 1.0), N, N0, eps=eps, eps_coarse=eps, dsolve="dense")
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


def main():
    lines = ["# FP64 oracle (oracle/excmg_oracle.py, DSOLVE dense) on the meshes of",
             "# paper_tables_gpu.txt; written by make_oracle_tables_large.py.",
             "# Rows: example mesh norm quantity value  |  example mesh iters c0,c1,... (per level)"]
    for name in sorted(SETUP):
        for N in MESHES[name]:
            vals, iters = errors(name, N)
            mesh = "x".join(str(n) for n in N)
            for (norm, qty), v in vals.items():
                lines.append(f"{name} {mesh} {norm} {qty} {v:.6e}")
            lines.append(f"{name} {mesh} iters {','.join(str(i) for i in iters)}")
            print(lines[-1], flush=True)
    with open(os.path.join(HERE, "oracle_tables_large.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
