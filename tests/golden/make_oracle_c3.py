"""Writes oracle_c3.txt: the FP64 oracle's complete EXCMG solve of the 1024x512x512
workload (box [0,1]^3, hx = 1/1024, hy = hz = 1/512; u = r^(5/3), f = (40/9) r^(-1/3),
g = u; 8 grids from 8x4x4; tolerance 1e-9 on levels >= 2, DSOLVE dense on the two
coarsest), with the ||f_h|| reading "lift": per-level CG step counts and relative
residuals, the errors of u_h against the exact solution, and the seconds each level
took on the CPU that ran it.

Calls only the oracle and the closed-form inputs.  About 25 GB of host memory and a few
minutes on one core.  Usage: python tests/golden/make_oracle_c3.py
"""
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1507_05063_gb300 import problems as P  # noqa: E402

N, N0, L, EPS = (1024, 512, 512), (8, 4, 4), (1.0, 1.0, 1.0), 1e-9


def main():
    f, g, u = P.make_inputs(P.PROBLEMS["r53"], N)
    t0 = time.perf_counter()
    res = O.excmg(f, g, L, N, N0, eps=EPS, eps_coarse=1e-12, dsolve="dense", want_utilde=False)
    secs = time.perf_counter() - t0
    uh = res["u"][-1]
    lines = ["# FP64 oracle EXCMG on 1024x512x512, u = r^(5/3), eps 1e-9 (levels >= 2), DSOLVE",
             "# dense, ||f_h|| reading lift; written by make_oracle_c3.py.",
             f"# host: {platform.machine()} {platform.processor() or ''}".rstrip(),
             "iters " + ",".join(str(i) for i in res["iters"]),
             "relres " + ",".join(f"{r:.6e}" for r in res["relres"]),
             f"err_L2 {O.l2_norm(uh - u):.6e}",
             f"err_Linf {O.linf_norm(uh - u):.6e}",
             f"seconds {secs:.1f}"]
    with open(os.path.join(HERE, "oracle_c3.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
