"""Runs one finest-grid CG solve with a fixed number of steps (or one residual or one
EXP_finite launch on that grid), for profilers.

    python -m paper_1507_05063_gb300.profile_cg [--N 512 256 128] [--steps 20]
        [--precision fp64|mixed] [--repeat 1] [--op cg|residual|exp_finite]

The problem is u = exp(x+y+z) on [0,1]^3 (f = 3u, g = u); CG starts from zero in the
interior.  The solve goes through excmg_cg (FP64: one k_cg_persistent<double> launch for
all steps; MIXED: float32 inner steps inside float64 refinement).  Prints the steps and
the CUDA-event time of the whole call.
"""
import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1507_05063_gb300 import excmg as X  # noqa: E402
from paper_1507_05063_gb300 import problems as P  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, nargs=3, default=[512, 256, 128])
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--op", default="cg", choices=["cg", "residual", "exp_finite"])
    a = ap.parse_args()
    N, L = tuple(a.N), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS["exp3"], N)
    fd = torch.from_numpy(f).cuda()
    start = g.copy()
    start[1:-1, 1:-1, 1:-1] = 0.0
    if a.op != "cg":
        # residual of the zero-interior start; EXP_finite from the exact solution sampled on
        # the grids with N/2 and N/4 cells
        u0 = torch.from_numpy(start).cuda()
        u2 = torch.from_numpy(P.make_inputs(P.PROBLEMS["exp3"], tuple(n // 2 for n in N))[2]).cuda()
        u4 = torch.from_numpy(P.make_inputs(P.PROBLEMS["exp3"], tuple(n // 4 for n in N))[2]).cuda()
        for _ in range(a.repeat):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if a.op == "residual":
                out, rn, bn = X.residual(fd, u0, L)
            else:
                out = X.exp_finite(u2, u4, L)
            e1.record()
            torch.cuda.synchronize()
            print(f"N={N} {a.op} ms={e0.elapsed_time(e1):.3f}", flush=True)
        assert np.isfinite(out.cpu().numpy()).all()
        return
    for _ in range(a.repeat):
        u = torch.from_numpy(start).cuda()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if a.precision == "fp64":
            st = X.cg(fd, u, L, eps=0.0, fixed_iters=[a.steps])
        else:
            st = X.cg(fd, u, L, eps=1e-30, precision="mixed", inner_tol=1e-30, max_iter=a.steps,
                      max_refine=1, mixed_min_nodes=1, allow_not_converged=True)
        e1.record()
        torch.cuda.synchronize()
        print(f"N={N} {a.precision} steps={st['iters'][0]} ms={e0.elapsed_time(e1):.3f}", flush=True)
    assert np.isfinite(u.cpu().numpy()).all()


if __name__ == "__main__":
    main()
