"""GPU regression over the paper's printed results on the meshes above the oracle's CPU
pins: the errors of the error tables of Section 5 at 64^3, 128^3, 256^3 (Example 4:
128x64x32, 256x128x64, 512x256x128), and Table 11's finest-grid CG step counts.

Each run is the GPU EXCMG (DSOLVE direct on levels 0-1) at the example's tolerance and
coarsest grid, under both readings of ||f_h|| in the stopping test of Algorithm 1
(options.rhs_norm: lift, forcing); w_h is EXP_finite of the GPU solutions on the two
next-coarser grids; the gradient is the GPU compact gradient.  Norms use the oracle's
discrete definitions (RMS over all nodes, max).  Checks per run and reading:

* against the FP64 oracle under the same reading (oracle_tables_large.txt,
  oracle_tables_large_forcing.txt, written by make_oracle_tables_large.py): every error
  within 1% and the same CG step counts -- the parity check, valid in every regime;
* against the paper: every printed row that a reading's oracle record reproduces to
  three digits (99 of the 144), the GPU under that reading reproduces to three digits.
"""
import collections

import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from paper_1507_05063_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# tolerance stated by each example's tables, and its coarsest grid (Section 5)
SETUP = {"ex1": (1e-14, (4, 4, 4)), "ex2": (1e-14, (4, 4, 4)), "ex3": (1e-11, (4, 4, 4)),
         "ex4": (1e-9, (8, 4, 2)), "ex5": (1e-12, (4, 4, 4)), "ex6": (1e-13, (4, 4, 4))}
L = (1.0, 1.0, 1.0)
DIGITS = 6e-3  # three printed significant digits


@pytest.fixture(scope="module")
def X():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05063_gb300 import excmg
    return excmg


def _oracle(reading):
    name = {"lift": "oracle_tables_large.txt", "forcing": "oracle_tables_large_forcing.txt"}[reading]
    vals, iters = {}, {}
    for row in read_golden(name):
        if row[2] == "iters":
            iters[(row[0], row[1])] = [int(v) for v in row[3].split(",")]
        else:
            vals[(row[0], row[1], row[2], row[3])] = float(row[4])
    return vals, iters


ORACLE = {r: _oracle(r) for r in ("lift", "forcing")}


def _groups():
    groups = collections.defaultdict(list)
    for ex, mesh, norm, qty, val, src in read_golden("paper_tables_gpu.txt"):
        groups[(ex, mesh)].append((norm, qty, float(val), src))
    return sorted(groups.items())


def _solve(X, f, g, N0, eps, reading):
    return X.solve(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), L, N0, eps=eps,
                   eps_coarse=eps, want_utilde=True, rhs_norm=reading)


def _errors(X, name, N, reading):
    eps, N0 = SETUP[name]
    prob = P.PROBLEMS[name]
    f, g, u = P.make_inputs(prob, N)
    res = _solve(X, f, g, N0, eps, reading)
    uh, ut = res["u"].cpu().numpy(), res["ut"].cpu().numpy()
    gx, gy, gz = (t.cpu().numpy() for t in X.grad(res["u"], L))
    ex, ey, ez = P.exact_gradient(prob, N)
    u2 = _solve(X, f[::2, ::2, ::2].copy(), g[::2, ::2, ::2].copy(), N0, eps, reading)["u"]
    u4 = _solve(X, f[::4, ::4, ::4].copy(), g[::4, ::4, ::4].copy(), N0, eps, reading)["u"]
    w = X.exp_finite(u2, u4, L).cpu().numpy()
    out = {
        ("L2", "u"): O.l2_norm(uh - u), ("Linf", "u"): O.linf_norm(uh - u),
        ("L2", "grad"): O.grad_l2_norm(gx - ex, gy - ey, gz - ez),
        ("Linf", "grad"): O.grad_linf_norm(gx - ex, gy - ey, gz - ez),
        ("L2", "ut"): O.l2_norm(ut - u), ("Linf", "ut"): O.linf_norm(ut - u),
        ("L2", "w"): O.l2_norm(w - uh), ("Linf", "w"): O.linf_norm(w - uh),
    }
    return out, res["stats"]


@pytest.mark.parametrize("key,rows", _groups(), ids=lambda v: "-".join(v) if isinstance(v, tuple) else "")
def test_gpu_reproduces_oracle_and_printed_errors(X, key, rows):
    """Both readings of ||f_h|| on the GPU: every error within 1% of the oracle's under the
    same reading (or within 5e-15, the rounding level of u) and the same step counts (+-1,
    or +-2% of the count on the long forcing runs); every printed row that one reading's oracle record reproduces to three digits,
    the GPU under that reading reproduces to three digits as well."""
    name, mesh = key
    N = tuple(int(v) for v in mesh.split("x"))
    got = {}
    for reading in ("lift", "forcing"):
        vals, iters = ORACLE[reading]
        e, st = _errors(X, name, N, reading)
        got[reading] = e
        want_iters = iters[key]
        assert len(st["iters"]) == len(want_iters)
        assert all(abs(a - b) <= max(1, 0.02 * b) for a, b in zip(st["iters"], want_iters)), \
            (reading, st["iters"], want_iters)
        for norm, qty, val, src in rows:
            o = vals[(name, mesh, norm, qty)]
            # 1%, or within 5e-15 where the error itself is at the rounding level of u
            assert e[(norm, qty)] == pytest.approx(o, rel=1e-2, abs=5e-15), (reading, src, norm, qty, o)
    for norm, qty, val, src in rows:
        for reading in ("lift", "forcing"):
            if abs(ORACLE[reading][0][(name, mesh, norm, qty)] / val - 1) <= DIGITS:
                assert got[reading][(norm, qty)] == pytest.approx(val, rel=DIGITS, abs=0), \
                    (reading, src, norm, qty, val)
                break


@pytest.mark.parametrize("name,mesh,iters,src", read_golden("paper_iterations.txt"))
def test_gpu_finest_grid_iterations(X, name, mesh, iters, src):
    """Table 11: EXCMG needs only 8-9 CG steps on the finest grid (w_h is a fifth-order
    approximation of u_h).  The GPU takes the oracle's count, and the printed one to a
    step where the oracle does; on Example 6 (eps = 1e-13, u only in H^5.5) both take 16:
    the relative residual stalls near 1.3e-13 from step 10 to 15 there."""
    eps, N0 = SETUP[name]
    N = tuple(int(v) for v in mesh.split("x"))
    f, g, _ = P.make_inputs(P.PROBLEMS[name], N)
    st = _solve(X, f, g, N0, eps, "lift")["stats"]
    want = ORACLE["lift"][1][(name, mesh)][-1]
    assert abs(st["iters"][-1] - want) <= 1, (st["iters"], want)
    if abs(want - int(iters)) <= 1:
        assert abs(st["iters"][-1] - int(iters)) <= 1, (st["iters"], iters)
    else:
        assert name == "ex6" and st["iters"][-1] <= 2 * int(iters), (st["iters"], iters)
