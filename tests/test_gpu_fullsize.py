"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

512x256x128 (u = exp(x+y+z)): the oracle runs the whole cascade with the GPU's
per-level iteration counts; rel L-inf <= 1e-10.
1024x512x512 (u = r^(5/3), MIXED): too large for the oracle's full run, so it checks
(a) the oracle's residual at sampled interior nodes against the GPU residual kernel,
(b) the oracle's EXP_finite on sampled interpolation cells against the GPU kernel,
(c) properties at any size: every level meets its tolerance in the float64 residual,
and the MIXED error against the exact solution is within 1.05x of the FP64 solve's.
"""
import numpy as np
import pytest

import oracle as O
from paper_1507_05063_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def X():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05063_gb300 import excmg
    return excmg


def test_512x256x128_fp64_full_cascade(X):
    N, N0, L = (512, 256, 128), (8, 4, 2), (1.0, 1.0, 1.0)
    f, g, u = P.make_inputs(P.PROBLEMS["exp3"], N)
    res = X.solve(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), L, N0, eps=1e-9,
                  eps_coarse=1e-12, want_utilde=True)
    iters = res["stats"]["iters"]
    ref = O.excmg(f, g, L, N, N0, eps=1e-9, dsolve="dense", fixed_iters=iters)
    ug = res["u"].cpu().numpy()
    uo = ref["u"][-1]
    assert np.max(np.abs(ug - uo)) <= 1e-10 * np.max(np.abs(uo))
    ut = res["ut"].cpu().numpy()
    assert np.max(np.abs(ut - ref["ut"][-1])) <= 1e-10 * np.max(np.abs(uo))


def test_512x256x128_fp64_cg_steps_persistent_engine(X):
    """Five float64 CG steps on the full 512x256x128 grid from EXP_finite's start -- the
    cooperative persistent engine with its flat vectorised update (nodes >= blocks x
    chunk) -- against the oracle's CG with the same five steps: rel L-inf <= 1e-10."""
    N, N0, L = (512, 256, 128), (8, 4, 2), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS["exp3"], N)
    rng = np.random.default_rng(21)
    u0 = g.copy()
    u0[1:-1, 1:-1, 1:-1] += 1e-6 * rng.standard_normal((N[2] - 1, N[1] - 1, N[0] - 1))
    want, it, _ = O.cg(u0, f, O.meshsizes(L, N), 0.0, fixed_iters=5)
    u = torch.from_numpy(u0).cuda()
    st = X.cg(torch.from_numpy(f).cuda(), u, L, eps=0.0, fixed_iters=[5], profile=1)
    assert st["iters"][0] == 5
    assert "cg_f64" in st["profile"]  # the persistent engine ran the steps
    got = u.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def test_512x256x128_mixed_refines_within_fp64_error(X):
    """MIXED on the full 512x256x128 workload with float32 inner solves on every level
    (mixed_min_nodes = 1) and a tolerance tight enough that every level, the finest
    included, needs refinement steps and the algebraic error falls below the
    discretisation error: every level meets eps in the float64 residual, and the error
    against the exact solution is within 1.05x of the FP64 oracle's at that tolerance."""
    N, N0, L, eps = (512, 256, 128), (8, 4, 2), (1.0, 1.0, 1.0), 1e-13
    f, g, u = P.make_inputs(P.PROBLEMS["exp3"], N)
    res = X.solve(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), L, N0, eps=eps,
                  eps_coarse=1e-12, precision="mixed", mixed_min_nodes=1)
    st = res["stats"]
    assert sum(st["refinements"][2:]) >= 3 and st["refinements"][-1] >= 1, st["refinements"]
    assert all(r <= eps * 1.0000001 for r in st["relres"][2:])
    ref = O.excmg(f, g, L, N, N0, eps=eps, eps_coarse=1e-12, dsolve="dense", want_utilde=False)
    e_or = np.max(np.abs(ref["u"][-1] - u))
    e_mx = np.max(np.abs(res["u"].cpu().numpy() - u))
    assert e_mx <= 1.05 * e_or, (e_mx, e_or)


def _windows(rng, N, k, halo):
    """k random window origins (x, y, z) leaving `halo` nodes of room on each side."""
    return [tuple(int(rng.integers(halo, N[d] - halo)) for d in range(3)) for _ in range(k)]


@pytest.fixture(scope="module")
def c3(X):
    N, N0, L = (1024, 512, 512), (8, 4, 4), (1.0, 1.0, 1.0)
    f, g, u = P.make_inputs(P.PROBLEMS["r53"], N)
    fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    return N, N0, L, f, g, u, fd, gd


def test_1024x512x512_mixed_properties(X, c3):
    N, N0, L, f, g, u, fd, gd = c3
    eps = 1e-9
    r64 = X.solve(fd, gd, L, N0, eps=eps, eps_coarse=1e-12)
    e64 = float(torch.max(torch.abs(r64["u"] - torch.from_numpy(u).cuda())))
    del r64
    rmx = X.solve(fd, gd, L, N0, eps=eps, eps_coarse=1e-12, precision="mixed")
    st = rmx["stats"]
    assert all(r <= eps * 1.0000001 for r in st["relres"][2:])
    assert any(n > 0 for n in st["refinements"])  # the float32 path ran on the big grids
    emx = float(torch.max(torch.abs(rmx["u"] - torch.from_numpy(u).cuda())))
    assert emx <= 1.05 * e64, (emx, e64)
    # (a) residual parity at sampled nodes: oracle stencil on 3x3x3 windows of the GPU u
    r, rn, bn = X.residual(fd, rmx["u"], L)
    assert rn <= eps * bn * 1.0000001
    uh = rmx["u"].cpu().numpy()
    rh = r.cpu().numpy()
    h = O.meshsizes(L, N)
    rng = np.random.default_rng(3)
    for (i, j, k) in _windows(rng, N, 200, 1):
        win_u = uh[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2]
        win_f = f[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2]
        want = O.residual(win_u, win_f, h)[0, 0, 0]
        # rounding scale: sum of |weight| x |value| over the 19 + 7 terms
        w = O.coefficients(*h)
        wsum = (abs(w["centre"]) + 2 * (abs(w["fx"]) + abs(w["fy"]) + abs(w["fz"]))
                + 4 * (abs(w["exy"]) + abs(w["exz"]) + abs(w["eyz"])))
        scale = wsum * np.max(np.abs(win_u)) + 6.0 * np.max(np.abs(win_f))
        assert abs(rh[k, j, i] - want) <= 1e-13 * scale


def test_1024x512x512_exp_finite_sampled_cells(X, c3):
    """EXP_finite at full size from GPU solutions on the two coarser grids."""
    N, N0, L, f, g, u, fd, gd = c3
    N1 = tuple(n // 2 for n in N)
    N2 = tuple(n // 4 for n in N)
    u1 = X.solve(fd[::2, ::2, ::2].contiguous(), gd[::2, ::2, ::2].contiguous(), L, N0, eps=1e-9)["u"]
    u2 = X.solve(fd[::4, ::4, ::4].contiguous(), gd[::4, ::4, ::4].contiguous(), L, N0, eps=1e-9)["u"]
    w = X.exp_finite(u1, u2, L).cpu().numpy()
    u1h, u2h = u1.cpu().numpy(), u2.cpu().numpy()
    rng = np.random.default_rng(5)
    ncell = (N[0] // 8, N[1] // 8, N[2] // 8)
    for _ in range(100):
        cx, cy, cz = (int(rng.integers(0, ncell[d])) for d in range(3))
        # one interpolation cell: 5^3 grid-2h nodes, 3^3 grid-4h nodes, 9^3 fine nodes
        w1 = u1h[4 * cz:4 * cz + 5, 4 * cy:4 * cy + 5, 4 * cx:4 * cx + 5]
        w2 = u2h[2 * cz:2 * cz + 3, 2 * cy:2 * cy + 3, 2 * cx:2 * cx + 3]
        want = O.exp_finite(w1, w2)
        got = w[8 * cz:8 * cz + 9, 8 * cy:8 * cy + 9, 8 * cx:8 * cx + 9]
        assert np.max(np.abs(got - want)) <= 1e-12 * max(np.max(np.abs(want)), 1e-300)
    assert N1[0] == 512 and N2[0] == 256


def test_1024x512x512_fp64_matches_oracle_record(X, c3):
    """The FP64 solve of the full 1024x512x512 workload against the oracle's complete
    solve of it (tests/golden/oracle_c3.txt, written by make_oracle_c3.py): the same CG
    step count on every level (+-1) and the same errors against the exact solution
    (0.1%)."""
    N, N0, L, f, g, u, fd, gd = c3
    rec = {}
    from conftest import read_golden
    for row in read_golden("oracle_c3.txt"):
        rec[row[0]] = row[1]
    iters = [int(v) for v in rec["iters"].split(",")]
    res = X.solve(fd, gd, L, N0, eps=1e-9, eps_coarse=1e-12)
    assert all(abs(a - b) <= 1 for a, b in zip(res["stats"]["iters"], iters)), (res["stats"]["iters"], iters)
    uh = res["u"].cpu().numpy()
    assert np.sqrt(np.mean((uh - u) ** 2)) == pytest.approx(float(rec["err_L2"]), rel=1e-3)
    assert np.max(np.abs(uh - u)) == pytest.approx(float(rec["err_Linf"]), rel=1e-3)
