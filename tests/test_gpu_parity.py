"""GPU path vs the FP64 CPU oracle, element by element on identical seeded inputs.

Every call goes through the C-ABI library (paper_1507_05063_gb300.excmg is a ctypes
binding).  Tolerance: the GPU FP64 solution must match the oracle to relative L-inf
1e-10 (the target stated for this solver); single kernels without an iteration match to
1e-12.  CG stops at a tolerance, and the GPU's reduction order differs from numpy's, so
solver parity replays the oracle's per-level iteration counts (or vice versa).
"""
import numpy as np
import pytest

import oracle as O
from paper_1507_05063_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-10
TOL_KERNEL = 1e-12


@pytest.fixture(scope="module")
def X():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05063_gb300 import excmg
    return excmg


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# --------------------------------------------------------------------------- kernels

@pytest.mark.parametrize("N,L", [((33, 17, 25), (1.0, 0.5, 2.0)), ((4, 4, 4), (1, 1, 1)),
                                 ((70, 9, 40), (1.0, 1.0, 1.0))])
def test_residual_kernel(X, N, L):
    rng = np.random.default_rng(1)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    u = rng.standard_normal(shape)
    f = rng.standard_normal(shape)
    h = O.meshsizes(L, N)
    r, rn, bn = X.residual(dev(f), dev(u), L)
    want = O.residual(u, f, h)
    got = host(r)
    assert rel_linf(got[1:-1, 1:-1, 1:-1], want) <= TOL_KERNEL
    assert np.all(got[0] == 0) and np.all(got[:, :, -1] == 0)
    assert rn == pytest.approx(np.linalg.norm(want), rel=1e-12)
    assert bn == pytest.approx(np.linalg.norm(O.rhs_vector(f, u, h)), rel=1e-12)


@pytest.mark.parametrize("N,tz", [((36, 10, 70), 0), ((36, 10, 70), 1), ((36, 10, 70), 5),
                                  ((36, 10, 70), 64), ((2, 6, 40), 64), ((30, 5, 9), 3),
                                  ((64, 64, 33), 40)])
def test_residual_norms_every_slab_depth(X, N, tz):
    """||r|| / ||b|| of a level's residual launch (b with its Dirichlet lift) at any slab
    depth: the lift at nodes next to an x face is formed after each tile's plane loop, one
    lane per plane in passes of 32 planes, so slabs deeper than 32, both x faces in one
    warp (nx <= 32) and a single interior column (nx = 2) all reach every such node once.
    history[0] of a zero-step CG is that ratio."""
    L = (1.0, 0.7, 2.0)
    rng = np.random.default_rng(9)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    f = rng.standard_normal(shape)
    start = rng.standard_normal(shape)
    h = O.meshsizes(L, N)
    want = np.linalg.norm(O.residual(start, f, h)) / np.linalg.norm(O.rhs_vector(f, start, h))
    st = X.cg(dev(f), dev(start), L, eps=0.0, fixed_iters=[0], history=1, tile_z=tz)
    assert st["iters"] == [0]
    assert st["history"][0] == pytest.approx(want, rel=1e-12, abs=0)


@pytest.mark.parametrize("N,L", [((32, 16, 24), (1.0, 1.0, 1.0)), ((64, 8, 8), (2.0, 1.0, 0.5)),
                                 ((8, 8, 8), (1, 1, 1))])
def test_exp_finite_kernel(X, N, L):
    rng = np.random.default_rng(2)
    N1 = tuple(n // 2 for n in N)
    N0 = tuple(n // 4 for n in N)
    u1 = rng.standard_normal((N1[2] + 1, N1[1] + 1, N1[0] + 1))
    u0 = rng.standard_normal((N0[2] + 1, N0[1] + 1, N0[0] + 1))
    g = rng.standard_normal((N[2] + 1, N[1] + 1, N[0] + 1))
    want = O.exp_finite(u1, u0)
    w = host(X.exp_finite(dev(u1), dev(u0), L))
    assert rel_linf(w, want) <= TOL_KERNEL
    wg = host(X.exp_finite(dev(u1), dev(u0), L, g=dev(g)))
    assert rel_linf(wg, O.with_boundary(want, g)) <= TOL_KERNEL


@pytest.mark.parametrize("N", [(16, 8, 24), (2, 2, 2), (34, 6, 10)])
def test_exp_true_kernel(X, N):
    rng = np.random.default_rng(3)
    N1 = tuple(n // 2 for n in N)
    uh = rng.standard_normal((N[2] + 1, N[1] + 1, N[0] + 1))
    u2h = rng.standard_normal((N1[2] + 1, N1[1] + 1, N1[0] + 1))
    got = host(X.exp_true(dev(uh), dev(u2h), (1, 1, 1)))
    assert rel_linf(got, O.extrapolate_true(uh, u2h)) <= TOL_KERNEL


@pytest.mark.parametrize("N,L", [((4, 5, 6), (1.0, 1.0, 1.0)), ((33, 40, 7), (1.0, 2.0, 0.3)),
                                 ((100, 12, 70), (1.0, 1.0, 1.0))])
def test_grad_kernel(X, N, L):
    rng = np.random.default_rng(4)
    u = rng.standard_normal((N[2] + 1, N[1] + 1, N[0] + 1))
    got = X.grad(dev(u), L)
    want = O.gradient(u, O.meshsizes(L, N))
    for gt, wt in zip(got, want):
        assert rel_linf(host(gt), wt) <= TOL_KERNEL


@pytest.mark.parametrize("N,L,k", [((32, 32, 32), (1, 1, 1), 7), ((40, 24, 16), (1.0, 0.6, 0.4), 12),
                                   ((33, 9, 65), (1, 1, 1), 3)])
def test_cg_fixed_iterations(X, N, L, k):
    rng = np.random.default_rng(5)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    f = rng.standard_normal(shape)
    g = rng.standard_normal(shape)
    start = g.copy()
    start[1:-1, 1:-1, 1:-1] = rng.standard_normal((N[2] - 1, N[1] - 1, N[0] - 1))
    want, it, _ = O.cg(start, f, O.meshsizes(L, N), 0.0, fixed_iters=k)
    u = dev(start)
    st = X.cg(dev(f), u, L, eps=0.0, fixed_iters=[k])
    assert st["iters"][0] == k
    assert rel_linf(host(u), want) <= TOL_SOLVE


def test_cg_tolerance_stop(X):
    N, L = (24, 24, 24), (1, 1, 1)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex3"], N)
    start = g.copy()
    start[1:-1, 1:-1, 1:-1] = 0.0
    want, it, rel = O.cg(start, f, O.meshsizes(L, N), 1e-10)
    u = dev(start)
    st = X.cg(dev(f), u, L, eps=1e-10)
    assert st["relres"][0] <= 1e-10
    assert abs(st["iters"][0] - it) <= 1
    assert rel_linf(host(u), want) <= 1e-8


# --------------------------------------------------------------------------- EXCMG

CASES = [("ex1", (32, 32, 32), (4, 4, 4), 1e-14, 1e-14),
         ("ex4", (64, 32, 16), (8, 4, 2), 1e-9, 1e-9),
         ("sin3", (32, 32, 32), (4, 4, 4), 1e-8, 1e-12),
         ("ex6", (32, 32, 32), (4, 4, 4), 1e-13, 1e-13)]


@pytest.mark.parametrize("name,N,N0,eps,epsc", CASES)
def test_excmg_replayed_iterations(X, name, N, N0, eps, epsc):
    """GPU EXCMG at the tolerance; the oracle replays its per-level iteration counts."""
    L = (1.0, 1.0, 1.0)
    f, g, u = P.make_inputs(P.PROBLEMS[name], N)
    res = X.solve(dev(f), dev(g), L, N0, eps=eps, eps_coarse=epsc, want_utilde=True)
    iters = res["stats"]["iters"]
    ref = O.excmg(f, g, L, N, N0, eps=eps, dsolve="dense", fixed_iters=iters)
    assert rel_linf(host(res["u"]), ref["u"][-1]) <= TOL_SOLVE
    assert rel_linf(host(res["ut"]), ref["ut"][-1]) <= TOL_SOLVE
    # the oracle run at the tolerance takes (nearly) the same counts
    free = O.excmg(f, g, L, N, N0, eps=eps, dsolve="dense")
    assert all(abs(a - b) <= 2 for a, b in zip(iters, free["iters"])), (iters, free["iters"])
    # discretisation errors agree to 3 significant digits
    e_gpu = np.max(np.abs(host(res["u"]) - u))
    e_ref = np.max(np.abs(free["u"][-1] - u))
    assert e_gpu == pytest.approx(e_ref, rel=1e-3, abs=0)


def test_excmg_oracle_fixed_counts_both_sides(X):
    """Both sides run the same prescribed iteration counts (FP64 fixed mode), DSOLVE as
    CG with counts, and DSOLVE as the direct solve (the counts of levels 0-1 unused)."""
    N, N0, L = (32, 16, 16), (8, 4, 4), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex3"], N)
    counts = [12, 9, 6]
    res = X.solve(dev(f), dev(g), L, N0, fixed_iters=counts, dsolve="cg")
    assert res["stats"]["iters"] == counts
    ref = O.excmg(f, g, L, N, N0, eps=0.0, fixed_iters=counts)
    assert rel_linf(host(res["u"]), ref["u"][-1]) <= TOL_SOLVE
    res = X.solve(dev(f), dev(g), L, N0, fixed_iters=counts)
    assert res["stats"]["iters"] == [0, 0, 6]
    ref = O.excmg(f, g, L, N, N0, eps=0.0, dsolve="dense", fixed_iters=counts)
    assert rel_linf(host(res["u"]), ref["u"][-1]) <= TOL_SOLVE


@pytest.mark.parametrize("N0,L", [((8, 4, 2), (1.0, 1.0, 1.0)),
                                  ((6, 10, 4), (1.2, 0.5, 2.0)),
                                  ((8, 6, 10), (1.0, 0.7, 1.3))])
def test_dsolve_direct_matches_dense_cholesky(X, N0, L):
    """DSOLVE (levels 0 and 1) by the sine transform equals the oracle's dense Cholesky
    solve: no CG steps there, residual at rounding level, and the 3-level cascade
    matches the oracle run with dense DSOLVE and the GPU's level-2 step count."""
    N = tuple(4 * n for n in N0)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex3"], N, L)
    res = X.solve(dev(f), dev(g), L, N0, eps=1e-10)
    st = res["stats"]
    assert st["levels"] == 3 and st["iters"][:2] == [0, 0]
    assert max(st["relres"][:2]) <= 1e-13
    ref = O.excmg(f, g, L, N, N0, eps=1e-10, dsolve="dense", fixed_iters=st["iters"])
    assert rel_linf(host(res["u"]), ref["u"][-1]) <= TOL_SOLVE
    # the CG variant of DSOLVE reaches the same answer to its tolerances
    rcg = X.solve(dev(f), dev(g), L, N0, eps=1e-10, dsolve="cg", eps_coarse=1e-13)
    assert min(rcg["stats"]["iters"][:2]) > 0
    assert rel_linf(host(rcg["u"]), ref["u"][-1]) <= 1e-8


def test_per_level_tolerance_replays_oracle(X):
    """eps_ratio: each level l >= 2 meets eps * r^(L-1-l) in the GPU's float64 residual,
    and the oracle run with the same per-level tolerances and step counts agrees."""
    N, N0, L = (64, 32, 16), (8, 4, 2), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex4"], N)
    eps, r = 1e-12, 64.0
    res = X.solve(dev(f), dev(g), L, N0, eps=eps, eps_ratio=r)
    st = res["stats"]
    nl = st["levels"]
    for l in range(2, nl):
        assert st["relres"][l] <= eps * r ** (nl - 1 - l) * 1.0000001
    ref = O.excmg(f, g, L, N, N0, eps=eps, dsolve="dense", eps_ratio=r, fixed_iters=st["iters"])
    assert rel_linf(host(res["u"]), ref["u"][-1]) <= TOL_SOLVE


@pytest.mark.parametrize("kind", ["quadratic", "linear"])
@pytest.mark.parametrize("name,N,N0,L", [("ex4", (64, 32, 16), (8, 4, 2), (1.0, 1.0, 1.0)),
                                         ("ex3", (48, 80, 32), (6, 10, 4), (1.2, 0.5, 2.0))])
def test_comparison_prolongation_matches_oracle(X, kind, name, N, N0, L):
    """prolong = quadratic / linear: with no CG steps above level 1 every level's u is its
    prolongation (boundary = g), element by element equal to the oracle's; at a tolerance
    the oracle replays the GPU's step counts.  48 cells along x leave a partial brick."""
    f, g, _ = P.make_inputs(P.PROBLEMS[name], N, L)
    nl = len(O.level_sizes(N, N0))
    zero = [0] * nl
    res = X.solve(dev(f), dev(g), L, N0, fixed_iters=zero, prolong=kind, profile=1)
    assert "prolong_cmp" in res["stats"]["profile"] and "exp_finite" not in res["stats"]["profile"]
    ref = O.excmg(f, g, L, N, N0, eps=0.0, dsolve="dense", fixed_iters=zero, prolong_kind=kind,
                  want_utilde=False)
    assert rel_linf(host(res["u"]), O.with_boundary(ref["w"][-1], g)) <= TOL_KERNEL
    res = X.solve(dev(f), dev(g), L, N0, eps=1e-10, prolong=kind)
    iters = res["stats"]["iters"]
    ref = O.excmg(f, g, L, N, N0, eps=1e-10, dsolve="dense", fixed_iters=iters,
                  prolong_kind=kind, want_utilde=False)
    assert rel_linf(host(res["u"]), ref["u"][-1]) <= TOL_SOLVE


def test_prolongation_ranking_on_finest_grid(X):
    """Section 3.3's first remark: the finest-grid CG needs far fewer steps from
    EXP_finite than from extrapolation + tri-quadratic, and those fewer than from the
    trilinear cascadic multigrid start (Example 1, 128^3, eps = 1e-12)."""
    N, N0, L = (128, 128, 128), (4, 4, 4), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex1"], N)
    fd, gd = dev(f), dev(g)
    its = {k: X.solve(fd, gd, L, N0, eps=1e-12, prolong=k)["stats"]["iters"][-1]
           for k in ("quartic", "quadratic", "linear")}
    assert its["quartic"] < its["quadratic"] < its["linear"], its
    assert 2 * its["quartic"] < its["linear"], its


def test_dsolve_large_coarse_grid_falls_back_to_cg(X):
    """A coarse grid whose interior does not fit one block's shared memory (31^3
    unknowns on level 1) is solved by CG to eps_coarse instead."""
    N0, L = (16, 16, 16), (1.0, 1.0, 1.0)
    N = (64, 64, 64)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex3"], N)
    res = X.solve(dev(f), dev(g), L, N0, eps=1e-10, eps_coarse=1e-12)
    st = res["stats"]
    assert st["iters"][0] == 0 and st["iters"][1] > 0  # 15^3 direct, 31^3 by CG
    assert st["relres"][1] <= 1e-12 and st["relres"][2] <= 1e-10
    ref = O.excmg(f, g, L, N, N0, eps=1e-10, dsolve="dense", fixed_iters=st["iters"])
    # level 1 differs from the oracle's exact level 1 by the CG tolerance only
    assert rel_linf(host(res["u"]), ref["u"][-1]) <= 1e-8


def test_excmg_table_errors(X):
    """GPU EXCMG reproduces the printed errors of Table 1/2 (Example 1, 32^3)."""
    N, L = (32, 32, 32), (1, 1, 1)
    prob = P.PROBLEMS["ex1"]
    f, g, u = P.make_inputs(prob, N)
    res = X.solve(dev(f), dev(g), L, (4, 4, 4), eps=1e-14, eps_coarse=1e-14, want_utilde=True)
    uh = host(res["u"])
    gx, gy, gz = (host(t) for t in X.grad(res["u"], L))
    ex, ey, ez = P.exact_gradient(prob, N)
    assert O.l2_norm(uh - u) == pytest.approx(1.09e-9, rel=6e-3, abs=0)
    assert O.linf_norm(uh - u) == pytest.approx(3.43e-9, rel=6e-3, abs=0)
    assert O.grad_linf_norm(gx - ex, gy - ey, gz - ez) == pytest.approx(5.18e-7, rel=6e-3, abs=0)
    assert O.linf_norm(host(res["ut"]) - u) == pytest.approx(1.77e-10, rel=6e-3, abs=0)


def test_pinned_host_inputs_read_in_place(X):
    """f and g in page-locked host memory: the kernels read them over the host link and
    the solution is bit-identical to the device-resident run; pageable host memory is
    refused on the host before any work (the binding raises, the library returns
    EXCMG_ERR_INVALID_ARG)."""
    N, N0, L = (64, 32, 16), (8, 4, 2), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex4"], N)
    ref = X.solve(dev(f), dev(g), L, N0, eps=1e-10, want_utilde=True)
    fp, gp = torch.from_numpy(f).pin_memory(), torch.from_numpy(g).pin_memory()
    got = X.solve(fp, gp, L, N0, eps=1e-10, want_utilde=True)
    torch.cuda.synchronize()
    assert got["stats"]["iters"] == ref["stats"]["iters"]
    assert np.array_equal(host(got["u"]), host(ref["u"]))
    assert np.array_equal(host(got["ut"]), host(ref["ut"]))
    with pytest.raises(ValueError):
        X.solve(torch.from_numpy(f), torch.from_numpy(g), L, N0)
    import ctypes
    grid = X.make_grid(L, N, N0)
    o, _keep = X.make_options()
    need = X.excmg_workspace_size(ctypes.byref(grid), ctypes.byref(o))
    ws = X.workspace(need, "cuda")
    u = torch.empty_like(ref["u"])
    fh = np.ascontiguousarray(f)  # pageable
    st = X.excmg_solve(ctypes.byref(grid), ctypes.c_void_p(fh.ctypes.data), ctypes.c_void_p(gp.data_ptr()),
                       ctypes.byref(o), ctypes.c_void_p(u.data_ptr()), None, ctypes.c_void_p(ws.data_ptr()),
                       ws.numel(), None, None)
    assert st == 1
    # the output must be device memory
    up = torch.empty(f.shape, dtype=torch.float64).pin_memory()
    st = X.excmg_solve(ctypes.byref(grid), ctypes.c_void_p(fp.data_ptr()), ctypes.c_void_p(gp.data_ptr()),
                       ctypes.byref(o), ctypes.c_void_p(up.data_ptr()), None, ctypes.c_void_p(ws.data_ptr()),
                       ws.numel(), None, None)
    assert st == 1


def _agree_while_large(got, want, floor=1e-8, rel=1e-6):
    """Residual histories of two implementations agree step by step while the residual
    is well above the rounding floor (below it the recursive residuals are noise)."""
    assert len(got) == len(want)
    for k, (a, b) in enumerate(zip(got, want)):
        if b > floor:
            assert a == pytest.approx(b, rel=rel, abs=0), (k, a, b)


def test_finest_level_residual_history_matches_oracle(X):
    """options.history: the finest level's relative residual after each CG step (the
    persistent engine on 129^3 nodes), step by step equal to the oracle's replay of the
    same counts; its last entry is the reported relative residual."""
    N, N0, L = (128, 128, 128), (4, 4, 4), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex1"], N)
    res = X.solve(dev(f), dev(g), L, N0, eps=1e-12, history=200, profile=1)
    st = res["stats"]
    assert "cg_f64" in st["profile"]
    h = res["history"]
    assert len(h) == st["iters"][-1] + 1 and h[-1] == st["relres"][-1] and h[-1] <= 1e-12
    want = []
    O.excmg(f, g, L, N, N0, eps=1e-12, dsolve="dense", fixed_iters=st["iters"], history=want,
            want_utilde=False)
    _agree_while_large(h, want)


@pytest.mark.parametrize("N,engine", [((16, 8, 4), "cg_cluster_f64"), ((64, 32, 16), "cg_resident_f64")])
def test_cg_residual_history_single_reduction_engines(X, N, engine):
    """The same history from the single-reduction engines (excmg_cg, fixed step count):
    their recursive residual follows the standard recurrence's in exact arithmetic."""
    rng = np.random.default_rng(5)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    f = rng.standard_normal(shape)
    start = rng.standard_normal(shape)
    L = (1.0, 1.0, 1.0)
    k = 25
    u = dev(start)
    st = X.cg(dev(f), u, L, eps=0.0, fixed_iters=[k], history=k + 1, profile=1)
    assert engine in st["profile"]
    want = []
    O.cg(start, f, O.meshsizes(L, N), 0.0, fixed_iters=k, history=want)
    assert len(st["history"]) == k + 1
    _agree_while_large(st["history"], want)


def test_profile_times_per_level(X):
    """options.profile: every launch's time is attributed to its level (the one DSOLVE
    launch that serves levels 0 and 1 counts to level 0); the levels add up to the total,
    which is the sum over kernel kinds."""
    N, N0, L = (64, 32, 16), (8, 4, 2), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex4"], N)
    st = X.solve(dev(f), dev(g), L, N0, eps=1e-10, profile=1, want_utilde=True)["stats"]
    assert len(st["ms_level"]) == st["levels"] == 4
    assert st["ms_level"][0] > 0 and st["ms_level"][1] == 0
    assert all(t > 0 for t in st["ms_level"][2:])
    assert sum(st["ms_level"]) == pytest.approx(st["ms_total"], rel=1e-9)
    assert st["ms_total"] == pytest.approx(sum(v["ms"] for v in st["profile"].values()), rel=1e-9)


def test_history_refused_where_not_supported(X):
    """MIXED precision has no single CG residual history: the workspace query refuses."""
    with pytest.raises(X.ExcmgError):
        f, g, _ = P.make_inputs(P.PROBLEMS["ex1"], (16, 16, 16))
        X.solve(dev(f), dev(g), (1, 1, 1), (4, 4, 4), precision="mixed", history=10)


# --------------------------------------------------------------------------- failure modes

def test_nan_in_f_reports_nonfinite(X):
    N = (16, 16, 16)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex1"], N)
    f[5, 6, 7] = np.nan
    with pytest.raises(X.ExcmgError) as ei:
        X.solve(dev(f), dev(g), (1, 1, 1), (4, 4, 4))
    assert ei.value.status == 4


def test_iteration_cap_reports_not_converged(X):
    N = (32, 32, 32)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex1"], N)
    res = X.solve(dev(f), dev(g), (1, 1, 1), (4, 4, 4), eps=1e-14, max_iter=2,
                  allow_not_converged=True)
    assert res["status"] == "EXCMG_ERR_NOT_CONVERGED"
    assert max(res["stats"]["iters"]) == 2


def test_workspace_reuse_gives_same_answer(X):
    N = (32, 32, 32)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex2"], N)
    fd, gd = dev(f), dev(g)
    a = X.solve(fd, gd, (1, 1, 1), (4, 4, 4), eps=1e-10)
    ws = X.workspace(X.solve_workspace_bytes((1, 1, 1), N, (4, 4, 4)), "cuda")
    ws.fill_(0xFF)  # garbage in the workspace must not matter
    b = X.solve(fd, gd, (1, 1, 1), (4, 4, 4), eps=1e-10, ws=ws)
    c = X.solve(fd, gd, (1, 1, 1), (4, 4, 4), eps=1e-10, ws=ws)
    assert torch.equal(a["u"], b["u"]) and torch.equal(b["u"], c["u"])
