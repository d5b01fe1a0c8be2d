"""GPU tests, through the C-ABI, of the two readings of ||f_h|| in the stopping test of
Algorithm 1 (options.rhs_norm), the float32 CG engine of the MIXED inner solves checked
element by element against the oracle's CG, the bounded device waits of the cooperative
CG launches (EXCMG_ERR_TIMEOUT), and the status of a CG loop allowed no step.
"""
import numpy as np
import pytest

import oracle as O
from paper_1507_05063_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-10  # GPU vs oracle after the same CG steps (float64)


@pytest.fixture(scope="module")
def X():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05063_gb300 import excmg
    return excmg


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.float64, order="C")).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------------------------ rhs_norm readings

@pytest.mark.parametrize("name,N,N0,eps", [("ex1", (32, 32, 32), (4, 4, 4), 1e-12),
                                           ("ex3", (32, 32, 32), (4, 4, 4), 1e-11),
                                           ("ex4", (64, 32, 16), (8, 4, 2), 1e-9)])
def test_forcing_reading_replays_oracle(X, name, N, N0, eps):
    """FORCING: the GPU's step counts at the tolerance equal the oracle's (+-1 per level),
    and replaying the GPU's counts on the oracle gives the same u_h to 1e-10."""
    L = (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS[name], N)
    res = X.solve(dev(f), dev(g), L, N0, eps=eps, eps_coarse=eps, rhs_norm="forcing",
                  dsolve="cg")
    free = O.excmg(f, g, L, N, N0, eps=eps, eps_coarse=eps, rhs_norm="forcing")
    it = res["stats"]["iters"]
    assert all(abs(a - b) <= 1 for a, b in zip(it, free["iters"])), (it, free["iters"])
    rep = O.excmg(f, g, L, N, N0, eps=eps, eps_coarse=eps, rhs_norm="forcing", fixed_iters=it)
    assert rel_linf(host(res["u"]), rep["u"][-1]) <= TOL_SOLVE
    # the relative residual is reported against the forcing norm and meets eps there
    assert res["stats"]["relres"][-1] <= eps * 1.0000001


def test_forcing_reading_is_tighter_than_lift(X):
    """Same problem, the two readings: FORCING's norm is the smaller (no lift), so it
    takes at least as many steps on every CG level and reaches the smaller algebraic
    error; the difference shows on the finest grid (Section 5's tables)."""
    N, N0, L, eps = (32, 32, 32), (4, 4, 4), (1.0, 1.0, 1.0), 1e-12
    f, g, _ = P.make_inputs(P.PROBLEMS["ex1"], N)
    a = X.solve(dev(f), dev(g), L, N0, eps=eps, rhs_norm="lift")["stats"]["iters"]
    b = X.solve(dev(f), dev(g), L, N0, eps=eps, rhs_norm="forcing")["stats"]["iters"]
    assert all(y >= x for x, y in zip(a[2:], b[2:])) and b[-1] > a[-1], (a, b)


def test_forcing_falls_back_to_lift_when_f_is_zero(X):
    """Example 2 has f = 0: RHS(f) vanishes, and FORCING takes the lift reading there
    (the oracle's stopping_norm does the same), so both readings take the same steps."""
    N, N0, L, eps = (32, 32, 32), (4, 4, 4), (1.0, 1.0, 1.0), 1e-12
    f, g, _ = P.make_inputs(P.PROBLEMS["ex2"], N)
    assert np.all(f == 0)
    a = X.solve(dev(f), dev(g), L, N0, eps=eps, rhs_norm="lift")
    b = X.solve(dev(f), dev(g), L, N0, eps=eps, rhs_norm="forcing")
    assert a["stats"]["iters"] == b["stats"]["iters"]
    assert np.array_equal(host(a["u"]), host(b["u"]))


def test_forcing_norm_of_one_residual(X):
    """excmg_cg with no step allowed reports the relative residual of its start against
    ||f_h|| under each reading, checked against the oracle's residual and two norms."""
    N, L = (24, 20, 16), (1.0, 0.8, 0.6)
    rng = np.random.default_rng(11)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    f = rng.standard_normal(shape)
    u0 = rng.standard_normal(shape)
    h = O.meshsizes(L, N)
    r = O.residual(u0, f, h)
    rn = np.sqrt(np.sum(r * r))
    for reading in ("lift", "forcing"):
        st = X.cg(dev(f), dev(u0), L, eps=1.0, fixed_iters=None, rhs_norm=reading, max_iter=0,
                  allow_not_converged=True)
        want = rn / O.stopping_norm(f, u0, h, reading)
        assert st["relres"][0] == pytest.approx(want, rel=1e-12), reading


# ------------------------------------------------------------------ float32 engine

@pytest.mark.parametrize("N,L,k", [((64, 48, 40), (1.0, 0.75, 0.6), 6),
                                   ((512, 256, 128), (1.0, 1.0, 1.0), 5)])
def test_float32_engine_against_oracle_cg(X, N, L, k):
    """One MIXED refinement with exactly k inner float32 CG steps (the engine that stages
    its stencil planes by tensor copies, with the right-hand side scaled in its first
    step) gives u0 + e_k, e_k the k-th CG iterate of A e = r0; the oracle's float64 CG
    from u0 reaches the same Krylov iterate after k steps.  Element by element, the
    corrections agree to float32 accuracy."""
    rng = np.random.default_rng(13)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    f, g, _ = P.make_inputs(P.PROBLEMS["exp3"], N, L)
    u0 = g.copy()
    u0[1:-1, 1:-1, 1:-1] += 1e-3 * rng.standard_normal((N[2] - 1, N[1] - 1, N[0] - 1))
    want, it, _ = O.cg(u0, f, O.meshsizes(L, N), 0.0, fixed_iters=k)
    u = dev(u0)
    st = X.cg(dev(f), u, L, precision="mixed", mixed_min_nodes=1, eps=1e-300, inner_tol=1e-30,
              max_iter=k, max_refine=1, allow_not_converged=True)
    assert st["iters"][0] == k and st["refinements"][0] == 1
    got = host(u)
    corr = want - u0
    assert np.max(np.abs((got - u0) - corr)) <= 2e-5 * np.max(np.abs(corr))
    assert np.array_equal(got[0], u0[0]) and np.array_equal(got[:, 0], u0[:, 0])  # boundary kept


# ------------------------------------------------------------------ bounded waits

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_barrier_wait_runs_out(X, precision):
    """A team that cannot fill (test_phantom_blocks: a member that is never launched)
    makes every grid barrier of the cooperative launch wait for a block that never
    arrives; with a 5 ms bound the kernel gives up, the call returns EXCMG_ERR_TIMEOUT,
    and the context stays usable: the same call without the phantom then solves."""
    import time
    N, L = (256, 128, 64), (1.0, 1.0, 1.0)  # 2.1 M nodes: the streaming cooperative engines
    f, g, _ = P.make_inputs(P.PROBLEMS["exp3"], N)
    u0 = g.copy()
    u0[1:-1, 1:-1, 1:-1] = 0.0  # far from the solution: CG steps are needed
    fd = dev(f)
    kw = dict(eps=1e-9, precision=precision, mixed_min_nodes=1)
    u = dev(u0)
    t0 = time.perf_counter()
    st = X.cg(fd, u, L, wait_timeout_ms=5.0, test_phantom_blocks=1, allow_timeout=True, **kw)
    assert st["status"] == "EXCMG_ERR_TIMEOUT"
    assert time.perf_counter() - t0 < 10.0
    u = dev(u0)
    st = X.cg(fd, u, L, **kw)
    assert st["status"] == "EXCMG_OK" and st["relres"][0] <= 1e-9 * 1.0000001


# ------------------------------------------------------------------ no step allowed

def test_max_iter_zero_reports_not_converged(X):
    """max_iter = 0 and a start that does not meet the tolerance: no step runs and the
    level is reported unconverged (EXCMG_ERR_NOT_CONVERGED), u unchanged."""
    N, L = (24, 24, 24), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex3"], N)
    u0 = g.copy()
    u0[1:-1, 1:-1, 1:-1] = 0.0
    u = dev(u0)
    st = X.cg(dev(f), u, L, eps=1e-9, max_iter=0, allow_not_converged=True)
    assert st["status"] == "EXCMG_ERR_NOT_CONVERGED" and st["iters"][0] == 0
    assert np.array_equal(host(u), u0)
    # from the converged solution it passes with no step
    X.cg(dev(f), u, L, eps=1e-9)
    st = X.cg(dev(f), u, L, eps=1e-9, max_iter=0)
    assert st["status"] == "EXCMG_OK" and st["iters"][0] == 0


# ------------------------------------------------------------------ launch-shape tuning

def test_autotune_fills_cache_and_keeps_the_solution(X):
    """options.autotune = 1 times candidate slab depths for every level from 2 up and
    caches the fastest per (grid, engine class, device); later solves (autotune = 0) use
    the cache.  The tuned and the modelled launch shapes solve the same problem to the
    same tolerance with the same error against the exact solution (+-1%)."""
    N, N0, L = (256, 128, 64), (8, 4, 2), (1.0, 1.0, 1.0)
    f, g, u = P.make_inputs(P.PROBLEMS["exp3"], N)
    fd, gd = dev(f), dev(g)
    X.excmg_tuning_clear()
    for prec in ("fp64", "mixed"):
        kw = dict(eps=1e-10, precision=prec, mixed_min_nodes=1 << 16)
        ref = X.solve(fd, gd, L, N0, autotune=-1, **kw)
        X.solve(fd, gd, L, N0, autotune=1, **kw)
        ents = [e for e in X.tuning_entries() if e["f32"] == (1 if prec == "mixed" else 0)]
        assert ents, prec
        for e in ents:
            assert e["res_tz"] >= 1 and e["res_ms"] > 0 and e["res_ms"] <= e["res_ms_model"] * 1.0001
            assert e["res_rows"] in (1, 4) and e["res_rows_model"] in (1, 4)
            if e["cg_tz"]:
                assert e["cg_ms"] > 0 and e["cg_ms"] <= e["cg_ms_model"] * 1.0001
        tuned = X.solve(fd, gd, L, N0, **kw)
        assert all(r <= 1e-10 * 1.0000001 for r in tuned["stats"]["relres"][2:])
        e_ref = np.max(np.abs(host(ref["u"]) - u))
        e_tun = np.max(np.abs(host(tuned["u"]) - u))
        assert e_tun == pytest.approx(e_ref, rel=1e-2)
    levels = {tuple(e["N"]) for e in X.tuning_entries()}
    assert (256, 128, 64) in levels and (64, 32, 16) in levels
    # a batch over tuned grids (some of whose single-solve CG engines are untiled, cached
    # without a CG slab depth) solves as the single solve does
    kw = dict(eps=1e-10, precision="fp64")
    single = X.solve(fd, gd, L, N0, **kw)
    bat = X.solve_batched([X.BatchedProblem(L, N, N0, fd, gd)] * 2, **kw)
    assert bat["status"] == "EXCMG_OK"
    for ub in bat["u"]:
        assert np.max(np.abs(host(ub) - u)) == pytest.approx(np.max(np.abs(host(single["u"]) - u)), rel=1e-2)
    X.excmg_tuning_clear()
    assert X.tuning_entries() == []


# ------------------------------------------------------------------ residual rows per thread

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_residual_rows_per_thread_agree(X, precision):
    """options.res_rows: the residual kernel with one and with four rows per thread forms
    every node's residual with the same grouping, so the two solves agree to rounding (the
    block sums of r.r and b.b add in another order); both meet the tolerance."""
    N, N0, L = (96, 64, 32), (6, 4, 2), (1.0, 0.9, 0.8)
    f, g, u = P.make_inputs(P.PROBLEMS["exp3"], N, L)
    fd, gd = dev(f), dev(g)
    kw = dict(eps=1e-10, precision=precision, mixed_min_nodes=1 << 15, autotune=-1)
    a = X.solve(fd, gd, L, N0, res_rows=1, **kw)
    b = X.solve(fd, gd, L, N0, res_rows=4, **kw)
    for r in (a, b):
        assert all(x <= 1e-10 * 1.0000001 for x in r["stats"]["relres"][2:])
    assert all(abs(x - y) <= 1 for x, y in zip(a["stats"]["iters"], b["stats"]["iters"]))
    ea, eb = np.max(np.abs(host(a["u"]) - u)), np.max(np.abs(host(b["u"]) - u))
    assert eb == pytest.approx(ea, rel=1e-2)
    with pytest.raises(X.ExcmgError):
        X.solve(fd, gd, L, N0, res_rows=2, **kw)
