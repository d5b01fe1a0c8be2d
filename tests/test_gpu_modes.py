"""GPU tests of the project additions, through the C-ABI: MIXED precision (float32 CG
inside float64 iterative refinement), the batched solve, and the adjoint.

Targets: MIXED reaches within 1.05x of the FP64 discretisation error; batched results
equal single solves to the CG tolerance; the adjoint matches the oracle's adjoint to
rel 1e-10 and central finite differences of GPU forward solves to rel 1e-6.
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


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.float64, order="C")).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


# --------------------------------------------------------------------------- MIXED

@pytest.mark.parametrize("name,N,N0,eps", [("exp3", (128, 64, 32), (8, 4, 2), 1e-9),
                                           ("ex1", (64, 64, 64), (4, 4, 4), 1e-12),
                                           ("r53", (64, 32, 32), (8, 4, 4), 1e-9)])
def test_mixed_error_within_fp64(X, name, N, N0, eps):
    L = (1.0, 1.0, 1.0)
    f, g, u = P.make_inputs(P.PROBLEMS[name], N)
    fd, gd = dev(f), dev(g)
    r64 = X.solve(fd, gd, L, N0, eps=eps)
    rmx = X.solve(fd, gd, L, N0, eps=eps, precision="mixed", mixed_min_nodes=1)
    e64 = np.max(np.abs(host(r64["u"]) - u))
    emx = np.max(np.abs(host(rmx["u"]) - u))
    assert emx <= 1.05 * e64, (emx, e64)
    l2_64 = np.sqrt(np.mean((host(r64["u"]) - u) ** 2))
    l2_mx = np.sqrt(np.mean((host(rmx["u"]) - u) ** 2))
    assert l2_mx <= 1.05 * l2_64
    assert any(r > 0 for r in rmx["stats"]["refinements"])  # the float32 path ran
    # every level met the tolerance in the float64 residual
    assert all(r <= eps * 1.0000001 for r in rmx["stats"]["relres"][2:])
    assert all(r <= 1e-12 * 1.0000001 for r in rmx["stats"]["relres"][:2])


def test_mixed_matches_oracle_to_tolerance(X):
    """Both solutions are within the CG tolerance of the discrete solution."""
    N, N0, L = (32, 32, 32), (4, 4, 4), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex3"], N)
    rmx = X.solve(dev(f), dev(g), L, N0, eps=1e-12, eps_coarse=1e-12, precision="mixed",
                  mixed_min_nodes=1)
    ref = O.excmg(f, g, L, N, N0, eps=1e-14, eps_coarse=1e-14)
    uo = ref["u"][-1]
    assert np.max(np.abs(host(rmx["u"]) - uo)) / np.max(np.abs(uo)) <= 1e-9


# --------------------------------------------------------------------------- batched

def _batch(seed, nprob, sizes):
    grids = P.batched_grids(nprob, seed, sizes=sizes)
    probs = []
    for i, (L, N, N0) in enumerate(grids):
        prob = P.trig_sum(seed + i, K=8, L=L)
        f, g, u = P.make_inputs(prob, N, L)
        probs.append((L, N, N0, f, g, u))
    return probs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_matches_single_solves(X, precision):
    probs = _batch(20151507, 6, (16, 32, 64))
    eps = 1e-10
    batch = [X.BatchedProblem(L, N, N0, dev(f), dev(g)) for L, N, N0, f, g, _ in probs]
    kw = dict(mixed_min_nodes=1) if precision == "mixed" else {}
    res = X.solve_batched(batch, eps=eps, precision=precision, **kw)
    for (L, N, N0, f, g, u), ub, st in zip(probs, res["u"], res["stats"]):
        single = X.solve(dev(f), dev(g), L, N0, eps=eps, precision=precision, **kw)
        a, b = host(ub), host(single["u"])
        # same algorithm, different reduction order: equal to far below the tolerance
        assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b)) + 1e-12
        assert st["relres"][-1] <= eps * 1.0000001


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_solves_large_problems_alone(X, precision):
    """excmg_solve_batched solves its problems of 2^18 nodes and more one after another as
    single solves (a 64^3 grid: 274,625 nodes) and batches the others: the large problem's
    result is the single solve's, bit for bit; the small ones agree with their single
    solves far below the tolerance; every problem meets it."""
    eps, L = 1e-10, (1.0, 1.0, 1.0)
    specs = [((64, 64, 64), (4, 4, 4)), ((32, 16, 16), (8, 4, 4)), ((16, 32, 16), (4, 8, 4))]
    probs = []
    for i, (N, N0) in enumerate(specs):
        f, g, _ = P.make_inputs(P.trig_sum(31 + i, K=8, L=L), N, L)
        probs.append((N, N0, f, g))
    kw = dict(eps=eps, precision=precision, autotune=-1)
    if precision == "mixed":
        kw["mixed_min_nodes"] = 1 << 12
    batch = [X.BatchedProblem(L, N, N0, dev(f), dev(g)) for N, N0, f, g in probs]
    res = X.solve_batched(batch, **kw)
    assert res["status"] == "EXCMG_OK"
    for k, ((N, N0, f, g), ub, st) in enumerate(zip(probs, res["u"], res["stats"])):
        single = X.solve(dev(f), dev(g), L, N0, **kw)
        a, b = host(ub), host(single["u"])
        if k == 0:
            assert np.array_equal(a, b)
            assert st["iters"] == single["stats"]["iters"]
        else:
            assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b)) + 1e-12
        assert st["relres"][-1] <= eps * 1.0000001


def test_batched_replays_oracle(X):
    """Each batched problem against the oracle run with the batch's iteration counts."""
    probs = _batch(7, 3, (16, 32))
    batch = [X.BatchedProblem(L, N, N0, dev(f), dev(g)) for L, N, N0, f, g, _ in probs]
    res = X.solve_batched(batch, eps=1e-10)
    for (L, N, N0, f, g, _), ub, st in zip(probs, res["u"], res["stats"]):
        ref = O.excmg(f, g, L, N, N0, eps=0.0, dsolve="dense", fixed_iters=st["iters"])
        uo = ref["u"][-1]
        assert np.max(np.abs(host(ub) - uo)) <= 1e-10 * np.max(np.abs(uo))


# --------------------------------------------------------------------------- adjoint

def test_adjoint_matches_oracle(X):
    N, L = (6, 5, 7), (1.0, 1.3, 0.8)
    h = O.meshsizes(L, N)
    rng = np.random.default_rng(3)
    dLdu = rng.standard_normal((N[2] + 1, N[1] + 1, N[0] + 1))
    df, dg, st = X.adjoint(dev(dLdu), L, eps=1e-15, max_iter=10000)
    wf, wg, _ = O.adjoint(dLdu, h, dense=True)
    assert np.max(np.abs(host(df) - wf)) <= 1e-10 * np.max(np.abs(wf))
    assert np.max(np.abs(host(dg) - wg)) <= 1e-10 * np.max(np.abs(wg))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_central_differences(X, precision):
    """dL/df, dL/dg of L = sum (u - u_t)^2 vs central differences of GPU forward solves
    (16^3, three grids), tight tolerances on both sides."""
    N, N0, L = (16, 16, 16), (4, 4, 4), (1.0, 1.0, 1.0)
    prob = P.trig_sum(20150705, K=8)
    f, g, _ = P.make_inputs(prob, N)
    rng = np.random.default_rng(1)
    ut = rng.standard_normal(f.shape) * 1e-2
    kw = dict(eps=1e-14, eps_coarse=1e-14)

    def loss(fa, ga):
        u = host(X.solve(dev(fa), dev(ga), L, N0, **kw)["u"])
        return float(np.sum((u - ut) ** 2)), u

    L0, u0 = loss(f, g)
    kwa = dict(mixed_min_nodes=1) if precision == "mixed" else {}
    df, dg, _ = X.adjoint(dev(2.0 * (u0 - ut)), L, eps=1e-14, precision=precision, **kwa)
    df, dg = host(df), host(dg)
    delta = 1e-3
    for m in [(8, 8, 8), (3, 12, 5), (1, 1, 1), (0, 7, 9), (15, 2, 16)]:
        fp, fm = f.copy(), f.copy()
        fp[m] += delta
        fm[m] -= delta
        fd = (loss(fp, g)[0] - loss(fm, g)[0]) / (2 * delta)
        assert df[m] == pytest.approx(fd, rel=1e-6, abs=1e-12)
    for m in [(0, 5, 5), (16, 3, 9), (7, 0, 2), (4, 16, 16)]:
        gp, gm = g.copy(), g.copy()
        gp[m] += delta
        gm[m] -= delta
        fd = (loss(f, gp)[0] - loss(f, gm)[0]) / (2 * delta)
        assert dg[m] == pytest.approx(fd, rel=1e-6, abs=1e-12)


# --------------------------------------------------------------------------- autograd

def test_autograd_backward_matches_adjoint_and_fd(X):
    from paper_1507_05063_gb300.autograd import excmg_solve
    N, N0, L = (16, 16, 16), (4, 4, 4), (1.0, 1.0, 1.0)
    f, g, _ = P.make_inputs(P.trig_sum(11, K=8), N)
    rng = np.random.default_rng(4)
    ut = torch.from_numpy(rng.standard_normal(f.shape) * 1e-2).cuda()
    fd = dev(f).requires_grad_(True)
    gd = dev(g).requires_grad_(True)
    kw = dict(eps=1e-14, eps_coarse=1e-14)
    u = excmg_solve(fd, gd, L, N0, **kw)
    loss = ((u - ut) ** 2).sum()
    loss.backward()
    gf = host(fd.grad)
    # central difference in f at two nodes, through the forward solve only
    for m in [(8, 7, 9), (0, 4, 4)]:
        delta = 1e-3
        vals = []
        for sgn in (1, -1):
            fp = f.copy()
            fp[m] += sgn * delta
            up = X.solve(dev(fp), dev(g), L, N0, **kw)["u"]
            vals.append(float(((up - ut) ** 2).sum()))
        assert gf[m] == pytest.approx((vals[0] - vals[1]) / (2 * delta), rel=1e-6, abs=1e-12)


def test_source_recovery_descends(X):
    """20 gradient-descent steps on f to match a target solution: the loss falls every
    step (exact line search: L is quadratic in f, so the optimal step is closed form)."""
    from paper_1507_05063_gb300.autograd import excmg_solve
    N, N0, L = (32, 32, 32), (4, 4, 4), (1.0, 1.0, 1.0)
    target = P.trig_sum(20150705, K=8)
    ft, g, _ = P.make_inputs(target, N)
    kw = dict(eps=1e-12, eps_coarse=1e-12)
    ut = X.solve(dev(ft), dev(g), L, N0, **kw)["u"]
    f = torch.zeros_like(ut)
    gd = dev(g)
    losses = []
    for _ in range(20):
        f.requires_grad_(True)
        u = excmg_solve(f, gd, L, N0, **kw)
        loss = ((u - ut) ** 2).sum()
        loss.backward()
        d = f.grad.detach()
        with torch.no_grad():
            # u is affine in f: u(f - t d) = u(f) - t J d, J d = u(d) - u(0) with g fixed
            Jd = X.solve(d, gd, L, N0, **kw)["u"] - X.solve(torch.zeros_like(d), gd, L, N0, **kw)["u"]
            resid = (u - ut).detach()
            t = float((resid * Jd).sum() / (Jd * Jd).sum())
            f = (f.detach() - t * d)
        losses.append(float(loss))
    assert all(b < a for a, b in zip(losses, losses[1:]))
    assert losses[-1] < 0.5 * losses[0]
