"""The three CG engines, each on grid sizes that select it, against the oracle.

excmg_cg (and every level of excmg_solve) runs a float64 grid's CG steps on one of:
  * k_cg_cluster   -- up to 2,000 nodes (and the small grids of batched solves, up to
                      20,000), one thread-block cluster of 1-16 CTAs;
  * k_cg_resident  -- from 2,000 nodes up to the largest grid whose boxes fit the shared
                      memory of the co-resident blocks (about 730,000 interior nodes on
                      GB300, never above 2^20), a cooperative grid with the vectors in
                      shared memory (3D boxes, partial boxes at the far faces);
  * k_cg_persistent -- larger grids, streaming from HBM.
The first two use the single-reduction recurrence (same iterates as the oracle's standard
recurrence in exact arithmetic), so the GPU and the oracle run the same number of steps
and agree to relative L-inf 1e-10.  The profile of each call names the engine that ran.
"""
import numpy as np
import pytest

import oracle as O

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
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _inputs(N, seed):
    rng = np.random.default_rng(seed)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    f = rng.standard_normal(shape)
    g = rng.standard_normal(shape)
    start = g.copy()
    start[1:-1, 1:-1, 1:-1] = rng.standard_normal((N[2] - 1, N[1] - 1, N[0] - 1))
    return f, start


# (cells, box lengths, engine, steps); comments: nodes and what the case exercises
ENGINE_CASES = [
    ((8, 4, 2), (1.0, 1.0, 1.0), "cg_cluster_f64", 10),       # 135: one CTA
    ((16, 8, 4), (1.0, 0.5, 0.25), "cg_cluster_f64", 15),     # 765: 8 CTAs of 4 warps
    ((24, 10, 6), (1.0, 0.7, 0.3), "cg_cluster_f64", 15),     # 1,925: last CTA partial
    ((32, 16, 8), (1.0, 1.0, 1.0), "cg_resident_f64", 20),    # 5,049
    ((40, 24, 12), (1.0, 0.8, 0.4), "cg_resident_f64", 20),   # 13,325
    ((64, 32, 16), (1.0, 1.0, 1.0), "cg_resident_f64", 20),   # 36,465
    ((50, 36, 22), (1.0, 0.9, 0.6), "cg_resident_f64", 20),   # 43,401: partial boxes
    ((128, 64, 32), (1.0, 1.0, 1.0), "cg_resident_f64", 12),  # 276,705
    ((160, 80, 40), (2.0, 1.0, 0.5), "cg_resident_f64", 8),   # 534,681: largest boxes
    ((208, 104, 52), (2.0, 1.0, 0.5), "cg_f64", 8),           # 1,163,085: streaming kernel
]


@pytest.mark.parametrize("N,L,engine,k", ENGINE_CASES)
def test_engine_fixed_steps(X, N, L, engine, k):
    f, start = _inputs(N, 11 + N[0])
    want, it, _ = O.cg(start, f, O.meshsizes(L, N), 0.0, fixed_iters=k)
    u = dev(start)
    st = X.cg(dev(f), u, L, eps=0.0, fixed_iters=[k], profile=1)
    assert engine in st["profile"], st["profile"].keys()
    assert st["iters"][0] == k
    assert rel_linf(u.cpu().numpy(), want) <= 1e-10


@pytest.mark.parametrize("N,L,engine", [((16, 8, 4), (1.0, 1.0, 1.0), "cg_cluster_f64"),
                                        ((40, 24, 12), (1.0, 0.8, 0.4), "cg_resident_f64"),
                                        ((64, 32, 16), (1.0, 1.0, 1.0), "cg_resident_f64"),
                                        ((50, 36, 22), (1.0, 0.9, 0.6), "cg_resident_f64")])
def test_engine_tolerance_stop(X, N, L, engine):
    """At a tolerance: the same stopping test on the recursive residual, so the step
    counts agree to one (rounding near the threshold) and both meet the tolerance."""
    f, start = _inputs(N, 3)
    h = O.meshsizes(L, N)
    eps = 1e-10
    want, it, rel = O.cg(start, f, h, eps)
    u = dev(start)
    st = X.cg(dev(f), u, L, eps=eps, profile=1)
    assert engine in st["profile"]
    assert st["relres"][0] <= eps
    assert abs(st["iters"][0] - it) <= 1
    # both are within the tolerance of the discrete solution: compare at that scale
    assert rel_linf(u.cpu().numpy(), want) <= 1e-7
    # the reported residual is the true one: recompute it from the GPU solution
    uh = u.cpu().numpy()
    r = O.residual(uh, f, h)
    b = O.rhs_vector(f, start, h)
    assert np.sqrt(np.sum(r * r)) <= 1.01 * eps * np.sqrt(np.sum(b * b))


def test_engine_zero_steps_from_solution(X):
    """Starting from the discrete solution the residual kernel stops the loop at once,
    whatever the engine: 0 steps, u unchanged."""
    for N in [(16, 8, 4), (64, 32, 16)]:
        f, start = _inputs(N, 7)
        h = O.meshsizes((1.0, 1.0, 1.0), N)
        sol, _, _ = O.cg(start, f, h, 1e-15, max_iter=5000)
        u = dev(sol)
        st = X.cg(dev(f), u, (1.0, 1.0, 1.0), eps=1e-8)
        assert st["iters"][0] == 0
        assert np.array_equal(u.cpu().numpy(), sol)
