"""Pins of the oracle's adjoint of the discrete solve (project addition, no paper
counterpart): central finite differences of forward solves, and an explicit dense
B^T A^{-1} product on a tiny grid."""
import numpy as np
import pytest

import oracle as O
from paper_1507_05063_gb300 import problems as P


def _solve(f, g, h):
    return O.dense_solve(g, f, h)


def _loss(u, ut):
    return float(np.sum((u - ut) ** 2))


@pytest.fixture(scope="module")
def setup():
    N, L = (5, 4, 6), (1.0, 1.3, 0.8)
    h = O.meshsizes(L, N)
    rng = np.random.default_rng(2)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    f = rng.standard_normal(shape)
    g = rng.standard_normal(shape)
    ut = rng.standard_normal(shape)
    return N, L, h, f, g, ut


def test_adjoint_matches_central_differences(setup):
    N, L, h, f, g, ut = setup
    u = _solve(f, g, h)
    dLdu = 2.0 * (u - ut)
    dLdf, dLdg, _ = O.adjoint(dLdu, h, dense=True)
    rng = np.random.default_rng(0)
    delta = 1e-4
    shape = f.shape
    for _ in range(12):
        m = tuple(int(rng.integers(0, s)) for s in shape)
        fp, fm = f.copy(), f.copy()
        fp[m] += delta
        fm[m] -= delta
        fd = (_loss(_solve(fp, g, h), ut) - _loss(_solve(fm, g, h), ut)) / (2 * delta)
        assert dLdf[m] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    bmask = np.ones(shape, dtype=bool)
    bmask[1:-1, 1:-1, 1:-1] = False
    bidx = np.argwhere(bmask)
    for m in bidx[rng.choice(len(bidx), 12, replace=False)]:
        m = tuple(m)
        gp, gm = g.copy(), g.copy()
        gp[m] += delta
        gm[m] -= delta
        fd = (_loss(_solve(f, gp, h), ut) - _loss(_solve(f, gm, h), ut)) / (2 * delta)
        assert dLdg[m] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # interior g entries are never read
    assert np.all(dLdg[1:-1, 1:-1, 1:-1] == 0)


def test_adjoint_dense_product(setup):
    """dL/df = -R^T A^{-1} (dL/du)_I with R the 7-point RHS operator, built densely."""
    N, L, h, f, g, ut = setup
    shape = f.shape
    rng = np.random.default_rng(5)
    dLdu = rng.standard_normal(shape)
    A = O.dense_matrix(N, h)
    n_all = f.size
    R = np.zeros((A.shape[0], n_all))
    for m in range(n_all):
        e = np.zeros(n_all)
        e[m] = 1.0
        R[:, m] = O.rhs(e.reshape(shape)).ravel()
    want = -(R.T @ np.linalg.solve(A, dLdu[1:-1, 1:-1, 1:-1].ravel())).reshape(shape)
    got, _, _ = O.adjoint(dLdu, h, dense=True)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12)
    got_cg, _, _ = O.adjoint(dLdu, h, eps=1e-15)
    np.testing.assert_allclose(got_cg, want, rtol=1e-9, atol=1e-10 * np.max(np.abs(want)))
