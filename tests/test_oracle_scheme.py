"""Pins of the oracle's compact scheme and CG (Section 2, eq. compact / FD; Algorithm 1)."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1507_05063_gb300 import problems as P


def _poly(coef):
    """u = sum c[p,q,r] x^p y^q z^r and its Laplacian, as callables."""
    def u(x, y, z):
        return sum(c * x ** p * y ** q * z ** r for (p, q, r), c in coef.items())

    def lap(x, y, z):
        out = 0.0
        for (p, q, r), c in coef.items():
            if p >= 2:
                out = out + c * p * (p - 1) * x ** (p - 2) * y ** q * z ** r
            if q >= 2:
                out = out + c * q * (q - 1) * x ** p * y ** (q - 2) * z ** r
            if r >= 2:
                out = out + c * r * (r - 1) * x ** p * y ** q * z ** (r - 2)
        return out
    return u, lap


def _grid(L, N):
    x, y, z = P.node_coords(L, N)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    return x, y, z, shape


def _scheme_residual(coef, L, N):
    u, lap = _poly(coef)
    x, y, z, shape = _grid(L, N)
    U = np.broadcast_to(u(x, y, z), shape).astype(np.float64)
    F = np.broadcast_to(lap(x, y, z) + np.zeros(shape), shape).astype(np.float64)
    h = O.meshsizes(L, N)
    r = O.residual(U, F, h)
    scale = np.max(np.abs(O.lhs(np.abs(U), h))) + np.max(np.abs(O.rhs(np.abs(F))))
    return np.max(np.abs(r)) / scale


@pytest.mark.parametrize("L,N", [((1.0, 1.0, 1.0), (6, 5, 7)), ((1.3, 0.7, 2.1), (8, 4, 6)),
                                 ((1.0, 1.0, 1.0), (12, 3, 5))])
def test_exact_for_total_degree_5(L, N):
    rng = np.random.default_rng(5)
    coef = {(p, q, r): rng.standard_normal()
            for p, q, r in itertools.product(range(6), repeat=3) if p + q + r <= 5}
    assert _scheme_residual(coef, L, N) < 1e-13


@pytest.mark.parametrize("mono", [(6, 0, 0), (0, 6, 0), (0, 0, 6), (4, 2, 0), (2, 4, 0)])
def test_not_exact_for_degree_6(mono):
    """Pure sixth derivatives leave an O(h^4) truncation error (eq. asy): the scheme is
    not exact beyond degree 5 (mixed monomials such as x^2 y^2 z^2 happen to be exact)."""
    assert _scheme_residual({mono: 1.0}, (1.3, 0.7, 2.1), (8, 4, 6)) > 1e-8


def test_weight_moments():
    """Zeroth and second moments of the seven weights: constants map to 0 and x^2, y^2,
    z^2 map to 12 = 6 * Laplacian (the printed RHS weights also sum to 6)."""
    h = (0.1, 0.17, 0.23)
    base = O.coefficients(*h)
    a, b, c = (1 / v ** 2 for v in h)
    assert base["centre"] == pytest.approx(-8 * (a + b + c))
    # weights sum to zero (constants are exact): centre + 2 faces + 4 edges per plane
    total = base["centre"] + 2 * (base["fx"] + base["fy"] + base["fz"]) + 4 * (
        base["exy"] + base["exz"] + base["eyz"])
    assert abs(total) < 1e-9 * abs(base["centre"])
    # second moments: sum w * dx^2 = 12 = 6 * (d^2/dx^2 of x^2)
    m_xx = (2 * base["fx"] + 4 * base["exy"] + 4 * base["exz"]) * h[0] ** 2
    m_yy = (2 * base["fy"] + 4 * base["exy"] + 4 * base["eyz"]) * h[1] ** 2
    m_zz = (2 * base["fz"] + 4 * base["exz"] + 4 * base["eyz"]) * h[2] ** 2
    assert m_xx == pytest.approx(12.0) and m_yy == pytest.approx(12.0) and m_zz == pytest.approx(12.0)


@pytest.mark.parametrize("N,L", [((4, 5, 6), (1.0, 1.0, 1.0)), ((6, 3, 4), (1.0, 3.0, 0.4))])
def test_negated_operator_is_spd(N, L):
    """Reading of eq. (FD): A = -(printed LHS) is symmetric positive definite."""
    h = O.meshsizes(L, N)
    M = O.dense_matrix(N, h)
    assert np.array_equal(M, M.T)
    ev = np.linalg.eigvalsh(M)
    assert ev.min() > 0


def test_symbol_ratio_bounds():
    """The negated 19-point symbol is 2 sum_d a_d X_d (6 - X_e - X_f) with X_d = 1 - cos t_d,
    so over sum_d a_d X_d it lies in [4, 12] for any aspect ratio: A is SPD and within 3x
    of the 7-point Laplacian's conditioning."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        h = np.exp(rng.uniform(-2.5, 2.5, 3))
        w = O.coefficients(*h)
        t = rng.uniform(0, np.pi, (3, 400))
        cx, cy, cz = np.cos(t)
        s19 = -(w["centre"] + 2 * w["fx"] * cx + 2 * w["fy"] * cy + 2 * w["fz"] * cz
                + 4 * w["exy"] * cx * cy + 4 * w["exz"] * cx * cz + 4 * w["eyz"] * cy * cz)
        s7 = sum((1 - c) / hh ** 2 for c, hh in zip((cx, cy, cz), h))
        ratio = s19 / s7
        assert ratio.min() >= 4 - 1e-9 and ratio.max() <= 12 + 1e-9


def test_rhs_vector_includes_lift_and_matches_dense():
    """b = LHS_IB g - RHS f and A u_I = b hold for the exact discrete solution."""
    N, L = (5, 4, 6), (1.0, 1.0, 1.0)
    h = O.meshsizes(L, N)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex1"], N, L)
    u = O.dense_solve(g, f, h)
    assert np.max(np.abs(O.residual(u, f, h))) < 1e-9 * np.max(np.abs(O.rhs_vector(f, g, h)))
    # A u_I - b = -(LHS(u) - RHS f)
    Au = O.apply_A(u[1:-1, 1:-1, 1:-1], h)
    np.testing.assert_allclose(Au, O.rhs_vector(f, g, h), rtol=1e-10, atol=1e-9)


@pytest.mark.parametrize("name,N,L", [("ex1", (6, 6, 6), (1, 1, 1)), ("ex4", (7, 5, 4), (1, 1, 1)),
                                      ("ex2", (4, 6, 5), (1.0, 2.0, 0.5))])
def test_cg_matches_dense_cholesky(name, N, L):
    h = O.meshsizes(L, N)
    f, g, _ = P.make_inputs(P.PROBLEMS[name], N, L)
    ud = O.dense_solve(g, f, h)
    start = g.copy()
    start[1:-1, 1:-1, 1:-1] = 0.0
    uc, it, rel = O.cg(start, f, h, 1e-14)
    assert rel <= 1e-14 and it > 0
    assert np.max(np.abs(uc - ud)) <= 1e-11 * np.max(np.abs(ud))


def test_cg_zero_iterations_when_start_is_solution():
    N, L = (6, 6, 6), (1, 1, 1)
    h = O.meshsizes(L, N)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex3"], N, L)
    ud = O.dense_solve(g, f, h)
    _, it, _ = O.cg(ud, f, h, 1e-9)
    assert it == 0


def test_polynomial_solution_reproduced_by_excmg():
    """For u of total degree <= 5 the FD solution equals u, so EXCMG returns u."""
    rng = np.random.default_rng(11)
    coef = {(p, q, r): rng.standard_normal()
            for p, q, r in itertools.product(range(6), repeat=3) if p + q + r <= 5}
    u, lap = _poly(coef)
    N, N0, L = (32, 16, 16), (8, 4, 4), (1.0, 1.0, 1.0)
    x, y, z, shape = _grid(L, N)
    U = np.broadcast_to(u(x, y, z), shape).astype(np.float64).copy()
    F = (np.broadcast_to(lap(x, y, z) + np.zeros(shape), shape)).astype(np.float64).copy()
    res = O.excmg(F, U, L, N, N0, eps=1e-13, eps_coarse=1e-13)
    assert np.max(np.abs(res["u"][-1] - U)) < 1e-10 * np.max(np.abs(U))
