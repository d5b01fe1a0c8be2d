"""Pins of the oracle's extrapolation / interpolation (Sections 3.2-3.3) and gradient."""
import itertools
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle as O
from conftest import read_golden
from paper_1507_05063_gb300 import problems as P


def test_quartic_weights_match_printed_equations():
    rows = {r[0]: [int(v) for v in r[2:]] for r in read_golden("quartic_weights.txt")}
    exact = O.quartic_weights_exact()  # t = 1/2, 3/2, 5/2, 7/2
    assert exact[0] == [Fraction(v) for v in rows["sifen1"]]
    assert exact[1] == [Fraction(v) for v in rows["sifen2"]]
    # reading: printed sifen3/sifen4 rows are swapped relative to the points they name
    assert exact[2] == [Fraction(v) for v in rows["sifen4"]]
    assert exact[3] == [Fraction(v) for v in rows["sifen3"]]
    for row in exact:
        assert sum(row) == 128


def test_triquartic_reproduces_triquartic_polynomials():
    M, idx = O.triquartic_cell_matrix()
    rng = np.random.default_rng(3)
    c = rng.standard_normal((5, 5, 5))

    def poly(x, y, z):
        return sum(c[p, q, r] * x ** p * y ** q * z ** r
                   for p, q, r in itertools.product(range(5), repeat=3))
    known = np.array([poly(i, j, k) for k in range(5) for j in range(5) for i in range(5)])
    got = M @ known
    want = np.array([poly(a / 2, b / 2, cc / 2) for cc, b, a in idx])
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-9)
    # and degree 5 in one variable is not reproduced
    known5 = np.array([float(i) ** 5 for k in range(5) for j in range(5) for i in range(5)])
    want5 = np.array([(a / 2) ** 5 for cc, b, a in idx])
    assert np.max(np.abs(M @ known5 - want5)) > 1e-3


def _levels_with_expansion(N2, seed):
    """u^i = U + A(x) (2^(2-i))^4 delta at the nodes of Z_i, A trilinear, U tri-quartic."""
    rng = np.random.default_rng(seed)
    cu = rng.standard_normal((5, 5, 5))
    ca = rng.standard_normal((2, 2, 2))
    L = (1.0, 1.0, 1.0)

    def U(x, y, z):
        return sum(cu[p, q, r] * x ** p * y ** q * z ** r
                   for p, q, r in itertools.product(range(5), repeat=3))

    def A(x, y, z):
        return sum(ca[p, q, r] * x ** p * y ** q * z ** r
                   for p, q, r in itertools.product(range(2), repeat=3))

    def on(N, fn):
        x, y, z = P.node_coords(L, N)
        return np.broadcast_to(fn(x, y, z), (N[2] + 1, N[1] + 1, N[0] + 1)).astype(np.float64)
    delta = 1e-3
    N1 = tuple(n // 2 for n in N2)
    N0 = tuple(n // 4 for n in N2)
    u0 = on(N0, lambda x, y, z: U(x, y, z) + 256 * delta * A(x, y, z))
    u1 = on(N1, lambda x, y, z: U(x, y, z) + 16 * delta * A(x, y, z))
    u2 = on(N2, lambda x, y, z: U(x, y, z) + delta * A(x, y, z))
    uexact = on(N2, U)
    return u0, u1, u2, uexact


@pytest.mark.parametrize("N2", [(16, 8, 24), (8, 8, 8)])
def test_exp_finite_exact_under_error_expansion(N2):
    """eqs. jiedian / zhongdian + tri-quartic: if u^i = U + A h_i^4 exactly (eq. asy
    without the O(h^6) term) with trilinear A and tri-quartic U, w^2 = u^2 everywhere."""
    u0, u1, u2, _ = _levels_with_expansion(N2, 1)
    w = O.exp_finite(u1, u0)
    np.testing.assert_allclose(w, u2, rtol=1e-12, atol=1e-10)
    # the values at the 125 known nodes of every cell (eqs. jiedian / zhongdian)
    W = O.extrapolate_fd(u1, u0)
    np.testing.assert_allclose(W, u2[::2, ::2, ::2], rtol=1e-12, atol=1e-10)


def test_exp_true_exact_under_error_expansion():
    """eqs. t1 / chenlin: u~ = U exactly when u_h = U + A h^4, u_2h = U + 16 A h^4."""
    _, u1, u2, uexact = _levels_with_expansion((16, 8, 24), 2)
    ut = O.extrapolate_true(u2, u1)
    np.testing.assert_allclose(ut, uexact, rtol=1e-12, atol=1e-10)


def test_exp_true_is_not_interpolation_free_of_d():
    """With a non-trilinear A the midpoint rule leaves an O(h^2)-relative defect (so the
    test above is not vacuous)."""
    rng = np.random.default_rng(4)
    u1 = rng.standard_normal((9, 9, 9))
    u2 = rng.standard_normal((17, 17, 17))
    ut = O.extrapolate_true(u2, u1)
    d = u2[::2, ::2, ::2] - u1
    # an x-edge midpoint by hand: u + (d_j + d_{j+1}) / 30
    k, j, i = 4, 6, 5
    want = u2[k, j, i] + (d[k // 2, j // 2, (i - 1) // 2] + d[k // 2, j // 2, (i + 1) // 2]) / 30
    assert ut[k, j, i] == pytest.approx(want, rel=1e-14)
    # a body centre by hand: mean over the four space diagonals
    k, j, i = 3, 5, 7
    corners = [(dk, dj, di) for dk in (0, 1) for dj in (0, 1) for di in (0, 1)]
    dsum = sum(d[(k - 1) // 2 + dk, (j - 1) // 2 + dj, (i - 1) // 2 + di] for dk, dj, di in corners)
    assert ut[k, j, i] == pytest.approx(u2[k, j, i] + dsum / 120, rel=1e-13)
    # corner by hand
    assert ut[4, 2, 6] == pytest.approx((16 * u2[4, 2, 6] - u1[2, 1, 3]) / 15, rel=1e-14)


def test_exp_finite_on_polynomial_fd_solution():
    """A degree-<=4 solution is reproduced by the scheme on every grid, so w_h = u_h."""
    rng = np.random.default_rng(9)
    coef = {(p, q, r): rng.standard_normal()
            for p, q, r in itertools.product(range(5), repeat=3) if p + q + r <= 4}

    def U(x, y, z):
        return sum(c * x ** p * y ** q * z ** r for (p, q, r), c in coef.items())
    L = (1.0, 2.0, 1.5)
    grids = [(8, 4, 4), (16, 8, 8), (32, 16, 16)]
    us = []
    for N in grids:
        x, y, z = P.node_coords(L, N)
        us.append(np.broadcast_to(U(x, y, z), (N[2] + 1, N[1] + 1, N[0] + 1)).astype(np.float64))
    w = O.exp_finite(us[1], us[0])
    np.testing.assert_allclose(w, us[2], rtol=1e-12, atol=1e-11)


def _poly1d_lines(deg, n, h, rng):
    c = rng.standard_normal(deg + 1)
    x = np.arange(n + 1) * h
    return np.polynomial.polynomial.polyval(x, c), np.polynomial.polynomial.polyval(
        x, np.polynomial.polynomial.polyder(c))


@pytest.mark.parametrize("n", [4, 5, 9, 16])
def test_gradient_exact_for_quartics(n):
    rng = np.random.default_rng(n)
    h = 0.37
    U, dU = _poly1d_lines(4, n, h, rng)
    D = O.excmg_oracle._derivative_lines(U[None, :], h)[0]
    np.testing.assert_allclose(D, dU, rtol=1e-11, atol=1e-10)
    U5, dU5 = _poly1d_lines(5, n, h, rng)
    D5 = O.excmg_oracle._derivative_lines(U5[None, :], h)[0]
    assert np.max(np.abs(D5 - dU5)) > 1e-8


def test_thomas_matches_dense_banded_solve():
    rng = np.random.default_rng(1)
    n, h = 23, 0.1
    U = rng.standard_normal((3, n + 1))
    D = O.excmg_oracle._derivative_lines(U, h)
    for line in range(3):
        ab = np.zeros((3, n - 1))
        ab[0, 1:] = 1 / 6
        ab[1, :] = 4 / 6
        ab[2, :-1] = 1 / 6
        rhs = (U[line, 2:] - U[line, :-2]) / (2 * h)
        rhs[0] -= D[line, 0] / 6
        rhs[-1] -= D[line, n] / 6
        x = scipy.linalg.solve_banded((1, 1), ab, rhs)
        np.testing.assert_allclose(D[line, 1:n], x, rtol=1e-12, atol=1e-12)


def test_gradient_3d_exact_for_tensor_quartics():
    rng = np.random.default_rng(7)
    cx, cy, cz = (rng.standard_normal(5) for _ in range(3))
    pv = np.polynomial.polynomial.polyval
    pd = np.polynomial.polynomial.polyder
    L, N = (1.0, 0.5, 2.0), (6, 5, 8)
    x, y, z = P.node_coords(L, N)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    u = np.broadcast_to(pv(x, cx) * pv(y, cy) * pv(z, cz), shape).astype(np.float64)
    gx, gy, gz = O.gradient(u, O.meshsizes(L, N))
    np.testing.assert_allclose(gx, np.broadcast_to(pv(x, pd(cx)) * pv(y, cy) * pv(z, cz), shape),
                               rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(gy, np.broadcast_to(pv(x, cx) * pv(y, pd(cy)) * pv(z, cz), shape),
                               rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(gz, np.broadcast_to(pv(x, cx) * pv(y, cy) * pv(z, pd(cz)), shape),
                               rtol=1e-10, atol=1e-9)


# ---- comparison prolongations (tri-quadratic after extrapolation; trilinear) ----

@pytest.mark.parametrize("P_", [2, 3])
def test_lagrange_cell_matrix_reproduces_its_degree_only(P_):
    """P nodes per direction reproduce every polynomial of degree < P in each variable at
    the half steps of the cell, and not x^P."""
    M, idx = O.lagrange_cell_matrix(P_)
    assert M.shape == ((2 * P_ - 1) ** 3 - P_ ** 3, P_ ** 3)
    rng = np.random.default_rng(P_)
    c = rng.standard_normal((P_, P_, P_))

    def poly(x, y, z):
        return sum(c[p, q, r] * x ** p * y ** q * z ** r
                   for p, q, r in itertools.product(range(P_), repeat=3))
    rng_nodes = range(P_)
    known = np.array([poly(i, j, k) for k in rng_nodes for j in rng_nodes for i in rng_nodes])
    want = np.array([poly(a / 2, b / 2, cc / 2) for cc, b, a in idx])
    np.testing.assert_allclose(M @ known, want, rtol=1e-12, atol=1e-12)
    knownP = np.array([float(i) ** P_ for k in rng_nodes for j in rng_nodes for i in rng_nodes])
    wantP = np.array([(a / 2) ** P_ for cc, b, a in idx])
    assert np.max(np.abs(M @ knownP - wantP)) > 1e-2
    # every row is a partition of unity
    np.testing.assert_allclose(M.sum(axis=1), 1.0, rtol=0, atol=1e-14)


def test_quadratic_weights_by_hand():
    """1D quadratic Lagrange on nodes 0, 1, 2 at t = 1/2: (3, 6, -1)/8; at 3/2: (-1, 6, 3)/8."""
    M, idx = O.lagrange_cell_matrix(3)
    row = {t: r for r, t in zip(M, idx)}
    np.testing.assert_array_equal(row[(0, 0, 1)][:3], [3 / 8, 6 / 8, -1 / 8])
    np.testing.assert_array_equal(row[(0, 0, 3)][:3], [-1 / 8, 6 / 8, 3 / 8])


def test_prolong_linear_is_trilinear_interpolation():
    """CMG prolongation: exact for trilinear functions on any grid; a body centre is the
    mean of its 8 corners."""
    rng = np.random.default_rng(5)
    ca = rng.standard_normal((2, 2, 2))
    L = (1.0, 0.5, 2.0)

    def A(x, y, z):
        return sum(ca[p, q, r] * x ** p * y ** q * z ** r
                   for p, q, r in itertools.product(range(2), repeat=3))
    N1, N2 = (6, 4, 2), (12, 8, 4)
    on = lambda N: np.broadcast_to(A(*P.node_coords(L, N)), (N[2] + 1, N[1] + 1, N[0] + 1))
    np.testing.assert_allclose(O.prolong_linear(on(N1)), on(N2), rtol=1e-13, atol=1e-13)
    u = rng.standard_normal((5, 4, 7))
    w = O.prolong_linear(u)
    assert w[3, 1, 5] == pytest.approx(u[1:3, 0:2, 2:4].mean(), rel=1e-14)
    np.testing.assert_array_equal(w[::2, ::2, ::2], u)


@pytest.mark.parametrize("N2", [(16, 8, 24), (8, 8, 8)])
def test_prolong_quadratic_exact_under_error_expansion(N2):
    """Extrapolation + tri-quadratic: if u^i = U + A h_i^4 with trilinear A and
    tri-quadratic U, w^2 = u^2 everywhere; with a tri-quartic U it is not (the
    interpolation is then the error, as the first remark of Section 3.3 says)."""
    rng = np.random.default_rng(7)
    L = (1.0, 1.0, 1.0)
    ca = rng.standard_normal((2, 2, 2))
    N1 = tuple(n // 2 for n in N2)
    N0 = tuple(n // 4 for n in N2)

    def levels(deg):
        cu = rng.standard_normal((deg + 1,) * 3)

        def fn(x, y, z, s):
            U = sum(cu[p, q, r] * x ** p * y ** q * z ** r
                    for p, q, r in itertools.product(range(deg + 1), repeat=3))
            A = sum(ca[p, q, r] * x ** p * y ** q * z ** r
                    for p, q, r in itertools.product(range(2), repeat=3))
            return U + s * 1e-3 * A
        on = lambda N, s: np.broadcast_to(fn(*P.node_coords(L, N), s),
                                          (N[2] + 1, N[1] + 1, N[0] + 1)).astype(np.float64)
        return on(N0, 256.0), on(N1, 16.0), on(N2, 1.0)
    u0, u1, u2 = levels(2)
    np.testing.assert_allclose(O.prolong_quadratic(u1, u0), u2, rtol=1e-12, atol=1e-11)
    u0, u1, u2 = levels(4)
    assert np.max(np.abs(O.prolong_quadratic(u1, u0) - u2)) > 1e-6


def test_prolongation_orders_on_example1():
    """||w_h - u_h||_2 on Example 1 (16^3 -> 32^3): EXP_finite is fifth order (Tables 1-2);
    extrapolation + tri-quadratic falls to the interpolation's third order; trilinear CMG
    to second order.  The finest-grid CG step counts follow the same ranking."""
    prob = P.PROBLEMS["ex1"]
    orders, iters = {}, {}
    for kind in ("quartic", "quadratic", "linear"):
        errs = []
        for N in [(16, 16, 16), (32, 32, 32)]:
            f, g, _ = P.make_inputs(prob, N)
            res = O.excmg(f, g, (1, 1, 1), N, (4, 4, 4), eps=1e-10, dsolve="dense",
                          want_utilde=False, prolong_kind=kind)
            w = O.with_boundary(res["w"][-1], g)
            errs.append(O.l2_norm(w - res["u"][-1]))
            iters[kind] = res["iters"][-1]
        orders[kind] = O.observed_order(errs[0], errs[1])
    assert 4.7 < orders["quartic"] < 5.4
    assert 2.5 < orders["quadratic"] < 3.4
    assert 1.6 < orders["linear"] < 2.3
    assert iters["quartic"] < iters["quadratic"] < iters["linear"]
