"""Plain FP64 CPU oracle for EXCMG + the 19-point fourth-order compact scheme.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference arm, never by the product path.  Nothing here is tuned: every
routine is the paper's definition written out with numpy slicing, in float64, so that a
reader can check it against the paper by eye.

Array convention: a node array on a grid of Nx x Ny x Nz cells has numpy shape
(Nz+1, Ny+1, Nx+1) and is indexed [k, j, i]; node (i, j, k) sits at (i hx, j hy, k hz)
(Section 2).  "Interior" arrays have shape (Nz-1, Ny-1, Nx-1).

Readings of the paper taken here (the CUDA path takes the same ones):
* Sign (Section 2, eq. FD): the printed left-hand side is negative definite; the SPD
  matrix is A = -(printed LHS restricted to the interior), b = -(printed RHS minus the
  boundary terms).  ``residual`` returns b - A u_I = LHS(u) - RHS(f).
* ||f_h|| in the stopping test of Algorithm 1 has two readings (``rhs_norm``), each pinned
  against the printed results it reproduces.  "lift" (the default): the 2-norm of the
  assembled right-hand side b of eq. (FD), Dirichlet lift included; it reproduces the
  finest-grid step counts of Table 11.  "forcing": the 2-norm of the right-hand side of
  eq. (compact) alone, (6 f + sum of the six face values)/2 at the interior nodes, which
  is how Section 2 defines f_h after eq. (FD); it reproduces the errors of Tables 1-10
  on the 128^3 meshes where the algebraic error shows.  Where that vector is zero
  (Example 2 has f = 0) the forcing reading falls back to the lift reading, since no
  relative test against a zero norm can ever pass.
* The WHILE loop of Algorithm 1 runs one CG step per pass; the test uses CG's
  recursively updated residual and is made before the first step.
* DSOLVE on the two coarsest grids is CG to a tight tolerance, or a dense Cholesky
  solve when asked (``dsolve='dense'``).
* Coarse-grid f and g are the finest-grid node values at the coarse nodes (nested
  grids, so injection equals evaluation).
* The quartic weights are computed from the Lagrange basis of Section 3.3; the printed
  labels of eqs. sifen3 and sifen4 are swapped relative to the points they name.
* w_h = EXP_finite(...) keeps the tri-quartic values on its boundary nodes (Table 1's
  ||w_h - u_h||_2 column is reproduced only so); CG starts from the interior values of
  w_h with the Dirichlet data on the boundary.
* Discrete norms: ||v||_2 = sqrt(mean over all nodes of v^2) (root mean square; Tables 1,
  3, 5 are reproduced only so), ||v||_inf = max |v|; for a gradient error e,
  sqrt(mean over all nodes of |e|^2) and the max over nodes and components.
"""

from __future__ import annotations

from fractions import Fraction

import numpy as np

__all__ = [
    "coefficients", "lhs", "rhs", "residual", "apply_A", "rhs_vector", "cg",
    "dense_matrix", "dense_solve", "quartic_weights", "quartic_weights_exact",
    "lagrange_basis", "triquartic_cell_matrix", "extrapolate_fd", "exp_finite", "with_boundary",
    "extrapolate_true", "gradient", "excmg", "level_sizes", "l2_norm", "linf_norm",
    "grad_l2_norm", "grad_linf_norm", "adjoint", "rhs_transpose", "lift_transpose",
    "meshsizes", "observed_order", "lagrange_cell_matrix", "prolong_quadratic",
    "prolong_linear", "prolong", "stopping_norm",
]


# --------------------------------------------------------------------------------------
# Section 2: the 19-point compact scheme, eq. (compact), and its matrix form, eq. (FD)
# --------------------------------------------------------------------------------------

def meshsizes(L, N):
    """hx = Lx/Nx, hy = Ly/Ny, hz = Lz/Nz (Section 2)."""
    return tuple(float(Ld) / int(Nd) for Ld, Nd in zip(L, N))


def coefficients(hx, hy, hz):
    """The seven distinct weights of the printed left-hand side of eq. (compact).

    a = 1/hx^2, b = 1/hy^2, c = 1/hz^2.  Centre -8(a+b+c); the x-face pair 4a-b-c,
    the y-face pair 4b-a-c, the z-face pair 4c-a-b; the four xy-edge neighbours (a+b)/2,
    the four xz-edge neighbours (a+c)/2 and the four yz-edge neighbours (b+c)/2.
    """
    a, b, c = 1.0 / hx**2, 1.0 / hy**2, 1.0 / hz**2
    return {
        "centre": -8.0 * (a + b + c),
        "fx": 4.0 * a - b - c,
        "fy": 4.0 * b - a - c,
        "fz": 4.0 * c - a - b,
        "exy": 0.5 * (a + b),
        "exz": 0.5 * (a + c),
        "eyz": 0.5 * (b + c),
    }


def _shift(u, dk, dj, di):
    """View of the full node array u at interior nodes offset by (di, dj, dk)."""
    nz, ny, nx = u.shape
    return u[1 + dk:nz - 1 + dk, 1 + dj:ny - 1 + dj, 1 + di:nx - 1 + di]


def lhs(u, h):
    """Printed left-hand side of eq. (compact) at every interior node.

    ``u`` is a full node array (boundary entries included); returns an interior array.
    """
    w = coefficients(*h)
    s = lambda dk, dj, di: _shift(u, dk, dj, di)  # noqa: E731
    out = w["centre"] * s(0, 0, 0)
    out = out + w["fx"] * (s(0, 0, 1) + s(0, 0, -1))
    out = out + w["fy"] * (s(0, 1, 0) + s(0, -1, 0))
    out = out + w["fz"] * (s(1, 0, 0) + s(-1, 0, 0))
    out = out + w["exy"] * (s(0, 1, 1) + s(0, -1, 1) + s(0, 1, -1) + s(0, -1, -1))
    out = out + w["exz"] * (s(1, 0, 1) + s(-1, 0, 1) + s(1, 0, -1) + s(-1, 0, -1))
    out = out + w["eyz"] * (s(1, 1, 0) + s(1, -1, 0) + s(-1, 1, 0) + s(-1, -1, 0))
    return out


def rhs(f):
    """Printed right-hand side of eq. (compact): (6 f_c + sum of the 6 face f) / 2.

    ``f`` is given on all nodes (face neighbours of interior nodes may be boundary
    nodes); returns an interior array.
    """
    s = lambda dk, dj, di: _shift(f, dk, dj, di)  # noqa: E731
    return 0.5 * (6.0 * s(0, 0, 0) + s(0, 0, 1) + s(0, 0, -1) + s(0, 1, 0)
                  + s(0, -1, 0) + s(1, 0, 0) + s(-1, 0, 0))


def residual(u, f, h):
    """b - A u_I for the SPD form A = -LHS_II of eq. (FD): equals LHS(u) - RHS(f).

    ``u`` carries the Dirichlet values on its boundary nodes.
    """
    return lhs(u, h) - rhs(f)


def _embed(v_interior):
    nz, ny, nx = v_interior.shape
    full = np.zeros((nz + 2, ny + 2, nx + 2))
    full[1:-1, 1:-1, 1:-1] = v_interior
    return full


def apply_A(v, h):
    """A v for interior vectors v, A = -(printed LHS with zero boundary values)."""
    return -lhs(_embed(v), h)


def rhs_vector(f, g, h):
    """Assembled right-hand side b of eq. (FD): b = LHS_IB g - RHS(f).

    ``g`` is a full node array whose boundary entries hold the Dirichlet data (its
    interior entries are ignored).
    """
    gb = np.array(g, dtype=np.float64, copy=True)
    gb[1:-1, 1:-1, 1:-1] = 0.0
    return lhs(gb, h) - rhs(f)


# --------------------------------------------------------------------------------------
# Algorithm 1, its WHILE loop: CG with the relative-residual stopping criterion
# --------------------------------------------------------------------------------------

def stopping_norm(f, g, h, rhs_norm="lift"):
    """||f_h||_2 of the WHILE test of Algorithm 1, under one of its two readings.

    "lift": f_h is the assembled right-hand side b = LHS_IB g - RHS(f) of eq. (FD).
    "forcing": f_h is the right-hand side vector of eq. (compact) as Section 2 defines it
    after eq. (FD), RHS(f) = (6 f + the six face values of f)/2 at the interior nodes;
    when it is zero (f = 0, Example 2) the lift reading is used instead.
    """
    if rhs_norm not in ("lift", "forcing"):
        raise ValueError(rhs_norm)
    if rhs_norm == "forcing":
        rf = rhs(f)
        norm = np.sqrt(np.sum(rf * rf))
        if norm > 0:
            return norm
    b = rhs_vector(f, g, h)
    return np.sqrt(np.sum(b * b))


def cg(u0, f, h, eps, max_iter=100000, fixed_iters=None, history=None, rhs_norm="lift"):
    """Unpreconditioned CG on A u_I = b from the initial guess u0 (the WHILE loop of Algorithm 1).

    One CG step per pass of the WHILE loop; the loop test ||r||_2 <= eps ||f_h||_2 is
    made before every step on CG's recursively updated residual r, with ||f_h|| from
    ``stopping_norm`` under the reading ``rhs_norm``.  ``fixed_iters`` replaces the test
    by an exact step count.  Returns (u, iterations, final recursive residual relative to
    ||f_h||); u keeps u0's boundary values.
    """
    u = np.array(u0, dtype=np.float64, copy=True)
    g = u  # boundary entries of u0 are the Dirichlet data
    bnorm = stopping_norm(f, g, h, rhs_norm)
    x = u[1:-1, 1:-1, 1:-1].copy()
    r = residual(u, f, h)
    p = r.copy()
    rr = np.sum(r * r)
    k = 0
    if history is not None:
        history.append(np.sqrt(rr) / bnorm if bnorm > 0 else 0.0)

    def keep_going():
        if fixed_iters is not None:
            return k < fixed_iters
        return np.sqrt(rr) > eps * bnorm and k < max_iter

    while keep_going():
        q = apply_A(p, h)
        alpha = rr / np.sum(p * q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = np.sum(r * r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        k += 1
        if history is not None:
            history.append(np.sqrt(rr) / bnorm if bnorm > 0 else 0.0)
    u[1:-1, 1:-1, 1:-1] = x
    relres = np.sqrt(rr) / bnorm if bnorm > 0 else 0.0
    return u, k, relres


def dense_matrix(n_cells, h):
    """Dense A (interior unknowns, x fastest) assembled column by column from A e_m."""
    nx, ny, nz = n_cells
    n = (nx - 1) * (ny - 1) * (nz - 1)
    M = np.zeros((n, n))
    for m in range(n):
        e = np.zeros(n)
        e[m] = 1.0
        M[:, m] = apply_A(e.reshape(nz - 1, ny - 1, nx - 1), h).ravel()
    return M


def dense_solve(g, f, h):
    """DSOLVE of Algorithm 1 (the two coarsest grids) as a dense Cholesky solve (tiny grids only)."""
    nz, ny, nx = f.shape
    M = dense_matrix((nx - 1, ny - 1, nz - 1), h)
    b = rhs_vector(f, g, h).ravel()
    Lc = np.linalg.cholesky(M)
    y = np.linalg.solve(Lc, b)
    x = np.linalg.solve(Lc.T, y)
    u = np.array(g, dtype=np.float64, copy=True)
    u[1:-1, 1:-1, 1:-1] = x.reshape(nz - 2, ny - 2, nx - 2)
    return u


# --------------------------------------------------------------------------------------
# Section 3.2 / 3.3: extrapolation and quartic / tri-quartic Lagrange interpolation
# --------------------------------------------------------------------------------------

def lagrange_basis(i, xi, nodes=(0, 1, 2, 3, 4)):
    """l_i^4(xi) = prod_{k != i} (xi - xi_k) / (xi_i - xi_k) (Section 3.3)."""
    out = 1.0
    for k, xk in enumerate(nodes):
        if k != i:
            out = out * (xi - xk) / (nodes[i] - xk)
    return out


def quartic_weights_exact():
    """Exact weights (times 128) of the quartic interpolant at the four quarter points
    of a two-element patch, eqs. sifen1-sifen4, from the Lagrange basis.

    Natural coordinates: the five known values sit at t = 0, 1, 2, 3, 4 (the nodes
    x_j, x_{j+1/2}, x_{j+1}, x_{j+3/2}, x_{j+2}); the quarter points at t = 1/2, 3/2,
    5/2, 7/2.  Row q holds 128 l_i(t_q) for i = 0..4.
    """
    rows = []
    for t in (Fraction(1, 2), Fraction(3, 2), Fraction(5, 2), Fraction(7, 2)):
        rows.append([128 * lagrange_basis(i, t, nodes=tuple(Fraction(k) for k in range(5)))
                     for i in range(5)])
    return rows


def quartic_weights():
    """Float version of ``quartic_weights_exact`` divided by 128, shape (4, 5)."""
    return np.array([[float(v) / 128.0 for v in row] for row in quartic_weights_exact()])


def triquartic_cell_matrix():
    """The tri-quartic interpolation of eq. (inter) on one interpolation cell.

    Returns (M, fine_idx): M has one row per fine node of the 9x9x9 cell that is NOT one
    of the 125 known nodes (604 rows) and one column per known node (125 columns, index
    (k*5 + j)*5 + i); row entries are N_m = l_i(xi) l_j(eta) l_k(zeta) at that fine
    node.  fine_idx lists the (c, b, a) = (z, y, x) local fine indices (0..8) of the
    rows.  Natural coordinates: xi = a/2 etc.
    """
    rows, fine_idx = [], []
    for c in range(9):
        for b in range(9):
            for a in range(9):
                if a % 2 == 0 and b % 2 == 0 and c % 2 == 0:
                    continue
                xi, eta, zeta = a / 2.0, b / 2.0, c / 2.0
                row = np.empty(125)
                for k in range(5):
                    for j in range(5):
                        for i in range(5):
                            row[(k * 5 + j) * 5 + i] = (lagrange_basis(i, xi)
                                                        * lagrange_basis(j, eta)
                                                        * lagrange_basis(k, zeta))
                rows.append(row)
                fine_idx.append((c, b, a))
    M = np.array(rows)
    assert M.shape == (604, 125)
    return M, fine_idx


def _parity_classes(u_fine, u_coarse, node_rule, mid_coef):
    """Walk the nodes of the finer of two nested grids by parity class (Section 3.3).

    Nodes with all-even indices are coarse nodes and get ``node_rule(u_fine, u_coarse)``.
    Every other node is the midpoint of an edge, a face or a coarse element; it gets
    u_fine + mid_coef * (d_a + d_b) along each segment through it whose two ends are
    coarse nodes (an edge: one segment; a face centre: the two face diagonals; an
    element centre: the four space diagonals), averaged over those segments, where
    d = u_fine - u_coarse at coarse nodes.
    """
    W = np.empty_like(u_fine)
    d = u_fine[::2, ::2, ::2] - u_coarse
    W[0::2, 0::2, 0::2] = node_rule(u_fine[0::2, 0::2, 0::2], u_coarse)

    def D(dz, dy, dx, sz, sy, sx):
        # d at the coarse corner offset (dz, dy, dx) in {0,1} along each odd axis;
        # s* says whether the axis is odd (True) for this class.
        zs = slice(dz, d.shape[0] - 1 + dz) if sz else slice(None)
        ys = slice(dy, d.shape[1] - 1 + dy) if sy else slice(None)
        xs = slice(dx, d.shape[2] - 1 + dx) if sx else slice(None)
        return d[zs, ys, xs]

    for sz in (False, True):
        for sy in (False, True):
            for sx in (False, True):
                n_odd = sz + sy + sx
                if n_odd == 0:
                    continue
                sel = (slice(1, None, 2) if sz else slice(0, None, 2),
                       slice(1, None, 2) if sy else slice(0, None, 2),
                       slice(1, None, 2) if sx else slice(0, None, 2))
                uf = u_fine[sel]
                # corners of the segment set: enumerate offsets on the odd axes
                odd_axes = [ax for ax, s in zip((0, 1, 2), (sz, sy, sx)) if s]
                corners = []
                for bits in range(1 << n_odd):
                    off = [0, 0, 0]
                    for t, ax in enumerate(odd_axes):
                        off[ax] = (bits >> t) & 1
                    corners.append(tuple(off))
                # segments: pairs of opposite corners (each counted once)
                segs = []
                for cnr in corners:
                    opp = tuple((1 - cnr[ax]) if ax in odd_axes else 0 for ax in range(3))
                    if (opp, cnr) not in segs:
                        segs.append((cnr, opp))
                vals = [uf + mid_coef * (D(*ca, sz, sy, sx) + D(*cb, sz, sy, sx))
                        for ca, cb in segs]
                W[sel] = sum(vals) / len(vals)
    return W


def extrapolate_fd(u1, u0):
    """w^2 at the nodes of Z1 from u^1 (grid Z1) and u^0 (grid Z0), Section 3.3.

    Coarse (Z0) nodes: eq. (jiedian), w = (17 u^1 - u^0)/16.  Edge midpoints: eq.
    (zhongdian), w = u^1 + (d_j + d_{j+1})/32 with d = u^1 - u^0.  Face centres: mean of
    eq. (zhongdian) along the two face diagonals.  Element centres: mean of eq.
    (zhongdian) along the four space diagonals.
    """
    return _parity_classes(u1, u0, lambda a, b: (17.0 * a - b) / 16.0, 1.0 / 32.0)


def extrapolate_true(uh, u2h):
    """EXP_true(u_h, u_2h), Section 3.3: eq. (t1) (16 u^1 - u^0)/15 at the coarse nodes
    and eq. (chenlin) u^1 + (d_j + d_{j+1})/30 (averaged over the face / space
    diagonals as for w^2) at all other nodes of the fine grid.  No interpolation."""
    return _parity_classes(uh, u2h, lambda a, b: (16.0 * a - b) / 15.0, 1.0 / 30.0)


def exp_finite(u2h, u4h):
    """EXP_finite(u_2h, u_4h) of Algorithm 1, the initial guess (Section 3.3), on all nodes of grid h.

    1. w^2 at the 125 known nodes of every interpolation cell (the nodes of grid 2h) by
       ``extrapolate_fd``;
    2. the remaining 604 fine nodes of every cell (2x2x2 coarse elements of grid 4h) by
       the tri-quartic interpolation eq. (inter) as a 604x125 matrix per cell
       (second remark of Section 3.3).
    Boundary nodes keep their interpolated values (the CG start replaces them by g).
    """
    W = extrapolate_fd(u2h, u4h)
    nz2, ny2, nx2 = W.shape
    assert (nz2 - 1) % 4 == 0 and (ny2 - 1) % 4 == 0 and (nx2 - 1) % 4 == 0, \
        "interpolation cells need an even number of coarse elements per direction"
    ncz, ncy, ncx = (nz2 - 1) // 4, (ny2 - 1) // 4, (nx2 - 1) // 4
    fine = np.empty((2 * nz2 - 1, 2 * ny2 - 1, 2 * nx2 - 1))
    fine[0::2, 0::2, 0::2] = W  # the 125 known values of every cell
    windows = np.lib.stride_tricks.sliding_window_view(W, (5, 5, 5))[::4, ::4, ::4]
    vals = windows.reshape(ncz * ncy * ncx, 125) @ triquartic_cell_matrix()[0].T
    vals = vals.reshape(ncz, ncy, ncx, 604)
    _, fine_idx = triquartic_cell_matrix()
    for col, (c, b, a) in enumerate(fine_idx):
        fine[c:c + 8 * ncz:8, b:b + 8 * ncy:8, a:a + 8 * ncx:8] = vals[..., col]
    return fine


# Comparison prolongations (the library's ``prolong`` option): what EXP_finite is measured
# against.  Section 3.3's first remark: the tri-quadratic interpolation of the earlier
# EXCMG (linear finite elements) is too inaccurate for the fourth-order scheme; Section 3:
# cascadic multigrid prolongs by linear interpolation alone.

def lagrange_cell_matrix(P):
    """Tensor-product Lagrange interpolation with P nodes per direction on one cell.

    The cell has P known nodes per direction at natural coordinates 0, 1, ..., P-1 and
    the fine nodes at the half steps 0, 1/2, ..., P-1.  Returns (M, fine_idx) like
    ``triquartic_cell_matrix``: one row per fine node that is not a known node, one
    column per known node (index (k*P + j)*P + i), entries l_i(xi) l_j(eta) l_k(zeta)
    with the P-point basis of ``lagrange_basis``.
    """
    nodes = tuple(range(P))
    nf = 2 * P - 1
    rows, fine_idx = [], []
    for c in range(nf):
        for b in range(nf):
            for a in range(nf):
                if a % 2 == 0 and b % 2 == 0 and c % 2 == 0:
                    continue
                row = np.empty(P ** 3)
                for k in range(P):
                    for j in range(P):
                        for i in range(P):
                            row[(k * P + j) * P + i] = (lagrange_basis(i, a / 2.0, nodes)
                                                        * lagrange_basis(j, b / 2.0, nodes)
                                                        * lagrange_basis(k, c / 2.0, nodes))
                rows.append(row)
                fine_idx.append((c, b, a))
    return np.array(rows), fine_idx


def _interpolate_cells(W, P):
    """Fine grid (half the spacing of W's grid) from the values W at its even nodes, by
    ``lagrange_cell_matrix(P)`` on every cell of (P-1)^3 elements of W's grid."""
    C = P - 1
    nz2, ny2, nx2 = W.shape
    assert (nz2 - 1) % C == 0 and (ny2 - 1) % C == 0 and (nx2 - 1) % C == 0, \
        "the grid must hold whole interpolation cells"
    ncz, ncy, ncx = (nz2 - 1) // C, (ny2 - 1) // C, (nx2 - 1) // C
    M, fine_idx = lagrange_cell_matrix(P)
    fine = np.empty((2 * nz2 - 1, 2 * ny2 - 1, 2 * nx2 - 1))
    fine[0::2, 0::2, 0::2] = W
    windows = np.lib.stride_tricks.sliding_window_view(W, (P, P, P))[::C, ::C, ::C]
    vals = windows.reshape(ncz * ncy * ncx, P ** 3) @ M.T
    vals = vals.reshape(ncz, ncy, ncx, len(fine_idx))
    for col, (c, b, a) in enumerate(fine_idx):
        fine[c:c + 2 * C * ncz:2 * C, b:b + 2 * C * ncy:2 * C, a:a + 2 * C * ncx:2 * C] = vals[..., col]
    return fine


def prolong_quadratic(u2h, u4h):
    """The extrapolation of EXP_finite (``extrapolate_fd``) at the nodes of grid 2h, then
    tri-quadratic interpolation on every cell of 2x2x2 elements of grid 2h."""
    return _interpolate_cells(extrapolate_fd(u2h, u4h), 3)


def prolong_linear(u2h):
    """Cascadic multigrid: trilinear interpolation of u_2h alone (no extrapolation)."""
    return _interpolate_cells(np.asarray(u2h, dtype=np.float64), 2)


def prolong(kind, u2h, u4h):
    """w_h of Algorithm 1 (the initial guess) by the named prolongation ('quartic' = EXP_finite)."""
    if kind == "quartic":
        return exp_finite(u2h, u4h)
    if kind == "quadratic":
        return prolong_quadratic(u2h, u4h)
    if kind == "linear":
        return prolong_linear(u2h)
    raise ValueError(kind)


def with_boundary(w, g):
    """Copy of w whose boundary nodes hold the Dirichlet data g (Section 2)."""
    out = np.array(g, dtype=np.float64, copy=True)
    out[1:-1, 1:-1, 1:-1] = w[1:-1, 1:-1, 1:-1]
    return out


# --------------------------------------------------------------------------------------
# Section 5, Example 1 text: the gradient by one-sided formulas and the compact
# (Collatz) tridiagonal system, solved by the Thomas algorithm
# --------------------------------------------------------------------------------------

def _derivative_lines(U, hd):
    """Derivative along the last axis of U (shape (..., N+1)) with step hd."""
    N = U.shape[-1] - 1
    D = np.empty_like(U)
    D[..., 0] = (-25.0 / 12.0 * U[..., 0] + 4.0 * U[..., 1] - 3.0 * U[..., 2]
                 + 4.0 / 3.0 * U[..., 3] - 0.25 * U[..., 4]) / hd
    D[..., N] = (25.0 / 12.0 * U[..., N] - 4.0 * U[..., N - 1] + 3.0 * U[..., N - 2]
                 - 4.0 / 3.0 * U[..., N - 3] + 0.25 * U[..., N - 4]) / hd
    # (1/6) D_{i-1} + (4/6) D_i + (1/6) D_{i+1} = (U_{i+1} - U_{i-1}) / (2 hd), i = 1..N-1
    n = N - 1
    a = c = 1.0 / 6.0
    bdiag = 4.0 / 6.0
    rhs_ = (U[..., 2:] - U[..., :-2]) / (2.0 * hd)
    rhs_[..., 0] -= a * D[..., 0]
    rhs_[..., n - 1] -= c * D[..., N]
    # Thomas: forward elimination, back substitution
    cp = np.empty(n)
    dp = np.empty_like(rhs_)
    cp[0] = c / bdiag
    dp[..., 0] = rhs_[..., 0] / bdiag
    for i in range(1, n):
        m = bdiag - a * cp[i - 1]
        cp[i] = c / m
        dp[..., i] = (rhs_[..., i] - a * dp[..., i - 1]) / m
    x = np.empty_like(rhs_)
    x[..., n - 1] = dp[..., n - 1]
    for i in range(n - 2, -1, -1):
        x[..., i] = dp[..., i] - cp[i] * x[..., i + 1]
    D[..., 1:N] = x
    return D


def gradient(u, h):
    """(u_x, u_y, u_z) on all nodes, each from the one-sided boundary formulas plus the
    compact tridiagonal system along every grid line of that direction."""
    hx, hy, hz = h
    ux = _derivative_lines(u, hx)
    uy = np.moveaxis(_derivative_lines(np.moveaxis(u, 1, -1), hy), -1, 1)
    uz = np.moveaxis(_derivative_lines(np.moveaxis(u, 0, -1), hz), -1, 0)
    return ux, uy, uz


# --------------------------------------------------------------------------------------
# Algorithm 1: EXCMG
# --------------------------------------------------------------------------------------

def level_sizes(N, N0):
    """Cell counts of every grid from the coarsest (N0) to the finest (N), halving."""
    N = tuple(int(v) for v in N)
    N0 = tuple(int(v) for v in N0)
    sizes = [N]
    while sizes[-1] != N0:
        cur = sizes[-1]
        if any(c % 2 for c in cur) or any(c <= c0 for c, c0 in zip(cur, N0)):
            raise ValueError(f"grid {N} is not N0={N0} times a power of two")
        sizes.append(tuple(c // 2 for c in cur))
    sizes.reverse()
    if len(sizes) < 3:
        raise ValueError("EXCMG needs at least three grids")
    if len({N[d] // N0[d] for d in range(3)}) != 1:
        raise ValueError("all directions must be refined by the same power of two")
    return sizes


def excmg(f, g, L, N, N0, eps, eps_coarse=1e-12, max_iter=100000, dsolve="cg",
          fixed_iters=None, want_utilde=True, eps_ratio=1.0, prolong_kind="quartic",
          history=None, rhs_norm="lift"):
    """EXCMG(A_h, f_h, L, eps) of Algorithm 1.

    ``f``, ``g``: finest-grid node arrays (g read on boundary nodes only).  ``L``: box
    lengths; ``N``: finest cells; ``N0``: coarsest cells.  Levels 0 and 1 are DSOLVE
    (CG to ``eps_coarse`` or dense Cholesky); every finer level starts CG from
    w_h = EXP_finite(u_2h, u_4h) and stops at ||r|| <= eps ||b||; ũ_h =
    EXP_true(u_h, u_2h).  ``fixed_iters`` (one count per level) replaces both tests.
    ``eps_ratio`` r: level l >= 2 of the nl levels stops at eps * r**(nl-1-l) (the
    uniform eps of Algorithm 1 when r = 1; r = 2**6 follows the sixth-order error of
    the extrapolated solution from level to level, Section 5's remark on uniform eps).
    ``prolong_kind``: 'quartic' (EXP_finite, the method), or the comparison
    prolongations 'quadratic' / 'linear' (``prolong``).  ``history``: a list that
    receives the finest level's relative residual before each CG step and after the
    last (the curve of the residual-history figure of Section 5).  ``rhs_norm``: the
    reading of ||f_h|| in every level's stopping test ("lift" or "forcing", see
    ``stopping_norm``).
    Returns a dict of per-level lists: 'u', 'w', 'ut', 'iters', 'relres', 'h', 'N'.
    """
    sizes = level_sizes(N, N0)
    out = {"u": [], "w": [], "ut": [], "iters": [], "relres": [], "h": [], "N": sizes}
    for l, Nl in enumerate(sizes):
        s = N[0] // Nl[0]
        fl = np.ascontiguousarray(f[::s, ::s, ::s])
        gl = np.ascontiguousarray(g[::s, ::s, ::s])
        hl = meshsizes(L, Nl)
        out["h"].append(hl)
        fixed = None if fixed_iters is None else fixed_iters[l]
        if l < 2:
            start = gl.copy()
            start[1:-1, 1:-1, 1:-1] = 0.0
            if dsolve == "dense":
                ul, it, rel = dense_solve(gl, fl, hl), 0, 0.0
            else:
                ul, it, rel = cg(start, fl, hl, eps_coarse, max_iter, fixed, rhs_norm=rhs_norm)
            w = None
        else:
            w = prolong(prolong_kind, out["u"][l - 1], out["u"][l - 2])
            eps_l = eps * eps_ratio ** (len(sizes) - 1 - l)
            hist = history if l == len(sizes) - 1 else None
            ul, it, rel = cg(with_boundary(w, gl), fl, hl, eps_l, max_iter, fixed, history=hist,
                             rhs_norm=rhs_norm)
        out["u"].append(ul)
        out["w"].append(w)
        out["iters"].append(it)
        out["relres"].append(rel)
        if l >= 1 and want_utilde:
            out["ut"].append(extrapolate_true(ul, out["u"][l - 1]))
        else:
            out["ut"].append(None)
    return out


# --------------------------------------------------------------------------------------
# Section 5: norms and observed order
# --------------------------------------------------------------------------------------

def l2_norm(v):
    """Discrete L2 norm: root mean square over all nodes."""
    v = np.asarray(v)
    return float(np.sqrt(np.sum(v * v) / v.size))


def linf_norm(v):
    return float(np.max(np.abs(v)))


def grad_l2_norm(ex, ey, ez):
    """Root mean square over all nodes of |e|^2 for a gradient error e."""
    return float(np.sqrt(np.sum(ex * ex + ey * ey + ez * ez) / ex.size))


def grad_linf_norm(ex, ey, ez):
    """Max over nodes and components."""
    return float(max(np.max(np.abs(ex)), np.max(np.abs(ey)), np.max(np.abs(ez))))


def observed_order(e_coarse, e_fine):
    """order = log2(||u_h - u|| / ||u_{h/2} - u||) (Section 5)."""
    return float(np.log2(e_coarse / e_fine))


# --------------------------------------------------------------------------------------
# Adjoint of the discrete solve (project addition; the paper has no adjoint)
# --------------------------------------------------------------------------------------

def rhs_transpose(lam, shape):
    """R^T lam: the transpose of ``rhs`` (interior -> all nodes)."""
    out = np.zeros(shape)
    nz, ny, nx = shape
    core = (slice(1, nz - 1), slice(1, ny - 1), slice(1, nx - 1))
    out[core] += 3.0 * lam
    for dk, dj, di in ((0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)):
        out[1 + dk:nz - 1 + dk, 1 + dj:ny - 1 + dj, 1 + di:nx - 1 + di] += 0.5 * lam
    return out


def lift_transpose(lam, h, shape):
    """LHS_IB^T lam: the transpose of the boundary part of the printed LHS, evaluated on
    boundary nodes (interior entries are zero)."""
    w = coefficients(*h)
    nz, ny, nx = shape
    out = np.zeros(shape)
    terms = [((0, 0, 0), w["centre"])]
    for o in ((0, 0, 1), (0, 0, -1)):
        terms.append((o, w["fx"]))
    for o in ((0, 1, 0), (0, -1, 0)):
        terms.append((o, w["fy"]))
    for o in ((1, 0, 0), (-1, 0, 0)):
        terms.append((o, w["fz"]))
    for o in ((0, 1, 1), (0, -1, 1), (0, 1, -1), (0, -1, -1)):
        terms.append((o, w["exy"]))
    for o in ((1, 0, 1), (-1, 0, 1), (1, 0, -1), (-1, 0, -1)):
        terms.append((o, w["exz"]))
    for o in ((1, 1, 0), (1, -1, 0), (-1, 1, 0), (-1, -1, 0)):
        terms.append((o, w["eyz"]))
    for (dk, dj, di), cw in terms:
        out[1 + dk:nz - 1 + dk, 1 + dj:ny - 1 + dj, 1 + di:nx - 1 + di] += cw * lam
    out[1:-1, 1:-1, 1:-1] = 0.0
    return out


def adjoint(dLdu, h, eps=1e-14, max_iter=100000, dense=False):
    """Gradients of L(u) through the discrete solve u_I = A^{-1} b(f, g), u_B = g.

    lam = A^{-1} (dL/du)_I  (CG, A is symmetric);  dL/df = -R^T lam;
    dL/dg = LHS_IB^T lam + (dL/du) on boundary nodes.  Returns (dLdf, dLdg, lam).
    """
    shape = dLdu.shape
    src = dLdu[1:-1, 1:-1, 1:-1]
    if dense:
        nz, ny, nx = shape
        M = dense_matrix((nx - 1, ny - 1, nz - 1), h)
        lam = np.linalg.solve(M, src.ravel()).reshape(src.shape)
    else:
        # A lam = src  <=>  LHS(lam_full) - RHS(f') = 0 with RHS(f') := -src; use cg on a
        # zero-boundary problem whose assembled b equals src.
        lam = _cg_interior(src, h, eps, max_iter)
    dLdf = -rhs_transpose(lam, shape)
    dLdg = lift_transpose(lam, h, shape)
    bmask = np.ones(shape, dtype=bool)
    bmask[1:-1, 1:-1, 1:-1] = False
    dLdg[bmask] += dLdu[bmask]
    return dLdf, dLdg, lam


def _cg_interior(b, h, eps, max_iter):
    """Plain CG for A x = b on interior vectors, from x = 0 (same steps as ``cg``)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.sum(r * r)
    bnorm = np.sqrt(rr)
    k = 0
    while np.sqrt(rr) > eps * bnorm and k < max_iter:
        q = apply_A(p, h)
        alpha = rr / np.sum(p * q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = np.sum(r * r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        k += 1
    return x
