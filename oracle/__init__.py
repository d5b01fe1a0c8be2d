"""Plain, slow FP64 CPU oracle for EXCMG with the 19-point compact scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, calls or links it, and this
package imports nothing from the product path.

Every function follows a passage of Pan, He & Hu, "An extrapolation cascadic multigrid
method combined with a fourth-order compact scheme for 3D Poisson equation"
(arXiv 1507.05063), cited by section / equation / algorithm in its docstring.

Parity status of each function (what pins it, in tests/test_oracle_*.py):

* ``lhs``, ``rhs``, ``residual``, ``apply_A``, ``rhs_vector``  -- pinned: exact on
  polynomials of total degree <= 5 for arbitrary hx, hy, hz; fails on degree 6;
  symmetric positive definite after negation (dense eigenvalues); Table 1/2 errors.
* ``cg``                      -- pinned: dense Cholesky on <= 6^3 interior grids.
* ``dense_solve``             -- pinned: numpy/LAPACK solve vs an independently
  assembled dense matrix; exactness on polynomial solutions.
* ``extrapolate_fd`` / ``extrapolate_true`` -- pinned: exact when the level solutions
  follow u + A(x) h^4 with trilinear A (the expansion of eq. asy), and Tables 1-6.
* ``quartic_weights``, ``triquartic_cell_matrix``, ``exp_finite`` -- pinned: the printed
  weights of eqs. sifen1-sifen4 (with the printed labels of sifen3/sifen4 swapped),
  exactness on tri-quartic polynomials, fifth order of w_h - u_h (Tables 1-10).
* ``gradient``                -- pinned: exact for degree <= 4 per direction; Thomas vs
  dense banded solve; Table 1/2 gradient errors.
* ``excmg``                   -- pinned end to end by Tables 1, 2, 5, 6 (Examples 1, 4).
* ``adjoint``                 -- pinned: central finite differences of ``excmg``-free
  forward solves, and an explicit dense B^T A^{-1} product on tiny grids.
"""

from .excmg_oracle import *  # noqa: F401,F403
