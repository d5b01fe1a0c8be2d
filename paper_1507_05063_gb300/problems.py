"""Seeded, closed-form input generators (no method arithmetic).

Each problem gives the exact solution u, the forcing f = u_xx + u_yy + u_zz and the
exact gradient as vectorised numpy functions of (x, y, z).  Inputs are evaluated on the
host in float64 (libm), once, and copied to the device, so the CUDA path and the CPU
oracle read bit-identical f and g.  This module holds none of the solver's arithmetic;
both the tests and the benchmark use it.

Problems:
* ``ex1`` .. ``ex6``  -- the six examples of Section 5 (Examples 1-6, in order of
  appearance: e^z sin(xy); e^{x+y} sin(sqrt2 z); the Gaussian; sin(2 pi x) sin(pi y)
  sin(pi z / 2); x^3 y^3 z^3 / r^3; xyz r).
* ``sin3``      -- sin(pi x) sin(pi y) sin(pi z), f = -3 pi^2 u, g = 0 (unit cube).
* ``exp3``      -- e^{x+y+z}, f = 3u.
* ``r53``       -- r^{5/3} = (x^2+y^2+z^2)^{5/6}, f = (40/9) r^{-1/3} (f := 0 at r = 0).
* ``trig_sum``  -- sum_k a_k sin(m_k pi x) sin(n_k pi y) sin(p_k pi z) with seeded
  a_k ~ N(0,1), m, n, p ~ U{1..8}; the sines vanish on boundaries of a box with integer
  sides, so g = 0.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional, Sequence, Tuple

import numpy as np

Array = np.ndarray


@dataclass
class Problem:
    name: str
    u: Callable[[Array, Array, Array], Array]
    f: Callable[[Array, Array, Array], Array]
    grad: Optional[Callable[[Array, Array, Array], Tuple[Array, Array, Array]]]
    L: Tuple[float, float, float] = (1.0, 1.0, 1.0)


def _r(x, y, z):
    return np.sqrt(x * x + y * y + z * z)


def _ex1():
    u = lambda x, y, z: np.exp(z) * np.sin(x * y)  # noqa: E731
    f = lambda x, y, z: np.exp(z) * np.sin(x * y) * (1.0 - x * x - y * y)  # noqa: E731
    g = lambda x, y, z: (np.exp(z) * y * np.cos(x * y), np.exp(z) * x * np.cos(x * y),  # noqa: E731
                         np.exp(z) * np.sin(x * y))
    return Problem("ex1", u, f, g)


def _ex2():
    s2 = np.sqrt(2.0)
    u = lambda x, y, z: np.exp(x + y) * np.sin(s2 * z)  # noqa: E731
    f = lambda x, y, z: np.zeros(np.broadcast(x, y, z).shape)  # noqa: E731
    g = lambda x, y, z: (np.exp(x + y) * np.sin(s2 * z), np.exp(x + y) * np.sin(s2 * z),  # noqa: E731
                         s2 * np.exp(x + y) * np.cos(s2 * z))
    return Problem("ex2", u, f, g)


def _ex3():
    def s(x, y, z):
        return (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
    u = lambda x, y, z: np.exp(-3.0 * s(x, y, z))  # noqa: E731
    f = lambda x, y, z: np.exp(-3.0 * s(x, y, z)) * (36.0 * s(x, y, z) - 18.0)  # noqa: E731
    g = lambda x, y, z: tuple(-6.0 * (c - 0.5) * np.exp(-3.0 * s(x, y, z)) for c in (x, y, z))  # noqa: E731
    return Problem("ex3", u, f, g)


def _ex4():
    pi = np.pi
    u = lambda x, y, z: np.sin(2 * pi * x) * np.sin(pi * y) * np.sin(0.5 * pi * z)  # noqa: E731
    f = lambda x, y, z: -5.25 * pi * pi * u(x, y, z)  # noqa: E731
    g = lambda x, y, z: (2 * pi * np.cos(2 * pi * x) * np.sin(pi * y) * np.sin(0.5 * pi * z),  # noqa: E731
                         pi * np.sin(2 * pi * x) * np.cos(pi * y) * np.sin(0.5 * pi * z),
                         0.5 * pi * np.sin(2 * pi * x) * np.sin(pi * y) * np.cos(0.5 * pi * z))
    return Problem("ex4", u, f, g)


def _safe_div(num, den):
    den = np.asarray(den, dtype=np.float64)
    out = np.zeros(np.broadcast(num, den).shape)
    np.divide(num, den, out=out, where=den > 0)
    return out


def _ex5():
    # u = P r^-3 with P = x^3 y^3 z^3;  f = 6xyz(x^2y^2+y^2z^2+z^2x^2)/r^3 - 48 P / r^5
    def u(x, y, z):
        return _safe_div(x ** 3 * y ** 3 * z ** 3, _r(x, y, z) ** 3)

    def f(x, y, z):
        r = _r(x, y, z)
        P = x ** 3 * y ** 3 * z ** 3
        q = x * x * y * y + y * y * z * z + z * z * x * x
        return _safe_div(6.0 * x * y * z * q, r ** 3) - _safe_div(48.0 * P, r ** 5)

    def grad(x, y, z):
        r = _r(x, y, z)
        P = x ** 3 * y ** 3 * z ** 3
        out = []
        for c, rest in ((x, y ** 3 * z ** 3), (y, x ** 3 * z ** 3), (z, x ** 3 * y ** 3)):
            out.append(_safe_div(3.0 * c * c * rest, r ** 3) - _safe_div(3.0 * P * c, r ** 5))
        return tuple(out)
    return Problem("ex5", u, f, grad)


def _ex6():
    def u(x, y, z):
        return x * y * z * _r(x, y, z)

    def f(x, y, z):
        return _safe_div(8.0 * x * y * z, _r(x, y, z))

    def grad(x, y, z):
        r = _r(x, y, z)
        return (y * z * r + _safe_div(x * x * y * z, r), x * z * r + _safe_div(x * y * y * z, r),
                x * y * r + _safe_div(x * y * z * z, r))
    return Problem("ex6", u, f, grad)


def _sin3():
    pi = np.pi
    u = lambda x, y, z: np.sin(pi * x) * np.sin(pi * y) * np.sin(pi * z)  # noqa: E731
    f = lambda x, y, z: -3.0 * pi * pi * u(x, y, z)  # noqa: E731
    g = lambda x, y, z: (pi * np.cos(pi * x) * np.sin(pi * y) * np.sin(pi * z),  # noqa: E731
                         pi * np.sin(pi * x) * np.cos(pi * y) * np.sin(pi * z),
                         pi * np.sin(pi * x) * np.sin(pi * y) * np.cos(pi * z))
    return Problem("sin3", u, f, g)


def _exp3():
    u = lambda x, y, z: np.exp(x + y + z)  # noqa: E731
    f = lambda x, y, z: 3.0 * np.exp(x + y + z)  # noqa: E731
    g = lambda x, y, z: (np.exp(x + y + z),) * 3  # noqa: E731
    return Problem("exp3", u, f, g)


def _r53():
    def u(x, y, z):
        return (x * x + y * y + z * z) ** (5.0 / 6.0)

    def f(x, y, z):
        r = _r(x, y, z)
        out = np.zeros(np.broadcast(x, y, z).shape)
        np.power(r, -1.0 / 3.0, out=out, where=r > 0)
        return (40.0 / 9.0) * out * (r > 0)

    def grad(x, y, z):
        r = _r(x, y, z)
        fac = np.zeros(np.broadcast(x, y, z).shape)
        np.power(r, -1.0 / 3.0, out=fac, where=r > 0)
        fac = (5.0 / 3.0) * fac * (r > 0)
        return fac * x, fac * y, fac * z
    return Problem("r53", u, f, grad)


PROBLEMS = {p.name: p for p in (_ex1(), _ex2(), _ex3(), _ex4(), _ex5(), _ex6(), _sin3(),
                                _exp3(), _r53())}


def trig_sum(seed: int, K: int = 8, L: Sequence[float] = (1.0, 1.0, 1.0)) -> Problem:
    """Seeded trig-sum source: f = sum_k a_k sin(m_k pi x) sin(n_k pi y) sin(p_k pi z),
    exact u = -sum_k a_k sin sin sin / (pi^2 (m_k^2 + n_k^2 + p_k^2)), g = 0."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(K)
    mnp = rng.integers(1, 9, size=(K, 3))
    pi = np.pi

    def f(x, y, z):
        out = np.zeros(np.broadcast(x, y, z).shape)
        for ak, (m, n, p) in zip(a, mnp):
            out = out + ak * np.sin(m * pi * x) * np.sin(n * pi * y) * np.sin(p * pi * z)
        return out

    def u(x, y, z):
        out = np.zeros(np.broadcast(x, y, z).shape)
        for ak, (m, n, p) in zip(a, mnp):
            lam = pi * pi * float(m * m + n * n + p * p)
            out = out - ak / lam * np.sin(m * pi * x) * np.sin(n * pi * y) * np.sin(p * pi * z)
        return out

    def grad(x, y, z):
        gx = np.zeros(np.broadcast(x, y, z).shape)
        gy = np.zeros_like(gx)
        gz = np.zeros_like(gx)
        for ak, (m, n, p) in zip(a, mnp):
            lam = pi * pi * float(m * m + n * n + p * p)
            c = -ak / lam
            sx, sy, sz = np.sin(m * pi * x), np.sin(n * pi * y), np.sin(p * pi * z)
            gx = gx + c * m * pi * np.cos(m * pi * x) * sy * sz
            gy = gy + c * n * pi * sx * np.cos(n * pi * y) * sz
            gz = gz + c * p * pi * sx * sy * np.cos(p * pi * z)
        return gx, gy, gz
    return Problem(f"trig_sum_{seed}", u, f, grad, tuple(float(v) for v in L))


def node_coords(L, N):
    """Broadcastable node coordinates (z, y, x order of axes) of a grid."""
    Lx, Ly, Lz = L
    Nx, Ny, Nz = N
    x = (np.arange(Nx + 1) * (Lx / Nx))[None, None, :]
    y = (np.arange(Ny + 1) * (Ly / Ny))[None, :, None]
    z = (np.arange(Nz + 1) * (Lz / Nz))[:, None, None]
    return x, y, z


def make_inputs(problem: Problem, N, L=None):
    """f, g (= exact u on all nodes; solvers read only its boundary) and exact u.

    Arrays have shape (Nz+1, Ny+1, Nx+1), float64, C-contiguous (x fastest).
    """
    L = problem.L if L is None else L
    x, y, z = node_coords(L, N)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    u = np.array(np.broadcast_to(problem.u(x, y, z), shape), dtype=np.float64, order="C")
    f = np.array(np.broadcast_to(problem.f(x, y, z), shape), dtype=np.float64, order="C")
    return f, u.copy(), u


def exact_gradient(problem: Problem, N, L=None):
    L = problem.L if L is None else L
    x, y, z = node_coords(L, N)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    return tuple(np.array(np.broadcast_to(c, shape), dtype=np.float64, order="C")
                 for c in problem.grad(x, y, z))


def batched_grids(nprob: int, seed: int, sizes=(32, 64, 128, 256)):
    """Per-problem (L, N, N0) for the batched workload: each N_d drawn uniformly from
    ``sizes``, each h_d = s_d / N_d with s_d in {1, 2} (so L_d in {1, 2}).  The coarsest
    grid halves N until its smallest side is 4 (even, so the interpolation cells fit)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nprob):
        N = tuple(int(v) for v in rng.choice(sizes, size=3))
        s = tuple(int(v) for v in rng.integers(1, 3, size=3))
        L = tuple(float(sd) for sd in s)
        k = 0
        while min(N) >> (k + 1) >= 4 and all((n >> (k + 1)) % 2 == 0 for n in N):
            k += 1
        N0 = tuple(n >> k for n in N)
        out.append((L, N, N0))
    return out
