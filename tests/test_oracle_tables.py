"""End-to-end pins: the oracle's EXCMG reproduces the errors printed in Tables 1-10."""
import collections

import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from paper_1507_05063_gb300 import problems as P

# tolerance of each table (Section 5 text / table captions) and coarsest grid
SETUP = {"ex1": (1e-14, (4, 4, 4)), "ex2": (1e-14, (4, 4, 4)), "ex3": (1e-11, (4, 4, 4)),
         "ex4": (1e-9, (8, 4, 2)), "ex5": (1e-12, (4, 4, 4)), "ex6": (1e-13, (4, 4, 4))}


def _rows():
    groups = collections.defaultdict(list)
    for ex, mesh, norm, qty, val, src in read_golden("paper_tables.txt"):
        groups[(ex, mesh)].append((norm, qty, float(val), src))
    return sorted(groups.items())


def errors_of_run(name, N):
    eps, N0 = SETUP[name]
    prob = P.PROBLEMS[name]
    f, g, u = P.make_inputs(prob, N)
    res = O.excmg(f, g, (1.0, 1.0, 1.0), N, N0, eps=eps, eps_coarse=eps)
    uh, ut, w = res["u"][-1], res["ut"][-1], res["w"][-1]
    gx, gy, gz = O.gradient(uh, res["h"][-1])
    ex, ey, ez = P.exact_gradient(prob, N)
    return {
        ("L2", "u"): O.l2_norm(uh - u), ("Linf", "u"): O.linf_norm(uh - u),
        ("L2", "grad"): O.grad_l2_norm(gx - ex, gy - ey, gz - ez),
        ("Linf", "grad"): O.grad_linf_norm(gx - ex, gy - ey, gz - ez),
        ("L2", "ut"): O.l2_norm(ut - u), ("Linf", "ut"): O.linf_norm(ut - u),
        ("L2", "w"): O.l2_norm(w - uh), ("Linf", "w"): O.linf_norm(w - uh),
    }


@pytest.mark.parametrize("key,rows", _rows(), ids=lambda v: "-".join(v) if isinstance(v, tuple) else "")
def test_reproduces_printed_errors(key, rows):
    name, mesh = key
    N = tuple(int(v) for v in mesh.split("x"))
    got = errors_of_run(name, N)
    for norm, qty, val, src in rows:
        # three printed significant digits
        assert got[(norm, qty)] == pytest.approx(val, rel=6e-3, abs=0), (src, norm, qty)


def test_observed_orders_example1():
    """Fourth order for u_h and grad u_h, sixth for u~_h, fifth for w_h - u_h (Section 5,
    Tables 1-2; order formula of Section 5)."""
    e16 = errors_of_run("ex1", (16, 16, 16))
    e32 = errors_of_run("ex1", (32, 32, 32))
    order = {k: O.observed_order(e16[k], e32[k]) for k in e16}
    assert 3.8 < order[("Linf", "u")] < 4.2
    assert 3.8 < order[("Linf", "grad")] < 4.2
    assert 5.4 < order[("Linf", "ut")] < 6.2
    assert 4.7 < order[("Linf", "w")] < 5.3


def test_harmonic_example_stops():
    """Example 2 has f = 0: the stopping test must use the assembled b (Dirichlet lift),
    else ||f_h|| = 0 and no tolerance is ever met; the forcing reading falls back to it."""
    N = (16, 16, 16)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex2"], N)
    assert np.all(f == 0)
    res = O.excmg(f, g, (1, 1, 1), N, (4, 4, 4), eps=1e-12, max_iter=500)
    assert all(it < 500 for it in res["iters"])
    assert res["relres"][-1] <= 1e-12
    res_f = O.excmg(f, g, (1, 1, 1), N, (4, 4, 4), eps=1e-12, max_iter=500, rhs_norm="forcing")
    assert res_f["iters"] == res["iters"]


def test_dense_dsolve_agrees_with_cg_dsolve():
    N = (16, 16, 16)
    f, g, _ = P.make_inputs(P.PROBLEMS["ex1"], N)
    a = O.excmg(f, g, (1, 1, 1), N, (4, 4, 4), eps=1e-13, eps_coarse=1e-14)
    b = O.excmg(f, g, (1, 1, 1), N, (4, 4, 4), eps=1e-13, dsolve="dense")
    assert np.max(np.abs(a["u"][1] - b["u"][1])) < 1e-12
    assert np.max(np.abs(a["u"][-1] - b["u"][-1])) < 1e-11


def test_per_level_tolerance():
    """eps_ratio r: level l >= 2 of nl levels stops at eps * r**(nl-1-l); r = 1 is the
    uniform tolerance of Algorithm 1 (identical run)."""
    N, N0, eps = (32, 32, 32), (4, 4, 4), 1e-12
    f, g, _ = P.make_inputs(P.PROBLEMS["ex1"], N)
    base = O.excmg(f, g, (1, 1, 1), N, N0, eps=eps, dsolve="dense")
    same = O.excmg(f, g, (1, 1, 1), N, N0, eps=eps, dsolve="dense", eps_ratio=1.0)
    assert base["iters"] == same["iters"]
    assert np.array_equal(base["u"][-1], same["u"][-1])
    r = 64.0
    res = O.excmg(f, g, (1, 1, 1), N, N0, eps=eps, dsolve="dense", eps_ratio=r)
    nl = len(res["N"])
    for l in range(2, nl):
        assert res["relres"][l] <= eps * r ** (nl - 1 - l)
    # looser coarse levels never take more steps than the uniform run there
    assert all(a <= b for a, b in zip(res["iters"][2:-1], base["iters"][2:-1]))


# ---- the larger meshes (64^3 ... 256^3), recorded by tests/golden/make_oracle_tables_large.py
# under the two readings of ||f_h|| in the stopping test of Algorithm 1

def _large(reading="lift"):
    name = {"lift": "oracle_tables_large.txt", "forcing": "oracle_tables_large_forcing.txt"}[reading]
    vals, iters = {}, {}
    for row in read_golden(name):
        if row[2] == "iters":
            iters[(row[0], row[1])] = [int(v) for v in row[3].split(",")]
        else:
            vals[(row[0], row[1], row[2], row[3])] = float(row[4])
    return vals, iters


def reading_of_rows():
    """Each printed row of paper_tables_gpu.txt -> the reading whose oracle record
    reproduces it to three digits ("lift" first, then "forcing"), or None."""
    lift, _ = _large("lift")
    force, _ = _large("forcing")
    out = {}
    for ex, mesh, norm, qty, val, _ in read_golden("paper_tables_gpu.txt"):
        key = (ex, mesh, norm, qty)
        v = float(val)
        if abs(lift[key] / v - 1) <= 6e-3:
            out[key] = "lift"
        elif abs(force[key] / v - 1) <= 6e-3:
            out[key] = "forcing"
        else:
            out[key] = None
    return out


def test_large_mesh_printed_rows_by_reading():
    """Of the 144 printed errors above the CPU pins, the lift reading reproduces 81 to
    three digits (the rows set by the discretisation and Table 11's step counts' runs),
    the forcing reading 96 (among them u and u~ of Examples 1, 3, 5, 6 at 128^3, where
    the algebraic error shows); 99 rows are reproduced by one or the other.  The other
    45 (u~ of Example 2, the 256^3 u and u~ rows, Example 4 from 256x128x64) lie where
    neither reading's algebraic error matches the print; the design notes list them
    with both values."""
    lift, _ = _large("lift")
    force, _ = _large("forcing")
    rows = read_golden("paper_tables_gpu.txt")
    assert len(rows) == 144
    n_lift = sum(abs(lift[tuple(r[:4])] / float(r[4]) - 1) <= 6e-3 for r in rows)
    n_force = sum(abs(force[tuple(r[:4])] / float(r[4]) - 1) <= 6e-3 for r in rows)
    by = reading_of_rows()
    assert (n_lift, n_force, sum(v is not None for v in by.values())) == (81, 96, 99)
    # the 128^3 rows of Examples 1 and 3 named in Tables 1-2 and table31/table32
    for key in (("ex1", "128x128x128", "Linf", "ut"), ("ex1", "128x128x128", "L2", "u"),
                ("ex3", "128x128x128", "L2", "u"), ("ex3", "128x128x128", "Linf", "u")):
        assert by[key] == "forcing", key


def test_large_mesh_oracle_takes_table11_step_counts():
    """Table 11: 8-9 CG steps on the finest grid.  The lift reading takes the printed
    count on Examples 1-5; Example 6 (eps = 1e-13) stalls near its tolerance.  The forcing
    reading takes 22 to 376 steps there (Example 2, f = 0, falls back to the lift)."""
    _, iters = _large("lift")
    _, iters_f = _large("forcing")
    for ex, mesh, n, _ in read_golden("paper_iterations.txt"):
        got = iters[(ex, mesh)][-1]
        if ex == "ex6":
            assert int(n) < got <= 2 * int(n)
        else:
            assert got == int(n), (ex, got, n)
        if ex == "ex2":
            assert iters_f[(ex, mesh)] == iters[(ex, mesh)]
        else:
            assert iters_f[(ex, mesh)][-1] > 2 * int(n)


@pytest.mark.parametrize("name,N,rows", [
    # printed value the forcing reading reproduces and the lift reading does not
    ("ex3", (64, 64, 64), [("L2", "ut", 1.87e-11), ("Linf", "ut", 6.63e-11)]),
    ("ex5", (64, 64, 64), [("L2", "ut", 8.57e-13)]),
])
def test_forcing_reading_live(name, N, rows):
    """The oracle run live under the forcing reading reproduces printed rows (table31,
    table32, table51) to three digits that the lift reading misses."""
    eps, N0 = SETUP[name]
    prob = P.PROBLEMS[name]
    f, g, u = P.make_inputs(prob, N)
    for reading in ("forcing", "lift"):
        res = O.excmg(f, g, (1.0, 1.0, 1.0), N, N0, eps=eps, eps_coarse=eps, dsolve="dense",
                      rhs_norm=reading)
        ut = res["ut"][-1]
        got = {("L2", "ut"): O.l2_norm(ut - u), ("Linf", "ut"): O.linf_norm(ut - u)}
        for norm, qty, val in rows:
            ok = abs(got[(norm, qty)] / val - 1) <= 6e-3
            assert ok == (reading == "forcing"), (reading, norm, qty, got[(norm, qty)], val)


@pytest.mark.slow
def test_forcing_reading_live_128():
    """Example 3 at 128^3 under the forcing reading (tens of seconds): u and u~ as
    table31/table32 print them, to three digits."""
    eps, N0 = SETUP["ex3"]
    N = (128, 128, 128)
    f, g, u = P.make_inputs(P.PROBLEMS["ex3"], N)
    res = O.excmg(f, g, (1.0, 1.0, 1.0), N, N0, eps=eps, eps_coarse=eps, dsolve="dense",
                  rhs_norm="forcing")
    uh, ut = res["u"][-1], res["ut"][-1]
    # u_h to the printed three digits; u~_h (an error of 3e-13, near the rounding of the
    # extrapolation) to 2.5%
    for got, val, tol in ((O.l2_norm(uh - u), 3.19e-10, 6e-3), (O.linf_norm(uh - u), 1.16e-9, 6e-3),
                          (O.l2_norm(ut - u), 3.05e-13, 2.5e-2), (O.linf_norm(ut - u), 1.04e-12, 2.5e-2)):
        assert abs(got / val - 1) <= tol, (got, val)


def test_stopping_norm_readings():
    """stopping_norm: lift = ||b|| of eq. (FD); forcing = ||RHS(f)|| of eq. (compact);
    forcing falls back to lift when RHS(f) = 0; both equal when g = 0 on the boundary."""
    rng = np.random.default_rng(7)
    N = (6, 5, 4)
    h = O.meshsizes((1.0, 1.0, 1.0), N)
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    f = rng.standard_normal(shape)
    g = rng.standard_normal(shape)
    b = O.rhs_vector(f, g, h)
    assert O.stopping_norm(f, g, h, "lift") == pytest.approx(np.sqrt(np.sum(b * b)), rel=1e-14)
    rf = O.rhs(f)
    assert O.stopping_norm(f, g, h, "forcing") == pytest.approx(np.sqrt(np.sum(rf * rf)), rel=1e-14)
    zero = np.zeros(shape)
    assert O.stopping_norm(zero, g, h, "forcing") == O.stopping_norm(zero, g, h, "lift") > 0
    assert O.stopping_norm(f, zero, h, "forcing") == pytest.approx(O.stopping_norm(f, zero, h, "lift"))
    with pytest.raises(ValueError):
        O.stopping_norm(f, g, h, "other")
