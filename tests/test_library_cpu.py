"""Host-side checks of the C-ABI library that need no GPU: it loads, exports every
symbol include/excmg.h declares, and rejects invalid arguments before any CUDA work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def X():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05063_gb300 import excmg
    return excmg


def test_exports_every_declared_symbol(X):
    header = open(os.path.join(ROOT, "include", "excmg.h")).read()
    declared = set(re.findall(r"\b(excmg_[a-z_]+)\s*\(", header))
    assert declared, "no declarations found"
    lib = ctypes.CDLL(X.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(X.EXPORTED)


def test_levels_and_workspace_queries(X):
    g = X.make_grid((1, 1, 1), (32, 32, 32), (4, 4, 4))
    assert X.excmg_num_levels(ctypes.byref(g)) == 4
    g2 = X.make_grid((1, 1, 1), (512, 256, 128), (8, 4, 2))
    assert X.excmg_num_levels(ctypes.byref(g2)) == 7
    o, _ = X.make_options()
    assert X.excmg_workspace_size(ctypes.byref(g2), ctypes.byref(o)) > 4 * 8 * 513 * 257 * 129
    om, _ = X.make_options(precision="mixed")
    assert 0 < X.excmg_workspace_size(ctypes.byref(g2), ctypes.byref(om)) < \
        X.excmg_workspace_size(ctypes.byref(g2), ctypes.byref(o))


@pytest.mark.parametrize("N,N0", [((32, 32, 32), (3, 3, 3)),      # odd coarsest
                                  ((32, 32, 30), (4, 4, 4)),      # not a power-of-two refinement
                                  ((16, 16, 16), (8, 8, 8)),      # only two grids
                                  ((32, 16, 16), (4, 4, 4))])     # unequal refinement ratios
def test_invalid_grids_rejected(X, N, N0):
    g = X.make_grid((1, 1, 1), N, N0)
    o, _ = X.make_options()
    assert X.excmg_num_levels(ctypes.byref(g)) == -1
    assert X.excmg_workspace_size(ctypes.byref(g), ctypes.byref(o)) == 0
    fake = ctypes.c_void_p(1 << 20)
    st = X.excmg_solve(ctypes.byref(g), fake, fake, ctypes.byref(o), ctypes.c_void_p(2 << 20),
                       None, fake, 1 << 30, None, None)
    assert st == 1


def test_invalid_options_rejected(X):
    g = X.make_grid((1, 1, 1), (32, 32, 32), (4, 4, 4))
    for kw in ({"precision": 7}, {"eps": -1.0}, {"max_iter": -3}, {"precision": "mixed", "inner_tol": 2.0},
               {"mixed_min_nodes": -1}, {"eps_ratio": -1.0}, {"eps_ratio": float("nan")},
               {"prolong": 7}, {"dsolve": 5}, {"precision": "mixed", "history": 8},
               {"res_rows": 2}, {"res_rows": -1}, {"autotune": 2}):
        o, _ = X.make_options(**kw)
        assert X.excmg_workspace_size(ctypes.byref(g), ctypes.byref(o)) == 0


def test_small_workspace_rejected(X):
    g = X.make_grid((1, 1, 1), (32, 32, 32), (4, 4, 4))
    o, _ = X.make_options()
    a, b = ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20)
    ws = ctypes.c_void_p(4 << 20)
    assert X.excmg_solve(ctypes.byref(g), a, b, ctypes.byref(o), ctypes.c_void_p(3 << 20), None,
                         ws, 1024, None, None) == 6
    # misaligned workspace
    assert X.excmg_solve(ctypes.byref(g), a, b, ctypes.byref(o), ctypes.c_void_p(3 << 20), None,
                         ctypes.c_void_p((4 << 20) + 8), 1 << 34, None, None) == 6


def test_bench_tables_cover_every_kernel_kind():
    """bench.py reports every kernel kind the library profiles (bytes, FP64 operations,
    symbol and source file per kind)."""
    import bench
    from paper_1507_05063_gb300 import excmg
    for k in excmg.KERNEL_NAMES:
        assert k in bench.ALGO and k in bench.KERNEL_SYMBOL and k in bench.KERNEL_SOURCE, k
        assert os.path.exists(os.path.join(ROOT, "paper_1507_05063_gb300", "csrc", bench.KERNEL_SOURCE[k]))


def test_history_option_sizes_the_workspace(X):
    """options.history adds its device copy to the workspace (history_len doubles, aligned);
    a history pointer with no length, and batched solves, are refused."""
    g = X.make_grid((1, 1, 1), (32, 32, 32), (4, 4, 4))
    o0, _ = X.make_options()
    o1, _k1 = X.make_options(history=100)
    base = X.excmg_workspace_size(ctypes.byref(g), ctypes.byref(o0))
    assert X.excmg_workspace_size(ctypes.byref(g), ctypes.byref(o1)) >= base + 800
    o1.history_len = 0
    assert X.excmg_workspace_size(ctypes.byref(g), ctypes.byref(o1)) == 0
    o2, _k2 = X.make_options(history=10)
    grids = (X.Grid * 2)(g, g)
    assert X.excmg_workspace_size_batched(2, grids, ctypes.byref(o2)) == 0


def test_default_options_match_the_header(X):
    """excmg_default_options writes the values its declaration lists, every field set."""
    o = X.Options()
    ctypes.memset(ctypes.byref(o), 0x5A, ctypes.sizeof(o))  # no field may keep this
    X.excmg_default_options(ctypes.byref(o))
    want = {"precision": 0, "eps": 1e-9, "eps_coarse": 1e-12, "max_iter": 100000,
            "inner_tol": 1e-4, "max_refine": 50, "tile_z": 0, "chunk": 0,
            "mixed_min_nodes": 0, "profile": 0, "dsolve": 0, "eps_ratio": 1.0,
            "prolong": 0, "history_len": 0}
    for name, v in want.items():
        assert getattr(o, name) == v, name
    assert not o.fixed_iters and not o.history
    header = open(os.path.join(ROOT, "include", "excmg.h")).read()
    doc = re.search(r"/\* Writes the defaults:(.*?)\*/", header, re.S).group(1)
    fields = [n for n, _ in X.Options._fields_]
    for name in fields:
        assert name in doc, "header's default list omits " + name
