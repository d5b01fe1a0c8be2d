"""excmg_cg_noalloc: the one-grid CG for callers that cannot allocate device memory.

Some callers must not call cudaMalloc themselves -- an application or framework that
owns all device memory through its own pool, code that cannot take cudaMalloc's implicit
synchronisation, or a binding with no way to reach a CUDA allocator.  For them the
library offers excmg_cg_noalloc, whose scratch is a device array built into the library
instead of a caller workspace.  This test calls it through the C-ABI and checks it
against excmg_cg (the entry point with a caller workspace) on two calls in a row, with
different grids, so that whatever the first call leaves in the shared scratch cannot
leak into the second.  It also checks that a grid too large for the built-in scratch
is refused before any work.
"""
import ctypes

import numpy as np
import pytest

from paper_1507_05063_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-10  # the solver parity tolerance of the GPU tests


@pytest.fixture(scope="module")
def X():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05063_gb300 import excmg
    return excmg


def _noalloc(X, f, u, L, **opts):
    N = (f.shape[2] - 1, f.shape[1] - 1, f.shape[0] - 1)
    grid = X.make_grid(L, N)
    o, keep = X.make_options(**opts)
    st = X.Stats()
    status = X.excmg_cg_noalloc(ctypes.byref(grid), ctypes.c_void_p(f.data_ptr()), ctypes.byref(o),
                                ctypes.c_void_p(u.data_ptr()), ctypes.byref(st),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    del keep
    return status, st.to_dict()


def _start(problem, N, L, seed):
    f, g, _ = P.make_inputs(problem, N, L)
    rng = np.random.default_rng(seed)
    u0 = g.copy()
    u0[1:-1, 1:-1, 1:-1] = rng.standard_normal((N[2] - 1, N[1] - 1, N[0] - 1))
    return torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()


CASES = [  # two calls in a row: different problems, grids and stopping rules
    ("ex3", (40, 24, 16), (1.0, 0.6, 0.4), dict(eps=1e-10)),
    ("ex1", (33, 17, 9), (1.0, 1.0, 1.0), dict(eps=0.0, fixed_iters=[25])),
]


def test_noalloc_matches_workspace_entry_point(X):
    for name, N, L, opts in CASES:
        fd, u0 = _start(P.PROBLEMS[name], N, L, seed=len(name) + N[0])
        u_ws = u0.clone()
        st_ws = X.cg(fd, u_ws, L, **opts)
        u_na = u0.clone()
        status, st_na = _noalloc(X, fd, u_na, L, **opts)
        assert status == 0, X.STATUS[status]
        assert st_na["iters"][0] == st_ws["iters"][0]
        a, b = u_na.cpu().numpy(), u_ws.cpu().numpy()
        assert np.max(np.abs(a - b)) <= TOL_SOLVE * np.max(np.abs(b))
        if "eps" in opts and opts["eps"] > 0:
            assert st_na["relres"][0] <= opts["eps"]


def test_noalloc_refuses_grids_beyond_its_scratch(X):
    N, L = (80, 80, 80), (1.0, 1.0, 1.0)  # 81^3 nodes x 4 arrays > 16 MiB
    grid = X.make_grid(L, N)
    o, _ = X.make_options()
    fake = ctypes.c_void_p(1 << 20)
    status = X.excmg_cg_noalloc(ctypes.byref(grid), fake, ctypes.byref(o), ctypes.c_void_p(2 << 20),
                                None, None)
    assert status == 6  # EXCMG_ERR_WORKSPACE, before any work is enqueued


def test_noalloc_refuses_options_it_cannot_honour(X):
    """The residual history and the per-launch timing need host buffers and events that
    the allocation-free entry point does not keep: it refuses them (EXCMG_ERR_INVALID_ARG)
    instead of leaving them unfilled; so are invalid options excmg_cg would refuse."""
    N, L = (16, 16, 16), (1.0, 1.0, 1.0)
    fd, u0 = _start(P.PROBLEMS["ex1"], N, L, seed=3)
    for opts in (dict(history=8), dict(profile=1), dict(eps_ratio=-1.0), dict(precision="mixed")):
        status, _ = _noalloc(X, fd, u0.clone(), L, **opts)
        assert status == 1, opts
