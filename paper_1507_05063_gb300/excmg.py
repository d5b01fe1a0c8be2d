"""Thin ctypes binding of libexcmg (include/excmg.h).

Argument marshalling only: every step of the solver runs in the CUDA library.  Arrays
are torch tensors on a CUDA device, float64, contiguous, shaped (Nz+1, Ny+1, Nx+1)
(x fastest).  Workspaces are torch uint8 tensors sized by the library's queries.
Importing this module loads ``libexcmg.so`` and raises ImportError if it is missing
(build it with ``python -m paper_1507_05063_gb300.build``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libexcmg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} not found: build the CUDA library first "
                      "(python -m paper_1507_05063_gb300.build)")
_lib = ctypes.CDLL(LIB_PATH)

MAX_LEVELS = 24
FP64, MIXED = 0, 1
KERNEL_NAMES = ["spmv_f64", "update_f64", "spmv_f32", "update_f32", "residual", "exp_finite",
                "init", "correct", "exp_true", "cg_f64", "cg_f32", "cg_cluster_f64", "cg_cluster_f32",
                "cg_resident_f64", "dsolve", "prolong_cmp"]
KERNEL_KINDS = len(KERNEL_NAMES)
STATUS = {0: "EXCMG_OK", 1: "EXCMG_ERR_INVALID_ARG", 2: "EXCMG_ERR_NOT_CONVERGED",
          3: "EXCMG_ERR_CUDA", 4: "EXCMG_ERR_NONFINITE", 5: "EXCMG_ERR_TIMEOUT",
          6: "EXCMG_ERR_WORKSPACE"}


class Grid(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("Nz", ctypes.c_int),
                ("Nx0", ctypes.c_int), ("Ny0", ctypes.c_int), ("Nz0", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("eps", ctypes.c_double),
                ("eps_coarse", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("fixed_iters", ctypes.POINTER(ctypes.c_int)), ("tile_z", ctypes.c_int),
                ("chunk", ctypes.c_int), ("mixed_min_nodes", ctypes.c_longlong),
                ("profile", ctypes.c_int), ("dsolve", ctypes.c_int), ("eps_ratio", ctypes.c_double),
                ("prolong", ctypes.c_int), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_len", ctypes.c_int), ("rhs_norm", ctypes.c_int),
                ("wait_timeout_ms", ctypes.c_double), ("test_phantom_blocks", ctypes.c_int),
                ("autotune", ctypes.c_int), ("res_rows", ctypes.c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int * 3), ("f32", ctypes.c_int), ("res_tz", ctypes.c_int),
                ("res_tz_model", ctypes.c_int), ("res_ms", ctypes.c_double),
                ("res_ms_model", ctypes.c_double), ("cg_tz", ctypes.c_int), ("cg_tz_model", ctypes.c_int),
                ("cg_ms", ctypes.c_double), ("cg_ms_model", ctypes.c_double),
                ("res_rows", ctypes.c_int), ("res_rows_model", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("N", (ctypes.c_int * 3) * MAX_LEVELS),
                ("iters", ctypes.c_int * MAX_LEVELS),
                ("refinements", ctypes.c_int * MAX_LEVELS),
                ("relres", ctypes.c_double * MAX_LEVELS), ("launches", ctypes.c_longlong),
                ("prof_ms", ctypes.c_double * KERNEL_KINDS),
                ("prof_launches", ctypes.c_longlong * KERNEL_KINDS),
                ("prof_nodes", ctypes.c_double * KERNEL_KINDS),
                ("ms_level", ctypes.c_double * MAX_LEVELS), ("ms_total", ctypes.c_double)]

    def to_dict(self):
        n = self.levels
        return {"levels": n, "N": [tuple(self.N[l]) for l in range(n)],
                "iters": list(self.iters[:n]), "refinements": list(self.refinements[:n]),
                "relres": list(self.relres[:n]), "launches": int(self.launches),
                "profile": {KERNEL_NAMES[k]: {"ms": float(self.prof_ms[k]),
                                              "launches": int(self.prof_launches[k]),
                                              "nodes": float(self.prof_nodes[k])}
                            for k in range(KERNEL_KINDS) if self.prof_launches[k] > 0},
                "ms_level": list(self.ms_level[:n]), "ms_total": float(self.ms_total)}


_P = ctypes.c_void_p
_GP = ctypes.POINTER(Grid)
_OP = ctypes.POINTER(Options)
_SP = ctypes.POINTER(Stats)
_D = ctypes.POINTER(ctypes.c_double)


def _sig(name, res, args):
    fn = getattr(_lib, name)
    fn.restype = res
    fn.argtypes = args
    return fn


excmg_default_options = _sig("excmg_default_options", None, [_OP])
excmg_status_string = _sig("excmg_status_string", ctypes.c_char_p, [ctypes.c_int])
excmg_num_levels = _sig("excmg_num_levels", ctypes.c_int, [_GP])
excmg_workspace_size = _sig("excmg_workspace_size", ctypes.c_size_t, [_GP, _OP])
excmg_workspace_size_batched = _sig("excmg_workspace_size_batched", ctypes.c_size_t,
                                    [ctypes.c_int, _GP, _OP])
excmg_workspace_size_adjoint = _sig("excmg_workspace_size_adjoint", ctypes.c_size_t, [_GP, _OP])
excmg_workspace_size_level = _sig("excmg_workspace_size_level", ctypes.c_size_t, [_GP, _OP])
excmg_solve = _sig("excmg_solve", ctypes.c_int,
                   [_GP, _P, _P, _OP, _P, _P, _P, ctypes.c_size_t, _SP, _P])
excmg_grad = _sig("excmg_grad", ctypes.c_int, [_GP, _P, _P, _P, _P, _P])
excmg_solve_batched = _sig("excmg_solve_batched", ctypes.c_int,
                           [ctypes.c_int, _GP, ctypes.POINTER(_P), ctypes.POINTER(_P), _OP,
                            ctypes.POINTER(_P), _P, ctypes.c_size_t, _SP, _P])
excmg_adjoint = _sig("excmg_adjoint", ctypes.c_int,
                     [_GP, _P, _OP, _P, _P, _P, ctypes.c_size_t, _SP, _P])
excmg_exp_finite = _sig("excmg_exp_finite", ctypes.c_int, [_GP, _P, _P, _P, _P, _P])
excmg_exp_true = _sig("excmg_exp_true", ctypes.c_int, [_GP, _P, _P, _P, _P])
excmg_cg = _sig("excmg_cg", ctypes.c_int, [_GP, _P, _OP, _P, _P, ctypes.c_size_t, _SP, _P])
excmg_residual = _sig("excmg_residual", ctypes.c_int,
                      [_GP, _P, _P, _P, _D, _D, _P, ctypes.c_size_t, _P])
excmg_cg_noalloc = _sig("excmg_cg_noalloc", ctypes.c_int, [_GP, _P, _OP, _P, _SP, _P])
excmg_tuning_entries = _sig("excmg_tuning_entries", ctypes.c_int, [ctypes.POINTER(Tuning), ctypes.c_int])
excmg_tuning_clear = _sig("excmg_tuning_clear", None, [])

EXPORTED = ["excmg_default_options", "excmg_status_string", "excmg_num_levels",
            "excmg_workspace_size", "excmg_workspace_size_batched",
            "excmg_workspace_size_adjoint", "excmg_workspace_size_level", "excmg_solve", "excmg_grad", "excmg_solve_batched",
            "excmg_adjoint", "excmg_exp_finite", "excmg_exp_true", "excmg_cg", "excmg_residual",
            "excmg_cg_noalloc", "excmg_tuning_entries", "excmg_tuning_clear"]


def tuning_entries():
    """The launch-shape cache (options.autotune) as a list of dicts."""
    n = excmg_tuning_entries(None, 0)
    arr = (Tuning * max(n, 1))()
    n = excmg_tuning_entries(arr, n)
    return [{"N": list(t.N), "f32": t.f32, "res_tz": t.res_tz, "res_tz_model": t.res_tz_model,
             "res_ms": t.res_ms, "res_ms_model": t.res_ms_model, "cg_tz": t.cg_tz,
             "cg_tz_model": t.cg_tz_model, "cg_ms": t.cg_ms, "cg_ms_model": t.cg_ms_model,
             "res_rows": t.res_rows, "res_rows_model": t.res_rows_model}
            for t in arr[:n]]


class ExcmgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


def _check(status, where, allow=()):
    if status != 0 and status not in allow:
        raise ExcmgError(status, where)
    return status


def make_grid(L, N, N0=(2, 2, 2)):
    return Grid(float(L[0]), float(L[1]), float(L[2]), int(N[0]), int(N[1]), int(N[2]),
                int(N0[0]), int(N0[1]), int(N0[2]))


DSOLVE = {"direct": 0, "cg": 1}
PROLONG = {"quartic": 0, "quadratic": 1, "linear": 2}
RHS_NORM = {"lift": 0, "forcing": 1}


def make_options(precision="fp64", eps=1e-9, eps_coarse=1e-12, max_iter=100000,
                 inner_tol=1e-4, max_refine=50, fixed_iters=None, tile_z=0, chunk=0, profile=0,
                 mixed_min_nodes=0, dsolve="direct", eps_ratio=1.0, prolong="quartic", history=0,
                 rhs_norm="lift", wait_timeout_ms=0.0, test_phantom_blocks=0, autotune=0, res_rows=0):
    o = Options()
    excmg_default_options(ctypes.byref(o))
    o.precision = {"fp64": FP64, "mixed": MIXED}[precision] if isinstance(precision, str) else int(precision)
    o.eps = float(eps)
    o.eps_coarse = float(eps_coarse)
    o.max_iter = int(max_iter)
    o.inner_tol = float(inner_tol)
    o.max_refine = int(max_refine)
    o.tile_z = int(tile_z)
    o.chunk = int(chunk)
    o.profile = int(profile)
    o.mixed_min_nodes = int(mixed_min_nodes)
    o.dsolve = DSOLVE[dsolve] if isinstance(dsolve, str) else int(dsolve)
    o.eps_ratio = float(eps_ratio)
    o.prolong = PROLONG[prolong] if isinstance(prolong, str) else int(prolong)
    o.rhs_norm = RHS_NORM[rhs_norm] if isinstance(rhs_norm, str) else int(rhs_norm)
    o.wait_timeout_ms = float(wait_timeout_ms)
    o.test_phantom_blocks = int(test_phantom_blocks)
    o.autotune = int(autotune)
    o.res_rows = int(res_rows)
    keep = {}
    if fixed_iters is not None:
        keep["fixed"] = (ctypes.c_int * len(fixed_iters))(*[int(v) for v in fixed_iters])
        o.fixed_iters = ctypes.cast(keep["fixed"], ctypes.POINTER(ctypes.c_int))
    if history:
        keep["history"] = (ctypes.c_double * int(history))()
        o.history = ctypes.cast(keep["history"], ctypes.POINTER(ctypes.c_double))
        o.history_len = int(history)
    return o, keep


def _history(keep, iters):
    """options.history as a list: ||r_k|| / ||b|| for k = 0 .. iters of the finest level."""
    h = keep.get("history")
    return None if h is None else list(h[:min(len(h), iters + 1)])


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("arrays must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("arrays must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _node_array(t: torch.Tensor, N, name, host_ok=False):
    shape = (N[2] + 1, N[1] + 1, N[0] + 1)
    if tuple(t.shape) != shape or t.dtype != torch.float64:
        raise ValueError(f"{name}: expected float64 tensor of shape {shape}, got "
                         f"{t.dtype} {tuple(t.shape)}")
    if host_ok and not t.is_cuda and t.is_pinned():
        if not t.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return ctypes.c_void_p(t.data_ptr())  # page-locked host memory, read by the kernels
    return _ptr(t)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def solve_workspace_bytes(L, N, N0, **opts) -> int:
    grid = make_grid(L, N, N0)
    o, _keep = make_options(**opts)
    return int(excmg_workspace_size(ctypes.byref(grid), ctypes.byref(o)))


def solve(f, g, L, N0, want_utilde=False, stream=None, ws=None, out=None, allow_not_converged=False,
          **opts):
    """Algorithm 1 on the GPU.  Returns dict(u, ut, stats, status).

    f and g may be CUDA tensors or pinned (page-locked) CPU tensors; the kernels read the
    latter over the host link.  u, u~ and the workspace are on the GPU."""
    N = (f.shape[2] - 1, f.shape[1] - 1, f.shape[0] - 1)
    grid = make_grid(L, N, N0)
    o, _keep = make_options(**opts)
    need = excmg_workspace_size(ctypes.byref(grid), ctypes.byref(o))
    if need == 0:
        raise ExcmgError(1, "excmg_workspace_size")
    dev = f.device if f.is_cuda else (out.device if out is not None else
                                      torch.device("cuda", torch.cuda.current_device()))
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    u = torch.empty(f.shape, dtype=f.dtype, device=dev) if out is None else out
    ut = torch.empty(f.shape, dtype=f.dtype, device=dev) if want_utilde else None
    st = Stats()
    status = excmg_solve(ctypes.byref(grid), _node_array(f, N, "f", True), _node_array(g, N, "g", True),
                         ctypes.byref(o), _node_array(u, N, "u"), _ptr(ut), _ptr(ws),
                         ws.numel(), ctypes.byref(st), _stream(stream))
    _check(status, "excmg_solve", allow=(2,) if allow_not_converged else ())
    sd = st.to_dict()
    out = {"u": u, "ut": ut, "stats": sd, "status": STATUS[status]}
    if "history" in _keep:
        out["history"] = _history(_keep, sd["iters"][-1])
    return out


def grad(u, L, stream=None):
    N = (u.shape[2] - 1, u.shape[1] - 1, u.shape[0] - 1)
    grid = make_grid(L, N)
    ux, uy, uz = (torch.empty_like(u) for _ in range(3))
    _check(excmg_grad(ctypes.byref(grid), _node_array(u, N, "u"), _ptr(ux), _ptr(uy), _ptr(uz),
                      _stream(stream)), "excmg_grad")
    return ux, uy, uz


def exp_finite(u2h, u4h, L, g=None, stream=None):
    N = (2 * (u2h.shape[2] - 1), 2 * (u2h.shape[1] - 1), 2 * (u2h.shape[0] - 1))
    grid = make_grid(L, N)
    w = torch.empty((N[2] + 1, N[1] + 1, N[0] + 1), dtype=torch.float64, device=u2h.device)
    _node_array(u2h, tuple(n // 2 for n in N), "u2h")
    _node_array(u4h, tuple(n // 4 for n in N), "u4h")
    if g is not None:
        _node_array(g, N, "g")
    _check(excmg_exp_finite(ctypes.byref(grid), _ptr(u2h), _ptr(u4h), _ptr(g), _ptr(w),
                            _stream(stream)), "excmg_exp_finite")
    return w


def exp_true(uh, u2h, L, stream=None):
    N = (uh.shape[2] - 1, uh.shape[1] - 1, uh.shape[0] - 1)
    grid = make_grid(L, N)
    _node_array(u2h, tuple(n // 2 for n in N), "u2h")
    ut = torch.empty_like(uh)
    _check(excmg_exp_true(ctypes.byref(grid), _node_array(uh, N, "uh"), _ptr(u2h), _ptr(ut),
                          _stream(stream)), "excmg_exp_true")
    return ut


def cg(f, u, L, stream=None, ws=None, allow_not_converged=False, allow_timeout=False, **opts):
    """CG on one grid from u's interior (u's boundary = g), in place.  Returns stats."""
    N = (f.shape[2] - 1, f.shape[1] - 1, f.shape[0] - 1)
    grid = make_grid(L, N)
    o, _keep = make_options(**opts)
    need = excmg_workspace_size_level(ctypes.byref(grid), ctypes.byref(o))
    if need == 0:
        raise ExcmgError(1, "excmg_workspace_size_level")
    if ws is None or ws.numel() < need:
        ws = workspace(need, f.device)
    st = Stats()
    status = excmg_cg(ctypes.byref(grid), _node_array(f, N, "f"), ctypes.byref(o),
                      _node_array(u, N, "u"), _ptr(ws), ws.numel(), ctypes.byref(st),
                      _stream(stream))
    _check(status, "excmg_cg", allow=((2,) if allow_not_converged else ()) + ((5,) if allow_timeout else ()))
    d = st.to_dict()
    d["status"] = STATUS[status]
    if "history" in _keep:
        d["history"] = _history(_keep, d["iters"][0])
    return d


def residual(f, u, L, stream=None):
    N = (f.shape[2] - 1, f.shape[1] - 1, f.shape[0] - 1)
    grid = make_grid(L, N)
    o, _keep = make_options()
    need = excmg_workspace_size_level(ctypes.byref(grid), ctypes.byref(o))
    ws = workspace(need, f.device)
    r = torch.empty_like(f)
    rn, bn = ctypes.c_double(), ctypes.c_double()
    _check(excmg_residual(ctypes.byref(grid), _node_array(f, N, "f"), _node_array(u, N, "u"),
                          _ptr(r), ctypes.byref(rn), ctypes.byref(bn), _ptr(ws), ws.numel(),
                          _stream(stream)), "excmg_residual")
    return r, rn.value, bn.value


@dataclass
class BatchedProblem:
    L: Sequence[float]
    N: Sequence[int]
    N0: Sequence[int]
    f: torch.Tensor
    g: torch.Tensor


def solve_batched(problems: List[BatchedProblem], stream=None, ws=None, allow_not_converged=False,
                  **opts):
    n = len(problems)
    grids = (Grid * n)(*[make_grid(p.L, p.N, p.N0) for p in problems])
    o, _keep = make_options(**opts)
    need = excmg_workspace_size_batched(n, grids, ctypes.byref(o))
    if need == 0:
        raise ExcmgError(1, "excmg_workspace_size_batched")
    dev = problems[0].f.device
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    us = [torch.empty_like(p.f) for p in problems]
    fp = (_P * n)(*[_node_array(p.f, p.N, "f").value for p in problems])
    gp = (_P * n)(*[_node_array(p.g, p.N, "g").value for p in problems])
    up = (_P * n)(*[_ptr(u).value for u in us])
    st = (Stats * n)()
    status = excmg_solve_batched(n, grids, fp, gp, ctypes.byref(o), up, _ptr(ws), ws.numel(),
                                 st, _stream(stream))
    _check(status, "excmg_solve_batched", allow=(2,) if allow_not_converged else ())
    return {"u": us, "stats": [s.to_dict() for s in st], "status": STATUS[status]}


def adjoint(dLdu, L, stream=None, ws=None, **opts):
    N = (dLdu.shape[2] - 1, dLdu.shape[1] - 1, dLdu.shape[0] - 1)
    grid = make_grid(L, N)
    o, _keep = make_options(**opts)
    need = excmg_workspace_size_adjoint(ctypes.byref(grid), ctypes.byref(o))
    if need == 0:
        raise ExcmgError(1, "excmg_workspace_size_adjoint")
    if ws is None or ws.numel() < need:
        ws = workspace(need, dLdu.device)
    dLdf, dLdg = torch.empty_like(dLdu), torch.empty_like(dLdu)
    st = Stats()
    _check(excmg_adjoint(ctypes.byref(grid), _node_array(dLdu, N, "dLdu"), ctypes.byref(o),
                         _ptr(dLdf), _ptr(dLdg), _ptr(ws), ws.numel(), ctypes.byref(st),
                         _stream(stream)), "excmg_adjoint")
    return dLdf, dLdg, st.to_dict()
