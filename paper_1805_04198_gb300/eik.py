"""Thin Python binding of libeik (include/eik.h).

Argument marshalling only: every step of the solvers runs in the CUDA kernels
of libeik.so.  PyTorch supplies device memory and the current stream.  There is
no fallback: if libeik.so is missing or cannot be loaded, every call raises.

Entry points mirror the C names:
    eik_fsm_workspace_size, eik_fsm, eik_dd_workspace_size, eik_dd_solve,
    eik_dd_batched_workspace_size, eik_dd_solve_batched, eik_dd_batched_autotune,
    eik_fsm_many_workspace_size, eik_fsm_many, eik_dd_adjoint_many_workspace_size,
    eik_dd_adjoint_many, eik_dd_shard_exchange_bytes, eik_dd_shard_start, eik_dd_shard_fine,
    eik_dd_shard_coarse, eik_set_wait_limit, eik_last_error, eik_version
plus the conveniences :func:`fsm` and :func:`dd_solve`, which allocate the
workspace and the output with torch and return host-side statistics.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeik.so")
_lock = threading.Lock()
_lib = None

EIK_F32, EIK_F64 = 0, 1
STATUS = {0: "EIK_OK", -1: "EIK_EINVAL", -2: "EIK_ENOMEM", -3: "EIK_ECUDA", -4: "EIK_EDEVICE_TIMEOUT",
          -5: "EIK_EUNSUPPORTED"}


class EikError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("dtype", ctypes.c_int), ("n", ctypes.c_int64 * 3),
                ("stride", ctypes.c_int64 * 3), ("h", ctypes.c_double)]


class FsmStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("converged", ctypes.c_int), ("error", ctypes.c_int),
                ("updates", ctypes.c_int64), ("launches", ctypes.c_int64)]


class DDParams(ctypes.Structure):
    _fields_ = [("tiles", ctypes.c_int * 3), ("coarse_ratio", ctypes.c_int), ("theta", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("tol", ctypes.c_double), ("max_fsm_sweeps", ctypes.c_int64),
                ("max_coarse_sweeps", ctypes.c_int64), ("theta_adaptive", ctypes.c_int),
                ("omega", ctypes.c_double * 3), ("sig_gamma", ctypes.c_double), ("sig_delta", ctypes.c_double),
                ("sig_x0", ctypes.c_double), ("theta_cap", ctypes.c_double)]


class DDStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("error", ctypes.c_int),
                ("causal_rounds_max", ctypes.c_int), ("fsm_sweeps_max", ctypes.c_int64),
                ("coarse_sweeps_max", ctypes.c_int64), ("fsm_cap_hits", ctypes.c_int64),
                ("coarse_cap_hits", ctypes.c_int64), ("last_delta", ctypes.c_double),
                ("fine_updates", ctypes.c_int64), ("coarse_updates", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("fine_solves_skipped", ctypes.c_int64)]


class AdjointStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("converged", ctypes.c_int), ("error", ctypes.c_int),
                ("launches", ctypes.c_int64)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("fine_queue", ctypes.c_int), ("coarse_queue", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("largest_first", ctypes.c_int)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double)]


def _as_dict(s):
    return {k: getattr(s, k) for k, _ in s._fields_}


def load():
    """Load libeik.so (built by __graft_entry__.build()); raise if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libeik.so not found at %s: run __graft_entry__.build() first" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        lib.eik_last_error.restype = ctypes.c_char_p
        lib.eik_version.restype = ctypes.c_int
        lib.eik_fsm_workspace_size.restype = ctypes.c_size_t
        lib.eik_fsm_workspace_size.argtypes = [ctypes.POINTER(Grid)]
        lib.eik_fsm.restype = ctypes.c_int
        lib.eik_fsm.argtypes = [ctypes.POINTER(Grid), vp, vp, vp, vp, ctypes.c_int64, vp, ctypes.c_size_t, vp, vp]
        lib.eik_dd_workspace_size.restype = ctypes.c_size_t
        lib.eik_dd_workspace_size.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(DDParams)]
        lib.eik_dd_solve.restype = ctypes.c_int
        lib.eik_dd_solve.argtypes = [ctypes.POINTER(Grid), vp, vp, vp, ctypes.POINTER(DDParams), vp, vp,
                                     ctypes.c_size_t, vp, vp]
        lib.eik_dd_adjoint_workspace_size.restype = ctypes.c_size_t
        lib.eik_dd_adjoint_workspace_size.argtypes = [ctypes.POINTER(Grid)]
        lib.eik_dd_adjoint.restype = ctypes.c_int
        lib.eik_dd_adjoint.argtypes = [ctypes.POINTER(Grid), vp, vp, vp, vp, vp, ctypes.c_int64, vp, ctypes.c_size_t,
                                       vp, vp]
        lib.eik_dd_coarse_state.restype = ctypes.c_int
        lib.eik_dd_coarse_state.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(DDParams), vp, ctypes.c_size_t, vp,
                                            vp, vp]
        lib.eik_dd_solve_noalloc.restype = ctypes.c_int
        lib.eik_dd_solve_noalloc.argtypes = [ctypes.POINTER(Grid), vp, vp, vp, ctypes.POINTER(DDParams), vp, vp, vp]
        pp = ctypes.POINTER(ctypes.c_void_p)
        lib.eik_dd_batched_workspace_size.restype = ctypes.c_size_t
        lib.eik_dd_batched_workspace_size.argtypes = [ctypes.c_int, ctypes.POINTER(Grid), ctypes.POINTER(DDParams)]
        lib.eik_dd_solve_batched.restype = ctypes.c_int
        lib.eik_dd_solve_batched.argtypes = [ctypes.c_int, ctypes.POINTER(Grid), pp, pp, pp,
                                             ctypes.POINTER(DDParams), pp, ctypes.POINTER(BatchConfig), vp,
                                             ctypes.c_size_t, vp, vp]
        lib.eik_dd_batched_autotune.restype = ctypes.c_int
        lib.eik_dd_batched_autotune.argtypes = [ctypes.c_int, ctypes.POINTER(Grid), pp, pp, pp,
                                                ctypes.POINTER(DDParams), pp, ctypes.c_int, vp, ctypes.c_size_t,
                                                ctypes.POINTER(BatchConfig), ctypes.POINTER(ctypes.c_double), vp]
        lib.eik_fsm_many_workspace_size.restype = ctypes.c_size_t
        lib.eik_fsm_many_workspace_size.argtypes = [ctypes.POINTER(Grid), ctypes.c_int]
        lib.eik_fsm_many.restype = ctypes.c_int
        lib.eik_fsm_many.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, vp, pp, pp, pp, ctypes.c_int64, vp,
                                     ctypes.c_size_t, vp, vp]
        lib.eik_dd_adjoint_many_workspace_size.restype = ctypes.c_size_t
        lib.eik_dd_adjoint_many_workspace_size.argtypes = [ctypes.POINTER(Grid), ctypes.c_int]
        lib.eik_dd_adjoint_many.restype = ctypes.c_int
        lib.eik_dd_adjoint_many.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, vp, pp, pp, pp, pp, vp,
                                            ctypes.c_int64, vp, ctypes.c_size_t, vp, vp]
        lib.eik_dd_shard_exchange_bytes.restype = ctypes.c_size_t
        lib.eik_dd_shard_exchange_bytes.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(DDParams),
                                                    ctypes.POINTER(ctypes.c_size_t)]
        lib.eik_dd_shard_start.restype = ctypes.c_int
        lib.eik_dd_shard_start.argtypes = [ctypes.POINTER(Grid), vp, vp, vp, ctypes.POINTER(DDParams), vp, vp,
                                           ctypes.c_size_t, vp]
        lib.eik_dd_shard_fine.restype = ctypes.c_int
        lib.eik_dd_shard_fine.argtypes = [ctypes.POINTER(Grid), vp, vp, vp, ctypes.POINTER(DDParams), vp, vp,
                                          ctypes.c_size_t, ctypes.c_int, ctypes.c_int, vp, vp]
        lib.eik_dd_shard_coarse.restype = ctypes.c_int
        lib.eik_dd_shard_coarse.argtypes = [ctypes.POINTER(Grid), vp, vp, vp, ctypes.POINTER(DDParams), vp, vp,
                                            ctypes.c_size_t, ctypes.c_int, vp, vp, vp]
        lib.eik_set_wait_limit.restype = ctypes.c_int
        lib.eik_set_wait_limit.argtypes = [ctypes.c_int64]
        lib.eik_profile_enable.restype = ctypes.c_int
        lib.eik_profile_enable.argtypes = [ctypes.c_int]
        lib.eik_profile_collect.restype = ctypes.c_int
        lib.eik_profile_collect.argtypes = [ctypes.POINTER(KernelTime), ctypes.c_int]
        _lib = lib
        return lib


def eik_last_error() -> str:
    return load().eik_last_error().decode(errors="replace")


def eik_version() -> int:
    return load().eik_version()


def eik_dd_shard_exchange_bytes(grid: Grid, params: DDParams):
    """(bytes of the exchange buffer, bytes of one subdomain's record)."""
    rec = ctypes.c_size_t(0)
    n = int(load().eik_dd_shard_exchange_bytes(ctypes.byref(grid), ctypes.byref(params), ctypes.byref(rec)))
    if n == 0:
        raise EikError(-1, eik_last_error())
    return n, int(rec.value)


def eik_dd_shard_start(grid, r, gamma, g, params, u_out, ws, stream=None):
    wsp, wsn = _aligned(ws)
    _check(load().eik_dd_shard_start(ctypes.byref(grid), _ptr(r), _ptr(gamma), _ptr(g), ctypes.byref(params),
                                     _ptr(u_out), wsp, wsn, _stream(stream)))


def eik_dd_shard_fine(grid, r, gamma, g, params, u_out, ws, row0, row1, xbuf, stream=None):
    wsp, wsn = _aligned(ws)
    _check(load().eik_dd_shard_fine(ctypes.byref(grid), _ptr(r), _ptr(gamma), _ptr(g), ctypes.byref(params),
                                    _ptr(u_out), wsp, wsn, int(row0), int(row1), _ptr(xbuf), _stream(stream)))


def eik_dd_shard_coarse(grid, r, gamma, g, params, u_out, ws, k, xbuf, stats_dev, stream=None):
    wsp, wsn = _aligned(ws)
    _check(load().eik_dd_shard_coarse(ctypes.byref(grid), _ptr(r), _ptr(gamma), _ptr(g), ctypes.byref(params),
                                      _ptr(u_out), wsp, wsn, int(k), _ptr(xbuf), _ptr(stats_dev), _stream(stream)))


def eik_set_wait_limit(iterations: int) -> None:
    """Polls a device-side wait may make before it reports EIK_EDEVICE_TIMEOUT
    (current device; 0 restores the default)."""
    _check(load().eik_set_wait_limit(int(iterations)))


def _check(code):
    if code != 0:
        raise EikError(code, eik_last_error())


def make_grid(t: torch.Tensor, h: float) -> Grid:
    """eik_grid describing tensor t of shape (nx,) (the 1-D method of
    eik_dd_solve only), (ny, nx) or (nz, ny, nx)."""
    if t.dim() not in (1, 2, 3):
        raise ValueError("expected a 1-D, 2-D or 3-D tensor")
    if t.dtype not in (torch.float32, torch.float64):
        raise ValueError("dtype must be float32 or float64")
    if t.stride(-1) != 1:
        raise ValueError("innermost dimension must be contiguous")
    d = t.dim()
    n = list(reversed(t.shape)) + [1] * (3 - d)
    st = list(reversed(t.stride())) + [0] * (3 - d)
    if d == 1:
        st[1] = st[2] = n[0]
    if d == 2:
        st[2] = st[1] * n[1]
    return Grid(d, EIK_F64 if t.dtype == torch.float64 else EIK_F32, (ctypes.c_int64 * 3)(*n),
                (ctypes.c_int64 * 3)(*st), float(h))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_like(ref, *ts):
    for t in ts:
        if t.device != ref.device or t.shape != ref.shape or t.stride() != ref.stride():
            raise ValueError("all arrays must share device, shape and strides")


def _workspace(nbytes, device):
    return torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)


def _aligned(ws):
    off = (-ws.data_ptr()) % 256
    return ctypes.c_void_p(ws.data_ptr() + off), ws.numel() - off


def eik_profile_enable(on: bool) -> bool:
    return bool(load().eik_profile_enable(1 if on else 0))


def eik_profile_collect() -> dict:
    """{kernel name: {launches, total_ms, max_ms}} of the launches timed since
    the last collect (waits for their events)."""
    lib = load()
    buf = (KernelTime * 64)()
    n = lib.eik_profile_collect(buf, 64)
    if n < 0:
        raise EikError(n, eik_last_error())
    return {buf[i].name.decode(): {"launches": buf[i].launches, "total_ms": buf[i].total_ms,
                                   "max_ms": buf[i].max_ms} for i in range(min(n, 64))}


def eik_fsm_workspace_size(grid: Grid) -> int:
    return int(load().eik_fsm_workspace_size(ctypes.byref(grid)))


def eik_fsm(grid, r, gamma, g, u, max_sweeps, ws, stats_dev, stream=None):
    """Direct C call: all tensors on the device, ws 256-byte aligned uint8."""
    lib = load()
    wsp, wsn = _aligned(ws)
    _check(lib.eik_fsm(ctypes.byref(grid), _ptr(r), _ptr(gamma), _ptr(g), _ptr(u), int(max_sweeps), wsp, wsn,
                       _ptr(stats_dev), _stream(stream)))


def eik_dd_workspace_size(grid: Grid, params: DDParams) -> int:
    return int(load().eik_dd_workspace_size(ctypes.byref(grid), ctypes.byref(params)))


def eik_dd_solve(grid, r, gamma, g, params, u_out, ws, stats_dev, stream=None):
    lib = load()
    wsp, wsn = _aligned(ws)
    _check(lib.eik_dd_solve(ctypes.byref(grid), _ptr(r), _ptr(gamma), _ptr(g), ctypes.byref(params), _ptr(u_out),
                            wsp, wsn, _ptr(stats_dev), _stream(stream)))


def eik_dd_coarse_state(grid, params, ws, U_out, W_out, stream=None):
    lib = load()
    wsp, wsn = _aligned(ws)
    _check(lib.eik_dd_coarse_state(ctypes.byref(grid), ctypes.byref(params), wsp, wsn, _ptr(U_out), _ptr(W_out),
                                   _stream(stream)))


def dd_step1_state(r, gamma, g, h, tiles, coarse_ratio, **kw):
    """U^0, W^0 after Step 1 and its causal sweep (eik_dd_shard_start, then
    eik_dd_coarse_state) on the fine grid: NaN / 255 off the coarse set."""
    grid = make_grid(r, h)
    p = dd_params(tiles, coarse_ratio, **kw)
    nbytes = eik_dd_workspace_size(grid, p)
    if nbytes == 0:
        raise EikError(-1, eik_last_error())
    ws = _workspace(nbytes, r.device)
    u = torch.empty_like(r)
    eik_dd_shard_start(grid, r, gamma.contiguous(), g, p, u, ws)
    Uc = torch.full_like(r, float("nan"))
    Wc = torch.full(r.shape, 255, dtype=torch.uint8, device=r.device)
    eik_dd_coarse_state(grid, p, ws, Uc, Wc)
    return Uc, Wc


def eik_dd_solve_noalloc(grid, r, gamma, g, params, u_out, stats_dev, stream=None):
    """eik_dd_solve with the library's static scratch instead of a workspace
    (for callers that cannot allocate device memory)."""
    lib = load()
    _check(lib.eik_dd_solve_noalloc(ctypes.byref(grid), _ptr(r), _ptr(gamma), _ptr(g), ctypes.byref(params),
                                    _ptr(u_out), _ptr(stats_dev), _stream(stream)))


NOALLOC_SCRATCH_BYTES = 32 << 20


def dd_params(tiles, coarse_ratio, theta=1.0, max_iter=10, tol=0.0, max_fsm_sweeps=100000,
              max_coarse_sweeps=8, theta_adaptive=False, omega=(1.0, 1.0, 1.0), sig_gamma=0.75, sig_delta=0.01,
              sig_x0=0.9, theta_cap=0.0) -> DDParams:
    t = list(tiles) + [1] * (3 - len(tiles))
    return DDParams((ctypes.c_int * 3)(*t), int(coarse_ratio), float(theta), int(max_iter), float(tol),
                    int(max_fsm_sweeps), int(max_coarse_sweeps), 1 if theta_adaptive else 0,
                    (ctypes.c_double * 3)(*omega), float(sig_gamma), float(sig_delta), float(sig_x0),
                    float(theta_cap))


def fsm(r, gamma, g, h, max_sweeps=100000, stream=None, sync=True):
    """Plain FSM on the whole grid.  Returns (u, stats dict)."""
    _check_like(r, g)
    if gamma.dtype != torch.uint8 or gamma.shape != r.shape:
        raise ValueError("gamma must be uint8 with r's shape")
    grid = make_grid(r, h)
    nbytes = eik_fsm_workspace_size(grid)
    if nbytes == 0:
        raise EikError(-1, eik_last_error())
    ws = _workspace(nbytes, r.device)
    u = torch.empty_like(r)
    st = torch.zeros(ctypes.sizeof(FsmStats), dtype=torch.uint8, device=r.device)
    eik_fsm(grid, r, gamma.contiguous(), g, u, max_sweeps, ws, st, stream)
    if not sync:
        return u, st
    s = FsmStats.from_buffer_copy(bytes(st.cpu().numpy()))
    if s.error:
        raise EikError(s.error, "device-side wait expired")
    return u, _as_dict(s)


def dd_solve(r, gamma, g, h, tiles, coarse_ratio, theta=1.0, max_iter=10, tol=0.0, max_fsm_sweeps=100000,
             max_coarse_sweeps=8, stream=None, sync=True, return_coarse=False, **adaptive):
    """Two-scale DD solve (Sec. 3.2; Sec. 3.1 for a 1-D r, where tiles =
    (N,) subintervals and coarse_ratio must be their width M).  Returns (u,
    stats dict), and with return_coarse (2-D) also the coarse state the solve
    leaves (eik_dd_coarse_state: U^k, or u^k at weight 0, and W = w^k) on the
    fine grid.  Keyword
    arguments theta_adaptive, omega, sig_gamma, sig_delta, sig_x0, theta_cap
    select the per-node weight of Sec. 4.2 (see dd_params)."""
    _check_like(r, g)
    if gamma.dtype != torch.uint8 or gamma.shape != r.shape:
        raise ValueError("gamma must be uint8 with r's shape")
    grid = make_grid(r, h)
    p = dd_params(tiles, coarse_ratio, theta, max_iter, tol, max_fsm_sweeps, max_coarse_sweeps, **adaptive)
    nbytes = eik_dd_workspace_size(grid, p)
    if nbytes == 0:
        raise EikError(-1, eik_last_error())
    ws = _workspace(nbytes, r.device)
    u = torch.empty_like(r)
    st = torch.zeros(ctypes.sizeof(DDStats), dtype=torch.uint8, device=r.device)
    eik_dd_solve(grid, r, gamma.contiguous(), g, p, u, ws, st, stream)
    coarse = ()
    if return_coarse:
        # the coarse state the workspace holds (U^k, or u^k at weight 0, and
        # W = w^k) at the coarse-set nodes (NaN and 255 elsewhere)
        Uc = torch.full_like(r, float("nan"))
        Wc = torch.full(r.shape, 255, dtype=torch.uint8, device=r.device)
        eik_dd_coarse_state(grid, p, ws, Uc, Wc, stream)
        coarse = (Uc, Wc)
    if not sync:
        return (u, st) + coarse
    s = DDStats.from_buffer_copy(bytes(st.cpu().numpy()))
    if s.error:
        raise EikError(s.error, "device-side wait expired")
    return (u, _as_dict(s)) + coarse


def eik_dd_adjoint_workspace_size(grid: Grid) -> int:
    return int(load().eik_dd_adjoint_workspace_size(ctypes.byref(grid)))


def eik_dd_adjoint(grid, r, gamma, u, dJdu, grad_r, max_sweeps, ws, stats_dev, stream=None):
    lib = load()
    wsp, wsn = _aligned(ws)
    _check(lib.eik_dd_adjoint(ctypes.byref(grid), _ptr(r), _ptr(gamma), _ptr(u), _ptr(dJdu), _ptr(grad_r),
                              int(max_sweeps), wsp, wsn, _ptr(stats_dev), _stream(stream)))


def adjoint(r, gamma, u, dJdu, h, max_sweeps=100000, stream=None, sync=True):
    """dJ/dr at the converged solution u for a scalar J with dJ/du given.
    Returns (grad_r, stats dict)."""
    _check_like(r, u, dJdu)
    grid = make_grid(r, h)
    nbytes = eik_dd_adjoint_workspace_size(grid)
    if nbytes == 0:
        raise EikError(-1, eik_last_error())
    ws = _workspace(nbytes, r.device)
    grad = torch.empty_like(r)
    st = torch.zeros(ctypes.sizeof(AdjointStats), dtype=torch.uint8, device=r.device)
    eik_dd_adjoint(grid, r, gamma.contiguous(), u, dJdu, grad, max_sweeps, ws, st, stream)
    if not sync:
        return grad, st
    s = AdjointStats.from_buffer_copy(bytes(st.cpu().numpy()))
    if s.error:
        raise EikError(s.error, "device-side wait expired")
    return grad, _as_dict(s)


class EikonalSolve(torch.autograd.Function):
    """u = Eikonal solution for slowness r (2-D), differentiable in r.

    forward runs the plain FSM (solver="fsm") or the two-scale DD solve
    (solver="dd", keyword arguments as for dd_solve) and keeps only the
    returned u for the backward pass; backward runs eik_dd_adjoint at that u,
    i.e. it differentiates the converged discrete system."""

    @staticmethod
    def forward(ctx, r, gamma, g, h, solver="fsm", dd_kwargs=None):
        if solver == "fsm":
            u, _ = fsm(r, gamma, g, h)
        else:
            u, _ = dd_solve(r, gamma, g, h, **(dd_kwargs or {}))
        ctx.save_for_backward(r, gamma, u)
        ctx.h = h
        return u

    @staticmethod
    def backward(ctx, grad_u):
        r, gamma, u = ctx.saved_tensors
        grad_r, _ = adjoint(r, gamma, u, grad_u.contiguous(), ctx.h)
        return grad_r, None, None, None, None, None


# --------------------------------------------------------------------------
# Batched DD (many independent 2-D problems)
# --------------------------------------------------------------------------
def _ptr_array(ts):
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def _struct_array(cls, items):
    return (cls * len(items))(*items)


def eik_dd_batched_workspace_size(grids, params) -> int:
    n = len(grids)
    return int(load().eik_dd_batched_workspace_size(n, _struct_array(Grid, grids), _struct_array(DDParams, params)))


def eik_dd_solve_batched(grids, r, gamma, g, params, u_out, config, ws, stats_dev, stream=None):
    """Direct C call; r, gamma, g, u_out are lists of device tensors."""
    lib = load()
    wsp, wsn = _aligned(ws)
    cfg = ctypes.byref(config) if config is not None else None
    _check(lib.eik_dd_solve_batched(len(grids), _struct_array(Grid, grids), _ptr_array(r), _ptr_array(gamma),
                                    _ptr_array(g), _struct_array(DDParams, params), _ptr_array(u_out), cfg, wsp, wsn,
                                    _ptr(stats_dev), _stream(stream)))


def eik_dd_batched_autotune(grids, r, gamma, g, params, u_out, tune_iters, ws, stream=None):
    """Returns (best BatchConfig, its time in ms)."""
    lib = load()
    wsp, wsn = _aligned(ws)
    best = BatchConfig()
    ms = ctypes.c_double(0.0)
    _check(lib.eik_dd_batched_autotune(len(grids), _struct_array(Grid, grids), _ptr_array(r), _ptr_array(gamma),
                                       _ptr_array(g), _struct_array(DDParams, params), _ptr_array(u_out),
                                       int(tune_iters), wsp, wsn, ctypes.byref(best), ctypes.byref(ms),
                                       _stream(stream)))
    return best, ms.value


class DDBatch:
    """A fixed batch of independent 2-D DD problems on one device.

    problems: list of dicts with keys r, gamma, g (device tensors, r and g of
    one float dtype for the whole batch), h, tiles, coarse_ratio and optionally
    theta, max_iter, tol, max_fsm_sweeps, max_coarse_sweeps and the per-node
    weight's theta_adaptive, omega, sig_gamma, sig_delta, sig_x0, theta_cap
    (see dd_params).  Owns the outputs
    `u` (list), the workspace and the device statistics.  run() enqueues one
    batched solve; capture() records it into a CUDA graph that replay() reruns."""

    def __init__(self, problems, config=None):
        if not problems:
            raise ValueError("empty batch")
        self.r = [p["r"] for p in problems]
        self.gamma = [p["gamma"].contiguous() for p in problems]
        self.g = [p["g"] for p in problems]
        for r, gm, g in zip(self.r, self.gamma, self.g):
            _check_like(r, g)
            if gm.dtype != torch.uint8 or gm.shape != r.shape:
                raise ValueError("gamma must be uint8 with r's shape")
        self.grids = [make_grid(p["r"], p["h"]) for p in problems]
        adaptive_keys = ("theta_adaptive", "omega", "sig_gamma", "sig_delta", "sig_x0", "theta_cap")
        self.params = [dd_params(p["tiles"], p["coarse_ratio"], p.get("theta", 1.0), p.get("max_iter", 10),
                                 p.get("tol", 0.0), p.get("max_fsm_sweeps", 100000), p.get("max_coarse_sweeps", 8),
                                 **{k: p[k] for k in adaptive_keys if k in p})
                       for p in problems]
        nbytes = eik_dd_batched_workspace_size(self.grids, self.params)
        if nbytes == 0:
            raise EikError(-1, eik_last_error())
        dev = self.r[0].device
        self.ws = _workspace(nbytes, dev)
        self.u = [torch.empty_like(r) for r in self.r]
        self.stats_dev = torch.zeros(ctypes.sizeof(DDStats) * len(problems), dtype=torch.uint8, device=dev)
        self.config = config
        self.graph = None

    def autotune(self, tune_iters=2, stream=None):
        best, ms = eik_dd_batched_autotune(self.grids, self.r, self.gamma, self.g, self.params, self.u, tune_iters,
                                           self.ws, stream)
        self.config = best
        return best, ms

    def run(self, stream=None):
        eik_dd_solve_batched(self.grids, self.r, self.gamma, self.g, self.params, self.u, self.config, self.ws,
                             self.stats_dev, stream)

    def capture(self):
        """Record one solve into a CUDA graph (warm-up run first)."""
        self.run()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def replay(self):
        if self.graph is None:
            raise RuntimeError("capture() first")
        self.graph.replay()

    def stats(self):
        raw = bytes(self.stats_dev.cpu().numpy())
        sz = ctypes.sizeof(DDStats)
        return [_as_dict(DDStats.from_buffer_copy(raw[i * sz:(i + 1) * sz])) for i in range(len(self.u))]


# --------------------------------------------------------------------------
# Many sources on one grid and one slowness
# --------------------------------------------------------------------------
def _rows(x):
    """List of per-problem tensors from a list or a stacked tensor."""
    return [x[i] for i in range(x.shape[0])] if isinstance(x, torch.Tensor) else list(x)


def fsm_many(r, gammas, gs, h, max_sweeps=100000, stream=None, sync=True):
    """Plain FSM for several source sets on one grid.  gammas, gs: stacked
    tensors [S, ...] (or lists) with r's shape.  Returns (u [S, ...], stats)."""
    gl, ggl = _rows(gammas), _rows(gs)
    for gm, gv in zip(gl, ggl):
        _check_like(r, gv)
        if gm.dtype != torch.uint8 or gm.shape != r.shape or not gm.is_contiguous():
            raise ValueError("each gamma must be contiguous uint8 with r's shape")
    grid = make_grid(r, h)
    n = len(gl)
    lib = load()
    nbytes = int(lib.eik_fsm_many_workspace_size(ctypes.byref(grid), n))
    if nbytes == 0:
        raise EikError(-1, eik_last_error())
    ws = _workspace(nbytes, r.device)
    u = torch.empty((n,) + tuple(r.shape), dtype=r.dtype, device=r.device)
    ul = [u[i] for i in range(n)]
    st = torch.zeros(ctypes.sizeof(FsmStats) * n, dtype=torch.uint8, device=r.device)
    wsp, wsn = _aligned(ws)
    _check(lib.eik_fsm_many(ctypes.byref(grid), n, _ptr(r), _ptr_array(gl), _ptr_array(ggl), _ptr_array(ul),
                            int(max_sweeps), wsp, wsn, _ptr(st), _stream(stream)))
    if not sync:
        return u, st
    raw = bytes(st.cpu().numpy())
    sz = ctypes.sizeof(FsmStats)
    stats = [_as_dict(FsmStats.from_buffer_copy(raw[i * sz:(i + 1) * sz])) for i in range(n)]
    if any(x["error"] for x in stats):
        raise EikError(-4, "device-side wait expired")
    return u, stats


def adjoint_many(r, gammas, us, dJdus, h, per_problem=False, max_sweeps=100000, stream=None, sync=True):
    """Sum over source sets of dJ_p/dr (added in source order) at converged
    solutions us [S, ...] with dJ_p/du given in dJdus [S, ...].  Returns
    (grad_sum, per-problem gradients [S, ...] or None, stats)."""
    gl, ul, dl = _rows(gammas), _rows(us), _rows(dJdus)
    for gm, uu, dj in zip(gl, ul, dl):
        _check_like(r, uu, dj)
        if gm.dtype != torch.uint8 or gm.shape != r.shape or not gm.is_contiguous():
            raise ValueError("each gamma must be contiguous uint8 with r's shape")
    grid = make_grid(r, h)
    n = len(gl)
    lib = load()
    nbytes = int(lib.eik_dd_adjoint_many_workspace_size(ctypes.byref(grid), n))
    if nbytes == 0:
        raise EikError(-1, eik_last_error())
    ws = _workspace(nbytes, r.device)
    gsum = torch.empty_like(r)
    per = torch.empty((n,) + tuple(r.shape), dtype=r.dtype, device=r.device) if per_problem else None
    st = torch.zeros(ctypes.sizeof(AdjointStats) * n, dtype=torch.uint8, device=r.device)
    wsp, wsn = _aligned(ws)
    gptr = _ptr_array([per[i] for i in range(n)]) if per_problem else None
    _check(lib.eik_dd_adjoint_many(ctypes.byref(grid), n, _ptr(r), _ptr_array(gl), _ptr_array(ul), _ptr_array(dl),
                                   gptr, _ptr(gsum), int(max_sweeps), wsp, wsn, _ptr(st), _stream(stream)))
    if not sync:
        return gsum, per, st
    raw = bytes(st.cpu().numpy())
    sz = ctypes.sizeof(AdjointStats)
    stats = [_as_dict(AdjointStats.from_buffer_copy(raw[i * sz:(i + 1) * sz])) for i in range(n)]
    if any(x["error"] for x in stats):
        raise EikError(-4, "device-side wait expired")
    return gsum, per, stats


class ManyDD:
    """Forward solve of many source sets on one grid by the two-scale DD
    (Sec. 3.2): one batched solve (eik_dd_solve_batched) whose problems share
    the slowness r and differ in gamma and g (stacked [S, ny, nx]).  Built once
    for r's storage; solve(r) reruns it (the batch holds r's address, so r
    must be that tensor or a view of the same storage).  Keyword arguments as
    for dd_params (theta, max_iter, tol, max_coarse_sweeps, ...)."""

    def __init__(self, r, gammas, gs, h, tiles, coarse_ratio, config=None, **params):
        self.ptr = r.data_ptr()
        self.shape = tuple(gammas.shape)
        probs = [dict(r=r, gamma=gammas[s], g=gs[s], h=h, tiles=tiles, coarse_ratio=coarse_ratio, **params)
                 for s in range(gammas.shape[0])]
        self.batch = DDBatch(probs, config=config)

    def solve(self, r):
        if r.data_ptr() != self.ptr:
            raise ValueError("ManyDD was built for another slowness tensor")
        self.batch.run()
        return torch.stack(self.batch.u)

    def stats(self):
        return self.batch.stats()


class EikonalSolveMany(torch.autograd.Function):
    """u[s] = Eikonal solution for slowness r and source set s (2-D), all
    source sets solved together; differentiable in r.  gammas, gs: stacked
    [S, ny, nx].  The forward is the plain FSM of every source in one call
    (eik_fsm_many), or the DD when `dd` is a ManyDD built for r.  Only the
    converged u is kept for the backward (no iterate of either solver), which
    sums the per-source gradients in the library (eik_dd_adjoint_many)."""

    @staticmethod
    def forward(ctx, r, gammas, gs, h, dd=None):
        if dd is None:
            u, _ = fsm_many(r, gammas, gs, h, sync=False)
        else:
            u = dd.solve(r)
        ctx.save_for_backward(r, gammas, u)
        ctx.h = h
        return u

    @staticmethod
    def backward(ctx, grad_u):
        r, gammas, u = ctx.saved_tensors
        gsum, _, _ = adjoint_many(r, gammas, u, grad_u.contiguous(), ctx.h, sync=False)
        return gsum, None, None, None, None


def parse_dd_stats(st: torch.Tensor) -> dict:
    return _as_dict(DDStats.from_buffer_copy(bytes(st.cpu().numpy())))
