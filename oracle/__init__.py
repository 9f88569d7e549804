"""FP64 CPU oracle for the two-scale DD Eikonal method (arXiv:1805.04198).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may load it; the product path never does.  It
shares no code with the CUDA library: the C source here is compiled on its own
with ``-ffp-contract=off`` so that no multiply-add is fused.

Functions (each follows the paper section named in its docstring):
  local_solve  Godunov local solve, Sec. 1.1 eq. (godonuv) / Alg. 3
  fsm          fast sweeping method, Sec. 1.1
  fmm          Dijkstra/fast marching on the same discrete system (Sec. 1.1)
  dd           two-scale domain decomposition, Sec. 3.2 Steps 1-4, Alg. 1-5
  adjoint      discrete adjoint of the converged Godunov system (no paper
               counterpart; checked by finite differences)
  theta_estimate  per-node weight of Sec. 4.2 (eqs. secthetaest, thetaest)
  model_problem   Sec. 4's model problem, eq. modelprob, with the bounds of
               Theorem 2's proof
  step4_box    Alg. 5 sweeps on one coarse box (Step 4 of Sec. 3.2)
  alg4_select  Alg. 4's choice among the copies of one coarse-set node
  theta_node   Sec. 4.2's weight of one node from its history
  dd_probe     dd with a per-iteration record of one node
  dd1          the one-dimensional method of Sec. 3.1 (Steps 1-4)
  dd_margins   dd() plus W^0 and the margins of Step 1's wind decisions (for
               tests of a lower-precision solve)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eik_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def _compile(out, extra):
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"] + extra + \
        ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (serial FP64, no FMA contraction)
    and liboracle_omp.so, the same source with OpenMP over the independent
    subdomain and shifted-grid solves (the all-cores CPU baseline)."""
    for out, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            _compile(out, extra)
    return _LIB


class DDParams(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_long * 3), ("h", ctypes.c_double),
                ("tiles", ctypes.c_int * 3), ("c", ctypes.c_int), ("theta", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_fsm_sweeps", ctypes.c_long), ("max_coarse_sweeps", ctypes.c_long),
                ("theta_adaptive", ctypes.c_int), ("omega", ctypes.c_double * 3),
                ("sig_gamma", ctypes.c_double), ("sig_delta", ctypes.c_double), ("sig_x0", ctypes.c_double),
                ("theta_cap", ctypes.c_double)]


class DD1Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_long), ("M", ctypes.c_long), ("h", ctypes.c_double), ("theta", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("tol", ctypes.c_double), ("max_fsm_sweeps", ctypes.c_long),
                ("max_coarse_sweeps", ctypes.c_long)]


class DD1Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("last_delta", ctypes.c_double),
                ("fsm_sweeps_max", ctypes.c_long), ("coarse_sweeps_max", ctypes.c_long),
                ("fsm_cap_hits", ctypes.c_long), ("coarse_cap_hits", ctypes.c_long),
                ("causal_rounds_max", ctypes.c_long), ("fine_updates", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DDStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("last_delta", ctypes.c_double),
                ("fsm_sweeps_max", ctypes.c_long), ("coarse_sweeps_max", ctypes.c_long),
                ("fsm_cap_hits", ctypes.c_long), ("coarse_cap_hits", ctypes.c_long),
                ("causal_rounds_max", ctypes.c_long), ("fine_updates", ctypes.c_longlong),
                ("coarse_updates", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load(omp=False):
    global _lib, _lib_omp
    with _lock:
        if omp:
            if _lib_omp is None:
                build()
                _lib_omp = _bind(ctypes.CDLL(_LIB_OMP))
            return _lib_omp
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _bind(lib):
    """Declare the argument and result types of the oracle's C functions."""
    dp = ctypes.POINTER(ctypes.c_double)
    bp = ctypes.POINTER(ctypes.c_ubyte)
    sp = ctypes.POINTER(ctypes.c_byte)
    lp = ctypes.POINTER(ctypes.c_long)
    lib.orc_local_solve.restype = ctypes.c_double
    lib.orc_local_solve.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, sp]
    lib.orc_fsm.restype = ctypes.c_long
    lib.orc_fsm.argtypes = [ctypes.c_int, lp, ctypes.c_double, dp, bp, dp, dp, sp, ctypes.c_long,
                            ctypes.POINTER(ctypes.c_int)]
    lib.orc_fmm.restype = None
    lib.orc_fmm.argtypes = [ctypes.c_int, lp, ctypes.c_double, dp, bp, dp, dp]
    lib.orc_dd.restype = ctypes.c_int
    lib.orc_dd.argtypes = [ctypes.POINTER(DDParams), dp, bp, dp, dp, dp, dp, ctypes.POINTER(DDStats)]
    lib.orc_theta_estimate.restype = ctypes.c_double
    lib.orc_theta_estimate.argtypes = [ctypes.POINTER(DDParams), ctypes.c_double, dp, ctypes.c_int,
                                       ctypes.c_double]
    ip = ctypes.POINTER(ctypes.c_int)
    lib.orc_step4_box.restype = ctypes.c_long
    lib.orc_step4_box.argtypes = [ctypes.c_int, lp, ctypes.c_double, dp, bp, dp, dp, dp, sp, sp, ip, dp,
                                  ctypes.c_long, dp, dp, ip]
    lib.orc_alg4_select.restype = ctypes.c_int
    lib.orc_alg4_select.argtypes = [ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, dp, sp, bp, sp]
    lib.orc_theta_node.restype = ctypes.c_double
    lib.orc_theta_node.argtypes = [ctypes.POINTER(DDParams), ctypes.c_int] + [ctypes.c_double] * 6
    lib.orc_dd_probe.restype = ctypes.c_int
    lib.orc_dd_probe.argtypes = [ctypes.POINTER(DDParams), dp, bp, dp, dp, dp, dp, ctypes.POINTER(DDStats),
                                 ctypes.c_long, dp]
    lib.orc_dd_margins.restype = ctypes.c_int
    lib.orc_dd_margins.argtypes = [ctypes.POINTER(DDParams), dp, bp, dp, dp, ctypes.POINTER(DDStats), sp, dp, dp, sp,
                                   dp, dp]
    lib.orc_dd1.restype = ctypes.c_int
    lib.orc_dd1.argtypes = [ctypes.POINTER(DD1Params), dp, bp, dp, dp, dp, dp, dp, sp,
                            ctypes.POINTER(DD1Stats)]
    lib.orc_adjoint.restype = None
    lib.orc_adjoint.argtypes = [ctypes.c_int, lp, ctypes.c_double, dp, bp, dp, dp, dp]
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _bp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))


def _sp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_byte))


def _shape_n(shape):
    """numpy shape (z, y, x) / (y, x) -> (d, n[3]) with n[0] = x extent."""
    d = len(shape)
    n = list(reversed(shape)) + [1] * (3 - d)
    return d, (ctypes.c_long * 3)(*n)


def _prep(r, gamma, g):
    r = np.ascontiguousarray(r, dtype=np.float64)
    gamma = np.ascontiguousarray(gamma, dtype=np.uint8)
    g = np.ascontiguousarray(np.broadcast_to(g, r.shape), dtype=np.float64)
    assert r.shape == gamma.shape
    return r, gamma, g


def local_solve(vm, vp, rh):
    """Godunov local solve (Sec. 1.1 / Alg. 3).  Returns (u~, wind tuple)."""
    lib = _load()
    d = len(vm)
    a = np.ascontiguousarray(vm, dtype=np.float64)
    b = np.ascontiguousarray(vp, dtype=np.float64)
    w = np.zeros(3, dtype=np.int8)
    u = lib.orc_local_solve(d, _dp(a), _dp(b), float(rh), _sp(w))
    return u, tuple(int(v) for v in w[:d])


def fsm(r, gamma, g, h, max_sweeps=100000, return_wind=False):
    """Fast sweeping method (Sec. 1.1).  Returns (u, sweeps, converged[, wind])."""
    lib = _load()
    r, gamma, g = _prep(r, gamma, g)
    d, n = _shape_n(r.shape)
    u = np.empty_like(r)
    w = np.zeros(r.shape + (3,), dtype=np.int8)
    conv = ctypes.c_int(0)
    s = lib.orc_fsm(d, n, float(h), _dp(r), _bp(gamma), _dp(g), _dp(u), _sp(w), int(max_sweeps),
                    ctypes.byref(conv))
    out = (u, int(s), bool(conv.value))
    if return_wind:
        out = out + (w[..., :d],)
    return out


def fmm(r, gamma, g, h):
    """Dijkstra / fast marching on the same scheme (cross-check of fsm)."""
    lib = _load()
    r, gamma, g = _prep(r, gamma, g)
    d, n = _shape_n(r.shape)
    u = np.empty_like(r)
    lib.orc_fmm(d, n, float(h), _dp(r), _bp(gamma), _dp(g), _dp(u))
    return u


def dd(r, gamma, g, h, tiles, c, theta=1.0, max_iter=10, tol=0.0, max_fsm_sweeps=100000,
       max_coarse_sweeps=80, return_coarse=False, theta_adaptive=False, omega=(1.0, 1.0, 1.0),
       sig_gamma=0.75, sig_delta=0.01, sig_x0=0.9, theta_cap=0.0, parallel=False):
    """Two-scale DD iteration (Sec. 3.2, Steps 1-4).

    tiles: subdomains per axis in (x, y[, z]) order.  Returns (u, stats dict,
    delta_log[, U]) where delta_log[k] = max |U^k - U^{k-1}|.  With
    theta_adaptive the weight of Alg. 5 is estimated per node (Sec. 4.2, eq.
    secthetaest damped by eq. thetaest; omega, sig_* its parameters) and
    `theta` is used where the estimate is undefined.  parallel=True runs the
    OpenMP build (same results; the subdomain and shifted-grid solves of a
    step on all host cores, or OMP_NUM_THREADS).
    """
    lib = _load(omp=parallel)
    r, gamma, g = _prep(r, gamma, g)
    d, n = _shape_n(r.shape)
    t = list(tiles) + [1] * (3 - len(tiles))
    p = DDParams(d, n, float(h), (ctypes.c_int * 3)(*t), int(c), float(theta), int(max_iter), float(tol),
                 int(max_fsm_sweeps), int(max_coarse_sweeps), 1 if theta_adaptive else 0,
                 (ctypes.c_double * 3)(*omega), float(sig_gamma), float(sig_delta), float(sig_x0),
                 float(theta_cap))
    u = np.empty_like(r)
    U = np.empty_like(r)
    log = np.empty(max_iter + 1, dtype=np.float64)
    st = DDStats()
    rc = lib.orc_dd(ctypes.byref(p), _dp(r), _bp(gamma), _dp(g), _dp(u), _dp(U), _dp(log), ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle dd: invalid parameters")
    out = (u, st.as_dict(), log)
    if return_coarse:
        out = out + (U,)
    return out


def dd_margins(r, gamma, g, h, tiles, c, theta=1.0, max_iter=0, tol=0.0, max_fsm_sweeps=100000,
               max_coarse_sweeps=80, U0=None, W0=None, parallel=False):
    """dd() with test hooks for comparing a lower-precision solve.  Returns
    (u, stats, W0_own, margin, copies, cmargin): W0_own (shape + (3,)) is this
    solve's W^0, margin (shape) at each coarse-set node the smallest margin of
    the Alg. 1 decisions behind its wind (NaN off the coarse set, +inf at Gamma
    and unreached nodes); copies (4 + shape) the subdomain copies of iteration
    0 at the coarse-set nodes by slot (NaN where absent) and cmargin (shape) the
    smallest margin of the decisions behind Alg. 4's choice there.  U0 (shape)
    and W0 (shape + (3,)), when given, replace this solve's U^0 and W^0 at the
    coarse-set nodes after Step 1."""
    lib = _load(omp=parallel)
    r, gamma, g = _prep(r, gamma, g)
    p = _params(r.shape, h, tiles, c, theta, max_iter, tol, max_fsm_sweeps, max_coarse_sweeps, False,
                (1.0, 1.0, 1.0), 0.75, 0.01, 0.9, 0.0)
    u = np.empty_like(r)
    W0_own = np.zeros(r.shape + (3,), dtype=np.int8)
    margin = np.empty_like(r)
    copies = np.empty((4,) + r.shape)
    cmargin = np.empty_like(r)
    U0_in = None if U0 is None else np.ascontiguousarray(U0, dtype=np.float64)
    W0_in = None if W0 is None else np.ascontiguousarray(W0, dtype=np.int8)
    null_d = ctypes.POINTER(ctypes.c_double)()
    null_s = ctypes.POINTER(ctypes.c_byte)()
    st = DDStats()
    rc = lib.orc_dd_margins(ctypes.byref(p), _dp(r), _bp(gamma), _dp(g), _dp(u), ctypes.byref(st), _sp(W0_own),
                            _dp(margin), null_d if U0_in is None else _dp(U0_in),
                            null_s if W0_in is None else _sp(W0_in), _dp(copies), _dp(cmargin))
    if rc != 0:
        raise ValueError("oracle dd_margins: invalid parameters")
    return u, st.as_dict(), W0_own, margin, copies, cmargin


def _params(shape, h, tiles, c, theta, max_iter, tol, max_fsm_sweeps, max_coarse_sweeps, theta_adaptive, omega,
            sig_gamma, sig_delta, sig_x0, theta_cap):
    d, n = _shape_n(shape)
    t = list(tiles) + [1] * (3 - len(tiles))
    return DDParams(d, n, float(h), (ctypes.c_int * 3)(*t), int(c), float(theta), int(max_iter), float(tol),
                    int(max_fsm_sweeps), int(max_coarse_sweeps), 1 if theta_adaptive else 0,
                    (ctypes.c_double * 3)(*omega), float(sig_gamma), float(sig_delta), float(sig_x0),
                    float(theta_cap))


def dd_probe(r, gamma, g, h, tiles, c, probe, theta=1.0, max_iter=10, tol=0.0, max_fsm_sweeps=100000,
             max_coarse_sweeps=80, theta_adaptive=False, omega=(1.0, 1.0, 1.0), sig_gamma=0.75, sig_delta=0.01,
             sig_x0=0.9, theta_cap=0.0):
    """dd (Sec. 3.2) with a record of the node at numpy index ``probe``: returns
    (u, stats, log) with log[k] = (u^k, C^k = C_H(nbrs U^k), weight used for
    U^{k+1}, U^k) at that node, NaN where iteration k did not compute it."""
    lib = _load()
    r, gamma, g = _prep(r, gamma, g)
    p = _params(r.shape, h, tiles, c, theta, max_iter, tol, max_fsm_sweeps, max_coarse_sweeps, theta_adaptive,
                omega, sig_gamma, sig_delta, sig_x0, theta_cap)
    u = np.empty_like(r)
    U = np.empty_like(r)
    dlog = np.empty(max_iter + 1, dtype=np.float64)
    plog = np.empty((max_iter + 1, 4), dtype=np.float64)
    st = DDStats()
    flat = int(np.ravel_multi_index(probe, r.shape))
    rc = lib.orc_dd_probe(ctypes.byref(p), _dp(r), _bp(gamma), _dp(g), _dp(u), _dp(U), _dp(dlog), ctypes.byref(st),
                          flat, _dp(plog))
    if rc != 0:
        raise ValueError("oracle dd_probe: invalid parameters")
    return u, st.as_dict(), plog


def step4_box(H, r, fixed, g, Uk, uk, wk, Wk, axes, theta, max_sweeps=80):
    """Alg. 5 sweeps on one coarse box (Step 4 of Sec. 3.2).  Arrays are numpy
    arrays of the box shape ((y, x) or (z, y, x)); wk, Wk carry a trailing axis
    of d wind components in (x, y[, z]) order; axes[...] has bit k set when the
    node lies on a coarse line of axis k; theta is a scalar or per node.
    Returns (U, C_H(nbrs U^k), sweeps, capped)."""
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    shape = r.shape
    d, n = _shape_n(shape)
    fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
    g = np.ascontiguousarray(np.broadcast_to(g, shape), dtype=np.float64)
    Uk = np.ascontiguousarray(Uk, dtype=np.float64)
    uk = np.ascontiguousarray(uk, dtype=np.float64)

    def winds(w):
        out = np.zeros(shape + (3,), dtype=np.int8)
        out[..., :d] = np.asarray(w, dtype=np.int8)
        return out

    wk3, Wk3 = winds(wk), winds(Wk)
    ax = np.ascontiguousarray(np.broadcast_to(axes, shape), dtype=np.int32)
    th = np.ascontiguousarray(np.broadcast_to(theta, shape), dtype=np.float64)
    U = np.empty(shape)
    C = np.empty(shape)
    capped = ctypes.c_int(0)
    s = lib.orc_step4_box(d, n, float(H), _dp(r), _bp(fixed), _dp(g), _dp(Uk), _dp(uk), _sp(wk3), _sp(Wk3),
                          ax.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(th), int(max_sweeps), _dp(U), _dp(C),
                          ctypes.byref(capped))
    return U, C, int(s), bool(capped.value)


def alg4_select(B, nc, u, w, echo, W, d=2):
    """Alg. 4's choice at one coarse-set node: index of the chosen copy."""
    lib = _load()
    ncopies = len(u)
    nca = (ctypes.c_int * 3)(*(list(nc) + [1] * (3 - len(nc))))
    ua = np.ascontiguousarray(u, dtype=np.float64)
    wa = np.zeros((ncopies, 3), dtype=np.int8)
    wa[:, :d] = np.asarray(w, dtype=np.int8)
    ea = np.ascontiguousarray(echo, dtype=np.uint8)
    Wa = np.zeros(3, dtype=np.int8)
    Wa[:d] = np.asarray(W, dtype=np.int8)
    return lib.orc_alg4_select(d, int(B), nca, ncopies, _dp(ua), _sp(wa), _bp(ea), _sp(Wa))


def theta_node(nhist, Ck, C1, C2, C3, uk, uprev, theta=0.2, omega=(1.0, 1.0, 1.0), sig_gamma=0.75, sig_delta=0.01,
               sig_x0=0.9, theta_cap=0.0, adaptive=True):
    """Sec. 4.2's weight of one node from its history (C^k .. C^{k-3}, u^k, u^{k-1})."""
    lib = _load()
    p = _params((1, 1), 1.0, (1, 1), 1, theta, 0, 0.0, 1, 1, adaptive, omega, sig_gamma, sig_delta, sig_x0,
                theta_cap)
    return lib.orc_theta_node(ctypes.byref(p), int(nhist), float(Ck), float(C1), float(C2), float(C3), float(uk),
                              float(uprev))


def dd1(r, gamma, g, h, N, M, theta=1.0, max_iter=10, tol=0.0, max_fsm_sweeps=100000, max_coarse_sweeps=1000):
    """The one-dimensional method of Sec. 3.1 on a fine grid of N*M+1 nodes
    (coarse node every M).  Returns (u, stats, logs) with logs a dict of
    (max_iter+1, N+1) arrays: U (U^k), u (u^k), W (W^k) and Upre (Step 4's
    result of iteration k before the causal sweep); unused rows are NaN / 0."""
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    gamma = np.ascontiguousarray(gamma, dtype=np.uint8)
    g = np.ascontiguousarray(np.broadcast_to(g, r.shape), dtype=np.float64)
    assert r.shape == (N * M + 1,)
    p = DD1Params(int(N), int(M), float(h), float(theta), int(max_iter), float(tol), int(max_fsm_sweeps),
                  int(max_coarse_sweeps))
    u = np.empty_like(r)
    logs = {k: np.full((max_iter + 1, N + 1), np.nan) for k in ("U", "u", "Upre")}
    Wl = np.zeros((max_iter + 1, N + 1), dtype=np.int8)
    st = DD1Stats()
    rc = lib.orc_dd1(ctypes.byref(p), _dp(r), _bp(gamma), _dp(g), _dp(u), _dp(logs["U"]), _dp(logs["u"]),
                     _dp(logs["Upre"]), _sp(Wl), ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle dd1: invalid parameters")
    logs["W"] = Wl
    return u, st.as_dict(), logs


def theta_estimate(du, dC, omega=(1.0, 1.0, 1.0), sig_gamma=0.75, sig_delta=0.01, sig_x0=0.9, theta_cap=0.0,
                   fallback=0.2):
    """Per-node weight of Sec. 4.2 from du = u^k - u^{k-1} and the last changes
    dC[s] of the coarse solver (eq. secthetaest, damping of eq. thetaest)."""
    lib = _load()
    p = DDParams(2, (ctypes.c_long * 3)(1, 1, 1), 1.0, (ctypes.c_int * 3)(1, 1, 1), 1, float(fallback), 0, 0.0, 1, 1,
                 1, (ctypes.c_double * 3)(*omega), float(sig_gamma), float(sig_delta), float(sig_x0),
                 float(theta_cap))
    a = np.ascontiguousarray(dC, dtype=np.float64)
    return lib.orc_theta_estimate(ctypes.byref(p), float(du), _dp(a), len(a), float(fallback))


def adjoint(r, gamma, u, dJdu, h):
    """dJ/dr of the converged discrete system at u for a scalar J with dJ/du given."""
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    gamma = np.ascontiguousarray(gamma, dtype=np.uint8)
    u = np.ascontiguousarray(u, dtype=np.float64)
    dJdu = np.ascontiguousarray(dJdu, dtype=np.float64)
    d, n = _shape_n(r.shape)
    out = np.zeros_like(r)
    lib.orc_adjoint(d, n, float(h), _dp(r), _bp(gamma), _dp(u), _dp(dJdu), _dp(out))
    return out


def model_problem(N, M, theta, max_iter):
    """The model problem of Sec. 4 and its weighted iteration, eq. modelprob.

    Strip [0, 1] x [0, H], H = 1/N, r = 1, Gamma = the bottom edge and the
    left edge with g = sqrt(x^2 + y^2); fine step h = H/M, coarse nodes
    X_ij = (iH, jh), i = 0..N, j = 0..M.  The coarse solver is the one printed
    with eq. modelprob: U_{i-1,j} + H for j < M, the two-term Godunov formula
    in U_{i-1,M} and U_{i,0} for j = M (min + H where the two differ by H or
    more, the causality branch of Sec. 3.2's C_H).  u^k_{.,i} is the fine FSM
    solution of subdomain [(i-1)H, iH] x [0, H] with U^k held fixed on its
    left column (the form the proof of Theorem 1 uses: u^k is computed from
    the values U^k) and g on its bottom row, read at x = iH; u^f is the FSM
    solution of the whole strip.  U^0 = C_H(U^0) (eq. modelprob's initial
    condition), the left column and bottom row of U stay at u^f (eqs. modelBC1,
    modelBC2), and for k >= 0, i = 1..N in order:
        U^{k+1}_ij = theta^{k+1}_ij [C_H(U^{k+1}_{i-1,j}) - C_H(U^k_{i-1,j})] + u^k_ij.

    ``theta`` is a constant or a callable theta(k1, i, j, mbar, Mbar) giving
    theta^{k1}_ij from the bounds of Theorem 2's proof,
        mbar = (U^k_ij - u^k_ij) / D,  Mbar = (u^f_ij - u^k_ij) / D,
        D = C_H(U^{k+1}_{i-1,j}) - C_H(U^k_{i-1,j})   (NaN where D = 0).

    Returns dict with arrays indexed [k][j, i]: U (k = 0..max_iter), u
    (k = 0..max_iter-1), mbar and Mbar (k = 1..max_iter at list index k-1),
    and uf [j, i].
    """
    H = 1.0 / N
    h = H / M
    nx = N * M + 1

    def g_at(l, m):
        return float(np.hypot(l * h, m * h))

    def strip(ncol, x0, left):
        r = np.ones((M + 1, ncol + 1))
        gam = np.zeros((M + 1, ncol + 1), np.uint8)
        gv = np.zeros((M + 1, ncol + 1))
        gam[:, 0] = 1
        gv[:, 0] = left
        gam[0, :] = 1
        gv[0, :] = [g_at(x0 + l, 0) for l in range(ncol + 1)]
        u, _, _ = fsm(r, gam, gv, h)
        return u

    ufull = strip(nx - 1, 0, [g_at(0, m) for m in range(M + 1)])
    uf = np.ascontiguousarray(ufull[:, ::M])

    def CH(a, i, j):
        if j < M:
            return a + H
        b = uf[0, i]
        if abs(a - b) >= H:
            return min(a, b) + H
        return 0.5 * (a + b + np.sqrt(2.0 * H * H - (a - b) ** 2))

    def fine(U):
        u = np.empty_like(U)
        u[:, 0] = U[:, 0]
        for i in range(1, N + 1):
            u[:, i] = strip(M, (i - 1) * M, U[:, i - 1])[:, M]
        u[0, :] = uf[0, :]
        return u

    U0 = np.empty((M + 1, N + 1))
    U0[:, 0] = uf[:, 0]
    U0[0, :] = uf[0, :]
    for i in range(1, N + 1):
        for j in range(1, M + 1):
            U0[j, i] = CH(U0[j, i - 1], i, j)
    Us, us, mb, Mb = [U0], [], [], []
    for k in range(max_iter):
        Uk = Us[-1]
        uk = fine(Uk)
        Un = np.empty_like(Uk)
        Un[:, 0] = uf[:, 0]
        Un[0, :] = uf[0, :]
        mk = np.full_like(Uk, np.nan)
        Mk = np.full_like(Uk, np.nan)
        for i in range(1, N + 1):
            for j in range(1, M + 1):
                D = CH(Un[j, i - 1], i, j) - CH(Uk[j, i - 1], i, j)
                if D != 0.0:
                    mk[j, i] = (Uk[j, i] - uk[j, i]) / D
                    Mk[j, i] = (uf[j, i] - uk[j, i]) / D
                t = theta(k + 1, i, j, mk[j, i], Mk[j, i]) if callable(theta) else theta
                Un[j, i] = t * D + uk[j, i]
        us.append(uk)
        mb.append(mk)
        Mb.append(Mk)
        Us.append(Un)
    return {"U": Us, "u": us, "mbar": mb, "Mbar": Mb, "uf": uf}
