"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a hand-derived value,
an independent algorithm (Dijkstra), an exact solution, a theorem of the paper,
or an invariant of the discrete scheme.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1805_04198_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
INF = math.inf


def _val(tok):
    return float(eval(tok, {"sqrt": math.sqrt, "inf": INF}))


def test_local_solve_2d_hand_values():
    """Sec. 3.2 closed form of C_H / Alg. 3 (with direction-of-travel winds)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "local_solve_2d.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) >= 8
    for vmx, vpx, vmy, vpy, rh, u, wx, wy in rows:
        got, w = O.local_solve([_val(vmx), _val(vmy)], [_val(vpx), _val(vpy)], _val(rh))
        want = _val(u)
        if math.isinf(want):
            assert math.isinf(got)
        else:
            assert got == pytest.approx(want, rel=1e-15, abs=1e-15)
            assert w == (int(wx), int(wy))


def test_local_solve_quadratic_residual():
    """The two- and three-term branches solve sum_j (u - a_j)^2 = (r h)^2."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        a = rng.uniform(0, 1, 3)
        rh = rng.uniform(0.05, 1.0)
        u2, w2 = O.local_solve([a[0], a[1]], [INF, INF], rh)
        if abs(a[0] - a[1]) < rh:
            assert (u2 - a[0]) ** 2 + (u2 - a[1]) ** 2 == pytest.approx(rh * rh, rel=1e-12)
            assert u2 > max(a[0], a[1])
        else:
            assert u2 == min(a[0], a[1]) + rh
        u3, w3 = O.local_solve(list(a), [INF] * 3, rh)
        if all(w3):
            assert sum((u3 - ai) ** 2 for ai in a) == pytest.approx(rh * rh, rel=1e-10)
            assert u3 > max(a)
        # causality: the solve never goes below its inputs plus nothing
        assert u3 > min(a)
        # 3-D with one axis missing reduces exactly to the 2-D solve
        u32, w32 = O.local_solve([a[0], a[1], INF], [INF] * 3, rh)
        assert u32 == u2 and w32[:2] == w2 and w32[2] == 0


def test_local_solve_3d_symmetric():
    """Equal minima on three axes: 3 (u - a)^2 = (rh)^2 -> u = a + rh/sqrt(3)."""
    u, w = O.local_solve([0.25, 0.25, 0.25], [INF, INF, INF], 0.3)
    assert u == pytest.approx(0.25 + 0.3 / math.sqrt(3), rel=1e-15)
    assert w == (1, 1, 1)
    u1, w1 = O.local_solve([0.5], [INF], 0.125)
    assert u1 == 0.625 and w1 == (1,)


@pytest.mark.parametrize("shape", [(17, 17), (33, 21), (9, 9, 9), (12, 7, 10)])
def test_fsm_equals_dijkstra(shape):
    """Sec. 1.1: the scheme is causal, so the FSM fixed point is the Dijkstra
    (fast marching) solution of the same discrete equations -- bitwise."""
    rng = np.random.default_rng(sum(shape))
    r = rng.uniform(0.5, 2.0, shape)
    gamma = (rng.uniform(size=shape) < 0.02).astype(np.uint8)
    gamma.flat[len(gamma.flat) // 3] = 1
    g = rng.uniform(0.0, 0.1, shape)
    u, sweeps, conv = O.fsm(r, gamma, g, 0.1)
    v = O.fmm(r, gamma, g, 0.1)
    assert conv
    assert np.array_equal(u, v)


def test_fsm_linear_data_exact():
    """r = 1, Gamma = {x = 0}, g = 0: u = x exactly (|a-b| = h is not < h, so
    every update is the one-term branch); h a power of two keeps it exact."""
    n = 65
    h = 1.0 / 64
    gamma = np.zeros((n, n), np.uint8)
    gamma[:, 0] = 1
    u, s, c = O.fsm(np.ones((n, n)), gamma, 0.0, h)
    x = np.arange(n) * h
    assert np.array_equal(u, np.broadcast_to(x[None, :], (n, n)))
    # 2^d sweeps suffice when characteristics do not turn (Sec. 1.1): one
    # ordering sweeps it, the next confirms nothing changes.
    assert c and s <= 4
    # constant r on a 3-D box with g = r * z on the face z = 0 ... linear in z
    gamma3 = np.zeros((9, 9, 9), np.uint8)
    gamma3[0] = 1
    u3, _, _ = O.fsm(np.full((9, 9, 9), 2.0), gamma3, 0.0, 0.25)
    z = np.arange(9) * 0.25 * 2.0
    assert np.array_equal(u3, np.broadcast_to(z[:, None, None], u3.shape))


def test_fsm_point_source_first_order():
    """r = 1, point source: u -> |x - x0| with observed order close to one
    (first-order scheme, log factor at the source)."""
    errs = []
    for n in (65, 129, 257, 513):
        h = 1.0 / (n - 1)
        m = n // 2
        gamma = np.zeros((n, n), np.uint8)
        gamma[m, m] = 1
        u, _, _ = O.fsm(np.ones((n, n)), gamma, 0.0, h)
        x = np.arange(n) * h
        ex = np.sqrt((x[None, :] - 0.5) ** 2 + (x[:, None] - 0.5) ** 2)
        assert np.all(u >= ex - 1e-12)  # the Godunov scheme overestimates distance
        errs.append(np.max(np.abs(u - ex)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(orders) > 0.7 and max(orders) < 1.1, orders


def test_fsm_invariants():
    """Monotone decrease across sweeps, u >= min g, comparison principle, and
    the discrete equation holds at every non-Gamma node of the fixed point."""
    rng = np.random.default_rng(7)
    shape = (25, 31)
    r1 = rng.uniform(0.5, 1.5, shape)
    r2 = r1 + rng.uniform(0.0, 0.5, shape)
    gamma = np.zeros(shape, np.uint8)
    gamma[3, 4] = gamma[20, 27] = 1
    g = np.full(shape, 0.2)
    prev = np.full(shape, INF)
    for k in range(1, 12):
        u, _, _ = O.fsm(r1, gamma, g, 0.05, max_sweeps=k)
        assert np.all(u <= prev)
        prev = u
    u1, _, _ = O.fsm(r1, gamma, g, 0.05)
    u2, _, _ = O.fsm(r2, gamma, g, 0.05)
    assert np.all(u1 >= 0.2) and np.all(u1 <= u2)
    # residual: the local solve at the final neighbours reproduces u bitwise
    ny, nx = shape
    for j in range(ny):
        for i in range(nx):
            if gamma[j, i]:
                continue
            vm = [u1[j, i - 1] if i > 0 else INF, u1[j - 1, i] if j > 0 else INF]
            vp = [u1[j, i + 1] if i < nx - 1 else INF, u1[j + 1, i] if j < ny - 1 else INF]
            ut, _ = O.local_solve(vm, vp, r1[j, i] * 0.05)
            assert ut == u1[j, i]


def _model_problem(N, M):
    """Sec. 4 model problem: strip [0,1] x [0,H], r = 1, Gamma = bottom and left
    edges with g = sqrt(x^2 + y^2); subdomains of width H = 1/N, M cells each."""
    h = 1.0 / (N * M)
    nx, ny = N * M + 1, M + 1
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    r = np.ones((ny, nx))
    gamma = np.zeros((ny, nx), np.uint8)
    gamma[0, :] = 1
    gamma[:, 0] = 1
    g = np.sqrt(x[None, :] ** 2 + y[:, None] ** 2)
    return r, gamma, g, h


@pytest.mark.parametrize("theta", [0.1, 0.5, 1.0])
def test_dd_theorem1_exactness(theta):
    """Theorem 1 (Sec. 4.1): on the model problem U^k_{i,j} = u^f_{i,j} for
    k >= i, for any theta -- bitwise, since both sides reach the same FP fixed
    point of the same local solves."""
    N, M = 8, 8
    r, gamma, g, h = _model_problem(N, M)
    uf, _, _ = O.fsm(r, gamma, g, h)
    for k in range(N + 1):
        u, st, log, U = O.dd(r, gamma, g, h, (N, 1), M, theta=theta, max_iter=k, tol=-1.0,
                             return_coarse=True)
        for i in range(N + 1):
            col = i * M
            same = np.array_equal(U[1:, col], uf[1:, col])
            if i <= k:
                assert same, (theta, k, i)
        if k == N:
            assert np.array_equal(u, uf)


def test_dd_theta1_unstable_on_model_problem():
    """Sec. 4: theta = 1 (plain parareal) has large, non-monotone errors on the
    model problem before exactness catches up; a small theta decreases steadily."""
    N, M = 10, 10
    r, gamma, g, h = _model_problem(N, M)
    uf, _, _ = O.fsm(r, gamma, g, h)
    e1, e01 = [], []
    for k in range(N):
        _, _, _, U1 = O.dd(r, gamma, g, h, (N, 1), M, theta=1.0, max_iter=k, tol=-1, return_coarse=True)
        _, _, _, U2 = O.dd(r, gamma, g, h, (N, 1), M, theta=0.1, max_iter=k, tol=-1, return_coarse=True)
        e1.append(np.max(np.abs(U1[:, ::M] - uf[:, ::M])))
        e01.append(np.max(np.abs(U2[:, ::M] - uf[:, ::M])))
    assert max(e1) > 2 * e1[0]          # theta = 1 error grows
    assert all(e01[i + 1] <= e01[i] * 1.0001 for i in range(len(e01) - 1))


def test_dd_single_subdomain_is_fsm():
    """One subdomain: every subdomain face is the domain boundary (never inflow),
    so Step 3 is the plain FSM on the whole grid and DD returns u^f bitwise."""
    rng = np.random.default_rng(3)
    n = 33
    r = rng.uniform(0.5, 2.0, (n, n))
    gamma = np.zeros((n, n), np.uint8)
    gamma[5, 9] = 1
    uf, _, _ = O.fsm(r, gamma, 0.0, 1 / 32)
    u, st, _ = O.dd(r, gamma, 0.0, 1 / 32, (1, 1), 8, theta=0.5, max_iter=2, tol=-1)
    assert np.array_equal(u, uf)


def test_dd_fixed_point_is_fine_solution():
    """A converged DD iterate reproduces the global fine FSM solution u^f
    (Sec. 5 reports errors against u^f): smooth r, point source, theta 0.2."""
    n = 129
    h = 1.0 / 128
    x = np.arange(n) * h
    r = 1.0 + 0.5 * np.sin(2 * np.pi * x[None, :] * 4) * np.sin(2 * np.pi * x[:, None] * 4)
    gamma = np.zeros((n, n), np.uint8)
    gamma[64, 64] = 1
    uf, _, _ = O.fsm(r, gamma, 0.0, h)
    u, st, log = O.dd(r, gamma, 0.0, h, (4, 4), 8, theta=0.2, max_iter=40, tol=1e-12, max_coarse_sweeps=8)
    assert st["converged"] == 1
    assert np.max(np.abs(u - uf)) < 1e-7


def test_speedup_bound_closed_form():
    """Sec. 4.3: the example N=20, M=100, d=2, 10 sweeps gives k << 266."""
    line = [l for l in open(os.path.join(GOLD, "paper_numbers.txt")) if l.startswith("speedup_bound")][0]
    kv = dict(t.split("=") for t in line.split()[1:])
    N, M, d, C = (int(kv[k]) for k in ("N", "M", "d", "C"))

    def A(n, dd):
        return C * 2 ** dd * (n + 1) ** dd

    bound = A(N * M, d) / (A(N, d) + A(M, d) + 2 ** d * M * (N + 1) ** 2)
    assert int(bound) == int(kv["value"])


def test_adjoint_matches_finite_differences():
    """dJ/dr of the converged discrete system against central differences of the
    FSM solution (J = 0.5 sum over receivers of (u - d)^2)."""
    rng = np.random.default_rng(11)
    n = 21
    h = 1.0 / 20
    r = 1.0 + 0.3 * rng.uniform(size=(n, n))
    gamma = np.zeros((n, n), np.uint8)
    gamma[10, 0] = 1
    rec = [(j, n - 1) for j in range(2, n - 2, 3)]
    d = rng.uniform(0.8, 1.2, len(rec))

    def J(rr):
        u, _, _ = O.fsm(rr, gamma, 0.0, h)
        return 0.5 * sum((u[p] - dd) ** 2 for p, dd in zip(rec, d)), u

    J0, u0 = J(r)
    dJdu = np.zeros_like(r)
    for p, dd in zip(rec, d):
        dJdu[p] = u0[p] - dd
    grad = O.adjoint(r, gamma, u0, dJdu, h)
    cells = [(j, i) for j in range(3, n - 3, 4) for i in range(3, n - 3, 4)]
    for c in cells:
        e = 1e-6
        rp = r.copy(); rp[c] += e
        rm = r.copy(); rm[c] -= e
        fd = (J(rp)[0] - J(rm)[0]) / (2 * e)
        assert grad[c] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_dd3_single_subdomain_is_fsm_and_converges():
    """3-D: one subdomain reproduces the plain FSM bitwise; with 4^3
    subdomains and theta = 0.2 the iteration settles on the fine solution."""
    n = 17
    h = 1.0 / 16
    x = np.arange(n) * h
    r = 1.0 + 0.3 * np.sin(2 * np.pi * x)[None, None, :] * np.cos(2 * np.pi * x)[:, None, None]
    r = np.ascontiguousarray(np.broadcast_to(r, (n, n, n)))
    gamma = np.zeros((n, n, n), np.uint8)
    gamma[8, 5, 8] = 1
    uf, _, _ = O.fsm(r, gamma, 0.0, h)
    u1, _, _ = O.dd(r, gamma, 0.0, h, (1, 1, 1), 4, theta=0.5, max_iter=1, tol=-1)
    assert np.array_equal(u1, uf)
    u, st, _ = O.dd(r, gamma, 0.0, h, (4, 4, 4), 4, theta=0.2, max_iter=40, tol=1e-12, max_coarse_sweeps=16)
    assert st["converged"] == 1
    assert np.max(np.abs(u - uf)) < 1e-10 * np.max(uf)


# --------------------------------------------------------------------------
# Per-node weight of Sec. 4.2 (eq. secthetaest damped by eq. thetaest)
# --------------------------------------------------------------------------
def test_theta_estimate_shape():
    """Properties the damping fixes whatever the rounding: at the midpoint
    t = x0 the sigmoid is exactly 1/2; the damped value lies between delta*t
    and t and tends to delta*t; negative estimates give 0; undefined ones the
    fallback; the weighted mean of the coarse-solver changes; the cap."""
    x0, dl = 0.9, 0.01
    # t = du / mean(dC) = x0 exactly
    v = O.theta_estimate(x0 * 0.5, [0.5], sig_x0=x0, sig_delta=dl)
    assert abs(v - 0.5 * (x0 + dl * x0)) <= 1e-15
    for t in (0.05, 0.3, 2.0, 7.5):
        v = O.theta_estimate(t, [1.0])
        assert dl * t < v < t
    assert abs(O.theta_estimate(400.0, [1.0]) / 400.0 - dl) < 1e-12
    assert O.theta_estimate(-0.3, [1.0]) == 0.0
    assert O.theta_estimate(0.3, [0.0], fallback=0.17) == 0.17
    assert O.theta_estimate(0.3, [], fallback=0.17) == 0.17
    assert O.theta_estimate(np.inf, [1.0], fallback=0.17) == 0.17
    # mean over the three terms; weights select terms
    assert O.theta_estimate(0.3, [0.5, 1.0, 1.5]) == O.theta_estimate(0.3, [1.0])
    assert O.theta_estimate(0.3, [1.0, 7.0, -3.0], omega=(1.0, 0.0, 0.0)) == O.theta_estimate(0.3, [1.0])
    assert O.theta_estimate(400.0, [1.0], theta_cap=1.0) == 1.0


def test_dd_adaptive_theta_first_update_and_theorem1():
    """The first weighted update has no history and uses the constant theta,
    so one iteration equals the constant-theta run bitwise; Theorem 1's
    exactness (U^k = u^f on columns i <= k) holds for any weights, adaptive
    ones included."""
    n = 65
    h = 1.0 / (n - 1)
    xs = np.arange(n) * h
    r = 1.0 + 0.5 * np.sin(8 * np.pi * xs)[None, :] * np.sin(8 * np.pi * xs)[:, None]
    gamma = np.zeros((n, n), np.uint8)
    gamma[20, 40] = 1
    g = np.zeros((n, n))
    a, _, _ = O.dd(r, gamma, g, h, (4, 4), 8, theta=0.2, max_iter=1, max_coarse_sweeps=8)
    b, _, _ = O.dd(r, gamma, g, h, (4, 4), 8, theta=0.2, max_iter=1, max_coarse_sweeps=8, theta_adaptive=True,
                   theta_cap=1.0)
    np.testing.assert_array_equal(a, b)
    N, M = 8, 8
    r, gamma, g, h = _model_problem(N, M)
    uf, _, _ = O.fsm(r, gamma, g, h)
    for k in (2, 5, N):
        _, _, _, U = O.dd(r, gamma, g, h, (N, 1), M, theta=0.5, max_iter=k, tol=-1.0, return_coarse=True,
                          theta_adaptive=True, theta_cap=1.0)
        for i in range(k + 1):
            assert np.array_equal(U[1:, i * M], uf[1:, i * M]), (k, i)


def _mp_mid(k1, i, j, mb, Mb):
    """A weight inside Theorem 2's interval (max(mbar, 0), Mbar)."""
    if not np.isfinite(Mb):
        return 0.0
    return 0.5 * (max(mb, 0.0) + Mb)


def test_model_problem_theorem1():
    """Theorem 1 (Sec. 4.1) on the model problem's own iteration, eq.
    modelprob: U^k = u^f on every column i <= k, bitwise, whatever the
    weights (constant 0.2, 1, or chosen per node)."""
    N, M = 10, 8
    for th in (0.2, 1.0, _mp_mid):
        R = O.model_problem(N, M, th, N)
        for k in range(N + 1):
            assert np.array_equal(R["U"][k][:, :k + 1], R["uf"][:, :k + 1]), (th, k)
        assert not np.array_equal(R["U"][1][:, 2:], R["uf"][:, 2:])


def test_model_problem_theorem2():
    """Theorem 2 (Sec. 4.1) at the paper's sizes H = 1/20, h = 1/1000: with
    every weight inside (max(mbar, 0), Mbar) the iterates decrease strictly
    and stay strictly above u^f on the columns i > k; the interval is never
    empty there and Mbar > 0.  Taking the weight Mbar itself puts the node on
    u^f, and a weight above it below u^f (the bound is sharp)."""
    N, M = 20, 50
    R = O.model_problem(N, M, _mp_mid, 5)
    uf = R["uf"]
    for k in range(1, 6):
        U, Up = R["U"][k], R["U"][k - 1]
        mb, Mb = R["mbar"][k - 1][1:, k + 1:], R["Mbar"][k - 1][1:, k + 1:]
        assert np.all(Mb > 0) and np.all(Mb > np.maximum(mb, 0.0)), k
        assert np.all(U[1:, k + 1:] < Up[1:, k + 1:]), k
        assert np.all(U[1:, k + 1:] > uf[1:, k + 1:]), k
    col = 2   # the first column whose coarse-solver change does not depend on upstream weights

    def at_bound(scale):
        def f(k1, i, j, mb, Mb):
            return scale * Mb if i == col else _mp_mid(k1, i, j, mb, Mb)
        return f

    U1 = O.model_problem(N, M, at_bound(1.0), 1)["U"][1]
    np.testing.assert_allclose(U1[1:, col], uf[1:, col], rtol=1e-14, atol=0)
    U1 = O.model_problem(N, M, at_bound(1.05), 1)["U"][1]
    assert np.all(U1[1:, col] < uf[1:, col])


def test_model_problem_theta_one_peaks():
    """Sec. 4 (figure for theta = 1, H = 1/20, h = 1/1000): with theta = 1 the
    error max|U^k - u^f| grows from the first iteration and peaks around
    k = 10 before Theorem 1 brings it to zero at k = N; a small weight
    (0.1) decreases it at every iteration."""
    N, M = 20, 50
    R = O.model_problem(N, M, 1.0, N)
    e = [np.abs(U - R["uf"]).max() for U in R["U"]]
    peak = int(np.argmax(e))
    assert 8 <= peak <= 12, peak
    assert all(e[k + 1] > e[k] for k in range(peak)), e
    assert e[1] > 10 * e[0] and e[N] == 0.0
    R = O.model_problem(N, M, 0.1, N)
    e = [np.abs(U - R["uf"]).max() for U in R["U"]]
    assert all(e[k + 1] <= e[k] for k in range(N)), e


@pytest.mark.parametrize("name,kw", [
    ("fast_strip", dict(n=101)),
    ("maze", dict(n=201)),
    ("checkerboard", dict(n=141, tiles=7)),
])
def test_dd_reaches_fine_solution_on_obstacles(name, kw):
    """Sec. 4, mazes and obstacles / random checkerboard: the iteration reaches
    the overall fine solution u^f on a fast obstacle (r = 0.01 on
    [0.26, 0.27] x [0, 0.6]), slow barriers (r = 1000) and a random 1/2
    checkerboard.  Within 30 iterations the relative max error falls below
    1e-9.  This fails if an inflow boundary value of a subdomain cannot be
    lowered by the subdomain's own solve (Step 3 sweeps every boundary node):
    the iteration then stalls at errors of 1e-3 to 0.3."""
    w = getattr(I, "workload_" + name)(**kw)
    uf, _, _ = O.fsm(w["r"], w["gamma"], w["g"], w["h"])
    u, st, _ = O.dd(w["r"], w["gamma"], w["g"], w["h"], w["tiles"], w["c"], theta=0.2, max_iter=30, tol=0.0)
    assert np.abs(u - uf).max() / np.abs(uf).max() < 1e-9


def test_parallel_oracle_build_equals_serial():
    """The OpenMP build of the oracle (the all-cores CPU baseline) runs the
    independent subdomain and shifted-grid solves in parallel and returns the
    serial build's results bitwise, statistics included."""
    n = 129
    h = 1.0 / (n - 1)
    r = I.sin_product((n, n), h, 0.5, 1.0 / 8)
    gamma, g = I.point_source((n, n), (40, 90))
    kw = dict(theta=0.3, max_iter=5, tol=0.0, max_coarse_sweeps=8)
    u0, s0, l0 = O.dd(r, gamma, g, h, (4, 4), 8, **kw)
    u1, s1, l1 = O.dd(r, gamma, g, h, (4, 4), 8, parallel=True, **kw)
    assert np.array_equal(u0, u1) and s0 == s1 and np.array_equal(l0, l1, equal_nan=True)


def test_dd_margins_hooks_leave_the_method_unchanged():
    """The test hooks of orc_dd_margins: without replacement the solution is
    orc_dd's bitwise, replacing U^0 / W^0 by the solve's own changes nothing,
    every coarse-set value of the first pass is one of the exported copies,
    and a copy exists only on the coarse set; the Step 1 margins are defined
    exactly on the coarse set and are never negative."""
    n, h = 97, 1.0 / 96
    r = I.sin_product((n, n), h, 0.5, 0.25)
    gam, g = I.point_source((n, n), (32, 64))  # a coarse node: every shifted grid sees it
    kw = dict(theta=0.0, max_coarse_sweeps=8)
    u, st, W0, mg, cp, cm = O.dd_margins(r, gam, g, h, (3, 3), 8, max_iter=0, **kw)
    u_ref, st_ref, _, U_ref = O.dd(r, gam, g, h, (3, 3), 8, max_iter=0, return_coarse=True, **kw)
    assert np.array_equal(u, u_ref) and st["fine_updates"] == st_ref["fine_updates"]
    cs = np.zeros((n, n), bool)
    cs[::8, :] = True
    cs[:, ::8] = True
    U0 = np.where(cs, U_ref, np.nan)  # max_iter = 0: the coarse state after Step 1
    u2, _, W0b, _, _, _ = O.dd_margins(r, gam, g, h, (3, 3), 8, max_iter=0, U0=U0, W0=W0, **kw)
    assert np.array_equal(u2, u) and np.array_equal(W0b, W0)
    assert np.all(np.any(cp[:, cs] == u[cs], axis=0))
    assert not np.any(np.isfinite(cp[:, ~cs]))
    assert np.all(np.isnan(mg[~cs])) and not np.any(np.isnan(mg[cs])) and np.all(mg[cs] >= 0)
    # a different W^0 changes the first pass (the hook is applied)
    W0x = -W0
    u3, _, _, _, _, _ = O.dd_margins(r, gam, g, h, (3, 3), 8, max_iter=0, U0=U0, W0=W0x, **kw)
    assert not np.array_equal(u3, u)
