"""The one-dimensional method of Sec. 3.1 (eik_dd_solve on a 1-D grid) against
the oracle's orc_dd1: FP64 bitwise in u and in every statistic the oracle
keeps, FP32 within the rounding bound of a sum along the path.

Cases: the Gaussian-bump example of Sec. 3.1 (N = 10), one-way flow from
x = 0, sources inside subintervals and on coarse nodes, a single subinterval,
one cell per subinterval, 2048 subintervals (more than one per thread), long
subintervals, max_iter = 0, weight 0, a tol stop, sweep caps that bind, and
no source at all."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1805_04198_gb300 import eik

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
STAT_KEYS = ("iters", "converged", "fsm_sweeps_max", "coarse_sweeps_max", "fsm_cap_hits", "coarse_cap_hits",
             "causal_rounds_max", "fine_updates")


def _bump(N, M):
    h = 1.0 / (N * M)
    x = np.arange(N * M + 1) * h
    r = 1.0 + 10.0 * np.exp(-(x - 0.75) ** 2 / (2 * 0.01 ** 2))
    gam = np.zeros(N * M + 1, np.uint8)
    gam[0] = gam[-1] = 1
    return r, gam, np.zeros(N * M + 1), h


def _random(N, M, seed, src):
    h = 1.0 / (N * M)
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.5, 2.0, N * M + 1)
    gam = np.zeros(N * M + 1, np.uint8)
    g = np.zeros(N * M + 1)
    for j in src:
        gam[j] = 1
        g[j] = rng.uniform(0.0, 0.1)
    return r, gam, g, h


CASES = {
    "bump_M100_theta0.1": (lambda: _bump(10, 100), 10, 100, dict(theta=0.1, max_iter=6)),
    "bump_M100_theta1": (lambda: _bump(10, 100), 10, 100, dict(theta=1.0, max_iter=6)),
    "bump_M20_theta0.5_k3": (lambda: _bump(10, 20), 10, 20, dict(theta=0.5, max_iter=3)),
    "one_way": (lambda: _random(8, 16, 1, [0]), 8, 16, dict(theta=0.2, max_iter=10)),
    "inner_sources_no_convergence": (lambda: _random(37, 27, 2, [5, 27 * 11, 27 * 20 + 13, 998]), 37, 27,
                          dict(theta=0.6, max_iter=60, tol=1e-12)),
    "single_subinterval": (lambda: _random(1, 500, 3, [250]), 1, 500, dict(theta=1.0, max_iter=3)),
    "one_cell_per_subinterval": (lambda: _random(300, 1, 4, [0, 150, 299]), 300, 1, dict(theta=0.5, max_iter=40)),
    "2048_subintervals": (lambda: _random(2048, 3, 5, [7, 3000, 6143]), 2048, 3, dict(theta=0.7, max_iter=12)),
    "long_subintervals": (lambda: _random(3, 100000, 6, [123457]), 3, 100000, dict(theta=1.0, max_iter=5)),
    "max_iter_0": (lambda: _random(16, 8, 7, [64]), 16, 8, dict(theta=1.0, max_iter=0)),
    "theta_0": (lambda: _random(20, 10, 8, [3, 199]), 20, 10, dict(theta=0.0, max_iter=25, tol=1e-14)),
    "caps_bind": (lambda: _random(12, 9, 9, [50]), 12, 9, dict(theta=0.9, max_iter=8, max_fsm_sweeps=1,
                                                              max_coarse_sweeps=1)),
    "no_source": (lambda: _random(6, 5, 10, []), 6, 5, dict(theta=0.5, max_iter=2)),
}


def _gpu(r, gam, g, h, N, M, dtype, **kw):
    R = torch.from_numpy(r).to(DEV, dtype)
    G = torch.from_numpy(gam).to(DEV)
    Gv = torch.from_numpy(g).to(DEV, dtype)
    return eik.dd_solve(R, G, Gv, h, (N,), M, **kw)


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_bitwise_against_oracle(name):
    make, N, M, kw = CASES[name]
    r, gam, g, h = make()
    kw = dict(kw)
    kw.setdefault("max_coarse_sweeps", 1000)
    u_o, st_o, _ = O.dd1(r, gam, g, h, N, M, **kw)
    u, st = _gpu(r, gam, g, h, N, M, torch.float64, **kw)
    np.testing.assert_array_equal(u.cpu().numpy(), u_o)
    for k in STAT_KEYS:
        assert st[k] == st_o[k], (k, st[k], st_o[k])
    if st_o["iters"] >= 1:
        assert st["last_delta"] == st_o["last_delta"]
    assert st["launches"] == 1 and st["error"] == 0


@pytest.mark.parametrize("name", ["bump_M100_theta1", "inner_sources_no_convergence", "2048_subintervals", "long_subintervals"])
def test_fp32_within_path_rounding(name):
    """FP32 against the oracle fed the FP32-rounded r: every node value is a
    sum of at most n terms r h along its path, so the error is within
    n * 2^-23 * max|u| (plus the same for the rounded g)."""
    make, N, M, kw = CASES[name]
    r, gam, g, h = make()
    r32 = r.astype(np.float32).astype(np.float64)
    g32 = g.astype(np.float32).astype(np.float64)
    kw = dict(kw)
    kw.setdefault("max_coarse_sweeps", 1000)
    u_o, st_o, _ = O.dd1(r32, gam, g32, h, N, M, **kw)
    u, st = _gpu(r32, gam, g32, h, N, M, torch.float32, **kw)
    u = u.cpu().numpy().astype(np.float64)
    fin = np.isfinite(u_o)
    assert np.array_equal(fin, np.isfinite(u))
    bound = (N * M + 1) * 2.0 ** -23 * np.max(np.abs(u_o[fin])) + 1e-7
    assert np.max(np.abs(u[fin] - u_o[fin])) <= bound
    assert st["iters"] == st_o["iters"]


def test_bump_example_converges_at_k3():
    """Sec. 3.1's example: the solve stopped at k = 3 is the fine solution."""
    r, gam, g, h = _bump(10, 100)
    uf, _, _ = O.fsm(r, gam, 0.0, h)
    u, st = _gpu(r, gam, g, h, 10, 100, torch.float64, theta=0.5, max_iter=3, max_coarse_sweeps=1000)
    assert st["iters"] == 3
    np.testing.assert_allclose(u.cpu().numpy(), uf, rtol=0, atol=1e-14)


def test_noalloc_entry_point_equals_dd_solve():
    r, gam, g, h = _random(37, 27, 2, [5, 27 * 11, 998])
    kw = dict(theta=0.6, max_iter=30, tol=1e-12, max_coarse_sweeps=1000)
    R = torch.from_numpy(r).to(DEV)
    G = torch.from_numpy(gam).to(DEV)
    Gv = torch.from_numpy(g).to(DEV)
    u, st = eik.dd_solve(R, G, Gv, h, (37,), 27, **kw)
    u2 = torch.empty_like(R)
    sd = torch.zeros(eik.ctypes.sizeof(eik.DDStats), dtype=torch.uint8, device=DEV)
    eik.eik_dd_solve_noalloc(eik.make_grid(R, h), R, G, Gv, eik.dd_params((37,), 27, **kw), u2, sd)
    torch.cuda.synchronize()
    assert torch.equal(u, u2) and eik.parse_dd_stats(sd) == st


def test_expired_barrier_reports_timeout_then_solves_exactly():
    """The grid barriers between the fine and coarse phases are bounded waits:
    with a one-poll limit some expires, the call ends with
    EIK_EDEVICE_TIMEOUT in its statistics, and with the default limit back
    the same context gives the oracle's result bitwise."""
    make, N, M, kw = CASES["2048_subintervals"]
    r, gam, g, h = make()
    kw = dict(kw, max_coarse_sweeps=1000)
    eik.eik_set_wait_limit(1)
    try:
        R = torch.from_numpy(r).to(DEV)
        u, sd = eik.dd_solve(R, torch.from_numpy(gam).to(DEV), torch.from_numpy(g).to(DEV), h, (N,), M,
                             sync=False, **kw)
        torch.cuda.synchronize()
        assert eik.parse_dd_stats(sd)["error"] == -4
    finally:
        eik.eik_set_wait_limit(0)
    u_o, st_o, _ = O.dd1(r, gam, g, h, N, M, **kw)
    u, st = _gpu(r, gam, g, h, N, M, torch.float64, **kw)
    assert st["error"] == 0
    np.testing.assert_array_equal(u.cpu().numpy(), u_o)
