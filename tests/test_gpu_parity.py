"""GPU path (through the C ABI) against the FP64 CPU oracle.

FP64 builds perform the same IEEE operations as the oracle, so their results
are compared bitwise.  FP32 builds are compared with the oracle run on the same
FP32-rounded inputs: relative max-norm error <= 1e-5 (the tolerance of the
method's FP32 storage).  Winds are compared through their effect: the DD
iterates, which depend on every Alg. 4 / Alg. 5 decision.
"""
import functools

import numpy as np
import pytest
import torch

import oracle as O
from paper_1805_04198_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL32 = 1e-5


def _t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def _rel(a, b):
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    return np.max(np.abs(a[fin] - b[fin])) / np.max(np.abs(b[fin]))


def _random_problem(shape, seed, nsrc=3):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.5, 2.0, shape)
    gamma = np.zeros(shape, np.uint8)
    for _ in range(nsrc):
        gamma[tuple(rng.integers(0, s) for s in shape)] = 1
    g = rng.uniform(0.0, 0.1, shape)
    return r, gamma, g


@pytest.mark.parametrize("shape", [(33, 33), (70, 100), (5, 200), (129, 40), (1, 1)])
def test_fsm_fp64_bitwise(gpu, shape):
    if shape == (1, 1):
        pytest.skip("degenerate 1x1 grid is rejected by validation (n >= 2)")
    r, gamma, g = _random_problem(shape, sum(shape))
    u_ref, s_ref, _ = O.fsm(r, gamma, g, 0.05)
    u, st = gpu.fsm(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), 0.05)
    assert st["converged"] == 1
    np.testing.assert_array_equal(u.cpu().numpy(), u_ref)


def test_fsm_sweep_cap_matches_oracle(gpu):
    """Stopped early by max_sweeps: the same sweeps in the same order."""
    r, gamma, g = _random_problem((60, 90), 5, nsrc=1)
    for k in (1, 2, 3, 5):
        u_ref, s_ref, c_ref = O.fsm(r, gamma, g, 0.05, max_sweeps=k)
        u, st = gpu.fsm(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), 0.05, max_sweeps=k)
        assert st["sweeps"] == s_ref
        np.testing.assert_array_equal(u.cpu().numpy(), u_ref)


def test_fsm_fp32(gpu):
    shape = (97, 257)
    r, gamma, g = _random_problem(shape, 9)
    r32 = r.astype(np.float32)
    g32 = g.astype(np.float32)
    u_ref, _, _ = O.fsm(r32.astype(np.float64), gamma, g32.astype(np.float64), 1.0 / 256)
    u, st = gpu.fsm(_t(r32, torch.float32), _t(gamma, torch.uint8), _t(g32, torch.float32), 1.0 / 256)
    assert _rel(u.cpu().numpy().astype(np.float64), u_ref) <= TOL32


def _dd_case(n, tiles, c, amp=0.5, eps=0.25, src=None):
    h = 1.0 / (n - 1)
    r = I.sin_product((n, n), h, amp, eps)
    gamma, g = I.point_source((n, n), src if src is not None else (n // 2, n // 2))
    return r, gamma, g, h


@pytest.mark.parametrize("n,tiles,c,theta,kmax", [
    (65, (4, 4), 8, 0.2, 6),
    (65, (4, 4), 16, 0.5, 4),     # c equal to the subdomain width (the paper's setting)
    (65, (2, 4), 8, 1.0, 3),      # theta = 1, anisotropic tiling
    (97, (3, 3), 16, 0.2, 5),     # 33-node subdomains: two blocks, ragged tail
    (129, (2, 2), 8, 0.3, 4),     # 65-node subdomains, c < S
    (73, (3, 3), 6, 0.2, 3),      # coarse ratio not a power of two
    (65, (4, 4), 8, 0.0, 6),      # weight 0: Alg. 4 hands u^k to the causal sweep, no Step 4 sweeps
    (97, (3, 3), 16, 0.0, 5),
])
def test_dd_fp64_bitwise(gpu, n, tiles, c, theta, kmax):
    r, gamma, g, h = _dd_case(n, tiles, c)
    for k in range(kmax + 1):
        u_ref, s_ref, _ = O.dd(r, gamma, g, h, tiles, c, theta=theta, max_iter=k, tol=0.0, max_coarse_sweeps=8)
        u, st = gpu.dd_solve(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), h, tiles, c,
                             theta=theta, max_iter=k, tol=0.0, max_coarse_sweeps=8)
        assert st["iters"] == s_ref["iters"] == k
        assert st["fsm_sweeps_max"] <= s_ref["fsm_sweeps_max"] + 4
        np.testing.assert_array_equal(u.cpu().numpy(), u_ref, err_msg="k=%d" % k)


@pytest.mark.parametrize("name,kw,ks", [
    ("fast_strip", dict(n=101), (0, 4, 12, 30)),
    ("maze", dict(n=201), (0, 4, 12, 30)),
    ("checkerboard", dict(n=141, tiles=7), (0, 4, 12, 30)),
    ("fast_strip", dict(n=501), (30,)),        # the paper's sizes, H = 1/10, h = 1/500
])
def test_dd_obstacles_fp64_bitwise(gpu, name, kw, ks):
    """Sec. 4 obstacle and random workloads (subdomain boundary values that
    the subdomain solve must lower): bitwise equal to the oracle, and at 30
    iterations within 1e-6 of the fine solution u^f (with the 8-sweep cap on
    Step 4 used here the oracle is 1.4e-9 away on the strips, 4e-13 on the
    maze and 7e-8 on the checkerboard)."""
    w = getattr(I, "workload_" + name)(**kw)
    args = (_t(w["r"], torch.float64), _t(w["gamma"], torch.uint8), _t(w["g"], torch.float64), w["h"],
            w["tiles"], w["c"])
    for k in ks:
        u_ref, s_ref, _ = O.dd(w["r"], w["gamma"], w["g"], w["h"], w["tiles"], w["c"], theta=0.2, max_iter=k,
                               tol=0.0, max_coarse_sweeps=8)
        u, st = gpu.dd_solve(*args, theta=0.2, max_iter=k, tol=0.0, max_coarse_sweeps=8)
        assert st["iters"] == s_ref["iters"] == k
        np.testing.assert_array_equal(u.cpu().numpy(), u_ref, err_msg="%s k=%d" % (name, k))
    uf, _, _ = O.fsm(w["r"], w["gamma"], w["g"], w["h"])
    assert _rel(u.cpu().numpy(), uf) < 1e-6


def test_dd_fp64_tol_stop_and_stats(gpu):
    r, gamma, g, h = _dd_case(65, (4, 4), 8, amp=0.3)
    u_ref, s_ref, log = O.dd(r, gamma, g, h, (4, 4), 8, theta=0.2, max_iter=40, tol=1e-9, max_coarse_sweeps=8)
    u, st = gpu.dd_solve(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), h, (4, 4), 8,
                         theta=0.2, max_iter=40, tol=1e-9, max_coarse_sweeps=8)
    assert st["converged"] == s_ref["converged"] == 1
    assert st["iters"] == s_ref["iters"]
    assert st["last_delta"] == s_ref["last_delta"]
    assert st["coarse_cap_hits"] == s_ref["coarse_cap_hits"]
    np.testing.assert_array_equal(u.cpu().numpy(), u_ref)


def test_dd_model_problem_theorem1(gpu):
    """Theorem 1 setting through the GPU path: bitwise equal to the oracle,
    which itself reproduces u^f on columns i <= k."""
    N, M = 8, 16
    h = 1.0 / (N * M)
    nx, ny = N * M + 1, M + 1
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    r = np.ones((ny, nx))
    gamma = np.zeros((ny, nx), np.uint8)
    gamma[0, :] = 1
    gamma[:, 0] = 1
    g = np.sqrt(x[None, :] ** 2 + y[:, None] ** 2)
    for k in (0, 3, 8):
        u_ref, _, _ = O.dd(r, gamma, g, h, (N, 1), M, theta=1.0, max_iter=k, tol=-1.0)
        u, _ = gpu.dd_solve(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), h, (N, 1), M,
                            theta=1.0, max_iter=k, tol=-1.0)
        np.testing.assert_array_equal(u.cpu().numpy(), u_ref)


def test_dd_c0_config_fp64(gpu):
    """257^2, eps = 1/16, point source at the centre, 4x4 subdomains, coarse
    ratio 8 (33^2 coarse grid), theta = 1, 10 iterations, FP64."""
    w = I.workload_c0()
    args = dict(theta=w["theta"], max_iter=w["max_iter"], tol=w["tol"], max_coarse_sweeps=8)
    u_ref, s_ref, _ = O.dd(w["r"], w["gamma"], w["g"], w["h"], w["tiles"], w["c"], **args)
    u, st = gpu.dd_solve(_t(w["r"], torch.float64), _t(w["gamma"], torch.uint8), _t(w["g"], torch.float64),
                         w["h"], w["tiles"], w["c"], **args)
    assert st["iters"] == s_ref["iters"]
    np.testing.assert_array_equal(u.cpu().numpy(), u_ref)


def test_dd_fp32_converged_against_oracle(gpu):
    """FP32 storage: the converged DD output agrees with the FP64 oracle on the
    same rounded inputs within 1e-5 relative max-norm."""
    r, gamma, g, h = _dd_case(129, (4, 4), 8, amp=0.5, eps=0.25)
    r32 = r.astype(np.float32)
    args = dict(theta=0.2, max_iter=40, tol=1e-7, max_coarse_sweeps=8)
    u_ref, s_ref, _ = O.dd(r32.astype(np.float64), gamma, g, h, (4, 4), 8, **args)
    u, st = gpu.dd_solve(_t(r32, torch.float32), _t(gamma, torch.uint8), _t(g, torch.float32), h, (4, 4), 8,
                         **args)
    assert s_ref["converged"] == 1
    assert _rel(u.cpu().numpy().astype(np.float64), u_ref) <= TOL32


@pytest.mark.parametrize("shape", [(300, 1100), (40, 2049)])
def test_fsm_multi_cta_fp64_bitwise(gpu, shape):
    """Grids wider than one CTA's 32 blocks run on many co-resident CTAs with
    global hand-offs: still the same sweeps, bitwise."""
    r, gamma, g = _random_problem(shape, shape[1])
    u_ref, s_ref, c_ref = O.fsm(r, gamma, g, 1.0 / 1024)
    u, st = gpu.fsm(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), 1.0 / 1024)
    assert st["converged"] == 1 and st["sweeps"] <= s_ref
    np.testing.assert_array_equal(u.cpu().numpy(), u_ref)


def test_fsm_full_size_fp32_against_oracle(gpu):
    """The full 4097^2 workload of the benchmark (Fourier-mode slowness, left
    edge source) through the plain FSM in FP32, against the FP64 oracle on the
    same rounded slowness, element by element."""
    w = I.workload_c1()
    r32 = w["r"].astype(np.float32)
    u_ref = _c1_oracle_fsm()
    u, st = gpu.fsm(_t(r32, torch.float32), _t(w["gamma"], torch.uint8), _t(w["g"], torch.float32), w["h"])
    assert st["converged"] == 1
    assert _rel(u.cpu().numpy().astype(np.float64), u_ref) <= TOL32


@pytest.mark.parametrize("n,tiles,c,kmax", [
    (65, (4, 4), 8, 6),
    (97, (3, 3), 16, 5),
    (129, (2, 2), 8, 4),
])
def test_dd_adaptive_theta_fp64_against_oracle(gpu, n, tiles, c, kmax):
    """Per-node weight of Sec. 4.2: the first weighted update uses the constant
    theta (bitwise); later ones use the estimate, which contains an exp whose
    last bit may differ between the device and the host library, hence the
    FP64 tolerance of 1e-11 relative."""
    r, gamma, g, h = _dd_case(n, tiles, c)
    kw = dict(theta=0.2, max_coarse_sweeps=8, theta_adaptive=True, theta_cap=1.0)
    for k in range(1, kmax + 1):
        u_ref, s_ref, _ = O.dd(r, gamma, g, h, tiles, c, max_iter=k, tol=0.0, **kw)
        u, st = gpu.dd_solve(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), h, tiles, c,
                             max_iter=k, tol=0.0, **kw)
        assert st["iters"] == s_ref["iters"] == k
        a = u.cpu().numpy()
        if k == 1:
            np.testing.assert_array_equal(a, u_ref)
        else:
            assert _rel(a, u_ref) <= 1e-11, k


def test_dd_adaptive_theta_validation(gpu):
    r = torch.ones((65, 65), dtype=torch.float64, device=DEV)
    G = torch.zeros((65, 65), dtype=torch.uint8, device=DEV)
    with pytest.raises(gpu.EikError):
        gpu.dd_solve(r, G, r, 1.0 / 64, (4, 4), 8, theta_adaptive=True, sig_gamma=0.0)
    r3 = torch.ones((17, 17, 17), device=DEV)
    G3 = torch.zeros((17, 17, 17), dtype=torch.uint8, device=DEV)
    with pytest.raises(gpu.EikError):
        gpu.dd_solve(r3, G3, r3, 1.0 / 16, (2, 2, 2), 4, theta_adaptive=True, omega=(0.0, 0.0, 0.0))


@pytest.mark.parametrize("n,tiles,c,kmax", [
    (17, (2, 2, 2), 4, 5),
    (25, (3, 2, 2), 4, 4),     # c < S on two axes
])
def test_dd3_adaptive_theta_fp64_against_oracle(gpu, n, tiles, c, kmax):
    """The per-node weight of Sec. 4.2 in the 3-D solve: bitwise at the
    first update, within 1e-11 (the estimate's exp) afterwards."""
    r, gamma, g, h = _dd3_case(n)
    kw = dict(theta=0.2, max_coarse_sweeps=8, theta_adaptive=True, theta_cap=1.0, omega=(1.0, 0.5, 0.25))
    for k in range(1, kmax + 1):
        u_ref, s_ref, _ = O.dd(r, gamma, g, h, tiles, c, max_iter=k, tol=0.0, **kw)
        u, st = gpu.dd_solve(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), h, tiles, c,
                             max_iter=k, tol=0.0, **kw)
        assert st["iters"] == s_ref["iters"] == k
        a = u.cpu().numpy()
        if k == 1:
            np.testing.assert_array_equal(a, u_ref)
        else:
            assert _rel(a, u_ref) <= 1e-11, k


# The DD workload of the benchmark: 4097^2, 16x16 subdomains, coarse ratio 16,
# theta 0, FP32, in the launch configuration bench.py times.
C1_DD = dict(theta=0.0, tol=1e-6, max_coarse_sweeps=8)   # the benchmark's solve


@functools.lru_cache(maxsize=1)
def _c1_oracle_fsm():
    w = I.workload_c1()
    r32 = w["r"].astype(np.float32)
    u_ref, s_ref, c_ref = O.fsm(r32.astype(np.float64), w["gamma"], w["g"], w["h"])
    assert c_ref
    return u_ref


def _godunov_2d(vmx, vpx, vmy, vpy, rh):
    """Godunov local solve (Sec. 1.1, eq. godonuv) written out in numpy, FP64."""
    a = np.minimum(vmx, vpx)
    b = np.minimum(vmy, vpy)
    with np.errstate(invalid="ignore"):
        d = a - b
        two = (a + b + np.sqrt(np.maximum(2.0 * rh * rh - d * d, 0.0))) / 2.0
        one = np.minimum(a, b) + rh
        return np.where(np.abs(d) < rh, two, one)


def test_dd_subdomain_shape_of_benchmark_fp64_bitwise(gpu):
    """The benchmark's subdomain shape (257x257) and coarse ratio (16) on a
    2049^2 grid of the same medium (8x8 subdomains; the 4097^2 grid's FP64
    coarse grids would not fit in shared memory), stopped after one pass
    (max_iter = 0) and after two iterations: FP64 bitwise equal to the oracle."""
    w = I.workload_c1(n=2049, tiles=8, c=16)
    for k in (0, 2):
        u_ref, s_ref, _ = O.dd(w["r"], w["gamma"], w["g"], w["h"], w["tiles"], w["c"], max_iter=k, **C1_DD)
        u, st = gpu.dd_solve(_t(w["r"], torch.float64), _t(w["gamma"], torch.uint8), _t(w["g"], torch.float64),
                             w["h"], w["tiles"], w["c"], max_iter=k, **C1_DD)
        assert st["iters"] == s_ref["iters"] == k and st["error"] == 0
        np.testing.assert_array_equal(u.cpu().numpy(), u_ref, err_msg="k=%d" % k)


def _wind_components(Wb):
    """Wind bytes of eik_dd_coarse_state -> components (ny, nx, 3), 0 where no
    coarse-set node (byte 255)."""
    comp = np.zeros(Wb.shape + (3,), np.int8)
    on = Wb != 255
    for a in range(2):
        comp[..., a] = np.where(on, ((Wb >> (2 * a)) & 3).astype(np.int8) - 1, 0)
    return comp


# Error bound of an FP32 coarse or copy value against FP64 (relative to max u):
# a path of at most 2 * 256 coarse (or 2 * 256 fine) local solves, each a few
# roundings of 2^-24.  A decision whose margin lies below twice this bound may
# be taken either way by the two precisions.
TIE32 = 2 * 512 * 3 * 2.0 ** -24


def test_dd_full_size_first_pass_fp32(gpu):
    """The first pass (Step 1, Steps 2-3, Alg. 4) of the 4097^2 benchmark solve
    in FP32 against the FP64 oracle on the rounded slowness, with an exact
    account of the decisions each side takes in its own precision (winds of
    Alg. 1 and Alg. 3, the Step 2 inflow test, Alg. 4's choice of copy):
    (a) every coarse node whose GPU wind W^0 differs from the oracle's own has
        an Alg. 1 decision margin below the FP32 error bound (a near tie);
    (b) the oracle then runs Steps 2-3 and Alg. 4 from the GPU's U^0 and W^0,
        i.e. with the same Step 2 decisions: every node off the coarse set
        agrees within 1e-5, and so does every coarse-set node except where
        Alg. 4 chose another copy; each of those holds one of the oracle's
        copies within 1e-5, its choice margin is below the FP32 error bound,
        and they are rare (at most 1e-4 of the nodes)."""
    w = I.workload_c1()
    r32 = w["r"].astype(np.float32)
    r64 = r32.astype(np.float64)
    dev_args = (_t(r32, torch.float32), _t(w["gamma"], torch.uint8), _t(w["g"], torch.float32), w["h"],
                w["tiles"], w["c"])
    u, st = gpu.dd_solve(*dev_args, max_iter=0, **C1_DD)
    Uc, Wc = gpu.dd_step1_state(*dev_args, max_iter=0, **C1_DD)
    a = u.cpu().numpy().astype(np.float64)
    U0 = Uc.cpu().numpy().astype(np.float64)
    W0 = _wind_components(Wc.cpu().numpy())
    args = (r64, w["gamma"], w["g"], w["h"], w["tiles"], w["c"])
    u_own, _, W0_own, margin, _, _ = O.dd_margins(*args, max_iter=0, parallel=True, **C1_DD)
    fin = np.isfinite(u_own)
    umax = np.max(u_own[fin])
    assert np.array_equal(np.isfinite(a), fin)
    cs = Wc.cpu().numpy() != 255
    # (a) Step 1 winds differ only at near ties
    flip = cs & np.any(W0 != W0_own, axis=-1)
    assert np.all(margin[flip] <= TIE32 * umax), (int(flip.sum()), float(np.max(margin[flip]) / umax))
    # (b) from the GPU's Step 1 on, the same decisions up to Alg. 4's near ties
    u_x, _, _, _, copies, cmargin = O.dd_margins(*args, max_iter=0, U0=U0, W0=W0, parallel=True, **C1_DD)
    err = np.abs(a - u_x) / umax
    off = err > TOL32
    assert not np.any(off & ~cs), (int((off & ~cs).sum()), float(err[~cs].max()))
    ys, xs = np.nonzero(off)
    other_copy = np.any(np.abs(copies[:, ys, xs] - a[ys, xs]) <= TOL32 * umax, axis=0)
    assert np.all(other_copy), int((~other_copy).sum())
    assert np.all(cmargin[ys, xs] <= TIE32 * umax), float(np.max(cmargin[ys, xs]) / umax)
    assert len(ys) <= 1e-4 * a.size, len(ys)


def test_dd_full_size_converged_solve(gpu):
    """4097^2 DD exactly as the benchmark runs it (theta = 0, stop at a coarse
    update below 1e-6, cap 42).  It converges, and then (a) at every node the
    output agrees with the FP64 oracle's full-grid fine solution u^f on the
    same rounded slowness within the FP32 tolerance 1e-5, and (b) every
    subdomain solve ends at its Gauss-Seidel fixed point: at each node strictly
    inside a subdomain (neighbours included, so that no neighbour took another
    subdomain's value in Alg. 4) u equals the Godunov local solve of its four
    neighbours, up to FP32 rounding."""
    w = I.workload_c1()
    r32 = w["r"].astype(np.float32)
    u, st = gpu.dd_solve(_t(r32, torch.float32), _t(w["gamma"], torch.uint8), _t(w["g"], torch.float32), w["h"],
                         w["tiles"], w["c"], max_iter=w["max_iter"], **C1_DD)
    assert st["converged"] == 1 and st["iters"] <= w["max_iter"]
    assert st["error"] == 0 and st["fsm_cap_hits"] == 0
    assert _rel(u.cpu().numpy().astype(np.float64), _c1_oracle_fsm()) <= TOL32
    U = u.cpu().numpy().astype(np.float64)
    n = U.shape[0]
    S = (n - 1) // w["tiles"][0]
    loc = np.arange(n) % S
    inner = (loc >= 2) & (loc <= S - 2)
    mask = inner[:, None] & inner[None, :] & (w["gamma"] == 0)
    rh = r32.astype(np.float64) * w["h"]
    inf = np.full((n, 1), np.inf)
    vmx = np.hstack([inf, U[:, :-1]])
    vpx = np.hstack([U[:, 1:], inf])
    vmy = np.vstack([inf.T, U[:-1, :]])
    vpy = np.vstack([U[1:, :], inf.T])
    ls = _godunov_2d(vmx, vpx, vmy, vpy, rh)
    m = mask & np.isfinite(U)
    assert m.sum() > 0.9 * mask.sum()
    rel = np.abs(U[m] - ls[m]) / np.abs(U[m])
    assert rel.max() <= TOL32


@pytest.mark.parametrize("shape", [(17, 20, 23), (33, 33, 33), (9, 40, 12)])
def test_fsm3_fp64_bitwise(gpu, shape):
    """3-D full-grid FSM (hyperplane sweeps over the whole grid): bitwise equal
    to the oracle's serial loop nest."""
    r, gamma, g = _random_problem(shape, sum(shape))
    u_ref, s_ref, c_ref = O.fsm(r, gamma, g, 0.05)
    u, st = gpu.fsm(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), 0.05)
    assert c_ref and st["converged"] == 1 and st["sweeps"] == s_ref
    np.testing.assert_array_equal(u.cpu().numpy(), u_ref)


def test_fsm3_sweep_cap_matches_oracle(gpu):
    r, gamma, g = _random_problem((21, 18, 25), 3, nsrc=1)
    for k in (1, 2, 5):
        u_ref, s_ref, _ = O.fsm(r, gamma, g, 0.05, max_sweeps=k)
        u, st = gpu.fsm(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), 0.05, max_sweeps=k)
        assert st["sweeps"] == s_ref == k
        np.testing.assert_array_equal(u.cpu().numpy(), u_ref)


def test_fsm3_fp32_against_oracle(gpu):
    n = 65
    h = 1.0 / (n - 1)
    r = I.sin_product((n, n, n), h, 0.4, 0.25).astype(np.float32)
    gamma, g = I.point_source((n, n, n), (n // 2, n // 3, n // 4))
    u_ref, _, _ = O.fsm(r.astype(np.float64), gamma, g, h)
    u, st = gpu.fsm(_t(r, torch.float32), _t(gamma, torch.uint8), _t(g, torch.float32), h)
    assert st["converged"] == 1
    assert _rel(u.cpu().numpy().astype(np.float64), u_ref) <= TOL32


def _dd3_case(n, amp=0.4, eps=0.25, src=None):
    h = 1.0 / (n - 1)
    r = I.sin_product((n, n, n), h, amp, eps)
    gamma, g = I.point_source((n, n, n), src if src is not None else (n // 2, n // 2, n // 2))
    return r, gamma, g, h


@pytest.mark.parametrize("n,tiles,c,theta,kmax", [
    (17, (2, 2, 2), 4, 0.5, 4),
    (17, (2, 2, 2), 8, 0.2, 3),    # c equal to the subdomain width
    (25, (3, 3, 3), 4, 0.5, 3),
    (17, (1, 2, 4), 2, 1.0, 2),    # anisotropic tiling, theta = 1
    (17, (2, 2, 2), 4, 0.0, 4),    # weight 0: Alg. 4 hands u^k to the causal sweep, no Step 4 sweeps
])
def test_dd3_fp64_bitwise(gpu, n, tiles, c, theta, kmax):
    r, gamma, g, h = _dd3_case(n, src=(n // 2, n // 3, n // 2))
    for k in range(kmax + 1):
        u_ref, s_ref, _ = O.dd(r, gamma, g, h, tiles, c, theta=theta, max_iter=k, tol=0.0, max_coarse_sweeps=16)
        u, st = gpu.dd_solve(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), h, tiles, c,
                             theta=theta, max_iter=k, tol=0.0, max_coarse_sweeps=16)
        assert st["iters"] == s_ref["iters"] == k
        assert st["fsm_sweeps_max"] == s_ref["fsm_sweeps_max"]
        np.testing.assert_array_equal(u.cpu().numpy(), u_ref, err_msg="k=%d" % k)


def test_dd3_fp32_converged_against_oracle(gpu):
    r, gamma, g, h = _dd3_case(33)
    r32 = r.astype(np.float32)
    # tol above the FP32 spacing of u ~ 1 so the FP32 run can meet it
    args = dict(theta=0.3, max_iter=30, tol=2e-6, max_coarse_sweeps=32)
    u_ref, s_ref, _ = O.dd(r32.astype(np.float64), gamma, g, h, (4, 4, 4), 8, **args)
    u, st = gpu.dd_solve(_t(r32, torch.float32), _t(gamma, torch.uint8), _t(g, torch.float32), h, (4, 4, 4), 8,
                         **args)
    assert s_ref["converged"] == 1 and st["converged"] == 1
    assert _rel(u.cpu().numpy().astype(np.float64), u_ref) <= TOL32


def test_dd3_fp32_box_shape_of_the_257_cube(gpu):
    """65^3 in 2^3 subdomains of 33^3 nodes with coarse ratio 8: the subdomain
    and coarse-grid box shapes of the 257^3 workload (every thread of the 3-D
    subdomain kernel owns three columns and uses every prefetch slot).  The
    converged FP32 solve against the oracle's FP64 full-grid solution u^f at
    every node."""
    n = 65
    h = 1.0 / (n - 1)
    r = I.sin_product((n, n, n), h, 0.4, 1.0 / 8)
    gamma, g = I.point_source((n, n, n), (32, 32, 32))
    r32 = r.astype(np.float32)
    uf, _, conv = O.fsm(r32.astype(np.float64), gamma, g, h)
    assert conv
    u, st = gpu.dd_solve(_t(r32, torch.float32), _t(gamma, torch.uint8), _t(g, torch.float32), h, (2, 2, 2), 8,
                         theta=0.0, max_iter=40, tol=1e-6, max_coarse_sweeps=8)
    assert st["converged"] == 1 and st["error"] == 0
    assert _rel(u.cpu().numpy().astype(np.float64), uf) <= TOL32


def test_dd3_full_size_257_against_oracle_fsm(gpu):
    """The 257^3 workload (8^3 subdomains, coarse ratio 8, FP32, weight 0,
    stop at a coarse update below 1e-6) in the launch configuration the
    benchmark times, run to convergence, against the oracle's FP64 full-grid
    FSM solution at every node."""
    w = I.workload_c2()
    r32 = w["r"].astype(np.float32)
    uf, _, conv = O.fsm(r32.astype(np.float64), w["gamma"], w["g"], w["h"])
    assert conv
    u, st = gpu.dd_solve(_t(r32, torch.float32), _t(w["gamma"], torch.uint8), _t(w["g"], torch.float32), w["h"],
                         w["tiles"], w["c"], theta=0.0, max_iter=80, tol=1e-6, max_coarse_sweeps=8)
    assert st["converged"] == 1 and st["error"] == 0
    assert _rel(u.cpu().numpy().astype(np.float64), uf) <= TOL32


# --------------------------------------------------------------------------
# Degenerate and extreme cases of the DD solve (FP64, bitwise against the
# oracle).
# --------------------------------------------------------------------------
def _dd_both(gpu, r, gamma, g, h, tiles, c, k, **kw):
    kw = dict(dict(theta=0.2, tol=0.0, max_coarse_sweeps=8), **kw)
    u_ref, s_ref, _ = O.dd(r, gamma, g, h, tiles, c, max_iter=k, **kw)
    u, st = gpu.dd_solve(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), h, tiles, c,
                         max_iter=k, **kw)
    assert st["iters"] == s_ref["iters"] and st["error"] == 0
    return u.cpu().numpy(), u_ref


def test_dd_without_sources_stays_infinite(gpu):
    """Gamma empty: nothing is ever reached; every node stays +inf."""
    n, h = 33, 1.0 / 32
    r = I.sin_product((n, n), h, 0.5, 0.25)
    a, ref = _dd_both(gpu, r, np.zeros((n, n), np.uint8), np.zeros((n, n)), h, (2, 2), 8, 3)
    assert np.isinf(ref).all()
    np.testing.assert_array_equal(a, ref)


def test_dd_everything_on_gamma_returns_g(gpu):
    """Gamma = every node: the solution is g, unchanged by every step."""
    n, h = 33, 1.0 / 32
    r = I.sin_product((n, n), h, 0.5, 0.25)
    g = np.random.default_rng(3).uniform(0.0, 1.0, (n, n))
    a, ref = _dd_both(gpu, r, np.ones((n, n), np.uint8), g, h, (2, 2), 8, 2)
    np.testing.assert_array_equal(ref, g)
    np.testing.assert_array_equal(a, g)


def test_dd_single_subdomain_is_the_fsm(gpu):
    """One subdomain: the first fine solve is the plain FSM of the whole grid."""
    n, h = 65, 1.0 / 64
    r, gamma, g, h = _dd_case(n, (1, 1), 8)
    a, ref = _dd_both(gpu, r, gamma, g, h, (1, 1), 8, 0)
    u_fsm, _ = gpu.fsm(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), h)
    np.testing.assert_array_equal(a, ref)
    np.testing.assert_array_equal(a, u_fsm.cpu().numpy())


def test_dd_largest_subdomain(gpu):
    """The widest FP64 subdomain whose sweep engine fits in shared memory: 288
    nodes (9 warps, 212 KB) on a 64 x 288 grid, coarse ratio 7.  A 1024-node
    subdomain is within the validated range but needs more shared memory than
    the device has: the call fails with EIK_EUNSUPPORTED before any work."""
    ny, nx = 64, 288
    h = 1.0 / (nx - 1)
    r = I.sin_product((ny, nx), h, 0.5, 0.1)
    gamma, g = I.point_source((ny, nx), (10, 150))
    for k in (0, 2):
        a, ref = _dd_both(gpu, r, gamma, g, h, (1, 1), 7, k)
        np.testing.assert_array_equal(a, ref)
    ny, nx = 64, 1024
    r = torch.ones((ny, nx), dtype=torch.float64, device=DEV)
    G = torch.zeros((ny, nx), dtype=torch.uint8, device=DEV)
    G[10, 500] = 1
    with pytest.raises(gpu.EikError) as e:
        gpu.dd_solve(r, G, torch.zeros_like(r), 1.0 / 1023, (1, 1), 3, max_iter=1)
    assert e.value.code == -5


@pytest.mark.parametrize("n,tiles,c,kmax", [(129, (4, 4), 8, 0), (97, (3, 3), 16, 3)])
def test_coarse_state_readback_fp64_bitwise(gpu, n, tiles, c, kmax):
    """eik_dd_coarse_state: after Step 1 (eik_dd_shard_start) U^0 and W^0 at
    every coarse-set node equal the oracle's; after a solve stopped at k (weight
    0.3) U equals the oracle's U^k; nodes off the coarse set are left
    untouched."""
    r, gamma, g, h = _dd_case(n, tiles, c)
    kw = dict(theta=0.3, tol=0.0, max_coarse_sweeps=8)
    dev_args = (_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), h, tiles, c)
    cs = np.zeros((n, n), bool)
    cs[::c, :] = True
    cs[:, ::c] = True
    U0, W0 = (x.cpu().numpy() for x in gpu.dd_step1_state(*dev_args, max_iter=kmax, **kw))
    _, _, W0_own, _, _, _ = O.dd_margins(r, gamma, g, h, tiles, c, max_iter=0, **kw)
    _, _, _, U0_ref = O.dd(r, gamma, g, h, tiles, c, max_iter=0, return_coarse=True, **kw)
    np.testing.assert_array_equal(U0[cs], U0_ref[cs])
    assert np.array_equal(_wind_components(W0), W0_own)
    assert np.all(np.isnan(U0[~cs])) and np.all(W0[~cs] == 255)
    u, st, Uc, _ = gpu.dd_solve(*dev_args, max_iter=kmax, return_coarse=True, **kw)
    _, _, _, U_ref = O.dd(r, gamma, g, h, tiles, c, max_iter=kmax, return_coarse=True, **kw)
    np.testing.assert_array_equal(Uc.cpu().numpy()[cs], U_ref[cs])


@pytest.mark.parametrize("dim,n,tiles,c,kmax", [
    (2, 65, (4, 4), 8, 10),
    (2, 97, (3, 3), 16, 10),
    (3, 17, (2, 2, 2), 4, 8),
])
def test_skipped_subdomain_solves_keep_results_bitwise(gpu, dim, n, tiles, c, kmax):
    """Subdomains whose Step 2 data did not change since their previous solve
    in the call are not solved again (fine_solves_skipped): once the
    iteration at weight 0 has settled, the solves are skipped, and the result
    after every k stays FP64 bitwise the oracle's, which solves every
    subdomain every time."""
    if dim == 2:
        r, gamma, g, h = _dd_case(n, tiles, c, src=(0, 0))
    else:
        r, gamma, g, h = _dd3_case(n, src=(0, 0, 0))
    kw = dict(theta=0.0, tol=0.0, max_coarse_sweeps=16)
    skipped = 0
    for k in range(kmax + 1):
        u_ref, s_ref, _ = O.dd(r, gamma, g, h, tiles, c, max_iter=k, **kw)
        u, st = gpu.dd_solve(_t(r, torch.float64), _t(gamma, torch.uint8), _t(g, torch.float64), h, tiles, c,
                             max_iter=k, **kw)
        assert st["iters"] == s_ref["iters"] == k
        np.testing.assert_array_equal(u.cpu().numpy(), u_ref, err_msg="k=%d" % k)
        assert st["fine_updates"] <= s_ref["fine_updates"]
        skipped = st["fine_solves_skipped"]
    assert skipped > 0
