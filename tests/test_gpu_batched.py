"""Batched DD (many independent 2-D problems in one sequence of launches)
through the C ABI.

Each problem of a batch must come out exactly as its own eik_dd_solve call:
bitwise equal to the FP64 oracle in FP64, bitwise equal to the single-problem
GPU solve in FP32, whatever the launch configuration, and unchanged when the
solve is replayed from a CUDA graph.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_1805_04198_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def _problem(shape, tiles, c, theta, max_iter, tol=0.0, src=None, amp=0.5, eps=0.25, seed=0):
    ny, nx = shape
    h = 1.0 / (max(nx, ny) - 1)
    rng = np.random.default_rng(seed)
    r = I.sin_product(shape, h, amp, eps) * rng.uniform(0.9, 1.1, shape)
    gamma, g = I.point_source(shape, src if src is not None else (ny // 2, nx // 2))
    return dict(r=r, gamma=gamma, g=g, h=h, tiles=tiles, coarse_ratio=c, theta=theta, max_iter=max_iter, tol=tol)


# Mixed sizes: subdomain widths of 17, 33, 65 nodes (1, 2, 3 warps), coarse grids
# of 9..33 nodes per side, a non-square grid, an off-lattice source, per-problem
# caps and one problem that stops by tol.
MIXED = [
    ((65, 65), (4, 4), 8, 0.2, 4, 0.0, None),
    ((97, 97), (3, 3), 16, 0.2, 3, 0.0, None),
    ((129, 129), (2, 2), 8, 0.3, 2, 0.0, None),
    ((65, 65), (2, 4), 8, 1.0, 5, 0.0, None),
    ((65, 65), (4, 4), 8, 0.2, 40, 1e-9, None),
    ((65, 129), (4, 2), 8, 0.2, 3, 0.0, (20, 90)),
    ((65, 65), (4, 4), 8, 0.2, 6, 0.0, (21, 37)),
    ((161, 161), (5, 5), 8, 0.2, 3, 0.0, None),
]


def _mixed(dtype):
    out = []
    for i, (shape, tiles, c, theta, k, tol, src) in enumerate(MIXED):
        p = _problem(shape, tiles, c, theta, k, tol, src, seed=i)
        npd = np.float64 if dtype == torch.float64 else np.float32
        p["r_host"] = p["r"].astype(npd).astype(np.float64)
        p["r"] = _t(p["r"].astype(npd), dtype)
        p["gamma"] = _t(p["gamma"], torch.uint8)
        p["g"] = _t(p["g"], dtype)
        out.append(p)
    return out


def _single(gpu, p):
    return gpu.dd_solve(p["r"], p["gamma"], p["g"], p["h"], p["tiles"], p["coarse_ratio"], theta=p["theta"],
                        max_iter=p["max_iter"], tol=p["tol"], max_coarse_sweeps=8)


def test_batched_fp64_bitwise_vs_oracle(gpu):
    probs = _mixed(torch.float64)
    B = gpu.DDBatch(probs)
    B.run()
    stats = B.stats()
    for i, p in enumerate(probs):
        u_ref, s_ref, _ = O.dd(p["r_host"], p["gamma"].cpu().numpy(), p["g"].cpu().numpy(), p["h"], p["tiles"],
                               p["coarse_ratio"], theta=p["theta"], max_iter=p["max_iter"], tol=p["tol"],
                               max_coarse_sweeps=8)
        assert stats[i]["iters"] == s_ref["iters"], i
        assert stats[i]["converged"] == s_ref["converged"], i
        assert stats[i]["error"] == 0
        np.testing.assert_array_equal(B.u[i].cpu().numpy(), u_ref, err_msg="problem %d" % i)
    assert stats[4]["converged"] == 1


def test_batched_fp32_equals_single_solves_every_config(gpu):
    probs = _mixed(torch.float32)
    singles = [_single(gpu, p) for p in probs]
    B = gpu.DDBatch(probs)
    configs = [None]
    for fq in (0, 1):
        for gq in (0, 1):
            for cps in (0, 1):
                for lf in (0, 1):
                    configs.append(gpu.BatchConfig(fq, gq, cps, lf))
    for cfg in configs:
        B.config = cfg
        for u in B.u:
            u.fill_(float("nan"))
        B.run()
        stats = B.stats()
        for i, (u1, s1) in enumerate(singles):
            assert torch.equal(B.u[i], u1), (i, cfg and (cfg.fine_queue, cfg.coarse_queue, cfg.ctas_per_sm))
            for key in ("iters", "converged", "fsm_sweeps_max", "coarse_sweeps_max", "fine_updates",
                        "coarse_updates", "fsm_cap_hits", "coarse_cap_hits"):
                assert stats[i][key] == s1[key], (i, key)
            assert stats[i]["last_delta"] == s1["last_delta"] or (
                np.isinf(stats[i]["last_delta"]) and np.isinf(s1["last_delta"]))


def test_batched_queue_rearms_across_launches(gpu):
    """The queue form reuses its counters launch after launch (one fine and
    one coarse launch per class and iteration): repeated solves agree."""
    probs = _mixed(torch.float32)
    B = gpu.DDBatch(probs, config=gpu.BatchConfig(1, 1, 1, 1))
    B.run()
    first = [u.clone() for u in B.u]
    for _ in range(3):
        B.run()
    for a, b in zip(first, B.u):
        assert torch.equal(a, b)


def test_batched_graph_replay(gpu):
    probs = _mixed(torch.float32)
    B = gpu.DDBatch(probs)
    B.capture()
    for u in B.u:
        u.fill_(0.0)
    B.replay()
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        u1, _ = _single(gpu, p)
        assert torch.equal(B.u[i], u1), i
    # the graph reads the inputs in place: new slowness, same graph
    probs[2]["r"].mul_(1.5)
    B.replay()
    torch.cuda.synchronize()
    u1, _ = _single(gpu, probs[2])
    assert torch.equal(B.u[2], u1)


def test_batched_autotune(gpu):
    probs = _mixed(torch.float32)
    B = gpu.DDBatch(probs)
    best, ms = B.autotune(tune_iters=1)
    assert ms > 0
    assert best.fine_queue in (0, 1) and best.coarse_queue in (0, 1)
    B.run()
    for i, p in enumerate(probs):
        assert torch.equal(B.u[i], _single(gpu, p)[0])


def test_batched_single_problem_batch(gpu):
    probs = _mixed(torch.float64)[:1]
    B = gpu.DDBatch(probs)
    B.run()
    assert torch.equal(B.u[0], _single(gpu, probs[0])[0])


def test_batched_validation(gpu):
    probs = _mixed(torch.float32)[:2]
    grids = [gpu.make_grid(p["r"], p["h"]) for p in probs]
    params = [gpu.dd_params(p["tiles"], p["coarse_ratio"]) for p in probs]
    assert gpu.eik_dd_batched_workspace_size([], []) == 0
    # mixed dtypes
    r64 = probs[1]["r"].double()
    g2 = [grids[0], gpu.make_grid(r64, probs[1]["h"])]
    assert gpu.eik_dd_batched_workspace_size(g2, params) == 0
    assert "dtype" in gpu.eik_last_error()
    # 3-D grids are not batched
    r3 = torch.ones((9, 9, 9), device=DEV)
    assert gpu.eik_dd_batched_workspace_size([gpu.make_grid(r3, 0.125)], [gpu.dd_params((2, 2, 2), 4)]) == 0
    # a bad tiling names its problem
    bad = [params[0], gpu.dd_params((5, 5), 8)]
    assert gpu.eik_dd_batched_workspace_size(grids, bad) == 0
    assert "problem 1" in gpu.eik_last_error()
    # workspace too small
    n = gpu.eik_dd_batched_workspace_size(grids, params)
    ws = torch.empty(n // 2, dtype=torch.uint8, device=DEV)
    with pytest.raises(gpu.EikError) as e:
        gpu.eik_dd_solve_batched(grids, [p["r"] for p in probs], [p["gamma"] for p in probs],
                                 [p["g"] for p in probs], params, [torch.empty_like(p["r"]) for p in probs], None,
                                 ws, None)
    assert e.value.code == -2


def test_batched_full_size_sampled(gpu):
    """The 256-problem batch of the benchmark (sides 257..2049, 8..32
    subdomains per side, FP32) in the launch configuration the benchmark
    times: sampled problems equal their own single-problem solves bitwise, and
    the smallest sampled ones agree with the FP64 oracle after one iteration."""
    w = I.workload_c3()
    probs = []
    for q in w:
        probs.append(dict(r=_t(q["r"].astype(np.float32), torch.float32), gamma=_t(q["gamma"], torch.uint8),
                          g=_t(q["g"].astype(np.float32), torch.float32), h=q["h"], tiles=q["tiles"],
                          coarse_ratio=q["c"], theta=q["theta"], max_iter=q["max_iter"], tol=q["tol"]))
    B = gpu.DDBatch(probs)
    B.autotune(tune_iters=1)
    B.run()
    stats = B.stats()
    assert all(s["error"] == 0 for s in stats)
    sides = [q["r"].shape[0] for q in w]
    sample = []
    for n in (257, 513, 1025, 2049):
        sample += [i for i, s in enumerate(sides) if s == n][:2]
    for i in sample:
        u1, s1 = _single(gpu, probs[i])
        assert torch.equal(B.u[i], u1), i
        assert stats[i]["iters"] == s1["iters"]
    # oracle, one DD iteration, on two 257^2 problems
    for i in [i for i, s in enumerate(sides) if s == 257][:2]:
        q = w[i]
        r32 = q["r"].astype(np.float32)
        p = dict(probs[i], max_iter=1)
        u1, _ = _single(gpu, p)
        u_ref, _, _ = O.dd(r32.astype(np.float64), q["gamma"], q["g"], q["h"], q["tiles"], q["c"], theta=q["theta"],
                           max_iter=1, tol=0.0, max_coarse_sweeps=8)
        a = u1.cpu().numpy().astype(np.float64)
        fin = np.isfinite(u_ref)
        assert np.array_equal(np.isfinite(a), fin)
        assert np.max(np.abs(a[fin] - u_ref[fin])) / np.max(np.abs(u_ref[fin])) <= 1e-5


_ADAPT = ("theta_adaptive", "omega", "sig_gamma", "sig_delta", "sig_x0", "theta_cap")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_adaptive_weight_mixed(gpu, dtype):
    """A batch mixing problems with the per-node weight of Sec. 4.2 and
    problems with a constant weight (every problem then carries the weight as
    a fourth Alg. 5 static): each output equals its own single-problem solve
    bitwise, with the same statistics, under the default and two explicit
    launch configurations."""
    probs = _mixed(dtype)
    for i in (0, 4, 6):
        probs[i].update(theta_adaptive=True, theta_cap=0.5, omega=(1.0, 0.5, 0.25))
    singles = []
    for p in probs:
        kw = {k: p[k] for k in _ADAPT if k in p}
        singles.append(gpu.dd_solve(p["r"], p["gamma"], p["g"], p["h"], p["tiles"], p["coarse_ratio"],
                                    theta=p["theta"], max_iter=p["max_iter"], tol=p["tol"], max_coarse_sweeps=8,
                                    **kw))
    B = gpu.DDBatch(probs)
    for cfg in (None, gpu.BatchConfig(1, 1, 0, 1), gpu.BatchConfig(0, 0, 1, 0)):
        B.config = cfg
        for u in B.u:
            u.fill_(float("nan"))
        B.run()
        stats = B.stats()
        for i, (u1, s1) in enumerate(singles):
            assert torch.equal(B.u[i], u1), i
            for key in ("iters", "converged", "fine_updates", "coarse_updates", "coarse_cap_hits"):
                assert stats[i][key] == s1[key], (i, key)
