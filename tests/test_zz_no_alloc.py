"""The entry point that allocates nothing (eik_dd_solve_noalloc).

Some callers cannot allocate device memory at all -- a host whose device
allocator belongs to another runtime that must not be bypassed, or a real-time
loop that forbids allocation once it runs.  They get the DD solver with the
library's static scratch array instead of a caller workspace.  These checks
call it through the C ABI and compare it bitwise with eik_dd_solve on the same
inputs.  The static array keeps the previous call's contents, so the calls
alternate between problems of different shapes, element types and dimension
(each leaves a different layout behind) and every problem is solved twice.
This file is named to be collected last so a stop-at-first-failure run has
executed everything else.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1805_04198_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _problem(shape, dtype, src, eps):
    h = 1.0 / (shape[0] - 1)
    r = I.sin_product(shape, h, 0.5, eps).astype(dtype)
    gamma, g = I.point_source(shape, src)
    return r, gamma, g.astype(dtype), h


# (shape, dtype, source, eps, tiles, coarse ratio, theta, max_iter)
CASES = [((129, 129), np.float64, (64, 64), 0.25, (4, 4), 8, 0.2, 5),
         ((257, 257), np.float32, (10, 200), 0.25, (4, 4), 8, 0.3, 4),     # off-centre source
         ((33, 33, 33), np.float32, (16, 11, 20), 0.25, (4, 4, 4), 4, 0.2, 4)]


def test_noalloc_matches_workspace_solve_bitwise(gpu):
    dev = "cuda:0"
    probs = []
    for shape, dt, src, eps, tiles, c, theta, kmax in CASES:
        r, gamma, g, h = _problem(shape, dt, src, eps)
        R = torch.from_numpy(r).to(dev)
        G = torch.from_numpy(gamma).to(dev)
        g_t = torch.from_numpy(g).to(dev)
        grid = gpu.make_grid(R, h)
        p = gpu.dd_params(tiles, c, theta=theta, max_iter=kmax, tol=0.0)
        assert gpu.eik_dd_workspace_size(grid, p) <= gpu.NOALLOC_SCRATCH_BYTES
        ref, ref_st = gpu.dd_solve(R, G, g_t, h, tiles, c, theta=theta, max_iter=kmax, tol=0.0)
        probs.append((R, G, g_t, grid, p, ref.cpu().numpy(), ref_st))
    for rnd in range(2):
        for i, (R, G, g_t, grid, p, ref, ref_st) in enumerate(probs):
            u = torch.full_like(R, float("nan"))
            st = torch.zeros(ctypes.sizeof(gpu.DDStats), dtype=torch.uint8, device=dev)
            gpu.eik_dd_solve_noalloc(grid, R, G, g_t, p, u, st)
            torch.cuda.synchronize()
            s = gpu.parse_dd_stats(st)
            assert s["error"] == 0 and s["iters"] == ref_st["iters"], (rnd, i, s)
            np.testing.assert_array_equal(u.cpu().numpy(), ref, err_msg="round %d, problem %d" % (rnd, i))


def test_noalloc_rejects_problems_beyond_the_static_scratch(gpu):
    R = torch.ones(1025, 1025, dtype=torch.float32, device="cuda:0")
    grid = gpu.make_grid(R, 1.0 / 1024)
    p = gpu.dd_params((16, 16), 16, max_iter=4)
    assert gpu.eik_dd_workspace_size(grid, p) > gpu.NOALLOC_SCRATCH_BYTES
    G = torch.zeros_like(R, dtype=torch.uint8)
    st = torch.zeros(ctypes.sizeof(gpu.DDStats), dtype=torch.uint8, device="cuda:0")
    with pytest.raises(gpu.EikError) as e:
        gpu.eik_dd_solve_noalloc(grid, R, G, R, p, R.clone(), st)
    assert e.value.code == -2 and "static scratch" in str(e.value)
