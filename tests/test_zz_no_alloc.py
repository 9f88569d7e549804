"""The entry point that allocates nothing (eik_dd_solve_noalloc).

Callers that cannot allocate device memory -- code recording a CUDA graph, or a
host whose device allocator belongs to another runtime -- get the DD solver
with the library's static scratch array instead of a caller workspace.  These
checks call it through the C ABI and compare it with eik_dd_solve on the same
inputs, twice in a row (the static array keeps the previous call's contents,
which must not leak into the next result).  This file is named to be
collected last so a stop-at-first-failure run has executed everything else.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1805_04198_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _problem(n, dtype, src):
    h = 1.0 / (n - 1)
    r = I.sin_product((n, n), h, 0.5, 0.25).astype(dtype)
    gamma, g = I.point_source((n, n), src)
    return r, gamma, g.astype(dtype), h


def test_noalloc_matches_workspace_solve_twice(gpu):
    dev = "cuda:0"
    cases = [(129, np.float64, (64, 64), (4, 4), 8, 0.2, 5, 0.0),   # FP64: compared bitwise
             (257, np.float32, (10, 200), (4, 4), 8, 0.3, 4, 1e-5)]  # FP32, off-centre source
    for n, dt, src, tiles, c, theta, kmax, tol in cases:
        r, gamma, g, h = _problem(n, dt, src)
        R = torch.from_numpy(r).to(dev)
        G = torch.from_numpy(gamma).to(dev)
        g_t = torch.from_numpy(g).to(dev)
        grid = gpu.make_grid(R, h)
        p = gpu.dd_params(tiles, c, theta=theta, max_iter=kmax, tol=0.0)
        assert gpu.eik_dd_workspace_size(grid, p) <= gpu.NOALLOC_SCRATCH_BYTES
        ref, ref_st = gpu.dd_solve(R, G, g_t, h, tiles, c, theta=theta, max_iter=kmax, tol=0.0)
        ref = ref.cpu().numpy()
        for call in range(2):
            u = torch.full_like(R, float("nan"))
            st = torch.zeros(ctypes.sizeof(gpu.DDStats), dtype=torch.uint8, device=dev)
            gpu.eik_dd_solve_noalloc(grid, R, G, g_t, p, u, st)
            torch.cuda.synchronize()
            s = gpu.parse_dd_stats(st)
            assert s["error"] == 0 and s["iters"] == ref_st["iters"], (call, s)
            got = u.cpu().numpy()
            if tol == 0.0:
                np.testing.assert_array_equal(got, ref, err_msg="call %d" % call)
            else:
                fin = np.isfinite(ref)
                assert np.array_equal(np.isfinite(got), fin)
                err = np.max(np.abs(got[fin] - ref[fin])) / np.max(np.abs(ref[fin]))
                assert err <= tol, (call, err)


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
