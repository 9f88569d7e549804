"""Many source sets on one grid and one slowness (eik_fsm_many,
eik_dd_adjoint_many) through the C ABI.

Each problem must come out exactly as its own eik_fsm / eik_dd_adjoint call
(bitwise, FP64 and FP32), in the one-CTA sweep form, the multi-CTA form and
the multi-CTA form split into several co-resident groups; the gradient sum
must equal the per-source gradients added in source order.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1805_04198_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=None):
    x = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return x if dtype is None else x.to(dtype)


def _sources(shape, nsrc, seed):
    rng = np.random.default_rng(seed)
    gam = np.zeros((nsrc,) + shape, np.uint8)
    g = np.zeros((nsrc,) + shape)
    for s in range(nsrc):
        for _ in range(1 + s % 3):
            j, i = rng.integers(0, shape[0]), rng.integers(0, shape[1])
            gam[s, j, i] = 1
            g[s, j, i] = rng.uniform(0.0, 0.05)
    return gam, g


@pytest.mark.parametrize("shape,nsrc,dtype", [
    ((70, 100), 5, torch.float64),     # one CTA per source
    ((40, 1100), 3, torch.float64),    # several co-resident CTAs per source
    ((20, 4097), 30, torch.float64),   # ... in more than one co-resident group
    ((65, 300), 7, torch.float32),
])
def test_fsm_many_equals_single(gpu, shape, nsrc, dtype):
    rng = np.random.default_rng(sum(shape))
    r = _t(rng.uniform(0.5, 2.0, shape), dtype)
    gam, g = _sources(shape, nsrc, nsrc)
    G, Gv = _t(gam), _t(g, dtype)
    h = 1.0 / 256
    u, st = gpu.fsm_many(r, G, Gv, h)
    for s in range(nsrc):
        u1, s1 = gpu.fsm(r, G[s].contiguous(), Gv[s].contiguous(), h)
        assert torch.equal(u[s], u1), s
        assert st[s]["sweeps"] == s1["sweeps"] and st[s]["converged"] == 1


def test_fsm_many_matches_oracle(gpu):
    shape = (33, 45)
    rng = np.random.default_rng(1)
    r = rng.uniform(0.5, 2.0, shape)
    gam, g = _sources(shape, 4, 2)
    u, _ = gpu.fsm_many(_t(r), _t(gam), _t(g), 0.1)
    for s in range(4):
        ref, _, _ = O.fsm(r, gam[s], g[s], 0.1)
        np.testing.assert_array_equal(u[s].cpu().numpy(), ref)


@pytest.mark.parametrize("shape,nsrc,dtype", [
    ((70, 100), 4, torch.float64),
    ((40, 1100), 3, torch.float64),
    ((65, 300), 5, torch.float32),
])
def test_adjoint_many_equals_single_and_ordered_sum(gpu, shape, nsrc, dtype):
    rng = np.random.default_rng(7 + nsrc)
    r = _t(rng.uniform(0.6, 1.6, shape), dtype)
    gam, _ = _sources(shape, nsrc, 3)
    G = _t(gam)
    h = 1.0 / 128
    u, _ = gpu.fsm_many(r, G, torch.zeros((nsrc,) + shape, dtype=dtype, device=DEV), h)
    dJ = _t(rng.uniform(-1, 1, (nsrc,) + shape) * (rng.uniform(size=(nsrc,) + shape) < 0.05), dtype)
    gsum, per, st = gpu.adjoint_many(r, G, u, dJ, h, per_problem=True)
    acc = None
    for s in range(nsrc):
        g1, _ = gpu.adjoint(r, G[s].contiguous(), u[s].contiguous(), dJ[s].contiguous(), h)
        assert torch.equal(per[s], g1), s
        assert st[s]["converged"] == 1
        acc = g1.clone() if acc is None else acc + g1
    assert torch.equal(gsum, acc)


def test_adjoint_many_oracle_fp64(gpu):
    shape = (40, 33)
    rng = np.random.default_rng(11)
    r = rng.uniform(0.6, 1.6, shape)
    gam, _ = _sources(shape, 3, 4)
    h = 1.0 / 64
    us = np.stack([O.fsm(r, gam[s], 0.0, h)[0] for s in range(3)])
    dJ = np.zeros((3,) + shape)
    dJ[:, :, -1] = rng.uniform(-1, 1, (3, shape[0]))
    gsum, per, _ = gpu.adjoint_many(_t(r), _t(gam), _t(us), _t(dJ), h, per_problem=True)
    ref = [O.adjoint(r, gam[s], us[s], dJ[s], h) for s in range(3)]
    for s in range(3):
        np.testing.assert_array_equal(per[s].cpu().numpy(), ref[s])
    np.testing.assert_array_equal(gsum.cpu().numpy(), (ref[0] + ref[1]) + ref[2])


def test_tomography_many_sources_full_size(gpu):
    """The 1025^2 tomography workload with all 64 sources through the
    many-source autograd Function: every forward solution equals its
    single-source solve and the gradient equals the single-source autograd
    gradients added in source order (FP32, bitwise)."""
    w = I.workload_c4()
    n, h = w["n"], w["h"]
    R = _t(w["r0"].astype(np.float32))
    S = len(w["src_rows"])
    gam = torch.zeros((S, n, n), dtype=torch.uint8, device=DEV)
    for s, row in enumerate(w["src_rows"]):
        gam[s, row, 0] = 1
    g0 = torch.zeros((S, n, n), device=DEV)
    rec = torch.tensor([j * n + n - 1 for j in w["rec_rows"]], device=DEV)
    d, _ = gpu.fsm_many(_t(w["r_true"].astype(np.float32)), gam, g0, h)
    d = d.reshape(S, -1)[:, rec].clone()
    rr = R.clone().requires_grad_(True)
    u = gpu.EikonalSolveMany.apply(rr, gam, g0, h)
    L = 0.5 * ((u.reshape(S, -1)[:, rec] - d) ** 2).sum()
    L.backward()
    acc = None
    for s in range(S):
        r1 = R.clone().requires_grad_(True)
        u1 = gpu.EikonalSolve.apply(r1, gam[s].contiguous(), torch.zeros_like(R), h)
        if s in (0, 31, 63):
            assert torch.equal(u1, u[s].detach())
        (0.5 * ((u1.flatten()[rec] - d[s]) ** 2).sum()).backward()
        acc = r1.grad.clone() if acc is None else acc + r1.grad
    assert torch.equal(rr.grad, acc)


def test_many_validation(gpu):
    r = torch.ones((9, 9), device=DEV)
    grid = gpu.make_grid(r, 0.1)
    lib = gpu.load()
    assert lib.eik_fsm_many_workspace_size(gpu.ctypes.byref(grid), 0) == 0
    assert lib.eik_dd_adjoint_many_workspace_size(gpu.ctypes.byref(grid), 0) == 0
    with pytest.raises(ValueError):
        gpu.fsm_many(r, torch.zeros((2, 9, 8), dtype=torch.uint8, device=DEV), torch.zeros((2, 9, 9), device=DEV),
                     0.1)


def test_dd_forward_of_many_sources(gpu):
    """The tomography gradient with the forward solved by the DD (ManyDD: one
    batched solve of every source, T = 4, c = 8): every source's u is its own
    eik_dd_solve bitwise and agrees with the plain FSM's within the FP32
    tolerance, and the gradient (the adjoint at that u) agrees with the one
    taken at the FSM's u within 1e-3 relative L2."""
    n, S = 257, 8
    h = 1.0 / (n - 1)
    r = _t(I.sin_product((n, n), h, 0.4, 1.0 / 8).astype(np.float32))
    gam = np.zeros((S, n, n), np.uint8)
    for s in range(S):
        gam[s, 16 + 32 * s, 0] = 1
    G, Gv = _t(gam), torch.zeros((S, n, n), dtype=torch.float32, device=DEV)
    rec = torch.arange(2, n, 4, device=DEV)
    kw = dict(theta=0.0, max_iter=40, tol=1e-6, max_coarse_sweeps=8)
    dd = gpu.ManyDD(r, G, Gv, h, (4, 4), 8, **kw)
    u_dd = dd.solve(r)
    torch.cuda.synchronize()
    assert all(st["converged"] == 1 for st in dd.stats())
    u_fsm, _ = gpu.fsm_many(r, G, Gv, h)
    for s in range(S):
        u1, _ = gpu.dd_solve(r, G[s].contiguous(), Gv[s].contiguous(), h, (4, 4), 8, **kw)
        assert torch.equal(u_dd[s], u1), s
    rel = ((u_dd - u_fsm).abs().max() / u_fsm.abs().max()).item()
    assert rel <= 1e-5, rel
    data = (u_fsm[:, rec, n - 1] * 1.01).detach()

    def grad(dd_arg):
        rr = r.detach().requires_grad_(True)
        u = gpu.EikonalSolveMany.apply(rr, G, Gv, h, dd_arg)
        (0.5 * ((u[:, rec, n - 1] - data) ** 2).sum()).backward()
        return rr.grad

    g_dd, g_fsm = grad(dd), grad(None)
    assert torch.isfinite(g_dd).all()
    diff = (torch.linalg.vector_norm(g_dd - g_fsm) / torch.linalg.vector_norm(g_fsm)).item()
    assert diff <= 1e-3, diff
