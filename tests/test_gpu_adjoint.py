"""The adjoint (gradient of a scalar J(u) with respect to the slowness r)
through the C ABI, against the FP64 oracle adjoint and finite differences."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1805_04198_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def _problem(shape, seed):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.6, 1.6, shape)
    gamma = np.zeros(shape, np.uint8)
    gamma[shape[0] // 2, 0] = 1
    gamma[shape[0] // 3, shape[1] // 2] = 1
    dJdu = np.zeros(shape)
    dJdu[:, -1] = rng.uniform(-1, 1, shape[0])      # receivers on the right edge
    dJdu[-1, ::7] = rng.uniform(-1, 1, len(range(0, shape[1], 7)))
    return r, gamma, dJdu


@pytest.mark.parametrize("shape", [(40, 33), (65, 129), (200, 1100)])
def test_adjoint_fp64_matches_oracle_bitwise(gpu, shape):
    r, gamma, dJdu = _problem(shape, sum(shape))
    h = 1.0 / 64
    u, _, _ = O.fsm(r, gamma, 0.0, h)
    ref = O.adjoint(r, gamma, u, dJdu, h)
    grad, st = gpu.adjoint(_t(r, torch.float64), _t(gamma, torch.uint8), _t(u, torch.float64),
                           _t(dJdu, torch.float64), h)
    assert st["converged"] == 1
    np.testing.assert_array_equal(grad.cpu().numpy(), ref)


def test_adjoint_fp32_against_oracle(gpu):
    r, gamma, dJdu = _problem((129, 257), 3)
    h = 1.0 / 256
    r32 = r.astype(np.float32)
    R = _t(r32, torch.float32)
    G = _t(gamma, torch.uint8)
    u32, _ = gpu.fsm(R, G, torch.zeros_like(R), h)
    u_np = u32.cpu().numpy().astype(np.float64)
    ref = O.adjoint(r32.astype(np.float64), gamma, u_np, dJdu, h)
    grad, st = gpu.adjoint(R, G, u32, _t(dJdu, torch.float32), h)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_autograd_matches_finite_differences(gpu):
    """EikonalSolve.apply + torch autograd: dJ/dr at 16 cells against central
    differences of the GPU forward solve (step 1e-4 on r), FP64."""
    rng = np.random.default_rng(5)
    n = 33
    h = 1.0 / 32
    r = _t(1.0 + 0.3 * rng.uniform(size=(n, n)), torch.float64)
    G = torch.zeros(n, n, dtype=torch.uint8, device=DEV)
    G[16, 0] = 1
    g = torch.zeros_like(r)
    rec = torch.tensor([(j * n + n - 1) for j in range(2, n - 2, 3)], device=DEV)
    d = _t(rng.uniform(0.8, 1.2, len(rec)), torch.float64)

    def loss(rr):
        u = gpu.EikonalSolve.apply(rr, G, g, h)
        return 0.5 * ((u.flatten()[rec] - d) ** 2).sum()

    rr = r.clone().requires_grad_(True)
    L = loss(rr)
    L.backward()
    grad = rr.grad.cpu().numpy()
    cells = [(int(a), int(b)) for a, b in rng.integers(4, n - 4, size=(16, 2))]
    for c in cells:
        e = 1e-4
        rp = r.clone(); rp[c] += e
        rm = r.clone(); rm[c] -= e
        fd = (loss(rp).item() - loss(rm).item()) / (2 * e)
        assert grad[c] == pytest.approx(fd, rel=1e-4, abs=1e-7), c


def test_tomography_gradient_full_size(gpu):
    """1025^2 tomography workload (two of the 64 sources): the FP32 gradient of
    0.5 sum (u_s(receiver) - d)^2 through autograd on the GPU.
    (a) against the FP64 oracle adjoint evaluated at the GPU's own forward
        solution and residuals: the adjoint alone, relative max error 1e-4;
    (b) against the all-FP64 oracle pipeline (its own forward solve): FP32 and
        FP64 forward solutions pick different neighbours at near-ties along the
        rays, so the gradients agree only to about 1e-2 (relative L2)."""
    w = I.workload_c4()
    n, h = w["n"], w["h"]
    r0 = w["r0"].astype(np.float32)
    R = _t(r0, torch.float32)
    g = torch.zeros_like(R)
    rec_rows = w["rec_rows"]
    total_gpu = np.zeros((n, n))
    total_at_gpu_u = np.zeros((n, n))
    total_fp64 = np.zeros((n, n))
    for s in (0, 37):
        gam = np.zeros((n, n), np.uint8)
        gam[w["src_rows"][s], 0] = 1
        ut, _, _ = O.fsm(w["r_true"], gam, 0.0, h)      # synthetic data, FP64 oracle forward
        d = ut[rec_rows, n - 1]
        G = _t(gam, torch.uint8)
        rr = R.clone().requires_grad_(True)
        u = gpu.EikonalSolve.apply(rr, G, g, h)
        rec = torch.tensor([j * n + n - 1 for j in rec_rows], device=DEV)
        L = 0.5 * ((u.flatten()[rec].double() - _t(d, torch.float64)) ** 2).sum()
        L.backward()
        total_gpu += rr.grad.cpu().numpy().astype(np.float64)
        ug = u.detach().cpu().numpy().astype(np.float64)
        dJdu = np.zeros((n, n))
        dJdu[rec_rows, n - 1] = ug[rec_rows, n - 1].astype(np.float32).astype(np.float64) - d
        total_at_gpu_u += O.adjoint(r0.astype(np.float64), gam, ug, dJdu, h)
        u0, _, _ = O.fsm(r0.astype(np.float64), gam, 0.0, h)
        dJdu0 = np.zeros((n, n))
        dJdu0[rec_rows, n - 1] = u0[rec_rows, n - 1] - d
        total_fp64 += O.adjoint(r0.astype(np.float64), gam, u0, dJdu0, h)
    err_adj = np.max(np.abs(total_gpu - total_at_gpu_u)) / np.max(np.abs(total_at_gpu_u))
    assert err_adj <= 1e-4, err_adj
    rel = np.linalg.norm(total_gpu - total_fp64) / np.linalg.norm(total_fp64)
    assert rel <= 2e-2, rel
