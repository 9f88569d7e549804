"""Failure detection on the GPU without a GPU fault: every device-side wait is
bounded, and an expired wait ends the call with EIK_EDEVICE_TIMEOUT in its
statistics instead of trapping.  The tests shorten the limit so that ordinary
waits expire, check the reported status, restore the limit and check that the
same context still produces the exact result."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1805_04198_gb300 import eik, inputs

pytestmark = pytest.mark.gpu
TIMEOUT = -4  # EIK_EDEVICE_TIMEOUT


def _case(n=257, src=(128, 128)):
    h = 1.0 / (n - 1)
    r = inputs.sin_product((n, n), h, 0.5, 1.0 / 16)
    gamma, g = inputs.point_source((n, n), src)
    return r, gamma, g, h


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def test_dd_expired_wait_reports_timeout_then_solves_exactly():
    """2-D DD (the coarse-grid engines hand columns between warps, the causal
    sweep uses grid barriers): with a one-poll limit some wait expires; the
    call returns, its statistics carry EIK_EDEVICE_TIMEOUT, and after the
    default limit is restored the same solve is bitwise the FP64 oracle's."""
    r, gamma, g, h = _case()
    kw = dict(theta=0.2, max_iter=4, tol=0.0, max_coarse_sweeps=8)
    rd, gd, vd = _dev(r, gamma, g)
    eik.eik_set_wait_limit(1)
    try:
        u, st = eik.dd_solve(rd, gd, vd, h, (4, 4), 8, sync=False, **kw)
        torch.cuda.synchronize()
        s = eik.DDStats.from_buffer_copy(bytes(st.cpu().numpy()))
        assert s.error == TIMEOUT
        with pytest.raises(eik.EikError) as ei:
            eik.dd_solve(rd, gd, vd, h, (4, 4), 8, **kw)
        assert ei.value.code == TIMEOUT
    finally:
        eik.eik_set_wait_limit(0)
    u2, st2 = eik.dd_solve(rd, gd, vd, h, (4, 4), 8, **kw)
    torch.cuda.synchronize()
    assert st2["error"] == 0
    u_ref, st_ref, _ = oracle.dd(r, gamma, g, h, (4, 4), 8, **kw)
    assert np.array_equal(u2.cpu().numpy(), u_ref)
    assert st2["iters"] == st_ref["iters"]


def test_fsm_multi_cta_expired_wait_reports_timeout_then_solves_exactly():
    """The plain FSM on a grid wide enough for the multi-CTA engine (CTAs hand
    block columns to each other through global memory)."""
    n = 1025
    r, gamma, g, h = _case(n, (512, 512))
    rd, gd, vd = _dev(r, gamma, g)
    eik.eik_set_wait_limit(1)
    try:
        with pytest.raises(eik.EikError) as ei:
            eik.fsm(rd, gd, vd, h)
        assert ei.value.code == TIMEOUT
    finally:
        eik.eik_set_wait_limit(0)
    u2, st2 = eik.fsm(rd, gd, vd, h)
    torch.cuda.synchronize()
    u_ref, sweeps, conv = oracle.fsm(r, gamma, g, h)
    assert np.array_equal(u2.cpu().numpy(), u_ref)
    assert st2["sweeps"] == sweeps
