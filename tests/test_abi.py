"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects invalid requests before any CUDA work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_04198_gb300 import _build, eik
    _build.build()
    return eik


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "eik.h")).read()
    declared = set(re.findall(r"\b(eik_[a-z0-9_]+)\s*\(", hdr))
    assert {"eik_fsm", "eik_dd_solve", "eik_last_error", "eik_version"} <= declared
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(so, name), name


def test_version(lib):
    assert lib.eik_version() >= 100


def _grid(lib, n=(65, 65), dtype=0, h=1 / 64, stride=None):
    st = stride or (1, n[0], n[0] * n[1])
    return lib.Grid(2, dtype, (ctypes.c_int64 * 3)(n[0], n[1], 1), (ctypes.c_int64 * 3)(*st), h)


def test_workspace_sizes_and_validation(lib):
    g = _grid(lib)
    assert lib.eik_fsm_workspace_size(g) > 0
    p = lib.dd_params((4, 4), 8)
    assert lib.eik_dd_workspace_size(g, p) > 0
    # tiles not dividing n-1
    assert lib.eik_dd_workspace_size(g, lib.dd_params((3, 4), 8)) == 0
    assert "tiles" in lib.eik_last_error()
    # coarse ratio not dividing the subdomain width
    assert lib.eik_dd_workspace_size(g, lib.dd_params((4, 4), 5)) == 0
    assert "coarse_ratio" in lib.eik_last_error()
    # bad spacing / dtype / stride
    assert lib.eik_fsm_workspace_size(_grid(lib, h=0.0)) == 0
    assert lib.eik_fsm_workspace_size(_grid(lib, dtype=7)) == 0
    assert lib.eik_fsm_workspace_size(_grid(lib, stride=(1, 10, 650))) == 0
    assert lib.eik_dd_workspace_size(g, lib.dd_params((4, 4), 8, max_iter=-1)) == 0


def test_calls_reject_null_and_small_workspace(lib):
    so = lib.load()
    g = _grid(lib)
    p = lib.dd_params((4, 4), 8)
    null = ctypes.c_void_p(0)
    rc = so.eik_dd_solve(ctypes.byref(g), null, null, null, ctypes.byref(p), null, null, 0, null, null)
    assert rc == -1
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: rejected before use
    rc = so.eik_dd_solve(ctypes.byref(g), fake, fake, fake, ctypes.byref(p), fake, fake, 16, null, null)
    assert rc == -2 and "workspace" in lib.eik_last_error()
    rc = so.eik_fsm(ctypes.byref(g), fake, fake, fake, fake, 0, fake, 1 << 30, null, null)
    assert rc == -1


def test_wait_limit_rejects_negative_before_cuda_work(lib):
    so = lib.load()
    assert so.eik_set_wait_limit(-1) == -1
    assert "iterations" in lib.eik_last_error()


def test_noalloc_scratch_size_matches_header(lib):
    """The binding's size check mirrors the header's #define."""
    hdr = open(os.path.join(ROOT, "include", "eik.h")).read()
    m = re.search(r"#define\s+EIK_NOALLOC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", hdr)
    assert m, "EIK_NOALLOC_SCRATCH_BYTES not found in eik.h"
    assert lib.NOALLOC_SCRATCH_BYTES == int(m.group(1)) << int(m.group(2))


def test_one_dimensional_requests(lib):
    """1-D grids go to the Sec. 3.1 solve: a valid request needs a few kB
    (control words, U, W and the end copies); coarse_ratio must be the
    subinterval width, at most 2048 subintervals, no per-node weight; the
    other entry points reject 1-D."""
    g = lib.Grid(1, 1, (ctypes.c_int64 * 3)(1001, 1, 1), (ctypes.c_int64 * 3)(1, 1001, 1001), 1e-3)
    assert 0 < lib.eik_dd_workspace_size(g, lib.dd_params((10,), 100)) <= 4096
    assert lib.eik_dd_workspace_size(g, lib.dd_params((10,), 50)) == 0
    assert "coarse_ratio" in lib.eik_last_error()
    assert lib.eik_dd_workspace_size(g, lib.dd_params((7,), 100)) == 0
    assert lib.eik_dd_workspace_size(g, lib.dd_params((10,), 100, theta_adaptive=True)) == 0
    big = lib.Grid(1, 0, (ctypes.c_int64 * 3)(2049 * 2 + 1, 1, 1), (ctypes.c_int64 * 3)(1, 1, 1), 1e-3)
    assert lib.eik_dd_workspace_size(big, lib.dd_params((2049,), 2)) == 0
    assert "2048" in lib.eik_last_error()
    ok = lib.Grid(1, 0, (ctypes.c_int64 * 3)(2048 * 2 + 1, 1, 1), (ctypes.c_int64 * 3)(1, 1, 1), 1e-3)
    assert 0 < lib.eik_dd_workspace_size(ok, lib.dd_params((2048,), 2)) <= 64 * 1024
    assert lib.eik_fsm_workspace_size(g) == 0
    with pytest.raises(lib.EikError, match="2-D"):
        lib.eik_dd_shard_exchange_bytes(g, lib.dd_params((10,), 100))
