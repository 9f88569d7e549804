"""The slab-sharded DD solve (eik_dd_shard_*) on one GPU: the slabs of a
two-process solve run in one process, each with its own workspace, exchange
buffer and output, and the exchange step copies the other slab's records
between the two buffers.  The assembled solution and the statistics equal
eik_dd_solve's bitwise."""
import numpy as np
import pytest
import torch

from paper_1805_04198_gb300 import eik, inputs, shard

pytestmark = pytest.mark.gpu


def _two_slab_solve(r, gamma, g, h, tiles, c, world=2, **params):
    procs = [shard.ShardedDD(r, gamma, g, h, tiles, c, q, world, exchange=lambda x, rb: None, **params)
             for q in range(world)]
    tx, ty = tiles
    rec = procs[0].record_bytes
    for p in procs:
        p.start()
    sts = None
    for k in range(procs[0].max_iter + 1):
        for p in procs:
            p.fine()
        # the exchange: every slab's records into every buffer
        for q, src in enumerate(procs):
            a, b = shard.slab_rows(ty, world, q)
            for dst in procs:
                if dst is not src:
                    dst.xbuf[a * tx * rec: b * tx * rec] = src.xbuf[a * tx * rec: b * tx * rec]
        sts = [p.coarse(k) for p in procs]
        local = ("launches", "fine_updates", "fsm_sweeps_max", "fsm_cap_hits",  # per process: its subdomains
                 "fine_solves_skipped")
        for st in sts[1:]:
            assert {kk: v for kk, v in st.items() if kk not in local} == \
                   {kk: v for kk, v in sts[0].items() if kk not in local}
        if sts[0]["converged"] or sts[0]["error"] or k == procs[0].max_iter:
            break
    torch.cuda.synchronize()
    ny = r.shape[0]
    sy = (ny - 1) // ty
    u = torch.empty_like(r)
    for q, p in enumerate(procs):
        a, b = shard.band_rows(ty, sy, ny, world, q)
        u[a:b] = p.u[a:b]
    # coarse-set nodes are computed by every process alike
    cs = np.zeros(r.shape, bool)
    cs[::c, :] = True
    cs[:, ::c] = True
    for p in procs[1:]:
        assert torch.equal(p.u.cpu()[torch.from_numpy(cs)], procs[0].u.cpu()[torch.from_numpy(cs)])
    st = dict(sts[0])
    st["fine_updates"] = sum(x["fine_updates"] for x in sts)
    st["fsm_cap_hits"] = sum(x["fsm_cap_hits"] for x in sts)
    st["fine_solves_skipped"] = sum(x["fine_solves_skipped"] for x in sts)
    st["fsm_sweeps_max"] = max(x["fsm_sweeps_max"] for x in sts)
    return u, st


@pytest.mark.parametrize("shape,tiles,c,dtype,theta,kmax,tol", [
    ((129, 129), (4, 4), 8, torch.float64, 0.2, 5, 0.0),
    ((193, 257), (4, 6), 16, torch.float64, 0.0, 6, 0.0),    # 6 subdomain rows over 2 slabs, weight 0
    ((241, 257), (4, 5), 8, torch.float32, 0.3, 40, 1e-6),   # slabs of 3 and 2 rows, stopped by tol
])
def test_two_slabs_equal_single_solve_bitwise(shape, tiles, c, dtype, theta, kmax, tol):
    h = 1.0 / (shape[1] - 1)
    r = inputs.sin_product(shape, h, 0.5, 0.25)
    gamma, g = inputs.point_source(shape, (shape[0] // 3, shape[1] // 2))
    R = torch.from_numpy(r).to("cuda:0", dtype)
    G = torch.from_numpy(gamma).cuda()
    g_t = torch.from_numpy(g).to("cuda:0", dtype)
    kw = dict(theta=theta, max_iter=kmax, tol=tol, max_coarse_sweeps=8)
    ref, st_ref = eik.dd_solve(R, G, g_t, h, tiles, c, **kw)
    u, st = _two_slab_solve(R, G, g_t, h, tiles, c, **kw)
    for key in ("iters", "converged", "error", "fine_updates", "coarse_updates", "fsm_sweeps_max",
                "fine_solves_skipped"):
        assert st[key] == st_ref[key], key
    np.testing.assert_array_equal(u.cpu().numpy(), ref.cpu().numpy())


def test_two_slabs_benchmark_workload_bitwise():
    """The 4097^2 benchmark solve (16 x 16 subdomains, coarse ratio 16, FP32,
    weight 0, stop at 1e-6) as two slabs of 8 subdomain rows."""
    w = inputs.workload_c1()
    R = torch.from_numpy(w["r"].astype(np.float32)).cuda()
    G = torch.from_numpy(w["gamma"]).cuda()
    g_t = torch.from_numpy(w["g"].astype(np.float32)).cuda()
    kw = dict(theta=0.0, max_iter=42, tol=1e-6, max_coarse_sweeps=8)
    ref, st_ref = eik.dd_solve(R, G, g_t, w["h"], w["tiles"], w["c"], **kw)
    u, st = _two_slab_solve(R, G, g_t, w["h"], w["tiles"], w["c"], **kw)
    assert st["iters"] == st_ref["iters"] and st["converged"] == 1
    assert torch.equal(u, ref)
