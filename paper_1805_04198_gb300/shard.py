"""Slab-sharded 2-D DD solve over several processes (one GPU each).

The subdomain solves of an iteration (Steps 2-3 of Sec. 3.2, independent for
every subdomain) are split by slabs of subdomain rows; every process keeps the
whole coarse state and runs Alg. 4, Step 4 and the causal sweep (Alg. 2) on it.
Per iteration each process solves its slab's subdomains, the processes
all-gather the subdomains' coarse-set copies (one record per subdomain, a slab's
records contiguous), and each runs the coarse phase on identical data, so the
update size that stops the iteration is identical on every process and needs no
reduction.  At the end the processes all-gather their slabs' rows of the fine
solution.

The kernels are libeik's (eik_dd_shard_start / _fine / _coarse, include/eik.h);
this module only partitions, moves bytes between processes
(torch.distributed) and drives the loop.
"""
from __future__ import annotations

import torch

from . import eik


def slab_rows(ty: int, world: int, rank: int):
    """Subdomain rows [row0, row1) of `rank` when ty rows are split over
    `world` processes as evenly as possible (the first ty % world slabs get
    one row more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    base, extra = divmod(ty, world)
    row0 = rank * base + min(rank, extra)
    return row0, row0 + base + (1 if rank < extra else 0)


def _pad_rows(ty: int, world: int) -> int:
    return -(-ty // world)


def allgather_records(xbuf: torch.Tensor, record_bytes: int, tx: int, ty: int, rank: int, world: int,
                      group=None) -> None:
    """Every slab's records into every process's xbuf.

    xbuf (uint8, tx * ty * record_bytes) holds this rank's slab at its own
    offset; after the call it holds every slab.  Slabs may differ by one row,
    so each is sent padded to the largest slab (all_gather_into_tensor wants
    equal parts)."""
    import torch.distributed as dist
    per_slab = _pad_rows(ty, world) * tx * record_bytes
    row0, row1 = slab_rows(ty, world, rank)
    send = torch.zeros(per_slab, dtype=torch.uint8, device=xbuf.device)
    n = (row1 - row0) * tx * record_bytes
    send[:n] = xbuf[row0 * tx * record_bytes: row1 * tx * record_bytes]
    recv = torch.empty(world * per_slab, dtype=torch.uint8, device=xbuf.device)
    dist.all_gather_into_tensor(recv, send, group=group)
    for q in range(world):
        a, b = slab_rows(ty, world, q)
        m = (b - a) * tx * record_bytes
        xbuf[a * tx * record_bytes: b * tx * record_bytes] = recv[q * per_slab: q * per_slab + m]


def band_rows(ty: int, sy: int, ny: int, world: int, rank: int):
    """Grid rows [y0, y1) that `rank` contributes to the assembled solution:
    its slab's rows, the slab's top boundary row (a coarse line, equal on every
    process) left to the slab above, except for the last slab."""
    row0, row1 = slab_rows(ty, world, rank)
    y0, y1 = row0 * sy, row1 * sy
    return y0, (ny if row1 == ty else y1)


def allgather_rows(u: torch.Tensor, ty: int, sy: int, rank: int, world: int, group=None) -> torch.Tensor:
    """The full solution from each process's band of rows of u (shape (ny, nx))."""
    import torch.distributed as dist
    ny, nx = u.shape
    rows_max = _pad_rows(ty, world) * sy + 1
    y0, y1 = band_rows(ty, sy, ny, world, rank)
    send = torch.zeros(rows_max, nx, dtype=u.dtype, device=u.device)
    send[: y1 - y0] = u[y0:y1]
    recv = torch.empty(world * rows_max, nx, dtype=u.dtype, device=u.device)
    dist.all_gather_into_tensor(recv, send, group=group)
    out = torch.empty_like(u)
    for q in range(world):
        a, b = band_rows(ty, sy, ny, world, q)
        out[a:b] = recv[q * rows_max: q * rows_max + (b - a)]
    return out


class ShardedDD:
    """One 2-D DD solve whose subdomain solves are split over the processes of
    a torch.distributed group (this process: rank `rank` of `world`, its GPU
    the device of r).

    exchange(xbuf, record_bytes) moves every slab's records into xbuf; the
    default all-gathers them over `group` (a NCCL group with device tensors; a
    gloo group gets host copies)."""

    def __init__(self, r, gamma, g, h, tiles, coarse_ratio, rank, world, group=None, exchange=None, **params):
        eik._check_like(r, g)
        self.r, self.gamma, self.g = r, gamma.contiguous(), g
        self.tiles, self.c = tuple(tiles), coarse_ratio
        self.rank, self.world, self.group = rank, world, group
        self.grid = eik.make_grid(r, h)
        self.params = eik.dd_params(tiles, coarse_ratio, **params)
        self.max_iter = self.params.max_iter
        nbytes = eik.eik_dd_workspace_size(self.grid, self.params)
        if nbytes == 0:
            raise eik.EikError(-1, eik.eik_last_error())
        self.ws = eik._workspace(nbytes, r.device)
        xbytes, self.record_bytes = eik.eik_dd_shard_exchange_bytes(self.grid, self.params)
        self.xbuf = torch.zeros(xbytes, dtype=torch.uint8, device=r.device)
        self.u = torch.empty_like(r)
        self.stats = torch.zeros(eik.ctypes.sizeof(eik.DDStats), dtype=torch.uint8, device=r.device)
        self.rows = slab_rows(tiles[1], world, rank)
        self._exchange = exchange or self._allgather

    def _allgather(self, xbuf, record_bytes):
        import torch.distributed as dist
        tx, ty = self.tiles
        if dist.get_backend(self.group) == "gloo" and xbuf.is_cuda:
            host = xbuf.cpu()
            allgather_records(host, record_bytes, tx, ty, self.rank, self.world, self.group)
            xbuf.copy_(host)
        else:
            allgather_records(xbuf, record_bytes, tx, ty, self.rank, self.world, self.group)

    def start(self):
        eik.eik_dd_shard_start(self.grid, self.r, self.gamma, self.g, self.params, self.u, self.ws)

    def fine(self):
        eik.eik_dd_shard_fine(self.grid, self.r, self.gamma, self.g, self.params, self.u, self.ws, self.rows[0],
                              self.rows[1], self.xbuf)

    def coarse(self, k) -> dict:
        eik.eik_dd_shard_coarse(self.grid, self.r, self.gamma, self.g, self.params, self.u, self.ws, k, self.xbuf,
                                self.stats)
        return eik.parse_dd_stats(self.stats)

    def run(self):
        """Returns (u of this process: all coarse-set nodes and its slab's
        nodes, statistics)."""
        self.start()
        st = None
        for k in range(self.max_iter + 1):
            self.fine()
            self._exchange(self.xbuf, self.record_bytes)
            st = self.coarse(k)
            if st["converged"] or st["error"] or k == self.max_iter:
                break
        if st["error"]:
            raise eik.EikError(st["error"], "device-side wait expired")
        return self.u, st

    def gather(self, u=None):
        """The full solution on every process (all-gather of the slabs' rows)."""
        import torch.distributed as dist
        u = self.u if u is None else u
        sy = (u.shape[0] - 1) // self.tiles[1]
        if dist.get_backend(self.group) == "gloo" and u.is_cuda:
            return allgather_rows(u.cpu(), self.tiles[1], sy, self.rank, self.world, self.group).to(u.device)
        return allgather_rows(u, self.tiles[1], sy, self.rank, self.world, self.group)
