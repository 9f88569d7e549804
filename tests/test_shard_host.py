"""Host logic of the slab-sharded DD solve on CPU: the partition of subdomain
rows, the all-gather of the subdomains' exchange records (slabs of unequal
size) and the assembly of the solution from each process's rows, with two gloo
ranks."""
import os
import socket
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1805_04198_gb300 import shard  # noqa: E402


def test_slab_rows_partition_every_row_once():
    for ty in range(1, 21):
        for world in range(1, 6):
            slabs = [shard.slab_rows(ty, world, q) for q in range(world)]
            assert slabs[0][0] == 0 and slabs[-1][1] == ty
            for (a0, a1), (b0, b1) in zip(slabs, slabs[1:]):
                assert a1 == b0
            sizes = [b - a for a, b in slabs]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


def test_band_rows_cover_the_grid_once():
    for ty, sy in ((5, 4), (16, 256), (7, 3)):
        ny = ty * sy + 1
        for world in (1, 2, 3):
            bands = [shard.band_rows(ty, sy, ny, world, q) for q in range(world)]
            covered = np.zeros(ny, int)
            for a, b in bands:
                covered[a:b] += 1
            assert np.all(covered == 1)


TX, TY, REC, SY, NX = 3, 5, 48, 4, 9


def _record_byte(tile, j):
    return (tile * 7 + j) % 251 + 1


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # exchange records: this rank fills its own slab, the rest is garbage
        xbuf = torch.full((TX * TY * REC,), 200 + rank, dtype=torch.uint8)
        row0, row1 = shard.slab_rows(TY, world, rank)
        for t in range(row0 * TX, row1 * TX):
            xbuf[t * REC:(t + 1) * REC] = torch.tensor([_record_byte(t, j) for j in range(REC)], dtype=torch.uint8)
        shard.allgather_records(xbuf, REC, TX, TY, rank, world)
        want = torch.tensor([_record_byte(t, j) for t in range(TX * TY) for j in range(REC)], dtype=torch.uint8)
        ok_records = bool(torch.equal(xbuf, want))
        # solution rows: this rank's band holds 1000 * y + x, other rows garbage
        ny = TY * SY + 1
        yy, xx = torch.meshgrid(torch.arange(ny, dtype=torch.float64), torch.arange(NX, dtype=torch.float64),
                                indexing="ij")
        full = 1000 * yy + xx
        u = torch.full((ny, NX), -7.0 - rank, dtype=torch.float64)
        a, b = shard.band_rows(TY, SY, ny, world, rank)
        u[a:b] = full[a:b]
        got = shard.allgather_rows(u, TY, SY, rank, world)
        out[rank] = (ok_records, bool(torch.equal(got, full)), (row0, row1))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_exchange_records_and_rows():
    """Slabs of 3 and 2 subdomain rows: every rank ends with every subdomain's
    record at its offset and with the whole solution."""
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][2] == (0, 3) and out[1][2] == (3, 5)
    for q in range(world):
        assert out[q][0], "records of rank %d" % q
        assert out[q][1], "rows of rank %d" % q
