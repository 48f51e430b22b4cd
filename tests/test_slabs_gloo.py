"""The y-slab halo exchange protocol over a torch.distributed process group,
on CPU with gloo (world sizes 2 and 3, periodic rings and walled ends): each
rank holds its slab's populations as a host array whose values name their
global row, population and column; after one exchange every halo row holds,
for the populations that cross into it, the neighbour's row it stands for.
The packing here follows the layout that include/lbm13.h states for
lbm13_halo_pack / lbm13_halo_unpack ([2 rows][4 populations][nx]; rows 2, 3 /
ny-4, ny-3 packed; rows 0, 1 / ny-2, ny-1 unpacked; v_y > 0 populations
cross northwards, v_y < 0 southwards)."""
import os
import socket

import numpy as np
import pytest

from paper_1401_0188_gb300 import slabs

UP = (2, 5, 6, 10)     # v_y > 0
DOWN = (4, 7, 8, 12)   # v_y < 0
NX = 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _value(grow, j, x):
    return 1000.0 * grow + 10.0 * j + 0.01 * x


def _rank(rank, world, ny, periodic, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        y0, y1 = slabs.split_rows(ny, world)[rank]
        hs, hn = slabs.slab_sides(world, periodic, rank)
        rows = slabs.global_rows(ny, y0, y1, hs, hn)
        n = len(rows)
        f = np.full((13, n, NX), np.nan)
        lo = 2 if hs else 0
        for r in range(lo, lo + (y1 - y0)):  # only the slab's own rows are known
            for j in range(13):
                f[j, r] = [_value(rows[r], j, x) for x in range(NX)]

        def pack(side):
            src = (2, 3) if side == slabs.SOUTH else (n - 4, n - 3)
            planes = DOWN if side == slabs.SOUTH else UP
            return torch.tensor(np.array([[f[j, r] for j in planes] for r in src]))

        def unpack(side, buf):
            dst = (0, 1) if side == slabs.SOUTH else (n - 2, n - 1)
            planes = UP if side == slabs.SOUTH else DOWN
            b = buf.numpy()
            for i, r in enumerate(dst):
                for k, j in enumerate(planes):
                    f[j, r] = b[i, k]

        slabs.exchange_over_group(rank, world, periodic, pack, unpack,
                                  lambda: torch.empty((2, 4, NX), dtype=torch.float64), dist)
        bad = []
        for side, rr, planes in ((slabs.SOUTH, (0, 1), UP), (slabs.NORTH, (n - 2, n - 1), DOWN)):
            if not (hs if side == slabs.SOUTH else hn):
                continue
            for r in rr:
                for j in planes:
                    want = [_value(rows[r], j, x) for x in range(NX)]
                    if not np.array_equal(f[j, r], want):
                        bad.append((side, r, j))
        q.put((rank, bad))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, True), (2, False), (3, True), (3, False)])
def test_halo_exchange_over_gloo(world, periodic):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ny = 4 * world + 3
    procs = [ctx.Process(target=_rank, args=(r, world, ny, periodic, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(not bad for _, bad in out), out


def test_slab_layout():
    assert slabs.split_rows(10, 2) == [(0, 5), (5, 10)]
    with pytest.raises(ValueError):
        slabs.split_rows(7, 2)
    assert slabs.exchange_pairs(3, False) == [(0, 1), (1, 2)]
    assert slabs.exchange_pairs(3, True) == [(0, 1), (1, 2), (2, 0)]
    assert slabs.neighbours(0, 3, False) == (None, 1)
    assert slabs.neighbours(2, 3, True) == (1, 0)
    assert slabs.slab_sides(3, False, 0) == (False, True)
    assert slabs.slab_sides(1, True, 0) == (True, True)
    assert slabs.global_rows(10, 0, 5, True, True) == [8, 9, 0, 1, 2, 3, 4, 5, 6]
