"""y-slab decomposition of one lattice with a two-row halo exchange per step.

An nx x ny lattice is split along y into K slabs of consecutive rows.  Slab k
holds its own rows plus two halo rows beyond each side that touches another
slab (LBM13_HALO): copies of the neighbour's two rows next to the boundary.
The D2Q13 stencil reaches two rows (Sec. 2: the (0, +-2) links), so two rows
carry everything a step pulls across a boundary, and only the four
populations whose v_y points across it need to move: after each step the
lower slab packs its top two rows of v_y > 0 populations for the upper slab's
south halo, and the upper slab packs its bottom two rows of v_y < 0
populations for the lower slab's north halo (lbm13_halo_pack / _unpack).  A
periodic y axis closes the slabs into a ring; walls at the bottom and top
stay with the first and last slab.  The step never writes halo rows and pulls
from them like any row, so the slabs reproduce the undivided lattice bit for
bit.

`SlabLattice` runs the K slabs on one device, in stream order; `RankSlab` is
the per-rank side of the same exchange over a torch.distributed process group
(one slab per rank, each on its own device), moving the packed halos by
send/recv.  `exchange_over_group` is that protocol with the packing passed in,
so the host logic can run on CPU tensors.
"""
from . import lbm13

SOUTH, NORTH = lbm13.HALO_SOUTH, lbm13.HALO_NORTH
TAG_UP, TAG_DOWN = 1, 2  # halo data moving to the slab above / below


def split_rows(ny, K):
    """Interior row ranges [(y0, y1), ...] of K slabs, as even as possible."""
    if K < 1 or ny < 4 * K:
        raise ValueError("need K >= 1 and at least four rows per slab")
    edges = [ny * k // K for k in range(K + 1)]
    return [(edges[k], edges[k + 1]) for k in range(K)]


def slab_sides(K, periodic, k):
    """(south is a halo side, north is a halo side) of slab k."""
    return (periodic or k > 0), (periodic or k < K - 1)


def exchange_pairs(K, periodic):
    """(lower, upper) slab pairs whose boundary is exchanged after a step."""
    pairs = [(k, k + 1) for k in range(K - 1)]
    if periodic:
        pairs.append((K - 1, 0))
    return pairs


def neighbours(rank, world, periodic):
    """(south neighbour, north neighbour) of a rank's slab (None at a wall)."""
    south = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    north = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return south, north


def slab_boundary(bnd, halo_south, halo_north):
    """The slab's boundary description: the global one with the sides it
    shares with a neighbour turned into halo sides."""
    b = dict(bnd)
    if halo_south:
        b["south"] = {"kind": lbm13.HALO, "u_t": 0.0, "T": 0.0}
    if halo_north:
        b["north"] = {"kind": lbm13.HALO, "u_t": 0.0, "T": 0.0}
    return b


def global_rows(ny, y0, y1, halo_south, halo_north):
    """Global row of each local row of a slab (halo rows wrap around for a
    periodic axis)."""
    lo = y0 - (2 if halo_south else 0)
    hi = y1 + (2 if halo_north else 0)
    return [y % ny for y in range(lo, hi)]


class SlabLattice:
    """K y-slabs of one nx x ny lattice on one device, stepped in stream
    order with a halo exchange after every step."""

    def __init__(self, nx, ny, K, params, bnd=None, precision=lbm13.FP64, stream=None):
        import torch
        bnd = bnd if bnd is not None else lbm13.boundary()
        self.nx, self.ny, self.K, self.precision = nx, ny, K, precision
        self.periodic = bnd["south"]["kind"] == lbm13.PERIODIC
        self.rows = split_rows(ny, K)
        self.sides = [slab_sides(K, self.periodic, k) for k in range(K)]
        self.slabs = []
        for k, ((y0, y1), (hs, hn)) in enumerate(zip(self.rows, self.sides)):
            n = (y1 - y0) + 2 * hs + 2 * hn
            self.slabs.append(lbm13.Lattice(nx, n, params, slab_boundary(bnd, hs, hn), precision=precision,
                                            stream=stream))
        nbytes = self.slabs[0].halo_bytes()
        dev = torch.device("cuda", self.slabs[0].device)
        self.pairs = exchange_pairs(K, self.periodic)
        self._bufs = [(torch.empty(nbytes, dtype=torch.uint8, device=dev),
                       torch.empty(nbytes, dtype=torch.uint8, device=dev)) for _ in self.pairs]

    def close(self):
        for s in self.slabs:
            s.close()

    def _local(self, k, field):
        import numpy as np
        (y0, y1), (hs, hn) = self.rows[k], self.sides[k]
        if field is None:
            return None
        a = np.broadcast_to(np.asarray(field, dtype=np.float64), (self.ny, self.nx))
        return np.ascontiguousarray(a[global_rows(self.ny, y0, y1, hs, hn)])

    def set_state(self, rho=None, ux=None, uy=None, T=None):
        """Equilibrium of global (ny, nx) fields (None = rest value); every
        slab, halo rows included, starts from its global rows."""
        for k, s in enumerate(self.slabs):
            s.set_state(*(self._local(k, f) for f in (rho, ux, uy, T)))

    def exchange(self):
        for (lo, up), (b_up, b_down) in zip(self.pairs, self._bufs):
            self.slabs[lo].halo_pack(NORTH, b_up)
            self.slabs[up].halo_unpack(SOUTH, b_up)
            self.slabs[up].halo_pack(SOUTH, b_down)
            self.slabs[lo].halo_unpack(NORTH, b_down)

    def step(self, n=1):
        for _ in range(int(n)):
            for s in self.slabs:
                s.step(1)
            self.exchange()

    @property
    def t(self):
        return self.slabs[0].t

    def _assemble(self, parts):
        import numpy as np
        out = []
        for (y0, y1), (hs, hn), a in zip(self.rows, self.sides, parts):
            lo = 2 if hs else 0
            out.append(a[:, lo:lo + (y1 - y0)])
        return np.concatenate(out, axis=1)

    def raw_state(self):
        """Stored populations of the whole lattice, [13][ny][nx] (interior rows of every slab)."""
        return self._assemble([s.get_raw_state() for s in self.slabs])

    def moments(self, mask=lbm13.ALL_MOMENTS):
        return self._assemble([s.moments(mask) for s in self.slabs])


def exchange_over_group(rank, world, periodic, pack, unpack, new_buffer, dist, group=None):
    """One halo exchange of rank's slab with its neighbours over a process
    group: pack(side) returns the packed rows next to halo side `side`,
    unpack(side, buf) writes a neighbour's packed rows into that halo,
    new_buffer() returns a receive buffer; dist is torch.distributed.  The
    operations are posted in one canonical order -- sends up then down,
    receives from below then from above -- so that transports that match
    messages between two ranks by order (NCCL) pair them correctly even in a
    ring of two, where each rank is the other's north and south neighbour;
    the tags say the same for transports that match by tag."""
    south, north = neighbours(rank, world, periodic)
    if world == 1:
        if periodic:  # a ring of one slab: its own rows feed its halos
            up, down = pack(NORTH), pack(SOUTH)
            unpack(SOUTH, up)
            unpack(NORTH, down)
        return
    ops, recv = [], []
    if north is not None:
        ops.append(dist.P2POp(dist.isend, pack(NORTH), north, group, TAG_UP))
    if south is not None:
        ops.append(dist.P2POp(dist.isend, pack(SOUTH), south, group, TAG_DOWN))
    if south is not None:
        recv.append((SOUTH, new_buffer()))
        ops.append(dist.P2POp(dist.irecv, recv[-1][1], south, group, TAG_UP))
    if north is not None:
        recv.append((NORTH, new_buffer()))
        ops.append(dist.P2POp(dist.irecv, recv[-1][1], north, group, TAG_DOWN))
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    for side, buf in recv:
        unpack(side, buf)


class RankSlab:
    """This rank's slab of an nx x ny lattice split over the ranks of a
    torch.distributed group (slab k on rank k, each rank on its own CUDA
    device), with the halos moved by send/recv after every step (NCCL keeps
    them in device memory)."""

    def __init__(self, nx, ny, params, bnd=None, precision=lbm13.FP64, group=None):
        import torch
        import torch.distributed as dist
        bnd = bnd if bnd is not None else lbm13.boundary()
        self.dist, self.group = dist, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        self.nx, self.ny = nx, ny
        self.periodic = bnd["south"]["kind"] == lbm13.PERIODIC
        (self.y0, self.y1) = split_rows(ny, self.world)[self.rank]
        self.hs, self.hn = slab_sides(self.world, self.periodic, self.rank)
        n = (self.y1 - self.y0) + 2 * self.hs + 2 * self.hn
        # on torch's current stream, which also orders the transfers
        self.lattice = lbm13.Lattice(nx, n, params, slab_boundary(bnd, self.hs, self.hn), precision=precision)
        self.nbytes = self.lattice.halo_bytes()
        self.device = torch.device("cuda", self.lattice.device)

    def set_state(self, rho=None, ux=None, uy=None, T=None):
        import numpy as np
        rows = global_rows(self.ny, self.y0, self.y1, self.hs, self.hn)
        loc = [None if f is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(f, dtype=np.float64), (self.ny, self.nx))[rows]) for f in (rho, ux, uy, T)]
        self.lattice.set_state(*loc)

    def exchange(self):
        import torch

        def pack(side):
            buf = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
            self.lattice.halo_pack(side, buf)
            return buf

        def unpack(side, buf):
            self.lattice.halo_unpack(side, buf)

        exchange_over_group(self.rank, self.world, self.periodic, pack, unpack,
                            lambda: torch.empty(self.nbytes, dtype=torch.uint8, device=self.device), self.dist,
                            self.group)

    def step(self, n=1):
        for _ in range(int(n)):
            self.lattice.step(1)
            self.exchange()
