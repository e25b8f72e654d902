"""Row-slab decomposition of one lattice over several GPUs (or several slabs on one).

The update of Sec. 3.6 is local except for streaming (Eq. streaming): a node
pulls f*_(1,0), f*_(-1,0) from its own row and f*_(0,1), f*_(0,-1) from the
rows below and above.  Cutting the lattice into horizontal slabs therefore
needs, per step and cut, the five components of f*_(0,1) of the row below the
cut (moving up) and of f*_(0,-1) of the row above it (moving down): 5 nx values
each way.  The C library keeps one halo row per neighbour and packs / unpacks
these messages (lbm_create_slab, lbm_halo_pack, lbm_halo_unpack in
include/lbm.h); this module splits the rows, names the neighbours and moves the
messages, either between ranks with torch.distributed point-to-point calls
(NCCL between GPUs, gloo on CPU) or between slabs held by one process.

Message order.  Every rank issues, in this order: its message to the slab above,
the receive from the slab below, its message to the slab below, the receive from
the slab above.  Between any two ranks the sends and receives then pair up in
issue order even when the two are each other's upper and lower neighbour (two
ranks on a periodic lattice), which is how NCCL matches point-to-point calls;
gloo additionally gets distinct tags for the two directions.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

from . import lbm as L

TAG_UP, TAG_DOWN = 11, 12


def slab_rows(ny: int, world: int, rank: int) -> Tuple[int, int]:
    """(first row, number of rows) of `rank`'s slab: rows split as evenly as possible."""
    if not (1 <= world <= ny) or not (0 <= rank < world):
        raise ValueError(f"need 1 <= world <= ny and 0 <= rank < world (ny={ny}, world={world}, rank={rank})")
    base, extra = divmod(ny, world)
    return rank * base + min(rank, extra), base + (1 if rank < extra else 0)


def neighbours(world: int, rank: int, periodic: bool) -> Tuple[Optional[int], Optional[int]]:
    """(rank below, rank above); None where a Dirichlet wall closes the lattice."""
    lower = (rank - 1) % world if (periodic or rank > 0) else None
    upper = (rank + 1) % world if (periodic or rank < world - 1) else None
    return lower, upper


def exchange(dist, rank: int, world: int, periodic: bool, to_lower, to_upper, from_lower, from_upper, group=None):
    """Send this rank's halo messages and receive its neighbours' (tensors, or None where
    there is no neighbour).  With one rank on a periodic lattice the slab is its own
    neighbour and the messages are copied locally."""
    lower, upper = neighbours(world, rank, periodic)
    if (to_lower is None) != (lower is None) or (to_upper is None) != (upper is None):
        raise ValueError("a message is needed exactly for each neighbour")
    if world == 1:
        if lower is not None:
            from_lower.copy_(to_upper)
            from_upper.copy_(to_lower)
        return
    ops = []
    if upper is not None:
        ops.append(dist.P2POp(dist.isend, to_upper, upper, group, TAG_UP))
    if lower is not None:
        ops.append(dist.P2POp(dist.irecv, from_lower, lower, group, TAG_UP))
    if lower is not None:
        ops.append(dist.P2POp(dist.isend, to_lower, lower, group, TAG_DOWN))
    if upper is not None:
        ops.append(dist.P2POp(dist.irecv, from_upper, upper, group, TAG_DOWN))
    for w in dist.batch_isend_irecv(ops):
        w.wait()


class Slab:
    """One slab's C context and its four message buffers (device memory)."""

    def __init__(self, nx, ny, dx, dt, cK, cmu, y_begin, rows, dirichlet=False, storage="f64",
                 track_displacement=False, stream=None, device=None):
        import torch
        self.nx, self.ny, self.y0, self.rows = int(nx), int(ny), int(y_begin), int(rows)
        self.periodic = not dirichlet
        st = L.STORAGE[storage] if isinstance(storage, str) else storage
        self.ctx = L.lbm_create_slab(nx, ny, dx, dt, cK, cmu, y_begin, rows,
                                     L.LBM_DIRICHLET if dirichlet else L.LBM_PERIODIC, st, track_displacement, stream)
        nb = L.lbm_halo_bytes(self.ctx)
        has_lo = not (dirichlet and y_begin == 0)
        has_hi = not (dirichlet and y_begin + rows == ny)
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        mk = (lambda: torch.empty(nb, dtype=torch.uint8, device=dev))
        self.to_lower = mk() if has_lo else None
        self.to_upper = mk() if has_hi else None
        self.from_lower = mk() if has_lo else None
        self.from_upper = mk() if has_hi else None

    def close(self):
        if self.ctx is not None:
            L.lbm_destroy(self.ctx)
            self.ctx = None

    def init(self, U0, dU0dx, dU0dy, u0=None):
        """Initial data of the slab's own rows, [5][rows][nx] (u0: [2][rows][nx])."""
        L.lbm_init(self.ctx, U0, dU0dx, dU0dy, None, u0)

    def pack(self):
        L.lbm_halo_pack(self.ctx, self.to_lower, self.to_upper)

    def unpack(self):
        L.lbm_halo_unpack(self.ctx, self.from_lower, self.from_upper)

    def step1(self):
        L.lbm_step(self.ctx, 1)

    def moments(self, out=None):
        import numpy as np
        if out is None:
            out = np.empty((10, self.rows, self.nx))
        L.lbm_moments(self.ctx, out)
        return out

    def energy(self) -> float:
        return L.lbm_energy(self.ctx)


def step_local(slabs: Sequence[Slab], n: int = 1):
    """Advance slabs that tile one lattice and live in this process (listed bottom to top)
    by n steps: pack, hand each message to its neighbour, unpack, step."""
    k = len(slabs)
    periodic = slabs[0].periodic
    for _ in range(n):
        for s in slabs:
            s.pack()
        for i, s in enumerate(slabs):
            lo, hi = neighbours(k, i, periodic)
            if lo is not None:
                s.from_lower.copy_(slabs[lo].to_upper)
            if hi is not None:
                s.from_upper.copy_(slabs[hi].to_lower)
        for s in slabs:
            s.unpack()
        for s in slabs:
            s.step1()


class DistributedSlab(Slab):
    """This rank's slab of an nx x ny lattice split over the ranks of a process group; the
    halo messages travel by torch.distributed point-to-point calls.  The context's stream
    must be torch's current stream, so that the calls are ordered after the pack."""

    def __init__(self, dist, nx, ny, dx, dt, cK, cmu, dirichlet=False, storage="f64", group=None, **kw):
        import torch
        self.dist, self.group = dist, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        y0, rows = slab_rows(ny, self.world, self.rank)
        super().__init__(nx, ny, dx, dt, cK, cmu, y0, rows, dirichlet, storage,
                         stream=torch.cuda.current_stream().cuda_stream, **kw)

    def step(self, n: int = 1):
        for _ in range(n):
            self.pack()
            exchange(self.dist, self.rank, self.world, self.periodic, self.to_lower, self.to_upper,
                     self.from_lower, self.from_upper, self.group)
            self.unpack()
            self.step1()

    def global_energy(self) -> float:
        """||f||_P^2 of the whole lattice: the slabs' sums added over the ranks (FP64)."""
        import torch
        t = torch.tensor([self.energy()], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, group=self.group)
        return float(t.item())


def row_block(a, y0: int, rows: int):
    """Rows [y0, y0 + rows) of a field array [..., ny, nx] (a helper for slab inputs)."""
    return a[..., y0:y0 + rows, :]


__all__: List[str] = ["slab_rows", "neighbours", "exchange", "Slab", "step_local", "DistributedSlab", "row_block"]
