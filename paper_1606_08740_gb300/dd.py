"""Domain decomposition of one stencil system over ranks (include/aar_dd.h): the slab plan and two
implementations of the communication the library calls back for.

The paper's parallel runs (Sec. 3.2, 3.3) give every process a subdomain: each sweep exchanges the
ghost region a stencil reaches, and each Anderson step makes one global reduction. Here a rank
owns a slab of whole z-planes; the library runs the iteration on the rank's GPU and calls back
for the two exchanges:

* ``slab_bounds`` / ``neighbours``: cut nz planes into ``world`` slabs (sizes differ by at most
  one, each at least the stencil radius) and name each slab's neighbours (periodic grids wrap).
* ``TorchDistComm``: halo exchange and sum over ranks through ``torch.distributed``, one rank per
  process (NCCL for CUDA tensors; gloo for CPU tensors).
* ``LocalGroup``: several slabs held by one process, one host thread per slab, exchanging by
  device copies between the slabs' buffers after a host barrier (no kernel waits on another).

This module moves bytes between ranks only: every step of the iteration runs in the library.
"""
from __future__ import annotations

import threading


def slab_bounds(nz: int, world: int, rank: int, radius: int = 1) -> tuple[int, int]:
    """[z_lo, z_hi) of rank's slab: nz planes in `world` consecutive slabs whose sizes differ by at
    most one. Raises ValueError when a slab would hold fewer than `radius` planes (its ghost
    planes would then span more than one neighbour)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    if nz < world * radius:
        raise ValueError(f"{nz} planes cannot give {world} slabs of at least {radius} planes")
    base, extra = divmod(nz, world)
    z_lo = rank * base + min(rank, extra)
    return z_lo, z_lo + base + (1 if rank < extra else 0)


def neighbours(rank: int, world: int, periodic: bool) -> tuple[int | None, int | None]:
    """(rank below, rank above); None where a zero Dirichlet end has no neighbour. On a periodic
    grid the lowest and highest slabs are neighbours (a single slab is its own)."""
    lo = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    hi = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return lo, hi


class _DevArray:
    """A device buffer given by pointer, as a __cuda_array_interface__ for torch.as_tensor."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "strides": None, "version": 3}


def _dev_tensor(ptr: int, n: int):
    import torch

    return torch.as_tensor(_DevArray(ptr, n), device="cuda")


def _stream(stream: int):
    import torch

    return torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()


# message tags: a slab's highest planes travel up (into the ghost planes below the slab above),
# its lowest planes travel down; every rank posts the upward pair first, so that two ranks that
# are each other's neighbours on both sides (two slabs of a periodic grid) match in order
_UP, _DOWN = 1, 2


class TorchDistComm:
    """Halo exchange and sum over ranks through torch.distributed (the default process group):
    one rank per process, NCCL for CUDA tensors, gloo for CPU tensors. The tensor-level methods
    work on any device; ``halo`` / ``allreduce`` are the library's callbacks (raw device pointers,
    ordered on the library's stream)."""

    def __init__(self, periodic: bool, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.lo, self.hi = neighbours(self.rank, self.world, periodic)

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi) -> None:
        """recv_lo <- the highest planes of the slab below, recv_hi <- the lowest planes of the slab
        above (untouched where there is no neighbour)."""
        dist = self.dist
        if self.world == 1:  # a periodic grid in one slab is its own neighbour on both sides
            if self.lo is not None:
                recv_lo.copy_(send_hi)
                recv_hi.copy_(send_lo)
            return
        peer = (lambda r: dist.get_global_rank(self.group, r)) if self.group is not None else (lambda r: r)
        ops = []
        if self.hi is not None:
            ops.append(dist.P2POp(dist.isend, send_hi, peer(self.hi), self.group, _UP))
        if self.lo is not None:
            ops.append(dist.P2POp(dist.irecv, recv_lo, peer(self.lo), self.group, _UP))
        if self.lo is not None:
            ops.append(dist.P2POp(dist.isend, send_lo, peer(self.lo), self.group, _DOWN))
        if self.hi is not None:
            ops.append(dist.P2POp(dist.irecv, recv_hi, peer(self.hi), self.group, _DOWN))
        for req in dist.batch_isend_irecv(ops):
            req.wait()

    def sum_(self, t) -> None:
        """t <- sum of t over ranks (the same values on every rank)."""
        self.dist.all_reduce(t, group=self.group)

    # ---- the library's callbacks (include/aar_dd.h)
    def halo(self, send_lo: int, send_hi: int, recv_lo: int, recv_hi: int, count: int, stream: int) -> None:
        import torch

        with torch.cuda.stream(_stream(stream)):
            self.exchange(_dev_tensor(send_lo, count), _dev_tensor(send_hi, count), _dev_tensor(recv_lo, count),
                          _dev_tensor(recv_hi, count))

    def allreduce(self, buf: int, count: int, stream: int) -> None:
        import torch

        with torch.cuda.stream(_stream(stream)):
            self.sum_(_dev_tensor(buf, count))


class LocalGroup:
    """Slabs of one grid solved by one process, one host thread per slab (for example several
    slabs on one GPU). Each exchange first makes every slab's stream finish the work queued before
    the call, then meets the other threads at a host barrier, then copies device to device."""

    def __init__(self, world: int, periodic: bool, timeout: float = 120.0):
        self.world = world
        self.periodic = periodic
        # a slab whose solve ended early leaves the others waiting: they give up after `timeout`
        # seconds (threading.BrokenBarrierError, which fails their callback: AAR_ERR_COMM)
        self.barrier = threading.Barrier(world, timeout=timeout)
        self.posted = [None] * world
        self.total = None

    def comm(self, rank: int) -> "LocalComm":
        return LocalComm(self, rank)


class LocalComm:
    def __init__(self, group: LocalGroup, rank: int):
        self.g = group
        self.rank = rank
        self.lo, self.hi = neighbours(rank, group.world, group.periodic)

    def halo(self, send_lo: int, send_hi: int, recv_lo: int, recv_hi: int, count: int, stream: int) -> None:
        import torch

        g, st = self.g, _stream(stream)
        st.synchronize()  # x_k of this slab is complete (and the previous exchange's copies are)
        g.posted[self.rank] = (send_lo, send_hi)
        g.barrier.wait()
        with torch.cuda.stream(st):
            if self.lo is not None:
                _dev_tensor(recv_lo, count).copy_(_dev_tensor(g.posted[self.lo][1], count))
            if self.hi is not None:
                _dev_tensor(recv_hi, count).copy_(_dev_tensor(g.posted[self.hi][0], count))
        st.synchronize()
        g.barrier.wait()  # every slab has read `posted` before it is replaced

    def allreduce(self, buf: int, count: int, stream: int) -> None:
        import torch

        g, st = self.g, _stream(stream)
        st.synchronize()
        g.posted[self.rank] = buf
        g.barrier.wait()
        if self.rank == 0:  # the sum in rank order, once, so that every slab gets the same values
            tot = _dev_tensor(g.posted[0], count).clone()
            for r in range(1, g.world):
                tot += _dev_tensor(g.posted[r], count)
            torch.cuda.current_stream().synchronize()
            g.total = tot
        g.barrier.wait()
        with torch.cuda.stream(st):
            _dev_tensor(buf, count).copy_(g.total)
        st.synchronize()
        g.barrier.wait()
