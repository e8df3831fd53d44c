"""Slab decomposition of a periodic domain along its last axis (y in 2D, z in 3D).

The Sec. 6 update of a periodic domain (Sec. 2.2) cut into slabs needs, per step and face, the
populations that cross the cut: one halo exchange of `crossing` planes (D2Q5, D3Q7: 1; D3Q19: 5)
with each neighbour, before the step.  The library's slab handles (LEE_BC_SLAB, include/lee_lbm.h)
pack what leaves into send buffers and unpack what enters from recv buffers; this module moves
the messages between slabs behind a small transport interface and runs the ring:

  SlabRing.step(n):  for each step: pack -> transport.exchange -> unpack -> one step.

Transports:
  DistTransport  one slab per rank of a torch.distributed group (NCCL on GPUs, gloo on CPU):
                 batched point-to-point sends to the lower and upper neighbour ranks (periodic).
  (slabs of one process on one device need no transport here: lee_lbm_slab_step runs the whole
  ring natively, copying each message into the receiver's own buffer.)

Nothing here computes: the halo messages are opaque buffers of the storage type.
"""
from __future__ import annotations

from typing import Protocol


def partition(n_planes: int, parts: int):
    """(first plane, planes) of each of `parts` slabs of an n_planes-plane axis, as even as
    possible (the first n_planes % parts slabs get one plane more)."""
    if parts < 1 or n_planes < parts:
        raise ValueError(f"cannot cut {n_planes} planes into {parts} slabs")
    base, extra = divmod(n_planes, parts)
    out, start = [], 0
    for k in range(parts):
        count = base + (1 if k < extra else 0)
        out.append((start, count))
        start += count
    return out


class HaloSlab(Protocol):
    """What a ring needs from a slab: pack / unpack its halo messages and take one step.
    `buffers()` returns (send_lo, send_hi, recv_lo, recv_hi) as tensors of equal size."""

    def pack(self) -> None: ...

    def unpack(self) -> None: ...

    def step1(self) -> None: ...

    def buffers(self): ...


class DistTransport:
    """Moves halo messages between the ranks of a torch.distributed group, one slab per rank in
    rank order along the cut (rank r + 1 above rank r, periodic).  send_lo goes down to the
    lower neighbour's recv_hi (tag 0), send_hi up to the upper neighbour's recv_lo (tag 1); all
    four operations are posted as one batch in the same order on every rank, so that NCCL (which
    matches by order) and gloo (by tag) pair them alike, also with two ranks, where the lower and
    the upper neighbour are the same rank."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def _global(self, r):
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi) -> None:
        if self.world == 1:  # the slab is the whole periodic domain
            recv_hi.copy_(send_lo)
            recv_lo.copy_(send_hi)
            return
        dist = self.dist
        lower = self._global((self.rank - 1) % self.world)
        upper = self._global((self.rank + 1) % self.world)
        ops = [dist.P2POp(dist.isend, send_lo, lower, self.group, 0),
               dist.P2POp(dist.isend, send_hi, upper, self.group, 1),
               dist.P2POp(dist.irecv, recv_hi, upper, self.group, 0),
               dist.P2POp(dist.irecv, recv_lo, lower, self.group, 1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class SlabRing:
    """One slab and the transport to its neighbours: n steps of the decomposed domain."""

    def __init__(self, slab: HaloSlab, transport):
        self.slab = slab
        self.transport = transport

    def step(self, n: int = 1) -> None:
        for _ in range(int(n)):
            self.slab.pack()
            self.transport.exchange(*self.slab.buffers())
            self.slab.unpack()
            self.slab.step1()


class _DeviceArray:
    """A device buffer of the library exposed through __cuda_array_interface__, so that
    torch.as_tensor sees it without a copy."""

    def __init__(self, ptr: int, nelem: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (nelem,), "typestr": typestr, "data": (ptr, False), "strides": None,
                                         "version": 3}


_TYPESTR = {"f64": "<f8", "f32": "<f4", "f16": "<f2"}


class GpuSlab:
    """A library slab handle (LEE_BC_SLAB) as a HaloSlab: pack / unpack / one step on the handle's
    stream, halo buffers as torch tensors over the handle's own device memory.  Create the solver
    on torch's current stream so that NCCL transfers, which torch orders after that stream, see
    the packed data."""

    def __init__(self, solver):
        import torch

        self.sv = solver
        crossing, plane, nbytes = solver.slab_info()
        ptrs = solver.slab_buffers()
        if solver.storage == "bf16":
            tens = [torch.as_tensor(_DeviceArray(p, nbytes // 2, "<i2"), device="cuda").view(torch.bfloat16)
                    for p in ptrs]
        else:
            tens = [torch.as_tensor(_DeviceArray(p, nbytes // int(_TYPESTR[solver.storage][-1]),
                                                 _TYPESTR[solver.storage]), device="cuda") for p in ptrs]
        self._bufs = tuple(tens)

    def pack(self):
        self.sv.slab_pack()

    def unpack(self):
        self.sv.slab_unpack()

    def step1(self):
        self.sv.step(1)

    def buffers(self):
        return self._bufs
