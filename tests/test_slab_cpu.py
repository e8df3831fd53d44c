"""Slab decomposition on CPU: the ring and its torch.distributed transport with 2 and 3 gloo ranks,
each rank owning one slab of a periodic domain cut along its last axis.

The slabs here are a test double that holds the library's state convention (post-collision
populations, Sec. 6 pull form): a step pulls every population from x - c_i -- across the cut from
the halo planes the transport filled -- and collides with the oracle.  The gathered field after n
steps must equal the oracle's own run of the whole periodic domain bit for bit (FP64, the same
per-cell arithmetic), which holds only if the partition, the neighbour pairing, the message
contents and the halo placement are all right.  The GPU slabs are checked the same way on one
GPU (tests/test_gpu_slab.py)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1601_08103_gb300 import inputs, slab


class OracleSlab:
    """Planes start .. start + count - 1 (along the last axis) of a periodic grid `shape`."""

    def __init__(self, name, shape, tau, g_post, start, count):
        import torch

        s = oracle.velset(name)
        self.name, self.tau, self.s = name, tau, s
        nx, ny, nz = shape
        self.dims = (nz, ny, nx) if s.D == 3 else (ny, nx)  # cut axis first (after the velocity axis)
        full = g_post.reshape((s.q,) + self.dims)
        self.own = full[:, start:start + count].copy()
        self.cut = s.c[:, s.D - 1]
        self.lo_ids = [i for i in range(s.q) if self.cut[i] == -1]  # leave downward
        self.hi_ids = [i for i in range(s.q) if self.cut[i] == 1]   # leave upward
        plane = int(np.prod(self.dims[1:]))
        n = len(self.hi_ids) * plane
        self.bufs = tuple(torch.zeros(n, dtype=torch.float64) for _ in range(4))
        self.halo_lo = np.zeros((s.q, 1) + self.dims[1:])
        self.halo_hi = np.zeros((s.q, 1) + self.dims[1:])

    def buffers(self):
        return self.bufs

    def pack(self):
        send_lo, send_hi = self.bufs[0].numpy(), self.bufs[1].numpy()
        send_lo[:] = np.concatenate([self.own[i, 0].ravel() for i in self.lo_ids])
        send_hi[:] = np.concatenate([self.own[i, -1].ravel() for i in self.hi_ids])

    def unpack(self):
        recv_lo, recv_hi = self.bufs[2].numpy(), self.bufs[3].numpy()
        plane = int(np.prod(self.dims[1:]))
        for k, i in enumerate(self.hi_ids):  # entering from below moves upward
            self.halo_lo[i, 0] = recv_lo[k * plane:(k + 1) * plane].reshape(self.dims[1:])
        for k, i in enumerate(self.lo_ids):
            self.halo_hi[i, 0] = recv_hi[k * plane:(k + 1) * plane].reshape(self.dims[1:])

    def step1(self):
        s = self.s
        ext = np.concatenate([self.halo_lo, self.own, self.halo_hi], axis=1)
        pulled = np.empty_like(self.own)
        for i in range(s.q):
            v = ext[i]
            # pull g_i(x - c_i): roll by +c_i along every axis; across the cut the rolled-in
            # values come from the halo planes, and whatever wraps around lands in the halos,
            # which are dropped
            axes = [0, 2, 1] if s.D == 3 else [0, 1]  # array axis of (cut, x) in 2D, (cut, x, y) in 3D
            comps = [s.c[i, s.D - 1], s.c[i, 0]] + ([s.c[i, 1]] if s.D == 3 else [])
            for ax, c in zip(axes, comps):
                if c:
                    v = np.roll(v, int(c), axis=ax)
            pulled[i] = v[1:-1]
        post = oracle.collide(self.name, self.tau, pulled.reshape(s.q, -1))
        self.own = post.reshape(self.own.shape)


def _free_port():
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    p = sk.getsockname()[1]
    sk.close()
    return p


CASES = [("D2Q5", (12, 10, 1), 0.6, 7), ("D2Q5_DI", (9, 11, 1), 0.5, 5), ("D3Q7", (6, 5, 7), 0.55, 4),
         ("D3Q19", (5, 4, 6), 0.8, 3)]


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    for ci, (name, shape, tau, n) in enumerate(CASES):
        s = oracle.velset(name)
        n_cut = shape[s.D - 1]
        rho, u, th = inputs.random_fields(shape, s.D, 70 + ci)
        g0 = oracle.equilibrium(name, rho, u, th)
        post0 = oracle.post_state(name, shape, tau, g0)  # the post-collision state at t = 0
        start, count = slab.partition(n_cut, world)[rank]
        ring = slab.SlabRing(OracleSlab(name, shape, tau, post0, start, count), slab.DistTransport())
        ring.step(n)
        np.save(os.path.join(out_dir, f"c{ci}_r{rank}.npy"), ring.slab.own)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_ring_over_gloo_equals_the_whole_domain(tmp_path, world):
    import torch.multiprocessing as mp

    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for ci, (name, shape, tau, n) in enumerate(CASES):
        s = oracle.velset(name)
        parts = [np.load(tmp_path / f"c{ci}_r{r}.npy") for r in range(world)]
        got = np.concatenate(parts, axis=1).reshape(s.q, -1)
        rho, u, th = inputs.random_fields(shape, s.D, 70 + ci)
        g = oracle.step(name, shape, tau, oracle.equilibrium(name, rho, u, th), n)
        want = oracle.post_state(name, shape, tau, g)
        assert np.array_equal(got, want), (name, world)


def test_single_slab_is_the_periodic_domain():
    """One slab with the transport of a one-rank group: its own faces are its neighbours."""

    class Solo:
        def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
            recv_hi.copy_(send_lo)
            recv_lo.copy_(send_hi)

    name, shape, tau, n = "D3Q19", (5, 4, 6), 0.7, 4
    s = oracle.velset(name)
    rho, u, th = inputs.random_fields(shape, s.D, 3)
    g0 = oracle.equilibrium(name, rho, u, th)
    ring = slab.SlabRing(OracleSlab(name, shape, tau, oracle.post_state(name, shape, tau, g0), 0, shape[2]), Solo())
    ring.step(n)
    want = oracle.post_state(name, shape, tau, oracle.step(name, shape, tau, g0, n))
    assert np.array_equal(ring.slab.own.reshape(s.q, -1), want)


def test_partition():
    assert slab.partition(10, 3) == [(0, 4), (4, 3), (7, 3)]
    assert slab.partition(384, 4) == [(0, 96), (96, 96), (192, 96), (288, 96)]
    assert sum(c for _, c in slab.partition(1001, 7)) == 1001
    with pytest.raises(ValueError):
        slab.partition(2, 3)
